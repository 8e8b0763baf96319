// The branch kernels and their launches for bitset width W = 1 (sub-branches of
// 0..32 vertices); see kc_branch_dev.cuh.
#define KC_BRANCH_INSTANTIATE
#include "kc_branch_dev.cuh"

KC_BRANCH_WIDTH(1)
