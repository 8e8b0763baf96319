"""Seeded synthetic inputs (graphs, batches, query traces); no k-clique arithmetic."""
from .graphs import *  # noqa: F401,F403
