"""Seeded synthetic inputs (forests and data) shared by the oracle tests, the CUDA
parity tests and the benchmark.  No star-forest arithmetic lives here."""
from . import rng
from .forests import (Forest, fig2, random_forest, one_to_one, pingpong, from_lists,
                      cfg1_plain_tiny, cfg2_halo, cfg4_batched, cfg5_powerlaw, zipf_forest, owned_plus_ghosts,
                      data)
from .rgg import cfg3_spmv

__all__ = ["rng", "Forest", "fig2", "random_forest", "one_to_one", "pingpong", "from_lists",
           "cfg1_plain_tiny", "cfg2_halo", "cfg3_spmv", "cfg4_batched", "cfg5_powerlaw",
           "zipf_forest", "owned_plus_ghosts", "data"]
