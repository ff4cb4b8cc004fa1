"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This package draws matrices and right-hand sides only; it contains none of
the solver's arithmetic.  See ``synth.randsvd`` for the recipe.
"""

from .randsvd import (randsvd_system, batched_systems, workloads, serving_pool,  # noqa: F401
                      poisson_arrivals)
