"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package draws random numbers only.  It holds none of the method's
arithmetic (no integrals, amplitudes or matrix elements), so that the CPU
oracle and the CUDA path stay independent while consuming identical inputs.
"""

from .inputs import (  # noqa: F401
    DotInputs,
    CONFIGS,
    make_inputs,
    scaled_sigma_b,
    perturbative_sigma_b,
    random_vectors,
    window_start,
)
