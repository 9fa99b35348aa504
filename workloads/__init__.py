"""Seeded synthetic inputs for the matrix-probing hot path.

This package only *generates inputs*: background models m0 = 1/c^2, source and
receiver positions, the source wavelet, model perturbations and probing trial
functions.  It contains none of the method's arithmetic (no stencil, no time
stepping, no symbol expansion), so that the FP64 oracle and the CUDA path can
both consume exactly the same arrays without sharing any computational code.

Every generator draws from ``numpy.random.Generator(PCG64(seed))`` and returns
float32 arrays, so both sides see bit-identical inputs.
"""
from .synth import (  # noqa: F401
    Workload,
    ricker,
    layered_background,
    linear_background,
    bandpassed_noise,
    random_sign_trials,
    gaussian_bumps,
    white_noise_trials,
    make_config,
    data_noise,
    mini_config,
    CONFIG_NAMES,
)
