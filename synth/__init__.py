"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This package only *generates data*: Poisson-noise movies of one moving
Gaussian-PSF spot (the experimental setup of Sec. 7.3: a spot moving under
near-constant-velocity dynamics, imaged through a Gaussian PSF, eq. 3, with
shot noise) and batches of such movies.  It contains no part of the particle
filter itself, so both the CUDA path and the FP64 oracle can consume its
output without sharing any of the method's arithmetic.
"""

from .movies import (  # noqa: F401
    Movie,
    MovieBatch,
    amplitude_for_snr,
    make_movie,
    make_movie_batch,
    preset,
    PRESETS,
)
