"""GB300-native SIR particle filter for single-spot tracking (PPF, Demirel et
al.): propagation, patch likelihood, normalisation, estimate and the
systematic / RPA (GS, SGS, LGS, one- and two-stage) / RNA / ARNA resampling steps as hand-written CUDA
kernels for sm_103a behind the C ABI of ``include/ppf.h``."""

from ._binding import (  # noqa: F401
    ARNA,
    BF16,
    ECUDA,
    EDEGENERATE,
    EINVAL,
    ENOMEM,
    ESTATE,
    ETIMEOUT,
    F16,
    F32,
    OK,
    PATH_AUTO,
    PATH_BINNED,
    PATH_DIRECT,
    RNA,
    RPA_GS,
    RPA_LGS,
    RPA2_GS,
    RPA2_LGS,
    RPA2_SGS,
    RPA_SGS,
    SCHEMES,
    SYSTEMATIC,
    BatchFilter,
    Estimate,
    fp32_peak,
    Model,
    ParticleFilter,
    PPFError,
    load,
    log_marginal_likelihood,
    lib_path,
    status_string,
)
from ._build import build  # noqa: F401
