"""GB300-native particle inference: likelihood weighting, SMC resampling and the
posterior reduction as sm_103a CUDA kernels behind a C ABI (include/ppl.h)."""
from .binding import *  # noqa: F401,F403
from .binding import lib, exported_symbols  # noqa: F401
