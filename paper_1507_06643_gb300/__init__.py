"""GB300-native DPDE timestep (Homman, Maillet, Roussel, Stoltz,
arXiv:1507.06643): CUDA kernels for sm_103a behind the C ABI of
include/dpde.h, with a thin ctypes binding in :mod:`.dpde`."""
from . import dpde  # noqa: F401
from .dpde import System, make_params, make_replica  # noqa: F401
