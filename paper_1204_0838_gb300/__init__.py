"""GB300-native (sm_103a) explicit 3D electromagnetic PIC step of the
perfect-dispersion Cartesian laser-wakefield method (Cowan, Kalmykov et al.,
J. Plasma Phys. 2012, arXiv:1204.0838): cubic-spline gather, Boris push,
Esirkepov cubic deposit, smoothed-curl field update and moving window, in
hand-written CUDA kernels behind the C-ABI of include/pic.h."""
from . import pic  # noqa: F401
from .pic import Sim  # noqa: F401
