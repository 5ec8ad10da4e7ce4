"""GB300-native (sm_103a) B-spline multilevel summation method (MSM) for electrostatics.

The method is the one of arXiv 2510.05961 (msmJAX): energy, potentials and
forces of N point charges in open, slab or periodic orthorhombic cells, plus a
hand-written adjoint for dE/dr, dE/dq and the virial, and a batched mode for
many systems. The compute path is the CUDA library ``lib/libmsm_gb300.so``
(C ABI in include/msm_gb300.h); this package is its thin Python binding.
"""
from .msm import LEVELS_BALL, LEVELS_SPECTRAL, SHORT_CLUSTER, Batch, MSMFunction, Plan, msm_energy, msm_outputs  # noqa: F401
