"""GB300-native (sm_103a) ghost-celled ideal-MHD patch advance.

The hyperbolic advance of grid patches that the AMR scheme of Carroll-Nellenback
et al. (Sec. 2.2-2.3) parallelises, with the ghost fill, CFL time step and
conservation sums that feed it, behind the C ABI of ``include/mhd_gpu.h``.
"""
from . import capi  # noqa: F401  (fails loudly if the CUDA library is missing)
from .patch import Patch, patch_shape, periodic_copies, update_box_schedule  # noqa: F401

__all__ = ["capi", "Patch", "patch_shape", "periodic_copies", "update_box_schedule"]
