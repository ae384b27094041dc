"""B300-native multi-body Nystrom operator library (arXiv 2606.31380, Lai & Li).

The compute path is the C-ABI shared library ``libqams.so`` (hand-written
CUDA for sm_103a, declared in ``include/qams.h``).  This package is only its
ctypes binding; there is no CPU fallback: importing it without the built
library, or calling it without a CUDA device, raises.
"""
from ._binding import (PREC_FF, PREC_FP32, PREC_FP64, PROF_ASSEMBLY, PROF_BLOCK_FP32,  # noqa: F401
                       PROF_BLOCK_FP64, PROF_BLOCK_TC, OPT_TC_MIN_RHS, OPT_TC_PAIR_MIN_RHS, OPT_PAIR_TARGETS, OPT_LATTICE, OPT_NEAR_FIELD, PROF_PAIRSUM_TC, PROF_PAIRSUM_LATTICE, PROF_LATTICE_PRODUCT32, PROF_LATTICE_PRODUCT64, PROF_PAIRSUM_FF, PROF_PAIRSUM_FP32, PROF_PAIRSUM_FP64, Context, QamsError,
                       Server, body_desc_array, body_nodes, footprint, kernel_launches, lib_path, load_library,
                       nearest_surface_point)

__all__ = ["Context", "Server", "QamsError", "PREC_FP64", "PREC_FP32", "PREC_FF", "load_library", "lib_path",
           "body_desc_array", "body_nodes", "footprint", "kernel_launches", "nearest_surface_point", "PROF_PAIRSUM_FP32", "PROF_PAIRSUM_FF",
           "PROF_PAIRSUM_FP64", "PROF_BLOCK_FP32", "PROF_BLOCK_FP64", "PROF_ASSEMBLY", "PROF_BLOCK_TC",
           "OPT_TC_MIN_RHS", "OPT_TC_PAIR_MIN_RHS", "OPT_PAIR_TARGETS", "OPT_LATTICE", "OPT_NEAR_FIELD", "PROF_PAIRSUM_TC",
           "PROF_PAIRSUM_LATTICE", "PROF_LATTICE_PRODUCT32", "PROF_LATTICE_PRODUCT64"]
