"""GB300-native matrix-free BCSR Hamiltonian (arXiv:1907.01005 hot path).

The compute path is libfe_mf.so (hand-written CUDA for sm_103a behind a C
ABI, include/fe_mf.h); this package is its ctypes binding.
"""
from ._capi import (FE_EDEVICE, FE_EINVAL, FE_ENOMEM, FE_EPATTERN, FE_ESTATE, FE_ECUDA,
                    FE_EUNSUPPORTED, FE_F32, FE_F64, FE_OK, FORM_CELLMAT, FORM_SUMFAC, FeError, check,
                    last_error, load)
from .api import (BCSR, Mesh, StepGraph, apply_H, apply_H_gram, apply_M, mmult, om_gradient, trace_dot, apply_H_gram_host, autotune, gram_PtP,
                  gram_PtY, gram_PtY_sym)

__all__ = ["Mesh", "BCSR", "apply_H", "apply_M", "mmult", "om_gradient", "trace_dot", "gram_PtY", "gram_PtY_sym", "gram_PtP", "apply_H_gram", "apply_H_gram_host",
           "StepGraph", "autotune", "FeError", "FE_F32", "FE_F64", "FORM_SUMFAC", "FORM_CELLMAT", "load", "check", "last_error"]
