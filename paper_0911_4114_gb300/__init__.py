"""GB300-native Fourier-basis Helmholtz FMM apply (Cecka & Darve, arXiv 0911.4114).

phi_i = sum_j q_j exp(i kappa |x_i - y_j|) / |x_i - y_j| through the C-ABI library
libhfmm.so (include/hfmm.h).  Importing this package loads nothing; the library is
loaded on first use and its absence is an error, never a fallback.
"""
from .plan import FmmBatch, FmmPlan  # noqa: F401

__all__ = ["FmmPlan", "FmmBatch"]
