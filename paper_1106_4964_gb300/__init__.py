"""GB300-native overlap-fermion library (hot path of arXiv:1106.4964).

``binding`` marshals Python arguments into the C ABI of ``libovgb.so``
(include/overlap.h); ``build`` compiles the CUDA sources for sm_103a.
"""
from .binding import (OV_BF16S, OV_DF64, OV_F16S, OV_F32, OV_F64, PREC, Context, Field, OverlapError,
                      declared_symbols, load, measure_fma_peak)

__all__ = ["Context", "Field", "OverlapError", "load", "declared_symbols", "OV_F64", "OV_F32", "OV_F16S",
           "OV_BF16S", "OV_DF64", "PREC", "measure_fma_peak"]
