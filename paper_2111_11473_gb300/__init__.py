"""Python binding of libthc.so, the GB300 THC-RR-CCSD residual library.

Argument marshalling only: every step of the residual, energy and solve runs
in the CUDA library behind the C ABI declared in ``include/thc.h``.  There is
no CPU fallback: if the library is not built, or no GPU is visible, the calls
raise.
"""
from .binding import (Context, Mlp, Report, ThcError, load_library, exported_symbols,
                      THC_PREC_FP64, THC_PREC_MIXED, THC_PREC_FP64_TC)

__all__ = ["Context", "Mlp", "Report", "ThcError", "load_library", "exported_symbols",
           "THC_PREC_FP64", "THC_PREC_MIXED", "THC_PREC_FP64_TC"]
