"""GB300 live Wigner Distribution Deconvolution (arXiv 2212.01309) behind a C ABI.

The compute path is libwdd.so (hand-written sm_103a CUDA kernels, declared in include/wdd.h);
`wdd` is its Python binding.  Build the library with `python -m paper_2212_01309_gb300.build`.
"""
from . import wdd  # noqa: F401
from .wdd import Plan, Params, WddError, make_params, params_from_acquisition  # noqa: F401

__all__ = ["wdd", "Plan", "Params", "WddError", "make_params", "params_from_acquisition"]
