"""GB300 (sm_103a) Artificial Retina: grid scan, truncated-Newton multistart
search and track extraction of arXiv:1709.08610 as hand-written CUDA kernels
behind a C ABI (include/retina.h).  ``retina`` is the Python binding; import it
explicitly (``from paper_1709_08610_gb300 import retina``) - it needs the
built library and raises if it is missing.
"""
__all__ = ["build", "retina"]
