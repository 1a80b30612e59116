"""GB300-native two-level spectral Schwarz PCG for SIMP linear elasticity
(M_EH / M_EH+Rot of arXiv 2006.13387), behind the C ABI of libtopsolve.so.

Import is cheap: the shared library is loaded on first use (api.Context).
"""
from .api import Context, Design, TopSolveError, design_from_problem  # noqa: F401
