"""GB300-native RACIPE ensemble solver (GRiNS, arXiv 2503.18356).

The compute path is the C-ABI library ``libgrins_racipe.so`` (hand-written
CUDA for sm_103a, built in this folder); ``api`` is its thin Python binding.
Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["api", "workloads"]
