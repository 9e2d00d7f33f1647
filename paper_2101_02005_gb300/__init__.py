"""GB300-native (sm_103a) hot path of the HELIOS-K 2.0 opacity method
(Grimm et al. 2021, arXiv:2101.02005): per-line strengths and widths, Voigt
profiles evaluated on every wavenumber bin inside the cut, summed into the
cross section sigma(nu), with batched and adjoint entry points.

The compute path is the C-ABI library ``libhk`` (hand-written CUDA in
``csrc/``); ``hk`` is its thin ctypes binding.  Importing this package does
not load the library; ``from paper_2101_02005_gb300 import hk`` does.
"""
__all__ = ["hk", "synth"]
