"""PSWF-LR reciprocal-space evaluation on B300 (sm_103a).

The compute path lives in the C-ABI library ``libpswf_lr.so`` (CUDA kernels
plus cuFFT); :mod:`paper_2606_06617_b300.lr` is the thin ctypes binding.
Importing this package does not load the library; the binding loads it on
first use and raises if it is missing.
"""
__all__ = ["lr", "workloads"]
