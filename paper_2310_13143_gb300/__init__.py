"""GB300 (sm_103a) SQP-ADMM solver for AC optimal power flow.

The compute path is the C-ABI library ``libacopf.so`` (CUDA kernels for
sm_103a, built by :mod:`paper_2310_13143_gb300.build`); :mod:`.binding` is its
thin ctypes wrapper.  :mod:`.gridgen` draws seeded synthetic inputs.
"""
__all__ = ["binding", "build", "gridgen"]
