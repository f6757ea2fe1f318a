"""GB300-native softened direct-sum n-body force path (sm_103a CUDA).

The compute runs in ``libnbody.so`` (hand-written CUDA behind a C ABI,
declared in ``include/nbody.h``); :mod:`paper_1211_2292_gb300.nbody` is the
thin ctypes binding, :mod:`paper_1211_2292_gb300.autograd` the
``torch.autograd.Function`` over the adjoint kernels, and
:mod:`paper_1211_2292_gb300.inputs` the seeded initial conditions.
"""
__all__ = ["inputs", "nbody"]
