"""CI-SCvx discretization/linearization on GB300 (sm_103a).

The compute lives in the C-ABI library ``libciscvx.so`` (CUDA kernels, see
``include/ciscvx.h``); :mod:`.api` is a thin ctypes binding with the same entry
point names, :mod:`.synth` the seeded synthetic robots and instances.
Importing the package loads nothing; :func:`api.load` opens the library.
"""
__all__ = ["api", "synth"]
