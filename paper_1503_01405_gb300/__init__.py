"""GB300-native phase-coherent dedispersion engine (PONDER, Sec. 3.7).

The compute path lives in ``libpond.so`` (C ABI, ``include/pond.h``); the
``pond`` module is its ctypes binding.  ``synth`` makes seeded test streams.
"""
__all__ = ["pond", "synth"]
