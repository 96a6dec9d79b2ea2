"""phtl: GB300-native (sm_103a) turn-by-turn macro-particle tracking.

The compute path lives in the CUDA library ``libphtl.so`` (sources in ``csrc/``,
C-ABI declared in ``include/phtl.h``); ``phtl.py`` is a thin ctypes binding that
passes PyTorch device pointers and streams through.  ``synth.py`` draws seeded
synthetic inputs.
"""
