"""GB300-native variable-density pressure multigrid (arXiv 1410.8568, Sec. 2.3).

The solver lives in the CUDA library ``libgbmg.so`` (sources in ``csrc/``,
C ABI in ``include/gbmg.h``).  ``gbmg`` is its thin ctypes binding; ``inputs``
builds the seeded synthetic density fields and right-hand sides.
"""
