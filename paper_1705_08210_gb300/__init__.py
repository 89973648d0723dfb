"""GB300-native (sm_103a) Proportional Similarity library.

The compute path is the C-ABI shared library ``libps.so`` built from
``csrc/``; ``ps`` is its thin ctypes binding and ``synth`` draws seeded
synthetic inputs.  Import ``paper_1705_08210_gb300.ps`` to load the library.
"""
__all__ = ["ps", "synth"]
