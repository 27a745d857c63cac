"""GB300-native (sm_103a) LHMM micro/macro hot path of arXiv 2512.13267.

The compute path is the C-ABI CUDA library ``liblhmm.so`` (built from
``csrc/``); ``lhmm`` is its thin ctypes binding and ``synth`` makes seeded
synthetic inputs.  Importing the package does not load the CUDA library.
"""
__all__ = ["lhmm", "synth"]
