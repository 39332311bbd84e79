"""GB300-native butterfly filtering (arXiv:1802.01685, Sect. 2.1-2.2).

The compute path is the CUDA library ``libbf.so`` behind the C ABI in
``include/bf.h``; ``paper_1802_01685_gb300.bf`` is its thin ctypes binding.
Importing this package loads nothing; ``bf`` loads the library on first use and
raises if it is missing.
"""
__all__ = ["bf", "synth"]
