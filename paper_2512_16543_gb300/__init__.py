"""GB300-native Woodbury + adaptive randomized SVD (WB-arSVD) RZF precoder updates.

The compute path lives in the CUDA library built from ``csrc/`` (C ABI declared in
``include/wbrzf.h``); ``binding`` is the thin ctypes layer over it.  ``channel`` is the seeded
synthetic-input generator.  Submodules are imported on demand so that importing the channel
generator never loads the CUDA library.
"""
__all__ = ["binding", "channel"]
__version__ = "0.1.0"
