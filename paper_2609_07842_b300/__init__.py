"""B300-native valency-bounding correction (VBC) force/energy evaluation.

The compute path is the CUDA library ``libvbc.so`` (C ABI declared in
``include/vbc.h``); ``paper_2609_07842_b300.vbc`` is its ctypes binding.
The binding is imported lazily so that ``paper_2609_07842_b300.inputs`` (the
seeded input generators) can be used without a GPU.
"""
__all__ = ["inputs", "vbc"]
