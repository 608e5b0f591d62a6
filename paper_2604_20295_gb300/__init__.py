"""GB300 (sm_103a) implementation of ETac's per-step tactile hot path (arXiv 2604.20295):
batched SDF contact and the decay + residual-network deformation propagation model, behind
the C ABI of ``include/etac.h``.

Submodules: ``inputs`` (seeded synthetic scenes, no method arithmetic), ``build`` (nvcc build
of libetac.so), ``etac`` (ctypes binding and ``TactileSim``).  Nothing is loaded at import
time; the binding raises when the library is missing.
"""
__all__ = ["inputs", "build", "etac"]
