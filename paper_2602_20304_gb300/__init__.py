"""GB300 (sm_103a) implementation of smooth, differentiable contact-manifold generation
(arXiv 2602.20304): a CUDA library behind a C ABI (``include/contact_manifold.h``), its
ctypes binding (``api``) and the batching layer on top (``engine``)."""

__all__ = ["api", "engine"]
