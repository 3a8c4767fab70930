"""GB300 (sm_103a) particle collision and projection operator of arXiv 2501.05340.

``pc``        binding of the C ABI (``include/pc.h``) of the CUDA library ``libpc.so``
``autograd``  differentiable multi-step rollouts on the hand-written adjoints
``inputs``    seeded synthetic workloads (no method arithmetic)
``build``     in-tree nvcc build of ``libpc.so``
"""
