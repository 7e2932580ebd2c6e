"""GB300-native batched RKCK / RKC integration of many independent small ODE
systems (Niemeyer & Sung, "GPU-Based Parallel Integration of Large Numbers
of Independent ODE Systems").

The compute path is ``libbatchode.so`` (hand-written CUDA for sm_103a behind
the C ABI of include/batchode.h); ``binding`` is its ctypes front end and
``workloads`` draws seeded synthetic inputs.
"""
__all__ = ["binding", "workloads", "build"]
