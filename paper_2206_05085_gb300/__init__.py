"""GB300-native (sm_103a) DVGOv2 volume-rendering training step.

The compute path is ``libdvgo.so`` (hand-written CUDA kernels behind a C
ABI, declared in ``include/dvgo.h``); ``_lib`` binds it with ctypes,
``ops`` wraps the forward/backward pairs as ``torch.autograd.Function``s and
``train`` strings one training iteration together.  Importing this package
does not load the library; the first op call does, and raises if the
library has not been built (there is no CPU fallback).
"""
__all__ = ["synth"]
