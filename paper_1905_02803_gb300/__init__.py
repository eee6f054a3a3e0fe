"""GB300-native 3D real-to-complex / complex-to-real transforms (P3DFFT method).

The compute path is the C-ABI library built from csrc/ (hand-written CUDA for
sm_103a); `p3dfft` is its thin ctypes binding.  Importing this package does
not load the library: the binding loads it on first use and raises if it is
missing, so no call can silently fall back to another implementation.
"""
__all__ = ["p3dfft", "inputs"]
