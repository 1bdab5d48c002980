"""GB300-native fused RHS + low-storage RK3 stage for the 3D compressible
Navier-Stokes equations (Jammy, Jacobs, Lusher & Sandham, arXiv:1709.09713).

The compute path is the CUDA library ``lib/libsbli.so`` (sm_103a); the
``sbli`` module is a thin ctypes binding over its C ABI (``include/sbli.h``).
Importing this package does not load the library; ``sbli.lib()`` does, and it
raises if the library has not been built.
"""

__all__ = ["sbli", "workloads"]
