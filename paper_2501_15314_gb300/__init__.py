"""GB300-native Laplacian-preconditioned Schur solver for the SIMPLE-based
direct-forcing immersed boundary method (arXiv 2501.15314).

* ``libibmschur.so`` (built from ``csrc/`` by ``build.py``): the C ABI of
  ``include/ibm_schur.h``, all computation in hand-written sm_103a kernels;
* ``_lib``: ctypes declarations with the C names;
* ``api``: torch-facing wrapper (device memory and streams from PyTorch);
* ``workloads``: seeded synthetic inputs.

Importing the package does not load the CUDA library; ``api`` does, and
raises if it is missing.
"""
__all__ = ["api", "workloads", "build"]
