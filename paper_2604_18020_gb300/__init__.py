"""Matrix-free 3D SIMP topology optimisation on one GB300 (sm_103a).

The compute path is libmfto.so (hand-written CUDA behind the C ABI of
include/mfto.h); ``mfto`` is its thin ctypes binding and ``workloads`` builds
seeded synthetic problems.  Submodules load lazily so that importing the
package needs neither a GPU nor the built library.
"""
__all__ = ["mfto", "workloads", "build"]
