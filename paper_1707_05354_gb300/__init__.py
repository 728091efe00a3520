"""GB300-native GPU LSM: a batched dynamic dictionary (arXiv 1707.05354).

The compute path is ``libgpulsm.so`` (hand-written sm_103a CUDA behind the C ABI
declared in ``include/gpulsm.h``).  ``gpulsm`` is the ctypes binding; importing
it loads the library and raises if it is missing.  ``workload`` holds the
seeded synthetic input generators.  This package file imports neither, so
that the generators can be used without a GPU.
"""

__all__ = ["gpulsm", "workload", "build"]
