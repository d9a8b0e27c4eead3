"""GB300-native resampling stage of the bootstrap particle filter.

The compute path is the C-ABI library ``libpf.so`` (hand-written sm_103a CUDA,
declared in ``include/pf.h``).  ``paper_1202_6163_gb300.pf`` is the thin ctypes
binding with the same entry-point names; it loads the library on first use and
raises if it has not been built.  ``workloads`` holds the seeded synthetic
input generators.
"""
