"""GB300-native two-level solver for B-spline IGA Poisson problems.

The compute path is the CUDA library ``libiga2l.so`` behind the C ABI in
``include/iga2l.h``; ``paper_2009_01499_gb300.iga2l`` is its thin ctypes
binding.  Importing this package does not load the library; the binding loads
it on first use and raises if it is missing.
"""
