"""GB300 (sm_103a) hot path of Clifford-based circuit cutting.

``ccs`` is a thin ctypes binding of ``libccs.so`` (declared in
``include/ccs.h``): argument marshalling only, every step of the path runs in
the library's CUDA kernels.  Importing the package does not load the library;
the first ``ccs`` call does, and fails loudly if it cannot.
"""
