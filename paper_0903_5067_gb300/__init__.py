"""GB300 (sm_103a) fluctuating D3Q19 lattice Boltzmann + bead-spring chain library.

The compute path is the CUDA shared library built from ``csrc/`` (C ABI declared in
``include/lb.h``); ``lb`` is its thin ctypes binding.  Importing this package does not load
the library; ``from paper_0903_5067_gb300 import lb`` does, and raises if it is missing.
"""
