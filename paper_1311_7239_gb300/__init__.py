"""GB300-native porous D2Q8 MRT lattice Boltzmann solver (Liu & He, arXiv 1311.7239).

The compute path is the CUDA library ``liblbm.so`` (sources in ``csrc/``, C-ABI in
``include/lbm.h``); ``paper_1311_7239_gb300.lbm`` is its thin ctypes binding.  Importing this
package loads nothing: the library is opened on first use and a missing library is an error.
"""
