"""GB300-native D2Q9 cascaded lattice Boltzmann step with consistent forcing
(Fei & Luo, arXiv:1705.11092).

The compute path is the CUDA library built from ``csrc/`` behind the C ABI of
``include/clbm.h``; ``clbm`` is its thin ctypes binding.  Importing this
package loads nothing; the library is loaded on first use and its absence is
an error, never a fallback.
"""
