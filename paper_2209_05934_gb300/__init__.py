"""GB300-native orbital-minimization (OMM) conjugate-gradient library.

The compute path is the CUDA library libomm_gb300.so (C ABI in include/omm.h);
`paper_2209_05934_gb300.omm` is its thin ctypes binding.
"""
