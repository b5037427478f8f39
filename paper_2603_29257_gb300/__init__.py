"""GB300-native TDA-risp (arXiv 2603.29257): FP64 CUDA kernels for sm_103a behind
the C ABI in include/tdarisp.h, with a thin ctypes binding (tdarisp.Context)
and a seeded synthetic-molecule generator (synth).

Importing the package does not load the CUDA library; tdarisp.lib() does, and
raises if it has not been built."""
