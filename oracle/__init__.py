"""CPU oracle for TDA-risp (arXiv 2603.29257) -- TEST INFRASTRUCTURE ONLY.

Plain FP64: Obara-Saika integrals in C (ints.c) and the method's
definitions in NumPy (tda.py).  Only tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg may import it.  It shares no code with the CUDA
library under paper_2603_29257_gb300/ and never imports it.
"""
