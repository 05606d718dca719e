"""B300-native Lancelot server evaluation: RNS-CKKS encrypted pair distances and masked
aggregation as hand-written sm_103a CUDA kernels behind a C ABI (include/lancelot.h).

`paper_2408_06197_b300.lancelot` is the thin ctypes binding of liblancelot.so; the native
library is loaded on first use and a missing or unloadable library raises immediately (there
is no CPU fallback).  `kgc` holds the plaintext key-generation-center selection rules.
"""
