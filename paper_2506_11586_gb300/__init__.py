"""GB300 (sm_103a) library for the homomorphic-convolution hot path of SecONNds
(arXiv 2506.11586): batched negacyclic NTT / INTT over RNS limbs and the
NTT-domain ciphertext x plaintext multiply-accumulate of its linear layers
(Sec. 6.2), plus the Z_P operations of SecONNds-P's layers (SIMD encoding,
key-switched slot rotations, the multiply-accumulate-rotate iteration; Sec.
6.1), behind a C ABI (include/hconv.h).

  build    -- compiles csrc/*.cu into _build/libhconv.so with nvcc
  _lib     -- ctypes binding with the C entry points' names
  inputs   -- seeded synthetic workloads (random numbers and shapes only)
  serving  -- Poisson-arrival driver of the library's request loop
  replicas -- one-process-per-GPU replica plumbing (barrier, max-over-ranks)
"""
