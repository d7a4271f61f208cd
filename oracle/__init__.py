"""CPU oracle for the homomorphic linear-layer path (TEST INFRASTRUCTURE).

Plain, slow, obviously-correct reference used only by ``tests/``, the package
``smoke()`` check and the benchmark's CPU-baseline leg.  It shares no code with
the CUDA library: its C core (``he_oracle.c``) has its own prime search, NTT,
ChaCha20 generator and big-integer CRT, and its packing module has its own plan
search.  The only thing both sides import is the seeded input generator module
``paper_2409_16675_gb300.workloads``.

Modules
  he        -- keygen / encrypt / decrypt / CPMul / CCMul / PPMul (Section 2, HE
               and Motivation; Section 3.2)
  packing   -- conventional (row-major) and correlated polynomial encodings and
               the partition-window search (Section 3.3, Eq. 1-2)
  protocol  -- the CryptoTrain-P linear layer (Section 3.2) composed from the two
"""
