"""CPU oracle for the GF(2)[x] product and its stages.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package.  It shares no code, table or
constant with the CUDA library under paper_1708_09746_gb300/, and never
imports it.

Modules:
  product  -- ctypes wrapper over gf2x_oracle.c: the plain carry-less product
              (definition of the method's output, Alg. 5), brute force, and
              the modular fingerprint.  Parity: pinned.
  stages   -- slow, step-by-step restatement of the paper's stages (tower
              field of Sec. 3.2, s_k of Def. 2.2, BasisCvt of Alg. 2/3,
              FFT_LCH of Alg. 1, changeRepr of Sec. 4.3, InterleavedCombine of
              Sec. 2.1) used to check the GPU stages one by one.  Parity:
              pinned by brute force and the paper's worked examples.
"""
