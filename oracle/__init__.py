"""Plain, slow CPU oracle for homomorphic CutMax (arXiv 2509.08383).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA library in ``paper_2509_08383_gb300``.

Contents
  ckks.py        ctypes wrapper of ckks_oracle.c (RNS-CKKS by definition)
  encoding.py    canonical-embedding encode / decode in numpy float64
  cutmax_fp64.py Alg. 1 (exact CutMax) and the FP64 mirror of Alg. 2
  circuit.py     Alg. 2 / Alg. 3 as a sequence of oracle CKKS operations
  bootstrap.py   CKKS bootstrapping on oracle operations
  build.py       compiles ckks_oracle.c with gcc
"""
