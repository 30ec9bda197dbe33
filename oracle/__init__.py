"""Oracle: plain, slow, CPU-only restatement of what the GEMM path computes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from here.  The CUDA
library never links, imports or calls this package, and this package never
imports the library: the two share no code.  The only module both sides use is
``cosma_inputs`` (seeded input generation, which holds none of the method).

Modules
  gemm      C = A B by its definition (naive partial-sum chain and compensated
            Dot2), sampled entries, Freivalds' check -- C core in gemm_oracle.c.
  pebble    red-blue pebble game simulator (Sec. 2.2) that replays a schedule
            given as data and counts its loads and stores.
  bounds    the paper's closed forms: Theorem 1, Theorem 2, eq. (a_opt, b_opt),
            eq. optTileShape, Table 2, the Corollary, and brute-force /
            exhaustive searches (FindSeqSchedule, FitRanks).
  mlp       FP64 forward/backward/Adam of the selector's 3-layer MLP.

Parity status per function is stated in each module's docstring.
"""
