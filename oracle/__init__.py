"""Oracle: plain, slow, FP64 CPU restatement of the QTT-FEM method.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only `tests/`, `__graft_entry__.smoke()`
and the CPU-baseline leg of `bench.py` may import it.  The CUDA library never
calls into it, and it shares no code with the CUDA path: the two meet only in
the seeded input descriptions of the `workloads` module.

Contents
--------
fem       O-1: sparse Q1 plane-stress finite elements (Sections 3.3-3.8),
          merged-node (conforming) and duplicated-node (concatenated)
          multi-patch systems, sparse direct solve.
indexing  Canonical and Z-order node numbering (Section 3.2).
tt        O-2: dense-reference tensor-train layer (Section 4): TT-SVD,
          full/dense expansion, MPO x MPS product, rounding, z-kron, norms,
          effective rank and parameter counts.
assembly  O-2: QTT assembly of K and f (Algorithm 1) built from 1D FE
          matrices compressed by TT-SVD and combined by z-kron.
amen      O-2: alternating minimal energy solver with residual enrichment
          (the solver the paper cites for K u = f; written from the
          Dolgov-Savostyanov 2014 formulation, see its module docstring).

Parity status
-------------
Every function is pinned by a `-m "not gpu"` test in tests/test_oracle_*.py
against something other than itself (closed forms, brute force, textbook
element matrices, convergence rates, invariants).  The paper's printed
figure values (memory, erank, R_d, N_d for the cantilever / SEN / L-shape
geometries) are parity unpinned: those geometries exist only in figures the
source does not contain.
"""
