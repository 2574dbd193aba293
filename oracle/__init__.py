"""CPU oracle for the matrix-free 3D SIMP hot path (arXiv 2604.18020).

TEST INFRASTRUCTURE ONLY.  A plain FP64 numpy restatement of the method,
written from the paper and pinned by the `-m "not gpu"` tests against
closed forms, invariants, brute force and the paper's printed values.  It
shares no code with the CUDA library and imports nothing from it.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.

Modules: fem (indexing, KE, K.v, assembly, Jacobi diagonal), filter (cone
filter), solve (Jacobi-PCG, dense solve), simp (compliance, sensitivities,
OC, SIMP loop), refine (FP64 iterative refinement around a low-precision
inner PCG), nn (3D-conv U-Net forward/backward).
"""
