"""CPU oracle of randomized strong recursive skeletonization (RSRS), arXiv 2311.01451.

TEST INFRASTRUCTURE.  This package is a plain, slow, FP64 restatement of the
method, written from the paper to check the CUDA library against.  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the library never does, and the two share no code (only the
seeded inputs of ``workloads``).

Modules:
    tree       -- quad/octree, neighbours, processing order, sample bound (Sec. 3, 4.4)
    operators  -- the matrices A (kernel, 7-point) and the sketches Y, Z (eq. rand_sample_setting)
    linalg     -- null, pseudoinverse, CPQR-based ID, LU (Sec. 2)
    rsrs       -- Algorithm 1, its factorization, solve and apply (eqs. Afact, Ainvfact)
    refine     -- FP64 iterative refinement, GMRES with the factor as preconditioner, and the
                  metrics of eq. (error)

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, brute force at tiny N and the paper's printed sample
counts.
"""
