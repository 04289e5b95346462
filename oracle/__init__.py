"""CPU FP64 oracle for the tensor Krylov solvers of the Sylvester tensor equation.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package.  The CUDA library never calls it and
shares no code with it; the two meet only in the seeded input generators of
paper_2405_09233_gb300.inputs, which hold none of the method's arithmetic.

Every routine here is a plain, slow restatement of the paper's definitions and
algorithms in numpy float64 (numpy/scipy library primitives such as a matrix
product, a dense solve, a least-squares solve or a complex Schur form serve as
single steps).  The T-product is computed from its block-circulant definition
(Definition 2.1), never by an FFT.

Modules:
  tproduct  -- bcirc/unfold/fold, T-product, transpose, identity, inner
               product, T-diamond, explicit DFT along mode 3 (§2)
  krylov    -- Sylvester operator M, tArnoldi, tFOM, tGMRES (§3, Algorithms 2-3)
  tubal     -- Normalize, Tubal-QR, Tubal Block Arnoldi, TBAS(m) (§5, Algorithms 6-8)
  schur     -- t-Schur and t-Bartels-Stewart (§4, Algorithms 4-5)

Parity pins: every function above is pinned in tests/test_oracle_*.py against
something other than itself (closed forms, library routines for the special
cases the paper reduces to, hand-computed examples, brute force, invariants
the paper proves).  No function here is "parity unpinned".
"""
from . import tproduct, krylov, tubal, schur  # noqa: F401
