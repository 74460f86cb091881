"""FP64 CPU oracle for summed total communicability (arXiv 1409.5000).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call,
link or execute anything in this package: only the tests, the smoke check
and the benchmark's CPU-baseline / reference arm do.  It shares no code
with the CUDA library; both sides consume the same seeded inputs.

Contents (each function cites the passage of the paper it follows):

* :mod:`oracle.communicability` -- dense e^A by scaling and squaring
  (eq. 3, eq. 4 written out), the m-step Lanczos (Krylov) approximation of
  e^A 1 with full reorthogonalisation ("Identification algorithm", the
  Krylov evaluation of e^A 1), the ensemble sum (eq. 5) and the top-k
  selection by a full sort ("Identification algorithm": the k largest EBTC).
* :mod:`oracle.adjoint` -- the Frechet derivative of the summed top-k
  score with respect to edge weights (dense, two independent ways, and the
  Krylov form used for checking at scale).  The paper has no gradient;
  this is an extension whose definition is the derivative itself.

Everything is plain numpy / scipy in float64; library primitives used as
steps are a sparse matrix-vector product, a dense symmetric eigensolver,
a dense matrix product and a sort.
"""
