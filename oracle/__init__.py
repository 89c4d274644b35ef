"""INV-ASKIT oracle: a plain, slow, FP64 CPU restatement of the method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs may import this package.  The product
(the CUDA library and its Python binding) never calls it, and the two share no
code: this package imports nothing from the product package and the product
imports nothing from here.

What is computed (Yu, March, Xiao, Biros, "INV-ASKIT", arXiv 1602.01376):

* ``kernel``   Gaussian kernel, eq. (gaussian) of Sec. I; the polynomial kernel of
               Sec. IV (degree and constant chosen here, selected by a context).
* ``tree``     balanced binary partition (Sec. II-A) and exact kNN lists (Sec. II-B).
* ``sampling`` nearest-neighbour row sampling plus uniform fill (Sec. II-B).
* ``linalg``   partial-pivoting LU (GETRF/GETRS of Alg. "Factorize"/"Solve") and
               column-pivoted QR with its interpolative decomposition (GEQP3 + GELS,
               Sec. II-B/II-C).
* ``askit``    skeletonization, nested projections P (eq. innerid), the dense
               definition of K~ (eqs. offdiag-askit, uv-askit) and the hierarchical
               MatVec (Skeletonize/Evaluate with the i-not-in-alpha criterion).
* ``nearfield`` the kNN-separated operator lambda I + K~ + S of eq. (askit): the
               Evaluate step with exact evaluation of the nodes holding a target's
               nearest neighbours, and the same matrix entry by entry.
* ``regression`` kernel regression for binary classification (Sec. III): weights
               from (lambda I + K~ + S) w = u, test labels sign(K(x, X) w).
* ``invaskit`` Alg. "Factorize" and Alg. "Solve" written literally with full P
               matrices (Sec. II-C, eqs. smw, hodlr, blocksmw), the dense reference
               solve, and the error metrics of eq. (error), Sec. III.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` against closed forms, library routines (LAPACK GEQP3 /
GETRF through scipy, numpy's dense solve, scipy's k-d tree), invariants and brute
force.  The uniform-fill random stream (splitmix64) is pinned to the published
reference outputs of that generator.
"""
from .kernel import gaussian_kernel, kernel_matrix, polynomial_kernel, PolynomialKernel, sqdist  # noqa: F401
from .tree import Tree, build_tree, knn_bruteforce, tree_depth, node_sizes  # noqa: F401
from .sampling import splitmix64, sample_rows  # noqa: F401
from .linalg import lu_factor, lu_solve, cpqr_id, back_substitute  # noqa: F401
from .askit import Skeletons, skeletonize, full_P, dense_Ktilde, matvec  # noqa: F401
from .invaskit import (  # noqa: F401
    Factorization,
    factorize,
    solve,
    dense_solve,
    eps_I,
    residual,
    eps_M_sampled,
    build_all,
)
