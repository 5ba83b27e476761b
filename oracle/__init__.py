"""CPU FP64 oracle for the MDS hot path: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import anything from this package; the CUDA product
path (``paper_2007_11919_gb300``) never does, and the two share no code.

Parity pins (each checked by a ``-m "not gpu"`` test in tests/test_oracle_pins.py):
  classical_mds        exact recovery of points in R^r, Eq. (1) invariant,
                       brute force against an independent Jacobi solver.
  double_center        zero row/column sums, equals the centred Gram matrix
                       for Euclidean input (Section 2 identity).
  gower_interpolate    landmarks reproduce X_1; equals LMDS (Prop. 1);
                       equals the closed-form PCA projection for Euclidean data.
  lmds_triangulate     Prop. 1 (against gower_interpolate).
  interpolation_mds    block-size invariance; p = 1 reduces to classical MDS;
                       Table 1 correlation band.
  procrustes           exact recovery of a planted orthogonal map + shift.
  divide_conquer_mds   exact recovery (up to one global orthogonal map) of
                       rank-r data; p = 1 reduces to classical MDS;
                       Table 1 correlation band.
  divide_conquer_parts exact recovery of rank-r data on a subset of parts.
  sign_convention      hand-built columns with a known largest entry (and
                       a tie) come out flipped or kept as expected.
  embed_new            equals interpolation_mds on the same points.
  (tests/test_oracle_variants.py, the variants of oracle/variants.py)
  affine_interpolation equals interpolation_mds (distance form) for
                       Euclidean rows; landmarks reproduce X_1.
  maxmin_landmarks     a hand-derived order on a line; picks distinct; the
                       gap of each new pick never grows; covering radius
                       within 2x of the brute-force optimal l-center.
  pivot_mds            pivots = all points is classical MDS; exact classical
                       MDS of a set made of two copies of a cloud, pivots one
                       copy (V_P^T V_P = I/2 exactly).
  fast_mds             n <= l is classical MDS; exact recovery of rank-r data
                       through one and two levels of division; each leaf's
                       aligned rows keep the covariance eigenvalues
                       lambda^j / n_j (orthogonal alignment).
No oracle function is "parity unpinned".
"""
from .mds import (RankError, classical_mds, divide_conquer_mds, divide_conquer_part, divide_conquer_parts,
                  double_center,
                  embed_new, gower_interpolate, interpolation_mds, lmds_triangulate, procrustes,
                  sign_convention, sq_dist)
from .compare import aligned_rel_error, column_correlations
from .jacobi import jacobi_eigh
from .variants import affine_interpolation, fast_mds, maxmin_landmarks, pivot_mds

__all__ = [
    "RankError", "classical_mds", "divide_conquer_mds", "divide_conquer_part", "divide_conquer_parts",
    "double_center",
    "embed_new", "gower_interpolate", "interpolation_mds", "lmds_triangulate", "procrustes",
    "sign_convention", "sq_dist", "aligned_rel_error", "column_correlations", "jacobi_eigh",
    "affine_interpolation", "fast_mds", "maxmin_landmarks", "pivot_mds",
]
