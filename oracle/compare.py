"""Comparison of two MDS configurations up to an orthogonal map.

TEST INFRASTRUCTURE ONLY (see ``oracle/mds.py``).  An MDS configuration is
unique only up to rotation, reflection and translation (Section 4.1 aligns
every configuration by a Procrustes transformation before comparing).  The
error of ``X`` against the reference ``X_ref`` is therefore measured after
the best orthogonal alignment of ``X`` onto ``X_ref``:

    err = || X T + 1 t^T - X_ref ||_F / || X_ref - 1 mean(X_ref)^T ||_F
"""
from __future__ import annotations

import numpy as np

from .mds import procrustes


def aligned_rel_error(X, X_ref) -> float:
    X = np.asarray(X, dtype=np.float64)
    X_ref = np.asarray(X_ref, dtype=np.float64)
    T, t = procrustes(X_ref, X)
    resid = X @ T + t[None, :] - X_ref
    scale = np.linalg.norm(X_ref - X_ref.mean(axis=0))
    return float(np.linalg.norm(resid) / scale)


def column_correlations(X, Y_dom) -> np.ndarray:
    """Correlation of each column of X, after Procrustes alignment onto the
    dominant columns Y_dom, with the matching column of Y_dom (Table 1's
    statistic)."""
    X = np.asarray(X, dtype=np.float64)
    Y_dom = np.asarray(Y_dom, dtype=np.float64)
    T, t = procrustes(Y_dom, X)
    Xa = X @ T + t[None, :]
    return np.array([np.corrcoef(Xa[:, i], Y_dom[:, i])[0, 1] for i in range(Y_dom.shape[1])])
