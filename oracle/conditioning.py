"""CPU oracle of the subspace conditioning tools (test infrastructure only).

Linear-dependence residual of Sec. IV C's discard test, written from its
definition: r_j = S_jj - s^T pinv(S_<j) s with s = S[0:j, j] and S_<j the
leading j x j block, the pseudo-inverse keeping eigenvalues above
eps * lambda_max.  Pinned in tests/test_conditioning_cpu.py against the
squared distance of explicit vectors from the span of the earlier ones
(least squares on the vectors themselves, an independent route).
"""
from __future__ import annotations

import numpy as np


def residuals(S: np.ndarray, eps: float = 1e-12) -> np.ndarray:
    S = np.triu(S) + np.triu(S, 1).T
    M = S.shape[0]
    r = np.zeros(M)
    for j in range(M):
        if j == 0:
            r[j] = S[0, 0]
            continue
        lam, W = np.linalg.eigh(S[:j, :j])
        keep = lam > eps * lam.max()
        w = W[:, keep].T @ S[:j, j]
        r[j] = S[j, j] - np.sum(w * w / lam[keep])
    return r
