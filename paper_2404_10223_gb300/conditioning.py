"""Conditioning tools for the subspace pencil (Sec. IV C): linear-dependence
discard and shot-noise emulation of the matrix elements.

The residual of state j against a set of states is the squared norm of its
component outside their span, `S_jj - s^T S_set^+ s` (computed on the GPU by
tnqe_dependence).  The paper discards a candidate whose residual is below a
threshold (1e-3 in its discussion) because it adds no new direction and only
worsens the conditioning of S.  Shot noise: a quantum evaluation of H_ij and
S_ij by Hadamard tests returns each element with a statistical error; the
emulation adds independent Gaussian errors (delta_H, delta_S) to every
element that is not known exactly (S_ii = 1 is), symmetrically, and re-solves.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def discard_dependent(ctx, S: np.ndarray, threshold: float = 1e-3, eps: float = 1e-12) -> Tuple[List[int], List[float]]:
    """Greedy scan in order: keep state j if its residual against the states kept so far is >= threshold.

    Returns (kept indices, residual of every state at the time it was tested)."""
    S = np.asarray(S, dtype=np.float64)
    kept: List[int] = [0]
    res = [float(S[0, 0])]
    for j in range(1, S.shape[0]):
        idx = kept + [j]
        r = ctx.dependence(S[np.ix_(idx, idx)], eps)[-1]
        res.append(float(r))
        if r >= threshold:
            kept.append(j)
    return kept, res


def shot_noise(H: np.ndarray, S: np.ndarray, rng: np.random.Generator, delta_H: float = 1e-4,
               delta_S: float = 1e-5) -> Tuple[np.ndarray, np.ndarray]:
    """Symmetric Gaussian errors on every estimated element; the diagonal of S (norms) stays exact."""
    M = H.shape[0]
    nH = rng.normal(0.0, delta_H, (M, M))
    nS = rng.normal(0.0, delta_S, (M, M))
    nH = np.triu(nH) + np.triu(nH, 1).T
    nS = np.triu(nS, 1) + np.triu(nS, 1).T
    return H + nH, S + nS


def noise_study(ctx, H: np.ndarray, S: np.ndarray, rng: np.random.Generator, trials: int = 50,
                eps_list: Sequence[float] = (1e-10, 1e-8, 1e-6, 1e-4), delta_H: float = 1e-4,
                delta_S: float = 1e-5) -> Dict[float, dict]:
    """Ground energy under emulated shot noise for several eigenvalue thresholds of S.

    For each eps: the noise-free energy and rank, and over the noisy trials the
    mean and standard deviation of E_0 - E_0(noise-free), the largest |deviation| and the ranks seen."""
    out = {}
    for eps in eps_list:
        E0, _, r0, _ = ctx.solve_ex(H, S, eps)
        dev, ranks = [], []
        for _ in range(trials):
            Hn, Sn = shot_noise(H, S, rng, delta_H, delta_S)
            E, _, r, _ = ctx.solve_ex(Hn, Sn, eps)
            dev.append(E[0] - E0[0])
            ranks.append(r)
        dev = np.array(dev)
        out[eps] = {"E0": float(E0[0]), "rank": int(r0), "mean_dev": float(dev.mean()), "std_dev": float(dev.std()),
                    "max_abs_dev": float(np.abs(dev).max()), "ranks": sorted(set(ranks))}
    return out
