"""Seeded synthetic inputs for the matrix-element hot path.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no rotation, no Hamiltonian, no contraction).  Both the
CUDA path (through the C ABI) and the CPU oracle consume exactly the arrays it
returns, so the two sides share bytes, not code.

What it produces (one "workload"):

* ``h1``  : N x N symmetric one-electron integrals; off-diagonal entries are
  N(0, 0.3^2), the diagonal is ``-1.0 - 0.3 p`` (p 0-based).
* ``eri`` : N^4 two-electron integrals in chemists' order (pq|rs), built as
  ``sum_L B^L_pq B^L_rs`` with ``B^L`` symmetric, entries N(0, 0.3^2).  This has
  the 8-fold permutational symmetry of real orbitals.
* ``mps`` : M matrix product states over N spatial-orbital sites with local
  dimension d = 4 (k = n_alpha + 2 n_beta).  Site tensor s has shape
  (chi_s, 4, chi_{s+1}) with chi_0 = chi_N = 1.  Every bond index carries a
  definite (n_alpha, n_beta) charge counted from the left; an entry
  A[l, k, r] is drawn N(0, 1) only when q(l) + q(k) = q(r) and is exactly 0
  otherwise (the particle-number block structure of the paper's numerics,
  Sec. Numerical details).  The tensors are then left-orthonormalised one
  charge block at a time (a QR per block) and the state is normalised, as
  the workload prescribes ("random N(0,1) real tensors, left-canonicalised
  and normalised").
* ``U``   : one orthogonal N x N orbital rotation per state, U = expm(K) with K
  antisymmetric, strictly-lower entries N(0, sigma_K^2); K_0 = 0 so U_0 = I.

Charge sectors per bond: labels go to the feasible (a, b) sectors by the
D'Hondt rule on Gaussian weights centred on the filling line
(a ~ n_alpha * bond / N), each sector capped at its exact Hilbert-space
dimension, then trimmed until every sector can be reached from both sides.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np
import scipy.linalg

LOCAL_CHARGE = ((0, 0), (1, 0), (0, 1), (1, 1))  # k -> (n_alpha, n_beta)


@dataclasses.dataclass
class MPSInput:
    tensors: List[np.ndarray]          # site s: (chi_s, 4, chi_{s+1}) float64, C-contiguous
    U: np.ndarray                      # (N, N) float64, orthogonal
    K: np.ndarray                      # generator, U = expm(K)
    chi: int                           # requested maximal bond dimension
    charges: List[List[Tuple[int, int]]]  # per bond b = 0..N: charge of every index

    @property
    def bond_dims(self) -> List[int]:
        return [1] + [t.shape[2] for t in self.tensors]


@dataclasses.dataclass
class Workload:
    name: str
    N: int
    n_alpha: int
    n_beta: int
    h1: np.ndarray
    eri: np.ndarray
    mps: List[MPSInput]
    cutoff: float = 1e-14
    seed: int = 0

    @property
    def M(self) -> int:
        return len(self.mps)

    def all_pairs(self) -> List[Tuple[int, int]]:
        return [(i, j) for i in range(self.M) for j in range(i, self.M)]


# ----------------------------------------------------------------------------- integrals
def draw_integrals(rng: np.random.Generator, N: int, L: int, std: float = 0.3):
    A = rng.normal(0.0, std, size=(N, N))
    h1 = np.triu(A, 1)
    h1 = h1 + h1.T
    h1[np.diag_indices(N)] = -1.0 - 0.3 * np.arange(N)
    B = np.empty((L, N, N))
    for l in range(L):
        A = rng.normal(0.0, std, size=(N, N))
        Bl = np.triu(A)
        B[l] = Bl + np.triu(Bl, 1).T
    eri = np.einsum("lpq,lrs->pqrs", B, B)
    return np.ascontiguousarray(h1), np.ascontiguousarray(eri)


def draw_rotation(rng: np.random.Generator, N: int, sigma: float) -> Tuple[np.ndarray, np.ndarray]:
    low = np.tril(rng.normal(0.0, sigma, size=(N, N)), -1)
    K = low - low.T
    return K, scipy.linalg.expm(K)


# ----------------------------------------------------------------------------- sectors
def _exact_dim(N: int, na: int, nb: int, b: int, a: int, bb: int) -> int:
    if a < 0 or bb < 0 or a > b or bb > b or na - a < 0 or nb - bb < 0:
        return 0
    if na - a > N - b or nb - bb > N - b:
        return 0
    left = math.comb(b, a) * math.comb(b, bb)
    right = math.comb(N - b, na - a) * math.comb(N - b, nb - bb)
    return min(left, right)


def bond_sectors(N: int, na: int, nb: int, chi: int) -> List[Dict[Tuple[int, int], int]]:
    """Charge-sector dimensions for bonds 0..N (see module docstring)."""
    dims: List[Dict[Tuple[int, int], int]] = []
    for b in range(N + 1):
        ex = {}
        for a in range(0, min(b, na) + 1):
            for bb in range(0, min(b, nb) + 1):
                e = _exact_dim(N, na, nb, b, a, bb)
                if e > 0:
                    ex[(a, bb)] = e
        total = min(chi, sum(ex.values()))
        ca, cb = na * b / N, nb * b / N
        s2 = 0.35 + 0.5 * b * (N - b) / N
        keys = sorted(ex)
        w = {q: math.exp(-((q[0] - ca) ** 2 + (q[1] - cb) ** 2) / (2.0 * s2)) for q in keys}
        d = {q: 0 for q in keys}
        for _ in range(total):
            best, bestv = None, -1.0
            for q in keys:
                if d[q] < ex[q]:
                    v = w[q] / (d[q] + 1)
                    if v > bestv:
                        best, bestv = q, v
            d[best] += 1
        dims.append({q: v for q, v in d.items() if v > 0})
    # trim until every sector is reachable from the left and from the right
    changed = True
    while changed:
        changed = False
        for b in range(N):
            left, right = dims[b], dims[b + 1]
            for q in list(right):
                cap = sum(left.get((q[0] - c[0], q[1] - c[1]), 0) for c in LOCAL_CHARGE)
                if right[q] > cap:
                    right[q] = cap
                    changed = True
                if right[q] == 0:
                    del right[q]
                    changed = True
            for q in list(left):
                cap = sum(right.get((q[0] + c[0], q[1] + c[1]), 0) for c in LOCAL_CHARGE)
                if left[q] > cap:
                    left[q] = cap
                    changed = True
                if left[q] == 0:
                    del left[q]
                    changed = True
    return dims


def _labels(sec: Dict[Tuple[int, int], int]) -> List[Tuple[int, int]]:
    out = []
    for q in sorted(sec):
        out += [q] * sec[q]
    return out


def draw_mps(rng: np.random.Generator, N: int, na: int, nb: int, chi: int,
             shuffle_bonds: bool = False) -> Tuple[List[np.ndarray], List[List[Tuple[int, int]]]]:
    secs = bond_sectors(N, na, nb, chi)
    labels = [_labels(s) for s in secs]
    if shuffle_bonds:
        for b in range(1, N):
            perm = rng.permutation(len(labels[b]))
            labels[b] = [labels[b][i] for i in perm]
    tensors = []
    for s in range(N):
        L, R = labels[s], labels[s + 1]
        mask = np.zeros((len(L), 4, len(R)), dtype=bool)
        for i, ql in enumerate(L):
            for k, qk in enumerate(LOCAL_CHARGE):
                for j, qr in enumerate(R):
                    if ql[0] + qk[0] == qr[0] and ql[1] + qk[1] == qr[1]:
                        mask[i, k, j] = True
        T = rng.normal(0.0, 1.0, size=mask.shape)
        T[~mask] = 0.0
        tensors.append(T)
    # blockwise left-orthonormalisation (QR inside each right charge block)
    for s in range(N - 1):
        L, R = labels[s], labels[s + 1]
        T = tensors[s].reshape(len(L) * 4, len(R))
        rowq = [(L[i][0] + LOCAL_CHARGE[k][0], L[i][1] + LOCAL_CHARGE[k][1])
                for i in range(len(L)) for k in range(4)]
        Rcarry = np.zeros((len(R), len(R)))
        for q in sorted(set(R)):
            cols = [j for j, qr in enumerate(R) if qr == q]
            rows = [r for r, qq in enumerate(rowq) if qq == q]
            Q, Rm = np.linalg.qr(T[np.ix_(rows, cols)])
            blk = np.zeros((T.shape[0], len(cols)))
            blk[rows, :] = Q
            T[:, cols] = blk
            Rcarry[np.ix_(cols, cols)] = Rm
        tensors[s] = T.reshape(len(L), 4, len(R))
        nxt = tensors[s + 1]
        tensors[s + 1] = np.einsum("ij,jkl->ikl", Rcarry, nxt)
    last = tensors[N - 1]
    tensors[N - 1] = last / np.linalg.norm(last)
    tensors = [np.ascontiguousarray(t) for t in tensors]
    return tensors, labels


# ----------------------------------------------------------------------------- workloads
def make_workload(N: int, n_alpha: int, n_beta: int, L: int, M: int, chi, sigma_K: float = 0.3,
                  seed: int = 0, name: str = "custom", cutoff: float = 1e-14,
                  shuffle_bonds: bool = False) -> Workload:
    rng = np.random.default_rng(seed)
    h1, eri = draw_integrals(rng, N, L)
    if isinstance(chi, (list, tuple)):
        chis = [int(c) for c in rng.choice(np.asarray(chi), size=M)]
    else:
        chis = [int(chi)] * M
    mps = []
    for j in range(M):
        if j == 0:
            K = np.zeros((N, N))
            U = np.eye(N)
        else:
            K, U = draw_rotation(rng, N, sigma_K)
        tensors, labels = draw_mps(rng, N, n_alpha, n_beta, chis[j], shuffle_bonds)
        mps.append(MPSInput(tensors=tensors, U=np.ascontiguousarray(U), K=K, chi=chis[j], charges=labels))
    return Workload(name=name, N=N, n_alpha=n_alpha, n_beta=n_beta, h1=h1, eri=eri, mps=mps,
                    cutoff=cutoff, seed=seed)


def workload(name: str, seed: int = 0) -> Workload:
    """The named workloads of the method's benchmark ladder.

    * ``n6_chi8``        : N=6, 3+3 electrons, L=12, M=3, chi=8 (oracle-sized)
    * ``n10_chi32``      : N=10, 5+5, L=20, M=6, chi=32
    * ``n14_mixed``      : N=14, 7+7, L=28, M=16, chi drawn from {32, 64, 128}
    * ``n14_chi128``     : N=14, 7+7, L=28, M=16, chi=128 for every state
    * ``n20_mixed``      : N=20, 10+10, L=40, M=24, chi drawn from {128, 256}, cutoff 1e-10
    """
    if name == "n6_chi8":
        return make_workload(6, 3, 3, 12, 3, 8, seed=seed, name=name)
    if name == "n10_chi32":
        return make_workload(10, 5, 5, 20, 6, 32, seed=seed, name=name)
    if name == "n14_mixed":
        return make_workload(14, 7, 7, 28, 16, [32, 64, 128], seed=seed, name=name)
    if name == "n14_chi128":
        return make_workload(14, 7, 7, 28, 16, 128, seed=seed, name=name)
    if name == "n20_mixed":
        return make_workload(20, 10, 10, 40, 24, [128, 256], seed=seed, name=name, cutoff=1e-10)
    raise KeyError(name)


def determinant_mps(N: int, occ_alpha: Sequence[int], occ_beta: Sequence[int]) -> List[np.ndarray]:
    """Bond-dimension-1 MPS of one occupation pattern (a Slater determinant in its own basis)."""
    ts = []
    for p in range(N):
        k = (1 if p in occ_alpha else 0) + (2 if p in occ_beta else 0)
        t = np.zeros((1, 4, 1))
        t[0, k, 0] = 1.0
        ts.append(t)
    return ts


# ----------------------------------------------------------------------------- rotation-proposal network
def draw_mlp_params(rng: np.random.Generator, n_in: int, n_h: int, n_out: int, out_scale: float = 0.1) -> np.ndarray:
    """Initial parameters of the proposal network, flat FP32 in the order W1, b1, W2, b2, W3, b3.

    He-style normal weights (variance 2 / fan_in) on the hidden layers, a
    small output layer (the first proposals stay close to "no change"), zero
    biases.
    """
    parts = [rng.normal(0.0, math.sqrt(2.0 / n_in), (n_h, n_in)), np.zeros(n_h),
             rng.normal(0.0, math.sqrt(2.0 / n_h), (n_h, n_h)), np.zeros(n_h),
             rng.normal(0.0, out_scale * math.sqrt(1.0 / n_h), (n_out, n_h)), np.zeros(n_out)]
    return np.concatenate([np.ravel(x) for x in parts]).astype(np.float32)
