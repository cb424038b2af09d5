"""Oracle B: a plain CPU FP64 MPS implementation of the matrix-element path.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Slow and direct on
purpose: numpy SVD / QR / eigh / tensordot are the only library steps.

Steps, each following the paper's definition in the paper's order:

1. ``givens_plan``: factor the relative rotation V = U_i^T U_j into
   nearest-neighbour Givens rotations (Eq. 11: "a QR factorization of the
   N x N orbital rotation matrix").  Reading (the paper fixes no order):
   column rotations J on adjacent columns zero V one row at a time,
   alternating the top row (sweeping right-to-left) and the bottom row
   (sweeping left-to-right) of the remaining block, so that
   V J_1 ... J_K = D = diag(1, .., det V, .., 1) and
   G(V) = G(D) G(J_K^T) ... G(J_1^T): the gates act in creation order and
   consecutive sweeps run in opposite directions.
2. ``gate16``: the two-site operator of one Givens rotation,
   g_{p,p+1}(theta) = exp[theta sum_s (a+_ps a_{p+1}s - a+_{p+1}s a_ps)]
   (Sec. II B, App. A3) with theta = atan2(s, c), built as the matrix
   exponential of that generator on the 16-dimensional two-site space.
3. ``apply_rotation``: contract the two-site tensor, apply the gate, SVD
   and keep k = #{l <= chi_rot : sigma_l > cutoff * sigma_1} singular values
   (Sec. II D, Eq. A5).  Sigma joins the side the canonical centre moves to:
   toward the sweep direction, and at the last gate of a sweep toward the
   next sweep's first bond.  No renormalisation unless requested.
4. ``rotate_integrals``: h -> U^T h U, (pq|rs) -> four-index transform, so
   that H expressed "in each orbital basis" (Sec. IV B) is available.
5. ``build_mpo``: an exact MPO of Eq. 1 (complementary-operator layout,
   channels keyed by the operator strings they carry).
6. ``contract``: transfer-matrix contraction <MPS_i| H |MPS_j'> and
   <MPS_i|MPS_j'> (Fig. 5b).
7. ``solve``: canonical orthogonalisation (projection method of Sec. IV C /
   App. A2) and the eigenvalue condition number kappa_1 (App. A2).
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg
import scipy.sparse

# ----------------------------------------------------------------------------- local operators
# local basis k = n_a + 2 n_b, |3> = a+_a a+_b |vac>
CDAG_A = np.zeros((4, 4))
CDAG_A[1, 0] = 1.0
CDAG_A[3, 2] = 1.0
CDAG_B = np.zeros((4, 4))
CDAG_B[2, 0] = 1.0
CDAG_B[3, 1] = -1.0          # a+_b a+_a |vac> = - |3>
PARITY = np.diag([1.0, -1.0, -1.0, 1.0])
ID4 = np.eye(4)


def local_ladder(spin: int, create: bool) -> np.ndarray:
    m = CDAG_A if spin == 0 else CDAG_B
    return m if create else m.T


# ----------------------------------------------------------------------------- Givens plan (Eq. 11)
# A rotation whose target pair (x, y) has norm below this is taken as the
# identity: entries of an orthogonal V that small are rounding noise, and
# rotating noise by O(1) angles would entangle a state that V leaves alone.
GIVENS_SKIP = 1e-14

def givens_plan(V: np.ndarray) -> Tuple[List[Tuple[int, float, float, str]], int, bool]:
    """Gates (a, c, s, sigma_side) in application order, the diagonal index m and det sign.

    A gate acts on sites (a, a+1) as G(J^T) for J = [[c, -s], [s, c]] placed
    at rows/columns (a, a+1).  Pairs with hypot(x, y) < GIVENS_SKIP give the
    identity rotation (c, s) = (1, 0).  ``sigma_side`` is "L" or "R": where the
    singular values go after the SVD of that gate.
    """
    N = V.shape[0]
    W = np.array(V, dtype=float, copy=True)
    gates: List[Tuple[int, float, float, str]] = []
    lo, hi = 0, N - 1
    top = True
    passes = []
    while lo < hi:
        this = []
        if top:
            for col in range(hi, lo, -1):          # zero W[lo, col] into column col-1
                a = col - 1
                x, y = W[lo, a], W[lo, a + 1]
                rho = math.hypot(x, y)
                c, s = (1.0, 0.0) if rho < GIVENS_SKIP else (x / rho, y / rho)
                ca, cb = W[:, a].copy(), W[:, a + 1].copy()
                W[:, a] = c * ca + s * cb
                W[:, a + 1] = -s * ca + c * cb
                this.append([a, c, s, "L"])
            lo += 1
        else:
            for col in range(lo, hi):               # zero W[hi, col] into column col+1
                a = col
                x, y = W[hi, a], W[hi, a + 1]
                rho = math.hypot(x, y)
                c, s = (1.0, 0.0) if rho < GIVENS_SKIP else (y / rho, -x / rho)
                ca, cb = W[:, a].copy(), W[:, a + 1].copy()
                W[:, a] = c * ca + s * cb
                W[:, a + 1] = -s * ca + c * cb
                this.append([a, c, s, "R"])
            hi -= 1
        passes.append(this)
        top = not top
    for n, this in enumerate(passes):
        if n + 1 < len(passes):                     # turn toward the next sweep
            this[-1][3] = "R" if this[-1][3] == "L" else "L"
        gates += [tuple(g) for g in this]
    m = lo
    neg = bool(W[m, m] < 0.0)
    return gates, m, neg


def plan_matrix(gates, m: int, neg: bool, N: int) -> np.ndarray:
    """Rebuild V = D J_K^T ... J_1^T from a plan (used by tests)."""
    P = np.eye(N)
    for a, c, s, _ in gates:
        J = np.eye(N)
        J[a, a], J[a, a + 1], J[a + 1, a], J[a + 1, a + 1] = c, -s, s, c
        P = P @ J
    D = np.eye(N)
    if neg:
        D[m, m] = -1.0
    return D @ P.T


# ----------------------------------------------------------------------------- two-site gate
def _four_mode_ops():
    """JW annihilators on the modes (a alpha, a beta, b alpha, b beta).

    Two-site index K = 4 k_a + k_b with k = n_alpha + 2 n_beta.
    """
    ops = []
    for j in range(4):
        m = np.zeros((16, 16))
        for K in range(16):
            ka, kb = divmod(K, 4)
            n = [ka & 1, ka >> 1, kb & 1, kb >> 1]
            if n[j] == 0:
                continue
            sign = (-1) ** sum(n[:j])
            n2 = list(n)
            n2[j] = 0
            K2 = 4 * (n2[0] + 2 * n2[1]) + (n2[2] + 2 * n2[3])
            m[K2, K] = sign
        ops.append(m)
    return ops


_C4 = _four_mode_ops()


def gate16(c: float, s: float) -> np.ndarray:
    theta = math.atan2(s, c)
    T = np.zeros((16, 16))
    for sp in range(2):
        ca, cb = _C4[sp], _C4[2 + sp]
        T += ca.T @ cb - cb.T @ ca
    return scipy.linalg.expm(theta * T)


# ----------------------------------------------------------------------------- gate application
def apply_rotation(tensors: Sequence[np.ndarray], V: np.ndarray, chi_rot: int, cutoff: float,
                   renormalize: bool = False, trace: Optional[list] = None):
    """Truncated G(V)|MPS> for a left-canonical MPS (centre on the last site).

    Returns (new tensors, total discarded weight sum sigma^2).  If ``trace`` is
    a list, each gate appends ``(k, sigma, rows)``: the kept count, the full
    singular-value list of its SVD and, for each kept left singular vector, the
    row (l, k1) of its largest entry (diagnostics only; the arithmetic is the
    same either way).
    """
    ts = [np.array(t, dtype=float, copy=True) for t in tensors]
    N = len(ts)
    norm0 = float(np.linalg.norm(ts[-1]))
    gates, m, neg = givens_plan(V)
    discarded = 0.0
    centre = N - 1
    for a, c, s, side in gates:
        A, B = ts[a], ts[a + 1]
        theta = np.tensordot(A, B, axes=([2], [0]))                 # (l, k1, k2, r)
        G = gate16(c, s).reshape(4, 4, 4, 4)                         # (k1', k2', k1, k2)
        theta = np.einsum("xyab,labr->lxyr", G, theta)
        chl, chr_ = A.shape[0], B.shape[2]
        mat = theta.reshape(chl * 4, 4 * chr_)
        try:
            u, sig, vt = scipy.linalg.svd(mat, full_matrices=False, lapack_driver="gesdd")
        except np.linalg.LinAlgError:
            u, sig, vt = scipy.linalg.svd(mat, full_matrices=False, lapack_driver="gesvd")
        if sig.size == 0 or sig[0] == 0.0:
            k = 1
        else:
            k = int(min(chi_rot, np.count_nonzero(sig > cutoff * sig[0])))
            k = max(k, 1)
        discarded += float(np.sum(sig[k:] ** 2))
        if trace is not None:
            trace.append((k, sig.copy(), np.argmax(np.abs(u[:, :k]), axis=0)))
        u, sk, vt = u[:, :k], sig[:k], vt[:k]
        if side == "L":
            ts[a] = (u * sk).reshape(chl, 4, k)
            ts[a + 1] = vt.reshape(k, 4, chr_)
            centre = a
        else:
            ts[a] = u.reshape(chl, 4, k)
            ts[a + 1] = (sk[:, None] * vt).reshape(k, 4, chr_)
            centre = a + 1
    if neg:                                                          # G(D): a+_m -> -a+_m, both spins
        ts[m] = ts[m] * np.array([1.0, -1.0, -1.0, 1.0])[None, :, None]
    if renormalize:
        nrm = float(np.linalg.norm(ts[centre]))
        if nrm > 0.0:
            ts[centre] = ts[centre] * (norm0 / nrm)
    return ts, discarded


def overlap(bra: Sequence[np.ndarray], ket: Sequence[np.ndarray]) -> float:
    E = np.ones((1, 1))
    for A, B in zip(bra, ket):
        E = np.einsum("ab,akx,bky->xy", E, A, B)
    return float(E[0, 0])


# ----------------------------------------------------------------------------- integrals
def rotate_integrals(h1: np.ndarray, eri: np.ndarray, U: np.ndarray):
    h = U.T @ h1 @ U
    g = np.tensordot(eri, U, axes=([0], [0]))          # (q r s p)
    g = np.tensordot(g, U, axes=([0], [0]))            # (r s p q)
    g = np.tensordot(g, U, axes=([0], [0]))            # (s p q r)
    g = np.tensordot(g, U, axes=([0], [0]))            # (p q r s)
    return h, np.ascontiguousarray(g)


# ----------------------------------------------------------------------------- MPO of Eq. 1
class MPO:
    """Site operators W_t as sparse (4 D_{t+1}) x (4 D_t) matrices.

    Row index w' * 4 + k (bra side), column w * 4 + k' (ket side).  Channel 0
    of every bond is the identity string (so the last bond also gives S);
    channel 1 of bonds >= 1 is the completed Hamiltonian.
    """

    def __init__(self, W: List[scipy.sparse.csr_matrix], dims: List[int]):
        self.W = W
        self.dims = dims


def _canonical_term(ops):
    """Stable sort of ladder operators by spin-orbital position with fermion sign."""
    n = len(ops)
    for i in range(n):
        for j in range(i + 1, n):
            if ops[i] == ops[j]:
                return None, 0                       # a+_x a+_x = a_x a_x = 0 (only adjacent after sort)
    order = sorted(range(n), key=lambda i: (ops[i][0], i))
    inv = 0
    for x in range(n):
        for y in range(x + 1, n):
            i, j = order[x], order[y]
            if i > j and ops[i][0] != ops[j][0]:
                inv += 1
    srt = tuple(ops[i] for i in order)
    # identical operators adjacent at the same position vanish
    for x in range(n - 1):
        if srt[x] == srt[x + 1]:
            return None, 0
    return srt, (-1 if inv % 2 else 1)


def build_mpo(h1: np.ndarray, eri: np.ndarray) -> MPO:
    N = h1.shape[0]
    half = N // 2
    terms = []
    for p in range(N):
        for q in range(N):
            if h1[p, q] != 0.0:
                for s in range(2):
                    terms.append((h1[p, q], [(2 * p + s, 1), (2 * q + s, -1)]))
    for p in range(N):
        for q in range(N):
            for r in range(N):
                for s_ in range(N):
                    v = eri[p, q, r, s_]
                    if v == 0.0:
                        continue
                    for s in range(2):
                        for t in range(2):
                            terms.append((0.5 * v, [(2 * p + s, 1), (2 * r + t, 1),
                                                    (2 * s_ + t, -1), (2 * q + s, -1)]))
    keys: List[Dict] = [dict() for _ in range(N + 1)]
    blocks: List[Dict] = [dict() for _ in range(N)]      # (kin, kout) -> [matrix, is_transition]

    def key(srt, b):
        n = len(srt)
        k = sum(1 for o in srt if o[0] // 2 < b)
        if k == 0:
            return ("I",)
        if k == n:
            return ("F",)
        if k == 1:
            return ("L", srt[:1])
        if k == 3:
            return ("R", srt[3:])
        return ("L", srt[:2]) if b <= half else ("R", srt[2:])

    for coef, ops in terms:
        srt, sign = _canonical_term(ops)
        if srt is None:
            continue
        sites = [o[0] // 2 for o in srt]
        path = [key(srt, b) for b in range(N + 1)]
        for t in range(N):
            L = ID4
            for o in srt:
                if o[0] // 2 == t:
                    L = L @ local_ladder(o[0] % 2, o[1] > 0)
            nafter = sum(1 for x in sites if x > t)
            M = L @ PARITY if nafter % 2 else L
            kin, kout = path[t], path[t + 1]
            trans = kin[0] in ("I", "L") and kout[0] in ("R", "F")
            ent = blocks[t].get((kin, kout))
            if trans:
                if ent is None:
                    blocks[t][(kin, kout)] = [coef * sign * M, True]
                else:
                    ent[0] = ent[0] + coef * sign * M
            else:
                if ent is None:
                    blocks[t][(kin, kout)] = [M, False]
                else:
                    assert np.array_equal(ent[0], M)
    for t in range(N):
        blocks[t][(("I",), ("I",))] = [ID4, False]
    # channel numbering: I = 0, F = 1, the rest in sorted order
    for t in range(N):
        for (kin, kout) in blocks[t]:
            keys[t].setdefault(kin, None)
            keys[t + 1].setdefault(kout, None)
    index = []
    for b in range(N + 1):
        ks = list(keys[b])
        rest = sorted((k for k in ks if k[0] not in ("I", "F")), key=repr)
        order = [("I",)] + ([("F",)] if ("F",) in keys[b] else []) + rest
        index.append({k: i for i, k in enumerate(order)})
    W = []
    for t in range(N):
        rows, cols, vals = [], [], []
        for (kin, kout), (M, _) in blocks[t].items():
            wi, wo = index[t][kin], index[t + 1][kout]
            nz = np.nonzero(M)
            for k, kp in zip(*nz):
                rows.append(wo * 4 + k)
                cols.append(wi * 4 + kp)
                vals.append(M[k, kp])
        W.append(scipy.sparse.csr_matrix((vals, (rows, cols)),
                                         shape=(4 * len(index[t + 1]), 4 * len(index[t]))))
    return MPO(W, [len(ix) for ix in index])


def mpo_dense(mpo: MPO) -> np.ndarray:
    """Contract the MPO into the full 4^N x 4^N matrix (tiny N only)."""
    N = len(mpo.W)
    # E[w, bra, ket] over the left block
    E = np.ones((1, 1, 1))
    for t in range(N):
        Wt = mpo.W[t].toarray().reshape(mpo.dims[t + 1], 4, mpo.dims[t], 4)  # (w', k, w, k')
        E = np.einsum("wxy,vkwl->vxkyl", E, Wt)
        d = E.shape[1] * 4
        E = E.reshape(E.shape[0], d, d)
    return E[1]


# ----------------------------------------------------------------------------- contraction
def contract(bra: Sequence[np.ndarray], mpo: MPO, ket: Sequence[np.ndarray]) -> Tuple[float, float]:
    """(<bra|H|ket>, <bra|ket>) by left-to-right transfer matrices (Fig. 5b)."""
    Lenv = np.ones((1, 1, 1))                              # (a, w, b)
    for t, (A, B) in enumerate(zip(bra, ket)):
        ci, D, cj = Lenv.shape
        X = np.tensordot(Lenv, B, axes=([2], [0]))          # (a, w, k', b')
        cj2 = B.shape[2]
        Xm = X.reshape(ci, D * 4, cj2).transpose(1, 0, 2).reshape(D * 4, ci * cj2)
        Y = mpo.W[t] @ Xm                                    # (w' k, a b')
        D2 = mpo.dims[t + 1]
        Y = Y.reshape(D2, 4, ci, cj2)
        Lenv = np.einsum("aks,wkab->swb", A, Y)
    return float(Lenv[0, 1, 0]), float(Lenv[0, 0, 0])


# ----------------------------------------------------------------------------- solve
def solve(H: np.ndarray, S: np.ndarray, eps: float = 1e-10):
    """Canonical orthogonalisation (Sec. IV C projection method).

    The upper triangle (i <= j) of H and S is authoritative.  Keeps the
    eigenvectors of S with lambda > eps * lambda_max, solves the projected
    standard problem, returns E ascending, C (M x rank, S-normalised, largest
    |entry| of each column positive), rank and kappa_1 = |c_1|^2 / sqrt(E_1^2 + 1).
    """
    Hs = np.triu(H) + np.triu(H, 1).T
    Ss = np.triu(S) + np.triu(S, 1).T
    lam, Wv = np.linalg.eigh(Ss)
    keep = lam > eps * lam[-1]
    X = Wv[:, keep] / np.sqrt(lam[keep])
    Ht = X.T @ Hs @ X
    E, Y = np.linalg.eigh(0.5 * (Ht + Ht.T))
    C = X @ Y
    for c in range(C.shape[1]):
        i = int(np.argmax(np.abs(C[:, c])))
        if C[i, c] < 0:
            C[:, c] = -C[:, c]
    kappa1 = float(np.dot(C[:, 0], C[:, 0]) / math.sqrt(E[0] ** 2 + 1.0))
    return E, C, int(keep.sum()), kappa1


# ----------------------------------------------------------------------------- whole path
class Context:
    """All-pairs H_ij, S_ij of M states, each in its own orbital basis."""

    def __init__(self, h1, eri, N, na, nb, chi_rot: int = 0, cutoff: float = 1e-14,
                 renormalize: bool = False):
        self.h1, self.eri, self.N, self.na, self.nb = h1, eri, N, na, nb
        self.chi_rot, self.cutoff, self.renormalize = chi_rot, cutoff, renormalize
        self.states: List[List[np.ndarray]] = []
        self.Us: List[np.ndarray] = []
        self._mpo: Dict[int, MPO] = {}

    def add_mps(self, tensors, U) -> int:
        self.states.append([np.asarray(t, dtype=float) for t in tensors])
        self.Us.append(np.asarray(U, dtype=float))
        return len(self.states) - 1

    def mpo(self, i: int) -> MPO:
        if i not in self._mpo:
            h, g = rotate_integrals(self.h1, self.eri, self.Us[i])
            self._mpo[i] = build_mpo(h, g)
        return self._mpo[i]

    def chi_of(self, j: int) -> int:
        return max(t.shape[2] for t in self.states[j][:-1]) if self.N > 1 else 1

    def rotate(self, i: int, j: int, trace: Optional[list] = None):
        if i == j:
            return self.states[j], 0.0
        V = self.Us[i].T @ self.Us[j]
        chi_rot = self.chi_rot if self.chi_rot > 0 else self.chi_of(j)
        return apply_rotation(self.states[j], V, chi_rot, self.cutoff, self.renormalize, trace)

    def pair(self, i: int, j: int):
        ket, disc = self.rotate(i, j)
        H, S = contract(self.states[i], self.mpo(i), ket)
        return H, S, disc

    def matrix_elements(self, pairs):
        out = [self.pair(i, j) for i, j in pairs]
        return np.array([o[0] for o in out]), np.array([o[1] for o in out])
