"""Oracle A: exact dense Fock-space evaluation of H_ij and S_ij (small N).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions (readings, stated because the paper leaves them open):

* Spin orbitals in Jordan-Wigner order 0a, 0b, 1a, 1b, ...  A d = 4 site of
  spatial orbital p has local index k = n_pa + 2 n_pb; the paper's Sec. II A
  lists the local states vac, up, down, updown as 00, 01, 10, 11, read here as
  the binary number n_b n_a.
* |k_0 ... k_{N-1}> = prod_p (a+_pa)^{n_pa} (a+_pb)^{n_pb} |vac>, p ascending.
* Eq. 1 read in chemists' notation with the usual 1/2:
  H = sum h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs,
  written equivalently as sum h E + 1/2 sum (pq|rs)(E_pq E_rs - d_qr E_ps)
  with E_pq = sum_s a+_ps a_qs.  No constant term.
* An orbital rotation V acts as G(V) a+_q G(V)^-1 = sum_p a+_p V_pq (Thouless,
  Sec. II B).  State j lives in basis U_j: |psi_j> = G(U_j) |MPS_j>.

Inside the (n_a, n_b) sector a state is stored as a matrix Psi[A, B] over
alpha and beta occupation sets in "block order",
(prod_{p in A} a+_pa)(prod_{p in B} a+_pb)|vac>; the interleaved-to-block
reordering sign is applied when converting from MPS amplitudes.  In block
order G(V) acts as Lambda^{n_a}(V) Psi Lambda^{n_b}(V)^T, where Lambda^n(V)
is the matrix of n x n minors (compound matrix).
"""
from __future__ import annotations

import itertools
from typing import List, Sequence, Tuple

import numpy as np
import scipy.sparse
import scipy.sparse.linalg


# ----------------------------------------------------------------------------- determinants
def occupation_sets(N: int, n: int) -> List[Tuple[int, ...]]:
    return list(itertools.combinations(range(N), n))


def _index(sets):
    return {s: i for i, s in enumerate(sets)}


def one_body_ops(N: int, n: int):
    """e[p][q] = matrix of sum a+_p a_q on the n-particle single-species space."""
    sets = occupation_sets(N, n)
    idx = _index(sets)
    dim = len(sets)
    e = [[None] * N for _ in range(N)]
    for p in range(N):
        for q in range(N):
            rows, cols, vals = [], [], []
            for c, A in enumerate(sets):
                if q not in A:
                    continue
                sign = (-1) ** A.index(q)                 # a_q past the orbitals below q
                rest = tuple(x for x in A if x != q)
                if p in rest:
                    continue
                sign *= (-1) ** sum(1 for x in rest if x < p)  # a+_p past the orbitals below p
                Ap = tuple(sorted(rest + (p,)))
                rows.append(idx[Ap])
                cols.append(c)
                vals.append(float(sign))
            e[p][q] = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(dim, dim))
    return e


class SectorHamiltonian:
    """H of Eq. 1 restricted to the (n_a, n_b) sector, applied matrix-free.

    H Psi = sum_ps h'_ps E_ps Psi + 1/2 sum_pq E_pq [ sum_rs (pq|rs) E_rs Psi ],
    h'_ps = h_ps - 1/2 sum_q (pq|qs).
    E_pq acts on the block-order matrix Psi[A, B] as e_pq Psi + Psi e_pq^T.
    """

    def __init__(self, h1: np.ndarray, eri: np.ndarray, na: int, nb: int):
        self.N = N = h1.shape[0]
        self.na, self.nb = na, nb
        self.ea = one_body_ops(N, na)
        self.eb = one_body_ops(N, nb) if nb != na else self.ea
        self.da = len(occupation_sets(N, na))
        self.db = len(occupation_sets(N, nb))
        self.h1 = h1
        self.eri = eri
        self.hp = h1 - 0.5 * np.einsum("pqqs->ps", eri)

    def E(self, p: int, q: int, Psi: np.ndarray) -> np.ndarray:
        return self.ea[p][q] @ Psi + (self.eb[p][q] @ Psi.T).T

    def apply(self, Psi: np.ndarray) -> np.ndarray:
        N = self.N
        phi = np.empty((N, N) + Psi.shape)
        for r in range(N):
            for s in range(N):
                phi[r, s] = self.E(r, s, Psi)
        out = np.einsum("ps,psab->ab", self.hp, phi)
        chi = np.einsum("pqrs,rsab->pqab", self.eri, phi)
        for p in range(N):
            for q in range(N):
                out += 0.5 * self.E(p, q, chi[p, q])
        return out

    def expectation(self, Psi_i: np.ndarray, Psi_j: np.ndarray) -> float:
        return float(np.sum(Psi_i * self.apply(Psi_j)))

    def ground_energy(self) -> float:
        dim = self.da * self.db
        op = scipy.sparse.linalg.LinearOperator(
            (dim, dim), matvec=lambda v: self.apply(v.reshape(self.da, self.db)).ravel(), dtype=float)
        if dim <= 400:
            dense = np.column_stack([op.matvec(np.eye(dim)[:, c]) for c in range(dim)])
            return float(np.linalg.eigvalsh(0.5 * (dense + dense.T))[0])
        val = scipy.sparse.linalg.eigsh(op, k=1, which="SA", tol=1e-12)[0]
        return float(val[0])


# ----------------------------------------------------------------------------- rotations
def compound_matrix(V: np.ndarray, n: int) -> np.ndarray:
    """Lambda^n(V)[A', A] = det V[A', A] over ascending n-subsets (Thouless, Sec. II B)."""
    N = V.shape[0]
    sets = occupation_sets(N, n)
    if n == 0:
        return np.ones((1, 1))
    S = np.array(sets)
    sub = V[S[:, None, :, None], S[None, :, None, :]]   # (dim, dim, n, n)
    return np.linalg.det(sub)


def rotate_sector(Psi: np.ndarray, V: np.ndarray, na: int, nb: int) -> np.ndarray:
    """Exact G(V)|Psi> in block order."""
    return compound_matrix(V, na) @ Psi @ compound_matrix(V, nb).T


# ----------------------------------------------------------------------------- MPS -> Fock
def mps_full_tensor(tensors: Sequence[np.ndarray]) -> np.ndarray:
    """Amplitudes Psi[k_0, ..., k_{N-1}] of Eq. 3 as a dense 4^N tensor."""
    acc = tensors[0][0]              # (4, chi_1)
    for t in tensors[1:]:
        acc = np.tensordot(acc, t, axes=([-1], [0]))
    return acc[..., 0]


def interleave_sign(A: Tuple[int, ...], B: Tuple[int, ...]) -> int:
    """Sign taking prod_p (a+_pa)^.(a+_pb)^. into (prod_A a+_a)(prod_B a+_b)."""
    inv = 0
    for p in A:
        inv += sum(1 for q in B if q < p)
    return -1 if inv % 2 else 1


def mps_to_sector(tensors: Sequence[np.ndarray], na: int, nb: int) -> np.ndarray:
    N = len(tensors)
    full = mps_full_tensor(tensors)
    SA, SB = occupation_sets(N, na), occupation_sets(N, nb)
    Psi = np.empty((len(SA), len(SB)))
    for ia, A in enumerate(SA):
        for ib, B in enumerate(SB):
            k = tuple((1 if p in A else 0) + (2 if p in B else 0) for p in range(N))
            Psi[ia, ib] = interleave_sign(A, B) * full[k]
    return Psi


def sector_weight(tensors: Sequence[np.ndarray], na: int, nb: int) -> float:
    full = mps_full_tensor(tensors)
    return float(np.sum(full * full))


# ----------------------------------------------------------------------------- matrix elements
def matrix_elements(h1, eri, na, nb, states: Sequence[Sequence[np.ndarray]], Us: Sequence[np.ndarray],
                    pairs=None, ham: SectorHamiltonian = None):
    """Exact H_ij = <psi_i|H|psi_j>, S_ij = <psi_i|psi_j> with psi_j = G(U_j)|MPS_j> (Eq. 10)."""
    if ham is None:
        ham = SectorHamiltonian(h1, eri, na, nb)
    psis = [rotate_sector(mps_to_sector(t, na, nb), U, na, nb) for t, U in zip(states, Us)]
    M = len(psis)
    if pairs is None:
        pairs = [(i, j) for i in range(M) for j in range(i, M)]
    H = np.array([ham.expectation(psis[i], psis[j]) for i, j in pairs])
    S = np.array([float(np.sum(psis[i] * psis[j])) for i, j in pairs])
    return H, S


# ----------------------------------------------------------------------------- full Fock (tiny N)
def jw_operators(N: int):
    """Dense Jordan-Wigner annihilators c_j on all 2N spin orbitals (Sec. II A).

    c_j = Z (x) ... (x) Z (x) sigma^- (x) 1 ..., spin-orbital j = 2p + s.
    Basis index: sum_j n_j 2^(2N-1-j) (spin orbital 0 most significant).
    """
    n = 2 * N
    Z = np.diag([1.0, -1.0])
    sm = np.array([[0.0, 1.0], [0.0, 0.0]])   # |0><1|
    I = np.eye(2)
    ops = []
    for j in range(n):
        m = np.ones((1, 1))
        for i in range(n):
            m = np.kron(m, Z if i < j else (sm if i == j else I))
        ops.append(m)
    return ops


def jw_hamiltonian(h1: np.ndarray, eri: np.ndarray) -> np.ndarray:
    """Dense H of Eq. 1 on the full 4^N Fock space, term by term."""
    N = h1.shape[0]
    c = jw_operators(N)
    cd = [x.T for x in c]
    dim = 4 ** N
    H = np.zeros((dim, dim))
    for p in range(N):
        for q in range(N):
            for s in range(2):
                H += h1[p, q] * cd[2 * p + s] @ c[2 * q + s]
    for p, q, r, s_ in itertools.product(range(N), repeat=4):
        v = eri[p, q, r, s_]
        if v == 0.0:
            continue
        for s in range(2):
            for t in range(2):
                H += 0.5 * v * cd[2 * p + s] @ cd[2 * r + t] @ c[2 * s_ + t] @ c[2 * q + s]
    return H


def full_vector(tensors: Sequence[np.ndarray]) -> np.ndarray:
    """MPS amplitudes mapped onto the JW qubit basis of ``jw_operators``.

    Local k = n_a + 2 n_b with the interleaved order equals the JW product
    order, so the qubit bits of site p are (n_pa, n_pb) in that order.
    """
    N = len(tensors)
    full = mps_full_tensor(tensors).reshape(-1)
    out = np.zeros(4 ** N)
    for kidx in range(4 ** N):
        ks = np.unravel_index(kidx, (4,) * N)
        bits = 0
        for p, k in enumerate(ks):
            bits = (bits << 2) | ((k & 1) << 1) | ((k >> 1) & 1)
        out[bits] = full[kidx]
    return out


def full_rotation(V: np.ndarray) -> np.ndarray:
    """Dense G(V) on the 4^N Fock space: exp of the one-body generator log(V) (det V = +1)."""
    import scipy.linalg
    N = V.shape[0]
    Kg = scipy.linalg.logm(V).real
    c = jw_operators(N)
    gen = np.zeros((4 ** N, 4 ** N))
    for p in range(N):
        for q in range(N):
            if Kg[p, q] == 0.0:
                continue
            for s in range(2):
                gen += Kg[p, q] * c[2 * p + s].T @ c[2 * q + s]
    return scipy.linalg.expm(gen)
