"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Every test here is CPU-only.  Each pin is chosen so that a plausible mistake
in the oracle (a sign convention, a dropped 1/2, a transposed rotation, a
wrong truncation count) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import fock as of
from oracle import mps as om
from paper_2404_10223_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_gates.json")))


def _rng(seed):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------------------- App. A3 gates
def _g2(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[1, 0, 0, 0], [0, c, -s, 0], [0, s, c, 0], [0, 0, 0, 1.0]])


def _big_to_local():
    """Permutation from 4-qubit big-endian (a_up, a_dn, b_up, b_dn) to K = 4 k_a + k_b."""
    P = np.zeros((16, 16))
    for big in range(16):
        n0, n1, n2, n3 = (big >> 3) & 1, (big >> 2) & 1, (big >> 1) & 1, big & 1
        P[4 * (n0 + 2 * n1) + (n2 + 2 * n3), big] = 1.0
    return P


def test_golden_gate_relations():
    f = np.array(GOLD["fswap_d2"], dtype=float)
    Z2 = np.kron(np.eye(2), np.diag([1.0, -1.0]))
    assert np.allclose(Z2 @ f, _g2(math.pi / 2), atol=1e-15)          # (1 x Z) f = g(pi/2)
    assert np.allclose(np.array(GOLD["givens_d2_pi_over_4"]), _g2(math.pi / 4), atol=1e-15)


@pytest.mark.parametrize("theta", [0.0, 0.37, -1.2, math.pi / 4, math.pi / 2, 2.9])
def test_gate16_is_paper_g4(theta):
    """Oracle gate (expm of the generator) equals g_4 = (1 x f x 1)(g x g)(1 x f x 1)."""
    f = np.array(GOLD["fswap_d2"], dtype=float)
    F = np.kron(np.kron(np.eye(2), f), np.eye(2))
    g4 = F @ np.kron(_g2(theta), _g2(theta)) @ F
    P = _big_to_local()
    G = om.gate16(math.cos(theta), math.sin(theta))
    assert np.abs(P @ g4 @ P.T - G).max() < 1e-14


# ----------------------------------------------------------------------------- Givens factorisation
@pytest.mark.parametrize("N", [2, 3, 4, 7, 14])
def test_givens_plan_reconstructs_V(N):
    K, U = inputs.draw_rotation(_rng(N), N, 0.7)
    gates, m, neg = om.givens_plan(U)
    assert len(gates) == N * (N - 1) // 2
    assert not neg
    assert np.abs(om.plan_matrix(gates, m, neg, N) - U).max() < 1e-13


def test_givens_plan_reflection_and_permutation():
    N = 5
    U = inputs.draw_rotation(_rng(1), N, 0.5)[1]
    R = np.eye(N)
    R[1, 1] = -1.0
    V = U @ R
    gates, m, neg = om.givens_plan(V)
    assert neg
    assert np.abs(om.plan_matrix(gates, m, neg, N) - V).max() < 1e-13
    Pm = np.eye(N)[[3, 0, 4, 1, 2]]
    gates, m, neg = om.givens_plan(Pm)
    for _, c, s, _ in gates:
        assert (abs(c), abs(s)) in ((1.0, 0.0), (0.0, 1.0))
    assert np.abs(om.plan_matrix(gates, m, neg, N) - Pm).max() < 1e-15


# ----------------------------------------------------------------------------- Hamiltonian
@pytest.mark.parametrize("N", [2, 3])
def test_mpo_equals_jordan_wigner_hamiltonian(N):
    h1, eri = inputs.draw_integrals(_rng(10 + N), N, 2 * N)
    Hm = om.mpo_dense(om.build_mpo(h1, eri))
    Hjw = of.jw_hamiltonian(h1, eri)
    P = np.zeros((4 ** N, 4 ** N))
    for kidx in range(4 ** N):
        bits = 0
        for k in np.unravel_index(kidx, (4,) * N):
            bits = (bits << 2) | ((k & 1) << 1) | ((k >> 1) & 1)
        P[bits, kidx] = 1.0
    assert np.abs(P @ Hm @ P.T - Hjw).max() < 1e-12


def test_sector_hamiltonian_matches_jordan_wigner():
    N, na, nb = 3, 2, 1
    h1, eri = inputs.draw_integrals(_rng(5), N, 6)
    Hjw = of.jw_hamiltonian(h1, eri)
    ham = of.SectorHamiltonian(h1, eri, na, nb)
    ts, _ = inputs.draw_mps(_rng(6), N, na, nb, 4)
    ts2, _ = inputs.draw_mps(_rng(7), N, na, nb, 4)
    a = of.full_vector(ts)
    b = of.full_vector(ts2)
    ref = a @ Hjw @ b
    got = ham.expectation(of.mps_to_sector(ts, na, nb), of.mps_to_sector(ts2, na, nb))
    assert abs(ref - got) < 1e-12


def _closed_shell_energy(h1, eri, nocc):
    occ = range(nocc)
    e = 2 * sum(h1[i, i] for i in occ)
    e += sum(2 * eri[i, i, j, j] - eri[i, j, j, i] for i in occ for j in occ)
    return e


@pytest.mark.parametrize("N", [4, 6, 10])
def test_closed_shell_energy_textbook(N):
    """<RHF|H|RHF> = 2 sum h_ii + sum_ij [2 (ii|jj) - (ij|ji)]: pins the 1/2 and index order."""
    h1, eri = inputs.draw_integrals(_rng(20 + N), N, 2 * N)
    n = N // 2
    det = inputs.determinant_mps(N, range(n), range(n))
    ref = _closed_shell_energy(h1, eri, n)
    Hb, Sb = om.contract(det, om.build_mpo(h1, eri), det)
    assert abs(Sb - 1.0) < 1e-15
    assert abs(Hb - ref) < 1e-11 * max(1.0, abs(ref))
    if N <= 6:
        ham = of.SectorHamiltonian(h1, eri, n, n)
        psi = of.mps_to_sector(det, n, n)
        assert abs(ham.expectation(psi, psi) - ref) < 1e-11


# ----------------------------------------------------------------------------- nonorthogonal determinants
def lowdin(h1, eri, Ui, Uj, occ_a, occ_b):
    """Generalised Slater-Condon rules for two determinants in bases U_i and U_j.

    |Phi> = G(U)|det(occ)>; orbital coefficient matrix C = U[:, occ].
    S = det(Ci_a^T Cj_a) det(Ci_b^T Cj_b); transition density
    rho = Cj (Ci^T Cj)^-1 Ci^T, <a+_p a_q>/S = rho[q, p]; Wick's theorem.
    """
    S = 1.0
    rhos = []
    for occ in (occ_a, occ_b):
        Ci, Cj = Ui[:, list(occ)], Uj[:, list(occ)]
        M = Ci.T @ Cj
        S *= np.linalg.det(M)
        rhos.append(Cj @ np.linalg.solve(M, Ci.T))
    rt = rhos[0] + rhos[1]
    e = sum(np.einsum("pq,qp->", h1, r) for r in rhos)
    e += 0.5 * np.einsum("pqrs,qp,sr->", eri, rt, rt)
    e -= 0.5 * sum(np.einsum("pqrs,sp,qr->", eri, r, r) for r in rhos)
    return e * S, S


def _sparse_rotation(rng, N, ngates, sigma=0.6):
    U = np.eye(N)
    for _ in range(ngates):
        a = int(rng.integers(0, N - 1))
        t = rng.normal(0, sigma)
        R = np.eye(N)
        R[a, a], R[a, a + 1], R[a + 1, a], R[a + 1, a + 1] = math.cos(t), math.sin(t), -math.sin(t), math.cos(t)
        U = R @ U
    return U


def test_lowdin_determinants_fock_and_mps():
    N, n = 6, 3
    rng = _rng(31)
    h1, eri = inputs.draw_integrals(rng, N, 12)
    occ = [(0, 1, 2), (0, 2, 4), (1, 3, 5)]
    Us = [np.eye(N), inputs.draw_rotation(rng, N, 0.4)[1], inputs.draw_rotation(rng, N, 0.4)[1]]
    dets = [inputs.determinant_mps(N, o, o) for o in occ]
    ctx = om.Context(h1, eri, N, n, n, chi_rot=64)
    for d, U in zip(dets, Us):
        ctx.add_mps(d, U)
    pairs = [(0, 0), (0, 1), (0, 2), (1, 2), (1, 1)]
    HA, SA = of.matrix_elements(h1, eri, n, n, dets, Us, pairs)
    HB, SB = ctx.matrix_elements(pairs)
    for (i, j), ha, sa, hb, sb in zip(pairs, HA, SA, HB, SB):
        assert abs(ha - hb) < 1e-11 and abs(sa - sb) < 1e-12
    # same occupation in two different bases: closed form
    for oc in [(0, 1, 2), (1, 2, 5)]:
        d = inputs.determinant_mps(N, oc, oc)
        H2, S2 = of.matrix_elements(h1, eri, n, n, [d, d], [Us[1], Us[2]], [(0, 1)])
        hl, sl = lowdin(h1, eri, Us[1], Us[2], oc, oc)
        # determinant sign: both sides share the same interleave sign, which cancels
        assert abs(S2[0] - sl) < 1e-12
        assert abs(H2[0] - hl) < 1e-11


@pytest.mark.parametrize("N", [10, 14])
def test_lowdin_determinants_large_N(N):
    """Closed form at sizes beyond Fock space, rotation sparse enough to stay lossless."""
    n = N // 2
    rng = _rng(40 + N)
    h1, eri = inputs.draw_integrals(rng, N, 2 * N)
    Ui = _sparse_rotation(rng, N, 4)
    Uj = _sparse_rotation(rng, N, 4)
    oc = tuple(range(n))
    d = inputs.determinant_mps(N, oc, oc)
    ctx = om.Context(h1, eri, N, n, n, chi_rot=256)
    ctx.add_mps(d, Ui)
    ctx.add_mps(d, Uj)
    H, S, disc = ctx.pair(0, 1)
    hl, sl = lowdin(h1, eri, Ui, Uj, oc, oc)
    assert disc < 1e-20
    assert abs(S - sl) < 1e-12
    assert abs(H - hl) < 1e-10 * max(1.0, abs(hl))


def test_signed_permutation_keeps_determinant_product():
    """FSWAP special case: a permuted determinant stays bond dimension 1 (App. A3, theta in {0, pi/2})."""
    N, n = 8, 4
    oc = (0, 2, 3, 6)
    d = inputs.determinant_mps(N, oc, (1, 2, 5, 7))
    P = np.eye(N)[[2, 0, 1, 5, 3, 7, 4, 6]]
    ts, disc = om.apply_rotation(d, P, chi_rot=1, cutoff=1e-14)
    assert disc < 1e-28
    assert max(t.shape[2] for t in ts) == 1
    assert abs(abs(om.overlap(ts, ts)) - 1.0) < 1e-14


# ----------------------------------------------------------------------------- App. D worked example
def _app_d_rotation(N):
    """Orbital rotation of App. D / Fig. 6 from pi/4 and pi/2 Givens gates (one spin species)."""
    h = N // 2
    U = np.eye(N)

    def g(a, t):
        nonlocal U
        R = np.eye(N)
        c, s = math.cos(t), math.sin(t)
        # single-particle matrix of g_{a,a+1}(t): a+_a -> c a+_a - s a+_{a+1}
        R[a, a], R[a + 1, a], R[a, a + 1], R[a + 1, a + 1] = c, -s, s, c
        U = R @ U

    for r in range(h):
        g(h - 1, math.pi / 4)
        # move the new particle right to site N-1-r and the new hole left to site r
        for a in range(h, N - 1 - r):
            g(a, math.pi / 2)
        for a in range(h - 2, r - 1, -1):
            g(a, math.pi / 2)
    return U


@pytest.mark.parametrize("N", [4, 6])
def test_app_d_maximal_schmidt_rank(N):
    U = _app_d_rotation(N)
    h = N // 2
    d = inputs.determinant_mps(N, range(h), range(h))
    ts, disc = om.apply_rotation(d, U, chi_rot=4 ** N, cutoff=1e-14)
    full = of.mps_full_tensor(ts).reshape(4 ** h, 4 ** h)
    sv = np.linalg.svd(full, compute_uv=False)
    rank = 2 ** N
    assert np.all(np.abs(sv[:rank] - 2.0 ** (-h)) < 1e-12)
    assert np.all(sv[rank:] < 1e-12)
    if N == GOLD["app_d_schmidt"]["N"]:
        assert rank == GOLD["app_d_schmidt"]["rank"]
        assert abs(2.0 ** (-h) - GOLD["app_d_schmidt"]["value"]) < 1e-15
    # the rotated MPS itself carries that rank on the central bond
    assert ts[h - 1].shape[2] == rank


# ----------------------------------------------------------------------------- rotations
def test_compound_matrix_equals_fock_exponential():
    N, na, nb = 3, 2, 1
    ts, _ = inputs.draw_mps(_rng(50), N, na, nb, 4)
    U = inputs.draw_rotation(_rng(51), N, 0.9)[1]
    full = of.full_vector(ts)
    ref = of.full_rotation(U) @ full
    Psi = of.rotate_sector(of.mps_to_sector(ts, na, nb), U, na, nb)
    # map block-order sector amplitudes back to JW amplitudes
    SA, SB = of.occupation_sets(N, na), of.occupation_sets(N, nb)
    got = np.zeros_like(ref)
    for ia, A in enumerate(SA):
        for ib, B in enumerate(SB):
            bits = 0
            for p in range(N):
                bits = (bits << 2) | ((1 if p in A else 0) << 1) | (1 if p in B else 0)
            got[bits] = of.interleave_sign(A, B) * Psi[ia, ib]
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("det_sign", [1, -1])
def test_mps_rotation_lossless_equals_compound(det_sign):
    N, na, nb = 6, 3, 2
    rng = _rng(60)
    ts, _ = inputs.draw_mps(rng, N, na, nb, 8)
    U = inputs.draw_rotation(rng, N, 0.8)[1]
    if det_sign < 0:
        R = np.eye(N)
        R[4, 4] = -1.0
        U = U @ R
    rot, disc = om.apply_rotation(ts, U, chi_rot=4 ** 3, cutoff=1e-14)
    ref = of.rotate_sector(of.mps_to_sector(ts, na, nb), U, na, nb)
    got = of.mps_to_sector(rot, na, nb)
    assert np.abs(got - ref).max() < 1e-12
    assert abs(om.overlap(rot, rot) - om.overlap(ts, ts)) < 1e-13     # norm preserved


def test_truncation_closed_form_two_sites():
    """N=2 closed shell |updown, vac> under one gate: Schmidt values c^2, cs, cs, s^2."""
    t = 0.41
    c, s = math.cos(t), math.sin(t)
    d = inputs.determinant_mps(2, (0,), (0,))
    U = np.array([[c, s], [-s, c]])                  # G(U) = g_{0,1}(t)
    for chi, kept in [(4, [c * c, c * s, c * s, s * s]), (1, [c * c]), (3, [c * c, c * s, c * s])]:
        ts, disc = om.apply_rotation(d, U, chi_rot=chi, cutoff=1e-14)
        allw = [c ** 4, (c * s) ** 2, (c * s) ** 2, s ** 4]
        assert abs(disc - (1.0 - sum(x * x for x in kept))) < 1e-14
        assert ts[0].shape[2] == chi
    # cutoff rule: relative threshold on sigma_1
    ts, disc = om.apply_rotation(d, U, chi_rot=4, cutoff=(c * s) / (c * c) * 1.0001)
    assert ts[0].shape[2] == 1


def test_renormalised_rotation_keeps_the_input_norm():
    """renormalize=True (App. A1's rescaling after truncation) restores the input norm.

    The input state has norm 0.7, so a norm / norm^2 slip fails: the plain
    truncated state has norm^2 = 0.49 - (discarded weight) (each SVD runs at
    the canonical centre, so the dropped sigma^2 are orthogonal losses), the
    renormalised one has norm^2 = 0.49 and is parallel to the plain one.
    """
    w = inputs.make_workload(6, 3, 3, 12, 2, 8, seed=4)
    ts = [t.copy() for t in w.mps[1].tensors]
    ts[-1] = 0.7 * ts[-1]
    V = w.mps[1].U
    plain, disc = om.apply_rotation(ts, V, chi_rot=4, cutoff=1e-14)
    renorm, disc2 = om.apply_rotation(ts, V, chi_rot=4, cutoff=1e-14, renormalize=True)
    assert disc > 1e-3 and disc == disc2                       # the case truncates
    n_plain = om.overlap(plain, plain)
    n_renorm = om.overlap(renorm, renorm)
    assert abs(n_plain - (0.49 - disc)) < 1e-12
    assert abs(n_renorm - 0.49) < 1e-12
    assert abs(om.overlap(renorm, plain) ** 2 - n_renorm * n_plain) < 1e-12
    # N = 2 closed form: chi = 1 keeps sigma_1 = c^2 of |updown, vac>; renormalised it is the unit vector
    t = 0.41
    c, s = math.cos(t), math.sin(t)
    d = inputs.determinant_mps(2, (0,), (0,))
    U = np.array([[c, s], [-s, c]])
    r1, _ = om.apply_rotation(d, U, chi_rot=1, cutoff=1e-14, renormalize=True)
    p1, _ = om.apply_rotation(d, U, chi_rot=1, cutoff=1e-14)
    assert abs(om.overlap(p1, p1) - c ** 4) < 1e-14
    assert abs(om.overlap(r1, r1) - 1.0) < 1e-14


def test_identity_rotation_is_plain_overlap():
    w = inputs.make_workload(6, 3, 3, 12, 2, 8, seed=3)
    ctx = om.Context(w.h1, w.eri, 6, 3, 3)
    ctx.add_mps(w.mps[0].tensors, w.mps[1].U)
    ctx.add_mps(w.mps[1].tensors, w.mps[1].U)
    H, S, disc = ctx.pair(0, 1)
    assert abs(S - om.overlap(w.mps[0].tensors, w.mps[1].tensors)) < 1e-14


def test_basis_invariance_of_energy():
    """<psi|H|psi> with psi = G(U)|MPS> in the reference basis = <MPS|H^(U)|MPS> (Sec. IV B)."""
    N, n = 6, 3
    rng = _rng(70)
    h1, eri = inputs.draw_integrals(rng, N, 12)
    ts, _ = inputs.draw_mps(rng, N, n, n, 8)
    U = inputs.draw_rotation(rng, N, 0.5)[1]
    ham = of.SectorHamiltonian(h1, eri, n, n)
    psi = of.rotate_sector(of.mps_to_sector(ts, n, n), U, n, n)
    ref = ham.expectation(psi, psi)
    h, g = om.rotate_integrals(h1, eri, U)
    Hm, Sm = om.contract(ts, om.build_mpo(h, g), ts)
    assert abs(ref - Hm) < 1e-11


# ----------------------------------------------------------------------------- whole path at N=6
@pytest.fixture(scope="module")
def n6():
    w = inputs.workload("n6_chi8")
    ham = of.SectorHamiltonian(w.h1, w.eri, 3, 3)
    return w, ham


def test_fock_equals_mps_lossless_n6(n6):
    w, ham = n6
    HA, SA = of.matrix_elements(w.h1, w.eri, 3, 3, [m.tensors for m in w.mps], [m.U for m in w.mps], ham=ham)
    ctx = om.Context(w.h1, w.eri, 6, 3, 3, chi_rot=64)
    for m in w.mps:
        ctx.add_mps(m.tensors, m.U)
    pairs = w.all_pairs()
    HB, SB = ctx.matrix_elements(pairs)
    assert np.abs(HA - HB).max() < 1e-10
    assert np.abs(SA - SB).max() < 1e-12
    # S_ii = 1 and Hermiticity computed both ways (different rotations)
    for i in range(w.M):
        assert abs(SB[pairs.index((i, i))] - 1.0) < 1e-13
    for i, j in [(0, 1), (0, 2), (1, 2)]:
        Hji, Sji, _ = ctx.pair(j, i)
        assert abs(Hji - HB[pairs.index((i, j))]) < 1e-10
        assert abs(Sji - SB[pairs.index((i, j))]) < 1e-12


def test_variational_bound_n6(n6):
    w, ham = n6
    ctx = om.Context(w.h1, w.eri, 6, 3, 3, chi_rot=64)
    for m in w.mps:
        ctx.add_mps(m.tensors, m.U)
    pairs = w.all_pairs()
    Hv, Sv = ctx.matrix_elements(pairs)
    H = np.zeros((w.M, w.M))
    S = np.zeros((w.M, w.M))
    for (i, j), h, s in zip(pairs, Hv, Sv):
        H[i, j] = H[j, i] = h
        S[i, j] = S[j, i] = s
    E, C, rank, k1 = om.solve(H, S)
    e_sector = ham.ground_energy()
    assert E[0] >= e_sector - 1e-10
    # full Fock space ground state lies at or below the sector's
    if w.N <= 4:
        Hjw = of.jw_hamiltonian(w.h1, w.eri)
        assert e_sector >= np.linalg.eigvalsh(Hjw)[0] - 1e-10


def test_full_fock_ground_state_below_sector():
    N = 3
    h1, eri = inputs.draw_integrals(_rng(80), N, 6)
    e_full = np.linalg.eigvalsh(of.jw_hamiltonian(h1, eri))[0]
    for na, nb in [(1, 1), (2, 1), (2, 2)]:
        assert of.SectorHamiltonian(h1, eri, na, nb).ground_energy() >= e_full - 1e-10


# ----------------------------------------------------------------------------- solve
def test_solve_special_cases():
    E, C, rank, k1 = om.solve(np.array([[-3.0]]), np.array([[0.25]]))
    assert rank == 1 and abs(E[0] + 12.0) < 1e-14
    assert abs(C[0, 0] - 2.0) < 1e-14
    assert abs(k1 - 4.0 / math.sqrt(145.0)) < 1e-14
    rng = _rng(90)
    M = 7
    A = rng.normal(size=(M, M))
    S = A @ A.T + M * np.eye(M)
    B = rng.normal(size=(M, M))
    H = B + B.T
    E, C, rank, k1 = om.solve(H, S)
    ref = scipy.linalg.eigh(H, S, eigvals_only=True)
    assert rank == M and np.abs(E - ref).max() < 1e-12
    assert np.abs(C.T @ S @ C - np.eye(M)).max() < 1e-12
    assert np.abs(H @ C - S @ C @ np.diag(E)).max() < 1e-11


def test_solve_drops_near_null_space():
    rng = _rng(91)
    M = 6
    Q = np.linalg.qr(rng.normal(size=(M, M)))[0]
    lam = np.array([1e-13, 1e-3, 0.1, 1.0, 2.0, 3.0])
    S = Q @ np.diag(lam) @ Q.T
    H = rng.normal(size=(M, M))
    H = H + H.T
    E, C, rank, k1 = om.solve(H, S, eps=1e-10)
    assert rank == 5
    X = Q[:, 1:] / np.sqrt(lam[1:])
    ref = np.linalg.eigvalsh(X.T @ H @ X)
    assert np.abs(E - ref).max() < 1e-12 * np.abs(ref).max()
