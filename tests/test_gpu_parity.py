"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle.

FP64 tolerances: max |dH_ij|, |dS_ij| <= 1e-10 and |dE| <= 1e-9 Ha.
"""
import math

import numpy as np
import pytest

from oracle import fock as of
from oracle import mps as om
from paper_2404_10223_gb300 import inputs
from paper_2404_10223_gb300 import tnqe

pytestmark = pytest.mark.gpu

TOL_HS = 1e-10
TOL_E = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2404_10223_gb300 import build as B
    import os
    if not os.path.exists(B.LIB):
        B.build()
    tnqe.load()


def gpu_ctx(w, **opts):
    ctx = tnqe.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff, **opts)
    for m in w.mps:
        ctx.add_mps(m.tensors, m.U)
    return ctx


def oracle_ctx(w, chi_rot=0, renormalize=False):
    o = om.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, chi_rot=chi_rot, cutoff=w.cutoff, renormalize=renormalize)
    for m in w.mps:
        o.add_mps(m.tensors, m.U)
    return o


def assemble(M, pairs, Hv, Sv):
    H = np.zeros((M, M))
    S = np.zeros((M, M))
    for (i, j), h, s in zip(pairs, Hv, Sv):
        H[i, j] = H[j, i] = h
        S[i, j] = S[j, i] = s
    return H, S


# ----------------------------------------------------------------------------- N = 6
def test_n6_lossless_equals_exact_fock():
    w = inputs.workload("n6_chi8")
    pairs = w.all_pairs()
    HA, SA = of.matrix_elements(w.h1, w.eri, 3, 3, [m.tensors for m in w.mps], [m.U for m in w.mps], pairs)
    with gpu_ctx(w, chi_rot=64) as g:
        HG, SG = g.matrix_elements(pairs)
    assert np.abs(HG - HA).max() <= TOL_HS
    assert np.abs(SG - SA).max() <= TOL_HS


@pytest.mark.parametrize("seed", [0, 1])
def test_n6_truncated_equals_oracle(seed):
    w = inputs.make_workload(6, 3, 3, 12, 4, 8, seed=seed, name="n6")
    pairs = w.all_pairs()
    HB, SB = oracle_ctx(w).matrix_elements(pairs)
    with gpu_ctx(w) as g:
        HG, SG = g.matrix_elements(pairs)
        EG, CG, rG, kG = g.solve(*assemble(w.M, pairs, HG, SG))
    assert np.abs(HG - HB).max() <= TOL_HS
    assert np.abs(SG - SB).max() <= TOL_HS
    EB, CB, rB, kB = om.solve(*assemble(w.M, pairs, HB, SB))
    assert rG == rB
    assert abs(EG[0] - EB[0]) <= TOL_E


# ----------------------------------------------------------------------------- N = 10
@pytest.fixture(scope="module")
def n10():
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    o = oracle_ctx(w)
    HB, SB = o.matrix_elements(pairs)
    return w, pairs, HB, SB


FORMS = [tnqe.TNQE_FORM_BLOCKS, tnqe.TNQE_FORM_DENSE]


@pytest.mark.parametrize("form", FORMS)
def test_n10_all_pairs_equal_oracle(n10, form):
    """FP64 contraction in charge blocks (default) and over the dense zero-padded tensors."""
    w, pairs, HB, SB = n10
    with gpu_ctx(w, contraction_form=form) as g:
        HG, SG = g.matrix_elements(pairs)
    dH = np.abs(HG - HB).max()
    dS = np.abs(SG - SB).max()
    assert dH <= TOL_HS, dH
    assert dS <= TOL_HS, dS


def test_n10_energy_equals_oracle(n10):
    w, pairs, HB, SB = n10
    with gpu_ctx(w) as g:
        HG, SG = g.matrix_elements(pairs)
        EG, CG, rG, kG = g.solve(*assemble(w.M, pairs, HG, SG))
    EB, CB, rB, kB = om.solve(*assemble(w.M, pairs, HB, SB))
    assert rG == rB
    assert abs(EG[0] - EB[0]) <= TOL_E
    assert abs(kG - kB) <= 1e-6 * max(1.0, abs(kB))


def test_n10_rotation_state_and_discarded_weight(n10):
    w = n10[0]
    o = oracle_ctx(w)
    with gpu_ctx(w) as g:
        for i, j in [(0, 3), (2, 5), (4, 1)]:
            dg = g.rotate(i, j)
            ket_g = g.get_rotated()
            ket_o, do = o.rotate(i, j)
            assert abs(dg - do) <= 1e-10
            # gauge-invariant comparison of the two rotated states
            f_go = om.overlap(ket_g, ket_o)
            assert abs(om.overlap(ket_g, ket_g) - om.overlap(ket_o, ket_o)) <= 1e-11
            assert abs(f_go - om.overlap(ket_o, ket_o)) <= 1e-11
            assert [t.shape[2] for t in ket_g] == [t.shape[2] for t in ket_o]


# ----------------------------------------------------------------------------- edge cases
def test_closed_form_determinants_n14():
    """chi = 1 determinants in sparse-rotated bases: Loewdin closed form (any N)."""
    from tests.test_oracle_pins import lowdin, _sparse_rotation
    N, n = 14, 7
    rng = np.random.default_rng(5)
    h1, eri = inputs.draw_integrals(rng, N, 2 * N)
    Us = [_sparse_rotation(rng, N, 4) for _ in range(3)]
    oc = tuple(range(n))
    det = inputs.determinant_mps(N, oc, oc)
    with tnqe.Context(h1, eri, N, n, n, chi_rot=64) as g:
        for U in Us:
            g.add_mps(det, U)
        pairs = [(0, 1), (0, 2), (1, 2), (1, 1)]
        HG, SG = g.matrix_elements(pairs)
    for (i, j), h, s in zip(pairs, HG, SG):
        hl, sl = lowdin(h1, eri, Us[i], Us[j], oc, oc)
        assert abs(s - sl) <= TOL_HS
        assert abs(h - hl) <= 1e-10 * max(1.0, abs(hl))


def test_reflection_identity_and_renormalisation():
    w = inputs.make_workload(6, 3, 2, 12, 3, 6, seed=11, name="n6b")
    R = np.eye(6)
    R[3, 3] = -1.0
    w.mps[1].U = w.mps[1].U @ R                      # det U = -1
    w.mps[2].U = w.mps[0].U.copy()                   # identical bases: identity rotation
    pairs = w.all_pairs()
    for renorm in (False, True):
        HB, SB = oracle_ctx(w, renormalize=renorm).matrix_elements(pairs)
        with gpu_ctx(w, renormalize_rotated=int(renorm)) as g:
            HG, SG = g.matrix_elements(pairs)
        assert np.abs(HG - HB).max() <= TOL_HS
        assert np.abs(SG - SB).max() <= TOL_HS
    # identity rotation reproduces the plain overlap
    k = pairs.index((0, 2))
    assert abs(SG[k] - om.overlap(w.mps[0].tensors, w.mps[2].tensors)) <= 1e-12


@pytest.mark.parametrize("form", FORMS)
def test_shuffled_bonds_and_ragged_dims(form):
    """Bond indices in arbitrary charge order and unequal chi_i, chi_j."""
    rng = np.random.default_rng(21)
    N, na, nb = 8, 4, 3
    h1, eri = inputs.draw_integrals(rng, N, 16)
    states = []
    for chi, sh in [(7, True), (13, False), (5, True)]:
        ts, _ = inputs.draw_mps(rng, N, na, nb, chi, shuffle_bonds=sh)
        U = inputs.draw_rotation(rng, N, 0.4)[1]
        states.append((ts, U))
    o = om.Context(h1, eri, N, na, nb)
    with tnqe.Context(h1, eri, N, na, nb, contraction_form=form) as g:
        for ts, U in states:
            o.add_mps(ts, U)
            g.add_mps(ts, U)
        pairs = [(0, 0), (0, 1), (0, 2), (1, 2), (2, 2)]
        HG, SG = g.matrix_elements(pairs)
    HB, SB = o.matrix_elements(pairs)
    assert np.abs(HG - HB).max() <= TOL_HS
    assert np.abs(SG - SB).max() <= TOL_HS


@pytest.mark.parametrize("form", FORMS)
def test_tiny_chains(form):
    for N, na, nb in [(1, 1, 0), (2, 1, 1), (3, 2, 1), (4, 0, 2), (3, 3, 3)]:
        rng = np.random.default_rng(N)
        h1, eri = inputs.draw_integrals(rng, N, 2)
        states = [inputs.draw_mps(rng, N, na, nb, 4)[0] for _ in range(2)]
        Us = [np.eye(N), inputs.draw_rotation(rng, N, 0.7)[1]]
        HA, SA = of.matrix_elements(h1, eri, na, nb, states, Us, [(0, 0), (0, 1), (1, 1)])
        with tnqe.Context(h1, eri, N, na, nb, chi_rot=64, contraction_form=form) as g:
            for t, U in zip(states, Us):
                g.add_mps(t, U)
            HG, SG = g.matrix_elements([(0, 0), (0, 1), (1, 1)])
        assert np.abs(HG - HA).max() <= TOL_HS
        assert np.abs(SG - SA).max() <= TOL_HS


def test_solve_matches_oracle_and_handles_null_space():
    rng = np.random.default_rng(3)
    M = 9
    Q = np.linalg.qr(rng.normal(size=(M, M)))[0]
    lam = np.array([1e-14, 1e-12, 1e-6, 1e-3, 0.1, 0.5, 1.0, 2.0, 3.0])
    S = Q @ np.diag(lam) @ Q.T
    B = rng.normal(size=(M, M))
    H = B + B.T
    w = inputs.workload("n6_chi8")
    with tnqe.Context(w.h1, w.eri, 6, 3, 3) as g:
        E, C, r, k = g.solve(H, S)
        E1, C1, r1, k1 = g.solve(np.array([[-3.0]]), np.array([[0.25]]))
    Eo, Co, ro, ko = om.solve(H, S)
    assert r == ro == 7
    # kept spectrum of S spans 1e-6..3: eigenvalue errors scale with cond = 3e6
    assert np.abs(E[:r] - Eo).max() <= 3e6 * 1e-15 * np.abs(Eo).max()
    assert np.all(np.isnan(E[r:]))
    assert np.abs(C[:, :r].T @ S @ C[:, :r] - np.eye(r)).max() <= 1e-8
    assert abs(k - ko) <= 1e-6 * abs(ko)
    # well-conditioned pencil: FP64-level agreement
    A = rng.normal(size=(M, M))
    S2 = A @ A.T + M * np.eye(M)
    with tnqe.Context(w.h1, w.eri, 6, 3, 3) as g:
        E2, C2, r2, k2 = g.solve(H, S2)
    Eo2 = om.solve(H, S2)[0]
    assert r2 == M and np.abs(E2 - Eo2).max() <= 1e-12 * np.abs(Eo2).max()
    assert r1 == 1 and abs(E1[0] + 12.0) <= 1e-14 and abs(k1 - 4.0 / math.sqrt(145.0)) <= 1e-14


def test_rejects_invalid_states():
    w = inputs.workload("n6_chi8")
    m = w.mps[1]
    with tnqe.Context(w.h1, w.eri, 6, 3, 3) as g:
        U = m.U.copy()
        U[0, 0] += 1e-6
        with pytest.raises(tnqe.TnqeError) as e:
            g.add_mps(m.tensors, U)
        assert e.value.status == 1
        bad = [t.copy() for t in m.tensors]
        bad[2][0, 0, :] += 0.3                       # breaks charge blocks / orthonormality
        with pytest.raises(tnqe.TnqeError):
            g.add_mps(bad, m.U)
        bad = [t.copy() for t in m.tensors]
        bad[1] *= 1.5                                # not left-orthonormal
        with pytest.raises(tnqe.TnqeError):
            g.add_mps(bad, m.U)
        with pytest.raises(tnqe.TnqeError):
            g.matrix_elements([(0, 5)])
        assert g.add_mps(m.tensors, m.U) == 0         # context still usable


# ----------------------------------------------------------------------------- full-size sampled pairs
def test_n14_mixed_sampled_pairs():
    """The benchmark workload (N=14, M=16, chi in {32,64,128}) on pairs the oracle finishes in seconds."""
    w = inputs.workload("n14_mixed")
    chis = [m.chi for m in w.mps]
    small = [k for k in range(w.M) if chis[k] == 32]
    mid = [k for k in range(w.M) if chis[k] == 64]
    pairs = [(small[0], small[1]), (small[0], mid[0]), (small[1], mid[1]), (small[2], small[2])]
    pairs = [(min(i, j), max(i, j)) for i, j in pairs]
    o = oracle_ctx(w)
    HB, SB = o.matrix_elements(pairs)
    with gpu_ctx(w) as g:
        HG, SG = g.matrix_elements(w.all_pairs())
    allp = w.all_pairs()
    for (i, j), hb, sb in zip(pairs, HB, SB):
        k = allp.index((i, j))
        assert abs(HG[k] - hb) <= TOL_HS, (i, j, HG[k], hb)
        assert abs(SG[k] - sb) <= TOL_HS
    # invariants at full size: S_ii = 1, finite everything
    for i in range(w.M):
        assert abs(SG[allp.index((i, i))] - 1.0) <= 1e-12
    assert np.all(np.isfinite(HG)) and np.all(np.isfinite(SG))


# ----------------------------------------------------------------------------- split precision
def test_tf32x3_contraction_error_against_fp64():
    """TF32x3 tensor-core contraction: errors stated as numbers against the FP64 path.

    Bounds (measured 1.9e-4 / 3.1e-6 / 1.5e-5 on this workload): FP32
    accumulation limits H_ii ~ 56 Ha to ~1e-5 relative.
    """
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    out = {}
    for prec in (0, 1):
        with gpu_ctx(w, precision=prec) as g:
            Hv, Sv = g.matrix_elements(pairs)
            E = g.solve(*assemble(w.M, pairs, Hv, Sv))[0]
        out[prec] = (Hv, Sv, E)
    (H0, S0, E0), (H1, S1, E1) = out[0], out[1]
    assert np.abs(H1 - H0).max() <= 1e-5 * np.abs(H0).max()
    assert np.abs(S1 - S0).max() <= 2e-5
    assert abs(E1[0] - E0[0]) <= 1e-4
    off = [k for k, (i, j) in enumerate(pairs) if i != j]
    assert np.abs(H1[off] - H0[off]).max() <= 1e-5


# Measured on n10_chi32 against the FP64 path (max|dH|, max|dS|, |dE|):
#   BF16X3 1.2e-2 / 4.5e-4 / 1.5e-2     BF16X6  8.6e-6 / 3.4e-7 / 1.1e-5
#   BF16X10 1.7e-7 / 6.7e-9 / 1.8e-7    BF16X15 4.6e-9 / 2.5e-10 / 7.6e-9
# The bounds below keep a margin of about five over those numbers.
SLICED_BOUNDS = {
    tnqe.TNQE_PREC_BF16X3: (5e-2, 2e-3, 5e-2),
    tnqe.TNQE_PREC_BF16X6: (5e-5, 2e-6, 5e-5),
    tnqe.TNQE_PREC_BF16X10: (1e-6, 5e-8, 1e-6),
    tnqe.TNQE_PREC_BF16X15: (3e-8, 2e-9, 5e-8),
}


def test_sliced_bf16_contraction_errors_against_fp64():
    """Sliced-BF16 tensor-core contractions: every mode's error stated and bounded."""
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    with gpu_ctx(w) as g:
        H0, S0 = g.matrix_elements(pairs)
        E0 = g.solve(*assemble(w.M, pairs, H0, S0))[0]
        for prec, (bh, bs, be) in SLICED_BOUNDS.items():
            g.set_precision(prec)
            Hv, Sv = g.matrix_elements(pairs)
            E = g.solve(*assemble(w.M, pairs, Hv, Sv))[0]
            assert np.abs(Hv - H0).max() <= bh, (prec, np.abs(Hv - H0).max())
            assert np.abs(Sv - S0).max() <= bs, (prec, np.abs(Sv - S0).max())
            assert abs(E[0] - E0[0]) <= be, (prec, abs(E[0] - E0[0]))


def test_sliced_bf16x15_against_exact_fock_n6():
    """The most accurate sliced mode against the dense Fock-space oracle (lossless rotations)."""
    w = inputs.workload("n6_chi8")
    pairs = w.all_pairs()
    Hf, Sf = of.matrix_elements(w.h1, w.eri, 3, 3, [m.tensors for m in w.mps], [m.U for m in w.mps], pairs)
    with gpu_ctx(w, chi_rot=64, precision=tnqe.TNQE_PREC_BF16X15) as g:
        Hv, Sv = g.matrix_elements(pairs)
    assert np.abs(Hv - Hf).max() <= 1e-8
    assert np.abs(Sv - Sf).max() <= 1e-9


def test_sliced_bf16_ragged_and_tiny_chains():
    """Ragged bond dimensions (tile tails in every GEMM) and N = 1, 2 chains in the sliced mode."""
    for name in ("n14_mixed",):
        w = inputs.workload(name)
        allp = w.all_pairs()
        pairs = [allp[k] for k in range(0, len(allp), 17)]
        with gpu_ctx(w) as g:
            H0, S0 = g.matrix_elements(pairs)
            g.set_precision(tnqe.TNQE_PREC_BF16X15)
            H1, S1 = g.matrix_elements(pairs)
        assert np.abs(H1 - H0).max() <= 3e-7
        assert np.abs(S1 - S0).max() <= 1e-8
    for N, na, nb in [(1, 1, 0), (2, 1, 1), (3, 2, 1)]:
        rng = np.random.default_rng(N)
        h1, eri = inputs.draw_integrals(rng, N, 2)
        states = [inputs.draw_mps(rng, N, na, nb, 4)[0] for _ in range(2)]
        Us = [np.eye(N), inputs.draw_rotation(rng, N, 0.7)[1]]
        HA, SA = of.matrix_elements(h1, eri, na, nb, states, Us, [(0, 0), (0, 1), (1, 1)])
        with tnqe.Context(h1, eri, N, na, nb, chi_rot=64, precision=tnqe.TNQE_PREC_BF16X15) as g:
            for t, U in zip(states, Us):
                g.add_mps(t, U)
            HG, SG = g.matrix_elements([(0, 0), (0, 1), (1, 1)])
        assert np.abs(HG - HA).max() <= 1e-9 and np.abs(SG - SA).max() <= 1e-10


def test_reversed_pair_order_matches_oracle():
    """(j, i) puts state j in the bra: equal to (i, j) up to truncation, and to the oracle's (j, i) exactly."""
    w = inputs.workload("n10_chi32")
    pairs = [(3, 1), (1, 3), (5, 0), (0, 5), (4, 4)]
    o = oracle_ctx(w)
    HB, SB = o.matrix_elements(pairs)
    with gpu_ctx(w) as g:
        HG, SG = g.matrix_elements(pairs)
    assert np.abs(HG - HB).max() <= TOL_HS and np.abs(SG - SB).max() <= TOL_HS



def test_hermiticity_and_norm_lossless():
    """Untruncated (chi_rot above every exact bond dimension): H_ij and H_ji, computed through different
    rotations (V and V^T), agree to 1e-12, S_ii = 1, and every rotation keeps the norm (nothing discarded)."""
    w = inputs.workload("n6_chi8")
    pairs = [(i, j) for i in range(w.M) for j in range(w.M)]
    with gpu_ctx(w, chi_rot=64) as g:
        Hv, Sv = g.matrix_elements(pairs)
        for i, j in pairs:
            if i != j:
                assert g.rotate(i, j) <= 1e-24
                ket = g.get_rotated()
                assert abs(om.overlap(ket, ket) - 1.0) <= 1e-13
    H = Hv.reshape(w.M, w.M)
    S = Sv.reshape(w.M, w.M)
    assert np.abs(H - H.T).max() <= 1e-12 and np.abs(S - S.T).max() <= 1e-12
    assert np.abs(np.diag(S) - 1.0).max() <= 1e-13


def test_pair_list_edge_cases():
    """An empty pair list, a list of unrotated pairs only, rotated pairs only, and a repeated pair."""
    w = inputs.workload("n10_chi32")
    o = oracle_ctx(w)
    with gpu_ctx(w) as g:
        H0, S0 = g.matrix_elements([])
        assert H0.size == 0 and S0.size == 0
        diag = [(k, k) for k in range(w.M)]
        Hd, Sd = g.matrix_elements(diag)
        rot = [(1, 4), (4, 1), (2, 3)]
        Hr, Sr = g.matrix_elements(rot)
        Hp, Sp = g.matrix_elements([(2, 3), (2, 3), (0, 0)])
        with pytest.raises(tnqe.TnqeError):
            g.matrix_elements([(0, w.M)])
    HB, SB = o.matrix_elements(diag + rot)
    assert np.abs(np.concatenate([Hd, Hr]) - HB).max() <= TOL_HS
    assert np.abs(np.concatenate([Sd, Sr]) - SB).max() <= TOL_HS
    assert Hp[0] == Hp[1] == Hr[2] and Sp[0] == Sp[1] == Sr[2] and Hp[2] == Hd[0]
