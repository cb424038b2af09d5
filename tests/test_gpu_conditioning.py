"""Conditioning tools on the GPU: dependence residuals against the oracle,
discard of near-duplicate states, the solve threshold, shot-noise emulation."""
import numpy as np
import pytest
import scipy.linalg

from oracle import conditioning as oc
from paper_2404_10223_gb300 import conditioning as cd
from paper_2404_10223_gb300 import inputs, tnqe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2404_10223_gb300 import build as B
    import os
    if not os.path.exists(B.LIB):
        B.build()
    tnqe.load()


def test_dependence_residuals_match_oracle():
    rng = np.random.default_rng(0)
    V = rng.normal(size=(40, 12))
    V[:, 7] = V[:, 1] - 0.5 * V[:, 3] + 1e-4 * rng.normal(size=40)
    V /= np.linalg.norm(V, axis=0)
    S = V.T @ V
    w = inputs.workload("n6_chi8")
    with tnqe.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta) as g:
        r = g.dependence(S, 1e-12)
    ro = oc.residuals(S, 1e-12)
    for j in range(12):   # both sides lose cond(S_<j) digits through the pseudo-inverse
        cond = np.linalg.cond(S[:j, :j]) if j else 1.0
        assert abs(r[j] - ro[j]) <= 1e-15 * cond + 1e-13, (j, r[j], ro[j], cond)
    assert r[7] < 1e-6 and np.all(np.delete(r, 7) > 1e-2)


def test_near_duplicates_are_discarded_and_the_energy_survives():
    w = inputs.workload("n10_chi32")
    rng = np.random.default_rng(7)
    states = [(m.tensors, m.U) for m in w.mps]
    # Near-duplicates: the same orbitals, the canonical-centre tensor perturbed by 1e-3 and
    # renormalised (charge blocks kept).  A perturbed rotation is no near-duplicate here: the
    # Givens network of V = I + O(1e-3) has O(1) angles between small entries, whose
    # truncations do not cancel (overlap 0.83 with the original at chi = 32).
    for j in (1, 4):
        t = [x.copy() for x in w.mps[j].tensors]
        last = t[-1]
        last += 1e-3 * rng.normal(size=last.shape) * (last != 0)
        last /= np.linalg.norm(last)
        states.append((t, w.mps[j].U))
    M = len(states)
    pairs = [(i, j) for i in range(M) for j in range(i, M)]
    with tnqe.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff) as g:
        for t, U in states:
            g.add_mps(t, U)
        Hv, Sv = g.matrix_elements(pairs)
        H = np.zeros((M, M))
        S = np.zeros((M, M))
        for (i, j), h, s in zip(pairs, Hv, Sv):
            H[i, j] = H[j, i] = h
            S[i, j] = S[j, i] = s
        kept, res = cd.discard_dependent(g, S, threshold=1e-3)
        assert kept == list(range(w.M))                  # the two copies go, the originals stay
        assert res[w.M] < 1e-3 and res[w.M + 1] < 1e-3
        # with truncated rotations S of a near-dependent set is not a Gram matrix (here it has an
        # eigenvalue near -1e-3), so the full solve is unreliable; the kept set is well conditioned
        assert np.abs(np.linalg.eigvalsh(S)).min() < 2e-3
        assert np.linalg.eigvalsh(S[np.ix_(kept, kept)]).min() > 0.5
        E_all = g.solve(H, S)[0][0]
        E_kept = g.solve(H[np.ix_(kept, kept)], S[np.ix_(kept, kept)])[0][0]
        assert abs(E_kept - E_all) < 1e-2
        # solve_ex at solve_eps is tnqe_solve
        E1 = g.solve_ex(H, S, 1e-10)[0]
        assert np.array_equal(np.nan_to_num(E1, nan=0.0), np.nan_to_num(g.solve(H, S)[0], nan=0.0))
        study = cd.noise_study(g, H[np.ix_(kept, kept)], S[np.ix_(kept, kept)], np.random.default_rng(3), trials=20)
    for eps, st in study.items():
        assert np.isfinite(st["std_dev"]) and st["max_abs_dev"] < 1e-2
        assert st["rank"] == len(kept)
