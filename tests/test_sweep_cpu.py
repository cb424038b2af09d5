"""Host logic of the generalized sweep (CPU), with the oracle as matrix-element backend.

Checks the variational bound against exact diagonalisation, monotone energies,
the growth schedule, the acceptance records, and that a proposer which never
moves is never accepted."""
import numpy as np
import pytest

from oracle import fock as of
from oracle import mps as om
from paper_2404_10223_gb300 import sweep as sw


class OracleBackend:
    def __init__(self, h1, eri, N, na, nb):
        self.args = (h1, eri, N, na, nb)
        self.reset()

    def reset(self):
        self.o = om.Context(*self.args)

    def add_mps(self, tensors, U):
        return self.o.add_mps(tensors, U)

    def matrix_elements(self, pairs):
        return self.o.matrix_elements(pairs)

    def energies(self, H, S):
        E, _, rank, _ = om.solve(H, S)
        return E[:rank]


CFG = sw.SweepConfig(N=4, n_alpha=2, n_beta=2, L=4, chi=4, M_max=3, sweeps=5, grow_every=2, R=3, sigma=0.2)


def test_plain_sweep_is_variational_monotone_and_follows_the_schedule():
    h1, eri = sw.hamiltonian(CFG)
    be = OracleBackend(h1, eri, CFG.N, CFG.n_alpha, CFG.n_beta)
    res = sw.run_sweep(CFG, seed=1, backend=be)
    assert res.M == [1, 1, 2, 2, 3]
    E = np.array(res.energies)
    assert np.all(np.diff(E) <= 1e-10)                      # acceptance and growth never raise the energy
    e_exact = of.SectorHamiltonian(h1, eri, CFG.n_alpha, CFG.n_beta).ground_energy()
    assert E[-1] >= e_exact - 1e-9                          # Rayleigh-Ritz bound
    steps = [r for r in res.records if r[0][-1] == 0.0]
    births = [r for r in res.records if r[0][-1] == 1.0]
    assert res.accepted == len(steps) and res.accepted > 0 and len(births) == 2
    for x, dK, drop in res.records:
        assert drop > CFG.tol and x.shape == (sw.n_features(CFG.N),)
        assert dK.shape == (CFG.N * (CFG.N - 1) // 2,)


def test_a_proposer_that_never_moves_is_never_accepted():
    """As an extra candidate a zero step never wins, and the random candidates are the plain run's:
    the learned run reproduces the plain run exactly."""
    h1, eri = sw.hamiltonian(CFG)
    be = OracleBackend(h1, eri, CFG.N, CFG.n_alpha, CFG.n_beta)
    n_k = CFG.N * (CFG.N - 1) // 2
    plain = sw.run_sweep(CFG, seed=2, backend=be)
    res = sw.run_sweep(CFG, seed=2, backend=be, proposer=lambda x: np.zeros((len(x), n_k)))
    assert res.learned_accepted == 0 and res.learned_births == 0
    assert res.proposals == (CFG.R + 1) * sum(res.M)
    assert res.energies == plain.energies and res.accepted == plain.accepted
    # in the replace mode the zero step takes the place of a random one
    rcfg = sw.SweepConfig(**{**CFG.__dict__, "learned_mode": "replace"})
    rep = sw.run_sweep(rcfg, seed=2, backend=be, proposer=lambda x: np.zeros((len(x), n_k)))
    assert rep.learned_accepted == 0 and rep.proposals == CFG.R * sum(rep.M)
    assert np.all(np.diff(rep.energies) <= 1e-10)


def test_a_good_extra_candidate_is_taken_and_never_hurts_a_step():
    """A proposer that returns a fixed nonzero step is an extra candidate: with the plain run's random
    candidates also on offer, the first sweep (one state) ends at an energy no higher than the plain
    run's, and the energies stay monotone."""
    h1, eri = sw.hamiltonian(CFG)
    be = OracleBackend(h1, eri, CFG.N, CFG.n_alpha, CFG.n_beta)
    n_k = CFG.N * (CFG.N - 1) // 2
    plain = sw.run_sweep(CFG, seed=3, backend=be)
    big = lambda x: np.tile(0.3 * np.ones(n_k) / np.sqrt(n_k), (len(x), 1))
    res = sw.run_sweep(CFG, seed=3, backend=be, proposer=big)
    assert res.energies[0] <= plain.energies[0] + 1e-10
    assert np.all(np.diff(res.energies) <= 1e-10)


def test_paired_summary_sign_test():
    rows = [{"sweeps_plain": 10, "sweeps_learned": s, "dE_final": d} for s, d in
            [(8, -1.0), (9, -0.5), (10, 0.0), (12, 0.2), (7, -0.1), (6, -0.3)]]
    out = sw.paired_summary(rows)
    assert (out["wins"], out["ties"], out["losses"]) == (4, 1, 1)
    assert abs(out["sign_test_p"] - 2 * (1 + 5) / 32) < 1e-12       # n = 5, k = 1
    assert abs(out["mean_sweep_difference"] - (-2 - 1 + 0 + 2 - 3 - 4) / 6) < 1e-12
    assert out["learned_lower_or_equal_final"] == 5


def test_sweeps_to_reach_and_training_rows():
    r = sw.SweepResult([-1.0, -1.5, -1.5, -2.0], [1, 1, 2, 2], 0, 0, 0, [], 0)
    assert sw.sweeps_to_reach(r, -1.5) == 2 and sw.sweeps_to_reach(r, -2.0) == 4 and sw.sweeps_to_reach(r, -3) == 5
    rec = [(np.ones(3), np.zeros(2), 2.0), (np.zeros(3), np.ones(2), 6.0)]
    X, T, w = sw.training_set(rec)
    assert X.shape == (2, 3) and T.shape == (2, 2) and np.allclose(w, [0.5, 1.5])
    K = sw.k_matrix(np.arange(6.0), 4)
    assert np.allclose(K, -K.T) and np.allclose(sw.k_vector(K), np.arange(6.0))
