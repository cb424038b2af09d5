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
    h1, eri = sw.hamiltonian(CFG)
    be = OracleBackend(h1, eri, CFG.N, CFG.n_alpha, CFG.n_beta)
    n_k = CFG.N * (CFG.N - 1) // 2
    plain = sw.run_sweep(CFG, seed=2, backend=be)
    res = sw.run_sweep(CFG, seed=2, backend=be, proposer=lambda x: np.zeros((len(x), n_k)))
    assert res.learned_accepted == 0
    assert res.proposals == CFG.R * sum(res.M)
    # zero steps take the place of random ones: never better than the plain run's first sweep
    assert res.energies[0] >= plain.energies[0] - 1e-9 or res.accepted <= plain.accepted
    assert np.all(np.diff(res.energies) <= 1e-10)


def test_sweeps_to_reach_and_training_rows():
    r = sw.SweepResult([-1.0, -1.5, -1.5, -2.0], [1, 1, 2, 2], 0, 0, 0, [])
    assert sw.sweeps_to_reach(r, -1.5) == 2 and sw.sweeps_to_reach(r, -2.0) == 4 and sw.sweeps_to_reach(r, -3) == 5
    rec = [(np.ones(3), np.zeros(2), 2.0), (np.zeros(3), np.ones(2), 6.0)]
    X, T, w = sw.training_set(rec)
    assert X.shape == (2, 3) and T.shape == (2, 2) and np.allclose(w, [0.5, 1.5])
    K = sw.k_matrix(np.arange(6.0), 4)
    assert np.allclose(K, -K.T) and np.allclose(sw.k_vector(K), np.arange(6.0))
