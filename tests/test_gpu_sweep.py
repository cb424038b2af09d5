"""Generalized sweep on the GPU: the same decisions as with the CPU oracle as
backend, the variational bound, and the learned proposal end to end (network
trained by the library's kernels on records of plain sweeps)."""
import numpy as np
import pytest

from oracle import fock as of
from oracle import mps as om
from paper_2404_10223_gb300 import sweep as sw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2404_10223_gb300 import build as B
    import os
    if not os.path.exists(B.LIB):
        B.build()


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


def test_sweep_on_gpu_takes_the_oracle_decisions():
    cfg = sw.SweepConfig(N=4, n_alpha=2, n_beta=2, L=4, chi=4, M_max=3, sweeps=4, R=3, sigma=0.2)
    h1, eri = sw.hamiltonian(cfg)
    gpu = sw.LibraryBackend(h1, eri, cfg.N, cfg.n_alpha, cfg.n_beta, use_graphs=0)
    rg = sw.run_sweep(cfg, 7, gpu)
    ro = sw.run_sweep(cfg, 7, OracleBackend(h1, eri, cfg.N, cfg.n_alpha, cfg.n_beta))
    gpu.close()
    assert rg.accepted == ro.accepted and rg.M == ro.M
    assert np.abs(np.array(rg.energies) - np.array(ro.energies)).max() <= 1e-9


def test_learned_proposal_end_to_end():
    cfg = sw.SweepConfig(N=6, n_alpha=3, n_beta=3, L=12, chi=8, M_max=4, sweeps=6, R=4, sigma=0.1)
    h1, eri = sw.hamiltonian(cfg)
    e_exact = of.SectorHamiltonian(h1, eri, cfg.n_alpha, cfg.n_beta).ground_energy()
    res = sw.experiment(cfg, train_seeds=range(1, 7), eval_seeds=range(101, 104), epochs=150, log=lambda *a: None)
    assert res["samples"] > 20
    assert res["loss_last"] < 0.5 * res["loss_first"]          # the Adam kernels fit the records
    for row in res["rows"]:
        assert row["E_plain"] >= e_exact - 1e-9 and row["E_learned"] >= e_exact - 1e-9
        assert 1 <= row["sweeps_learned"] <= cfg.sweeps + 1
    # the paired comparison is reported, not gated (the run of one seed is chaotic; a small training
    # set shows no reliable gain): wins, ties and losses cover the seeds and the sign test is a p-value
    print({k: res[k] for k in ("wins", "ties", "losses", "sign_test_p", "mean_sweep_difference", "mean_dE_final")})
    assert res["wins"] + res["ties"] + res["losses"] == len(res["rows"])
    assert 0.0 < res["sign_test_p"] <= 1.0 and np.isfinite(res["mean_dE_final"])
