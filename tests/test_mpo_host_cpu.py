"""The library's host-built Hamiltonian MPO (Eq. 1 in second quantisation,
Sec. II A) against the oracle, on the CPU: the dense operator at N <= 4 equals
the Jordan-Wigner Hamiltonian, transfer contractions at N = 10 equal the
oracle MPO's, integrals without the (pq|rs) = (rs|pq) symmetry still give the
Jordan-Wigner operator, and repeated builds are bitwise identical."""
import numpy as np
import pytest
import scipy.sparse

from oracle import fock as of
from oracle import mps as om
from paper_2404_10223_gb300 import build, inputs, tnqe

pytestmark = pytest.mark.skipif(not __import__("os").path.exists(build.LIB),
                                reason="library not built")


def lib_mpo(h1, eri, N):
    """The library's MPO as an oracle MPO object (rows k * D' + w' -> w' * 4 + k)."""
    dims, sites = tnqe.tnqe_mpo_host(h1, eri, N)
    W = []
    for t, (rp, col, val) in enumerate(sites):
        dout, din = dims[t + 1], dims[t]
        A = scipy.sparse.csr_matrix((val, col, rp), shape=(4 * dout, 4 * din)).tocoo()
        r = A.row
        W.append(scipy.sparse.csr_matrix((A.data, ((r % dout) * 4 + r // dout, A.col)), shape=A.shape))
    return om.MPO(W, dims)


def interleave_perm(N):
    """Permutation from site order (k = n_alpha + 2 n_beta per site) to the JW bit order."""
    P = np.zeros((4 ** N, 4 ** N))
    for kidx in range(4 ** N):
        bits = 0
        for k in np.unravel_index(kidx, (4,) * N):
            bits = (bits << 2) | ((k & 1) << 1) | ((k >> 1) & 1)
        P[bits, kidx] = 1.0
    return P


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_library_mpo_equals_jordan_wigner_hamiltonian(N):
    h1, eri = inputs.draw_integrals(np.random.default_rng(40 + N), N, 2 * N)
    m = lib_mpo(h1, eri, N)
    assert m.dims[0] == 1 and m.dims[N] == 2
    P = interleave_perm(N)
    Hjw = of.jw_hamiltonian(h1, eri)
    assert np.abs(P @ om.mpo_dense(m) @ P.T - Hjw).max() <= 1e-12 * max(1.0, np.abs(Hjw).max())


def test_integrals_without_pair_symmetry():
    """The builder adds (pq|rs) and (rs|pq) as one operator string with the summed coefficient."""
    N = 3
    rng = np.random.default_rng(7)
    h1, _ = inputs.draw_integrals(rng, N, 2 * N)
    eri = rng.normal(size=(N, N, N, N))             # no symmetry at all
    P = interleave_perm(N)
    Hjw = of.jw_hamiltonian(h1, eri)
    assert np.abs(P @ om.mpo_dense(lib_mpo(h1, eri, N)) @ P.T - Hjw).max() <= 1e-12 * np.abs(Hjw).max()


def test_transfer_contractions_equal_the_oracle_mpo_n10():
    w = inputs.workload("n10_chi32")
    ml = lib_mpo(w.h1, w.eri, w.N)
    mo = om.build_mpo(w.h1, w.eri)
    for i, j in [(0, 0), (0, 1), (2, 4)]:
        Hl, Sl = om.contract(w.mps[i].tensors, ml, w.mps[j].tensors)
        Ho, So = om.contract(w.mps[i].tensors, mo, w.mps[j].tensors)
        assert abs(Hl - Ho) <= 1e-10 * max(1.0, abs(Ho)) and abs(Sl - So) <= 1e-12


def test_builds_are_bitwise_identical():
    h1, eri = inputs.draw_integrals(np.random.default_rng(3), 8, 16)
    d1, s1 = tnqe.tnqe_mpo_host(h1, eri, 8)
    d2, s2 = tnqe.tnqe_mpo_host(h1, eri, 8)
    assert d1 == d2
    for a, b in zip(s1, s2):
        for x, y in zip(a, b):
            assert x.tobytes() == y.tobytes()


def test_rejects_bad_arguments():
    with pytest.raises(tnqe.TnqeError):
        tnqe.tnqe_mpo_host(np.zeros((1, 1)), np.zeros((1, 1, 1, 1)), 0)
