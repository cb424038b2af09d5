"""The library's host steps of the path on the CPU, against the oracle:
a1, the nearest-neighbour Givens plan of a relative rotation V = U_i^T U_j
(Eq. 11, App. A3; rebuilds V, signed permutations give angles 0 and pi/2) and
the 16 x 16 two-site gate of each rotation, and a2, the integrals in a state's
basis (h' = U^T h U and the four-index transform of (pq|rs))."""
import math
import numpy as np
import pytest
import scipy.linalg

from oracle import mps as om
from paper_2404_10223_gb300 import build, inputs, tnqe

pytestmark = pytest.mark.skipif(not __import__("os").path.exists(build.LIB), reason="library not built")


def rand_orth(rng, N, det=1):
    K = rng.normal(size=(N, N))
    U = scipy.linalg.expm(0.7 * (K - K.T))
    if det < 0:
        U[:, -1] *= -1.0
    return U


def as_oracle(gates):
    return [(a, c, s, "L" if side == 0 else "R") for a, c, s, side in gates]


@pytest.mark.parametrize("N", [2, 6, 10, 14, 20])
@pytest.mark.parametrize("det", [1, -1])
def test_givens_plan_equals_the_oracle_plan(N, det):
    V = rand_orth(np.random.default_rng(100 + N), N, det)
    gl, neg_site = tnqe.tnqe_givens_host(V)
    go, m, neg = om.givens_plan(V)
    assert len(gl) == len(go) == N * (N - 1) // 2
    for (a, c, s, side), (ao, co, so, sido) in zip(as_oracle(gl), go):
        assert a == ao and side == sido
        assert abs(c - co) <= 1e-13 and abs(s - so) <= 1e-13
    assert neg_site == (m if neg else -1)
    assert (neg_site >= 0) == (det < 0)
    assert np.abs(om.plan_matrix(as_oracle(gl), m, neg_site >= 0, N) - V).max() <= 1e-13


def test_signed_permutation_gives_right_angles():
    rng = np.random.default_rng(9)
    N = 8
    V = np.eye(N)[rng.permutation(N)] * rng.choice([-1.0, 1.0], size=N)[:, None]
    gl, neg_site = tnqe.tnqe_givens_host(V)
    for _, c, s, _ in gl:
        assert (abs(c), abs(s)) in ((1.0, 0.0), (0.0, 1.0))
    go, m, neg = om.givens_plan(V)
    assert np.abs(om.plan_matrix(as_oracle(gl), m, neg_site >= 0, N) - V).max() == 0.0


def test_identity_rotation_has_identity_gates():
    gl, neg_site = tnqe.tnqe_givens_host(np.eye(7))
    assert neg_site == -1 and all((c, s) == (1.0, 0.0) for _, c, s, _ in gl)


def test_integrals_in_a_basis_equal_the_oracle():
    rng = np.random.default_rng(5)
    N = 8
    h1, eri = inputs.draw_integrals(rng, N, 2 * N)
    U = rand_orth(rng, N)
    hl, gl = tnqe.tnqe_rotate_integrals_host(h1, eri, U)
    ho, go = om.rotate_integrals(h1, eri, U)
    assert np.abs(hl - ho).max() <= 1e-13 * np.abs(ho).max()
    assert np.abs(gl - go).max() <= 1e-13 * np.abs(go).max()
    hb, gb = tnqe.tnqe_rotate_integrals_host(hl, gl, U.T)        # and back
    assert np.abs(hb - h1).max() <= 1e-12 * np.abs(h1).max()
    assert np.abs(gb - eri).max() <= 1e-12 * np.abs(eri).max()


@pytest.mark.parametrize("theta", [0.0, 0.37, -1.2, math.pi / 4, math.pi / 2, 2.9])
def test_two_site_gate_equals_the_oracle_gate(theta):
    """The oracle's gate is pinned to the paper's g_4 form (test_oracle_pins)."""
    G = tnqe.tnqe_gate_host(math.cos(theta), math.sin(theta))
    assert np.abs(G - om.gate16(math.cos(theta), math.sin(theta))).max() <= 1e-14
    assert np.abs(G @ G.T - np.eye(16)).max() <= 1e-14


def test_gate_rejects_non_rotation():
    with pytest.raises(tnqe.TnqeError):
        tnqe.tnqe_gate_host(1.0, 0.5)
