"""Pins of the conditioning oracle and host logic of the noise emulation (CPU)."""
import numpy as np

from oracle import conditioning as oc
from paper_2404_10223_gb300 import conditioning as cd


def test_residual_is_squared_distance_from_the_span():
    rng = np.random.default_rng(0)
    V = rng.normal(size=(9, 6))
    V[:, 4] = 0.3 * V[:, 0] - 2.0 * V[:, 2] + 1e-3 * rng.normal(size=9)   # nearly dependent
    S = V.T @ V
    r = oc.residuals(S)
    for j in range(6):
        if j == 0:
            d = V[:, 0] @ V[:, 0]
        else:
            coef, *_ = np.linalg.lstsq(V[:, :j], V[:, j], rcond=None)
            d = np.sum((V[:, j] - V[:, :j] @ coef) ** 2)
        # the Gram route loses cond(S_<j) digits against the vectors' own least squares
        cond = np.linalg.cond(S[:j, :j]) if j else 1.0
        assert abs(r[j] - d) <= 1e-15 * cond * np.abs(S).max() + 1e-13, (j, r[j], d, cond)
    assert r[4] < 1e-4 < r[3]


def test_residual_special_cases():
    assert np.allclose(oc.residuals(np.eye(5)), 1.0)
    S = np.ones((3, 3))                      # three copies of one normalised state
    assert np.allclose(oc.residuals(S), [1.0, 0.0, 0.0], atol=1e-14)


def test_shot_noise_keeps_symmetry_and_exact_norms():
    rng = np.random.default_rng(1)
    H = rng.normal(size=(5, 5))
    H = H + H.T
    S = np.eye(5) + 0.1 * np.ones((5, 5))
    np.fill_diagonal(S, 1.0)
    Hn, Sn = cd.shot_noise(H, S, rng, 1e-4, 1e-5)
    assert np.allclose(Hn, Hn.T) and np.allclose(Sn, Sn.T)
    assert np.all(np.diag(Sn) == 1.0)
    assert 1e-6 < np.abs(Hn - H).max() < 1e-3 and 1e-7 < np.abs(Sn - S).max() < 1e-4
