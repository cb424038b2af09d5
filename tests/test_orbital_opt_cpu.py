"""Host logic of the bond co-optimisation (CPU): golden-section search and the basis update."""
import math

import numpy as np

from paper_2404_10223_gb300 import orbital_opt as oo


def test_golden_section_finds_minima():
    x, fx, n = oo.golden_section(lambda t: (t - 0.3) ** 2 + 1.0, -1.0, 2.0, tol=1e-9)
    assert abs(x - 0.3) < 1e-7 and abs(fx - 1.0) < 1e-12 and n < 80
    x, fx, _ = oo.golden_section(math.cos, 0.0, 2 * math.pi, tol=1e-9)
    assert abs(x - math.pi) < 1e-6


def test_embed_is_orthogonal_and_local():
    J = np.array([[math.cos(0.4), -math.sin(0.4)], [math.sin(0.4), math.cos(0.4)]])
    R = oo.embed(J, 6, 2)
    assert np.allclose(R @ R.T, np.eye(6))
    assert np.allclose(R[2:4, 2:4], J) and np.allclose(np.delete(np.delete(R, [2, 3], 0), [2, 3], 1), np.eye(4))
