"""Bond orbital co-optimisation on the GPU (Sec. II D): xi(theta) against the
oracle's gate + SVD, recovery of a planted rotation and of a planted FSWAP with
the physical state unchanged, and a whole right-to-left pass."""
import math

import numpy as np
import pytest

from oracle import fock as of
from oracle import mps as om
from paper_2404_10223_gb300 import inputs
from paper_2404_10223_gb300 import orbital_opt as oo

pytestmark = pytest.mark.gpu
N, NA, NB, CHI = 6, 3, 3, 8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2404_10223_gb300 import build as B
    import os
    if not os.path.exists(B.LIB):
        B.build()


def codes(labels):
    return [a * 16 + b for a, b in labels]


def oracle_xi(A, B, theta, chi):
    t = np.tensordot(A, B, axes=([2], [0]))
    G = om.gate16(math.cos(theta), math.sin(theta)).reshape(4, 4, 4, 4)
    t = np.einsum("xyab,labr->lxyr", G, t)
    sig = np.linalg.svd(t.reshape(A.shape[0] * 4, 4 * B.shape[2]), compute_uv=False)
    return float(np.sum(sig[chi:] ** 2) / np.sum(sig ** 2))


def state(ts, U):
    return of.rotate_sector(of.mps_to_sector(ts, NA, NB), U, NA, NB)


def planted(theta_star, seed):
    """A state whose bond (2, 3) carries a rotation that raises its Schmidt rank above CHI.

    The centre is moved to site 3 by lossless zero-angle steps, then the gate at
    angle theta_star is applied without truncation; returns tensors, charges."""
    rng = np.random.default_rng(seed)
    ts, labels = inputs.draw_mps(rng, N, NA, NB, CHI)
    ts = [t.copy() for t in ts]
    qs = [codes(l) for l in labels]
    for p, th in ((4, 0.0), (3, 0.0), (2, theta_star)):
        opt = oo.BondOptimizer(ts[p], ts[p + 1], qs[p], qs[p + 1], qs[p + 2], 64)
        xi, An, Bn, q = opt.apply(th)
        assert xi < 1e-13
        ts[p], ts[p + 1] = An, Bn
        qs[p + 1] = [int(x) for x in q]
    return ts, qs


def test_xi_matches_oracle():
    ts, qs = planted(0.6, 1)
    opt = oo.BondOptimizer(ts[2], ts[3], qs[2], qs[3], qs[4], CHI)
    for th in (-1.2, -0.6, 0.0, 0.3, 1.5):
        assert abs(opt.xi(th) - oracle_xi(ts[2], ts[3], th, CHI)) <= 1e-10


@pytest.mark.parametrize("theta_star", [0.6, -0.35, math.pi / 2])
def test_planted_rotation_is_undone_and_the_state_kept(theta_star):
    ts, qs = planted(theta_star, 2)
    U0 = np.eye(N)
    before = state(ts, U0)
    r = oo.optimize_bond(ts[2], ts[3], qs[2], qs[3], qs[4], CHI, U0, 2)
    assert r.xi0 > 1e-4                       # the planted rotation does cost truncation at CHI
    assert r.xi < 1e-12 and r.A.shape[2] <= CHI
    # the state is unchanged: G(U_new) |MPS_new> = G(U0) |MPS>
    new = list(ts)
    new[2], new[3] = r.A, r.B
    after = state(new, r.U)
    assert abs(np.vdot(before, after) / (np.linalg.norm(before) * np.linalg.norm(after)) - 1.0) < 1e-10
    assert abs(np.linalg.norm(after) - np.linalg.norm(before)) < 1e-10
    # the angle found undoes the planted one (mod pi: theta and theta + pi differ by a parity sign)
    d = (r.theta + theta_star) % math.pi
    assert min(d, math.pi - d) < 1e-4


def test_right_to_left_pass_never_raises_xi():
    rng = np.random.default_rng(5)
    ts, labels = inputs.draw_mps(rng, N, NA, NB, CHI)
    new, qs, U, recs = oo.optimize_mps_bonds(ts, [codes(l) for l in labels], np.eye(N), CHI)
    assert len(recs) == N - 1
    for r in recs:
        assert r.xi <= r.xi0 + 1e-15
    a, b = state(ts, np.eye(N)), state(new, U)
    assert abs(abs(np.vdot(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b)) - 1.0) < 1e-10
