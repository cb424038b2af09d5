"""The allocation-free single-gate entry point against the allocating path.

tnqe_apply_gate_noalloc serves callers that cannot call cudaMalloc (programs
whose device memory is all handed out by their own pool reserved at start-up,
host loops that must not pay the latency and implicit synchronisation of
cudaMalloc / cudaFree): it keeps all of its working storage in one static
device array.  These tests call it through the C ABI and compare what
it produces with the ordinary tnqe_rotate path, on consecutive calls that
share that static array.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

from oracle import mps as om
from paper_2404_10223_gb300 import inputs
from paper_2404_10223_gb300 import tnqe

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    from paper_2404_10223_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    tnqe.load()


def codes(labels):
    return [a * 16 + b for a, b in labels]


def rot2(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, s], [-s, c]])


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def noalloc_gate(A, B, qL, qM, qR, c, s, side, chi_max, cutoff=1e-14):
    import torch
    chl, chm, chr_ = A.shape[0], A.shape[2], B.shape[2]
    dA, dB = dev(A), dev(B)
    Ao = torch.zeros(chl * 4 * chi_max, dtype=torch.float64, device="cuda")
    Bo = torch.zeros(chi_max * 4 * chr_, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    k, qo, disc = tnqe.tnqe_apply_gate_noalloc(dA.data_ptr(), dB.data_ptr(), chl, chm, chr_, qL, qM, qR, c, s, side,
                                               chi_max, cutoff, 60, Ao.data_ptr(), Bo.data_ptr(), 0)
    An = Ao[: chl * 4 * k].cpu().numpy().reshape(chl, 4, k)
    Bn = Bo[: k * 4 * chr_].cpu().numpy().reshape(k, 4, chr_)
    return An, Bn, k, qo, disc


def existing_rotation(h1, eri, N, na, nb, states, chi_rot):
    with tnqe.Context(h1, eri, N, na, nb, chi_rot=chi_rot) as g:
        for ts, U in states:
            g.add_mps(ts, U)
        disc = g.rotate(0, 1)
        return g.get_rotated(), disc


def single_gate_of(V):
    gates, m, neg = om.givens_plan(V)
    real = [(a, c, s, side) for a, c, s, side in gates if (c, s) != (1.0, 0.0)]
    assert len(real) == 1 and not neg
    return real[0]


def test_truncating_gate_matches_rotate_on_two_calls():
    """N = 2: the whole state is the two-site tensor, so truncation is gauge-free."""
    rng = np.random.default_rng(7)
    h1, eri = inputs.draw_integrals(rng, 2, 4)
    for call, theta in enumerate([0.7, -1.1]):
        ts, labels = inputs.draw_mps(rng, 2, 1, 1, 4)
        states = [(inputs.draw_mps(rng, 2, 1, 1, 4)[0], np.eye(2)), (ts, rot2(theta))]
        ref, disc_ref = existing_rotation(h1, eri, 2, 1, 1, states, chi_rot=2)
        a, c, s, side = single_gate_of(rot2(theta))
        An, Bn, k, qo, disc = noalloc_gate(ts[0], ts[1], codes(labels[0]), codes(labels[1]), codes(labels[2]),
                                           c, s, 0 if side == "L" else 1, chi_max=2)
        assert k == ref[0].shape[2], call
        assert np.all(np.diff(qo) >= 0)
        th_new = np.tensordot(An, Bn, axes=([2], [0]))
        th_ref = np.tensordot(ref[0], ref[1], axes=([2], [0]))
        assert np.abs(th_new - th_ref).max() <= TOL, call
        assert abs(disc - disc_ref) <= TOL, call


def test_lossless_gate_inside_chain_matches_rotate_on_two_calls():
    rng = np.random.default_rng(9)
    N, na, nb = 5, 3, 2
    h1, eri = inputs.draw_integrals(rng, N, 10)
    for call, (bond, theta) in enumerate([(1, 0.45), (2, -0.8)]):
        ts, labels = inputs.draw_mps(rng, N, na, nb, 8)
        V = np.eye(N)
        V[bond:bond + 2, bond:bond + 2] = rot2(theta)
        a, c, s, side = single_gate_of(V)
        assert a == bond
        ref, disc_ref = existing_rotation(h1, eri, N, na, nb, [(ts, np.eye(N)), (ts, V)], chi_rot=128)
        An, Bn, k, qo, disc = noalloc_gate(ts[a], ts[a + 1], codes(labels[a]), codes(labels[a + 1]),
                                           codes(labels[a + 2]), c, s, 0 if side == "L" else 1, chi_max=128)
        new = list(ts)
        new[a], new[a + 1] = An, Bn
        nn, rr, nr = om.overlap(new, new), om.overlap(ref, ref), om.overlap(new, ref)
        assert abs(nn - rr) <= TOL and abs(nr - rr) <= TOL, call
        assert disc <= 1e-20 and disc_ref <= 1e-20
        assert k == ref[a].shape[2], call


def test_rejects_oversized_bonds():
    with pytest.raises(tnqe.TnqeError) as e:
        tnqe.tnqe_apply_gate_noalloc(1, 1, 129, 2, 2, [0] * 129, [0, 0], [0, 0], 1.0, 0.0, 0, 2, 1e-14, 60, 1, 1)
    assert e.value.status == 1 and "128" in str(e.value)
