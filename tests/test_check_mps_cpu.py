"""The host checks tnqe_add_mps makes on a state (tnqe_check_mps), on the CPU:
valid workload states pass; each rejection reason is reported with its message."""
import numpy as np
import pytest

from paper_2404_10223_gb300 import build, inputs, tnqe

pytestmark = pytest.mark.skipif(not __import__("os").path.exists(build.LIB), reason="library not built")


@pytest.mark.parametrize("name", ["n6_chi8", "n10_chi32", "n14_mixed"])
def test_workload_states_are_valid(name):
    w = inputs.workload(name)
    for m in w.mps:
        assert tnqe.tnqe_check_mps(m.tensors, m.U, w.n_alpha, w.n_beta) == (0, "")


def _state():
    w = inputs.workload("n6_chi8")
    m = w.mps[1]
    return w, [t.copy() for t in m.tensors], m.U.copy()


def test_non_orthogonal_basis():
    w, ts, U = _state()
    U[0, 0] += 1e-6
    st, msg = tnqe.tnqe_check_mps(ts, U, w.n_alpha, w.n_beta)
    assert st == 1 and "orthogonal" in msg


def test_entry_outside_the_charge_blocks():
    w, ts, U = _state()
    A = ts[2]
    l, k, r = [int(x[0]) for x in np.nonzero(A == 0.0)]     # a structural zero
    A[l, k, r] = 0.3
    st, msg = tnqe.tnqe_check_mps(ts, U, w.n_alpha, w.n_beta)
    assert st == 1 and "block structure" in msg


def test_bond_index_without_weight():
    w, ts, U = _state()
    ts[3][:, :, 0] = 0.0
    st, msg = tnqe.tnqe_check_mps(ts, U, w.n_alpha, w.n_beta)
    assert st == 1 and "no weight" in msg


def test_site_not_left_orthonormal():
    w, ts, U = _state()
    ts[1] *= 1.5
    st, msg = tnqe.tnqe_check_mps(ts, U, w.n_alpha, w.n_beta)
    assert st == 1 and "left-orthonormal" in msg


def test_wrong_particle_sector():
    w, ts, U = _state()
    st, msg = tnqe.tnqe_check_mps(ts, U, w.n_alpha - 1, w.n_beta)
    assert st == 1 and "sector" in msg


def test_bond_dimensions_at_the_ends():
    w, ts, U = _state()
    ts[0] = np.concatenate([ts[0], ts[0]], axis=0)            # left bond of dimension 2
    st, msg = tnqe.tnqe_check_mps(ts, U, w.n_alpha, w.n_beta)
    assert st == 1 and "must be 1" in msg


def test_bad_electron_numbers():
    w, ts, U = _state()
    assert tnqe.tnqe_check_mps(ts, U, 7, 0)[0] == 1


def test_errors_are_reported_in_site_order():
    """A block-structure violation at an early site is reported before a column
    without weight at a later site and before a non-orthonormal site, and the
    site number in the message is the earliest offending one."""
    w, ts, U = _state()
    A = ts[1]
    l, k, r = [int(x[0]) for x in np.nonzero(A == 0.0)]
    A[l, k, r] = 0.3                                          # site 1: outside the blocks
    ts[3][:, :, 0] = 0.0                                      # site 3: a bond index with no weight
    ts[4] *= 1.5                                              # site 4: not left-orthonormal
    st, msg = tnqe.tnqe_check_mps(ts, U, w.n_alpha, w.n_beta)
    assert st == 1 and "block structure" in msg and "site 1" in msg
    w, ts, U = _state()
    ts[2][:, :, 0] = 0.0                                      # site 2: no weight
    ts[1] *= 1.5                                              # site 1: not left-orthonormal (checked later)
    st, msg = tnqe.tnqe_check_mps(ts, U, w.n_alpha, w.n_beta)
    assert st == 1 and "no weight" in msg and "site 2" in msg


def test_states_of_the_benchmark_workload_are_valid():
    """The N = 14, chi = 128 states pass (the sites are checked on host threads)."""
    w = inputs.workload("n14_chi128")
    for m in w.mps[:4]:
        assert tnqe.tnqe_check_mps(m.tensors, m.U, w.n_alpha, w.n_beta) == (0, "")
