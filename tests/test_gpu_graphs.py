"""CUDA-graph capture and replay of whole matrix-element calls (GPU).

The first call for a (pair list, states, options) combination runs eagerly, the
second runs eagerly and captures its launch sequence, and identical later calls
replay the graph.  Replays
must reproduce the eager results bit for bit (the kernels are deterministic),
and any change of states or options must stop a stale graph from running.
"""
import numpy as np
import pytest

from paper_2404_10223_gb300 import inputs
from paper_2404_10223_gb300 import tnqe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2404_10223_gb300 import build as B
    import os
    if not os.path.exists(B.LIB):
        B.build()
    tnqe.load()


def ctx_for(w, **opts):
    g = tnqe.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff, **opts)
    for m in w.mps:
        g.add_mps(m.tensors, m.U)
    return g


@pytest.mark.parametrize("prec", [tnqe.TNQE_PREC_FP64, tnqe.TNQE_PREC_TF32X3, tnqe.TNQE_PREC_BF16X15])
def test_replay_equals_eager(prec):
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    with ctx_for(w, precision=prec, use_graphs=0) as e:
        He, Se = e.matrix_elements(pairs)
        assert e.graph_count() == 0
    with ctx_for(w, precision=prec, use_graphs=1) as g:
        H0, S0 = g.matrix_elements(pairs)          # eager
        assert g.graph_count() == 0
        H1, S1 = g.matrix_elements(pairs)          # eager + capture
        assert g.graph_count() == 1
        H2, S2 = g.matrix_elements(pairs)          # replay
        H3, S3 = g.matrix_elements(pairs)          # replay again
        prof = g.last_profile()
    for H, S in ((H0, S0), (H1, S1), (H2, S2), (H3, S3)):
        assert np.array_equal(H, He) and np.array_equal(S, Se)
    assert prof[9] > 0 and prof[0] > 0 and prof[1] > 0    # timings and launch count survive a replay


def test_graphs_follow_state_and_option_changes():
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    sub = pairs[:7]
    with ctx_for(w, use_graphs=1) as g:
        for _ in range(2):
            g.matrix_elements(pairs)
            g.matrix_elements(sub)
        assert g.graph_count() == 2                # one graph per pair list
        g.set_precision(tnqe.TNQE_PREC_BF16X15)
        Hb, _ = g.matrix_elements(sub)
        Hb1, _ = g.matrix_elements(sub)
        assert g.graph_count() == 3                # and per precision
        Hb2, _ = g.matrix_elements(sub)
        assert np.array_equal(Hb, Hb1) and np.array_equal(Hb, Hb2)
        # a new state drops every graph; the old pair list still gives the old values
        extra = inputs.workload("n10_chi32").mps[1]
        g.add_mps(extra.tensors, extra.U)
        assert g.graph_count() == 0
        Hc, _ = g.matrix_elements(sub)
        assert np.array_equal(Hc, Hb)
        g.clear_graphs()
        assert g.graph_count() == 0
        # reset + different states under the same ids: nothing stale may run
        g.reset_mps()
        w2 = inputs.make_workload(N=w.N, n_alpha=w.n_alpha, n_beta=w.n_beta, L=20, M=3, chi=[16, 16, 16], seed=11)
        for m in w2.mps:
            g.add_mps(m.tensors, m.U)
        p2 = w2.all_pairs()
        Hd, Sd = g.matrix_elements(p2)
        g.matrix_elements(p2)
        Hd2, Sd2 = g.matrix_elements(p2)
        assert g.graph_count() == 1
    with tnqe.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff, precision=tnqe.TNQE_PREC_BF16X15,
                      use_graphs=0) as e:
        for m in w2.mps:
            e.add_mps(m.tensors, m.U)
        He, Se = e.matrix_elements(p2)
    assert np.array_equal(Hd, He) and np.array_equal(Hd2, He) and np.array_equal(Sd2, Se)


def test_replay_with_device_outputs_and_own_stream():
    torch = pytest.importorskip("torch")
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    s = torch.cuda.Stream()
    Hd = torch.zeros(len(pairs), dtype=torch.float64, device="cuda")
    Sd = torch.zeros(len(pairs), dtype=torch.float64, device="cuda")
    with ctx_for(w, precision=tnqe.TNQE_PREC_BF16X15, use_graphs=1, cuda_stream=s.cuda_stream) as g:
        Hh, Sh = g.matrix_elements(pairs)
        for _ in range(4):
            Hd.zero_()
            torch.cuda.synchronize()
            g.matrix_elements(pairs, Hd.data_ptr(), Sd.data_ptr())
            torch.cuda.synchronize()
            assert np.array_equal(Hd.cpu().numpy(), Hh) and np.array_equal(Sd.cpu().numpy(), Sh)
        assert g.graph_count() == 1


def test_autotune_and_manual_shapes_give_identical_results():
    """Launch shapes change tiling only: each output keeps its summation order, so results are bit-identical."""
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    with ctx_for(w, precision=tnqe.TNQE_PREC_BF16X15) as g:
        H0, S0 = g.matrix_elements(pairs)
        cfg, times = g.autotune(pairs)
        assert cfg[0] in (64, 128) and cfg[1] in (64, 128) and cfg[2] in (2, 4, 8)
        assert np.all(times > 0)
        H1, S1 = g.matrix_elements(pairs)
        for shape in ((64, 64, 4), (64, 128, 1), (128, 64, 2)):
            g.set_tuning(*shape)
            H2, S2 = g.matrix_elements(pairs)
            assert np.array_equal(H2, H0) and np.array_equal(S2, S0), shape
        with pytest.raises(tnqe.TnqeError):
            g.set_tuning(96, 128, 8)
    assert np.array_equal(H1, H0) and np.array_equal(S1, S0)


def test_multi_wave_call_is_captured_and_replayed():
    """With a workspace limit that splits the pairs into several waves, the charge-block FP64 form runs
    the waves in stream order without host synchronisation: the call is captured, and eager, captured
    and replayed results equal the single-wave results bit for bit."""
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    with ctx_for(w, use_graphs=0) as e:
        He, Se = e.matrix_elements(pairs)
    # one pair's workspace at n10_chi32 is a few MB: 40 MB gives several waves
    with ctx_for(w, use_graphs=1, workspace_limit=40 << 20) as g:
        outs = [g.matrix_elements(pairs) for _ in range(4)]
        assert g.graph_count() == 1
        prof = g.last_profile()
    for H, S in outs:
        assert np.array_equal(H, He) and np.array_equal(S, Se)
    assert prof[1] > 0 and prof[2] > 0 and prof[3] > 0


def test_block_stage_cta_sizes_give_identical_results():
    """The charge-block stages' CTA size changes only the launch shape, never a summation order."""
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    res = []
    with ctx_for(w) as g:
        for t in (64, 128, 256):
            g.set_block_tuning(t, t, t)
            res.append(g.matrix_elements(pairs))
    for H, S in res[1:]:
        assert np.array_equal(H, res[0][0]) and np.array_equal(S, res[0][1])


def test_autotune_cache_file(tmp_path):
    """tnqe_autotune times the candidates once per pair-list class and stores the choice; a new context
    with the same cache file takes the stored shapes without timing."""
    w = inputs.workload("n10_chi32")
    pairs = w.all_pairs()
    path = str(tmp_path / "tune.txt")
    with ctx_for(w, autotune_cache=path) as g:
        cfg1, times1 = g.autotune(pairs)
        H1, S1 = g.matrix_elements(pairs)
    assert all(c in (64, 128, 256) for c in cfg1) and times1.max() > 0
    lines = open(path).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith("tnqe-tune N=10 prec=0 form=0 ")
    with ctx_for(w, autotune_cache=path) as g:
        cfg2, times2 = g.autotune(pairs)
        H2, S2 = g.matrix_elements(pairs)
    assert cfg2 == cfg1 and times2.max() == 0.0
    assert len(open(path).read().splitlines()) == 1
    assert np.array_equal(H1, H2) and np.array_equal(S1, S2)
    # another class (a different pair list) is tuned and appended
    with ctx_for(w, autotune_cache=path) as g:
        g.autotune(pairs[:5])
    assert len(open(path).read().splitlines()) == 2
