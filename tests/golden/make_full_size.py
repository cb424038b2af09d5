"""Write the oracle's values for the full-size workloads (expected values of the GPU parity tests).

Calls only ``oracle/`` (the CPU FP64 MPS path) and the seeded input
generator; nothing here touches the CUDA library.  Run once on a CPU host:

    python tests/golden/make_full_size.py n14        # all 136 pairs of n14_chi128 (about an hour on 8 cores)
    python tests/golden/make_full_size.py n20        # two rotated pairs of n20_mixed (chi 128 and 256)

Output (next to this script):

* ``n14_chi128_oracle.npz``: for every pair (i, j), i <= j, of the N = 14,
  7+7 electron, M = 16, chi = 128 workload: ``pairs``, ``H``, ``S``,
  ``discarded`` (sum of the discarded sigma^2 of the rotation of state j into
  basis i, Sec. II D / Eq. A5), ``gap`` (the smallest relative gap
  (sigma_k - sigma_{k+1}) / sigma_1 over the gates whose cut is set by chi
  rather than by the cutoff; +inf if no gate truncates at chi) and
  ``margin`` (the smallest relative distance (|sigma_l - cutoff sigma_1|) /
  sigma_1 of a singular value from the cutoff threshold), and the solve of
  the assembled pencil (canonical orthogonalisation, Sec. IV C): ``E``,
  ``rank``.
* ``n20_mixed_oracle.npz``: the same per-pair fields for the pairs listed in
  ``N20_PAIRS`` of the N = 20, 10+10 electron, M = 24, chi in {128, 256},
  cutoff 1e-10 workload.

Pairs are spread over worker processes (started with ``spawn``), two BLAS
threads each; a worker builds the MPO of a basis once for all pairs with
that bra.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

# rotated pairs of n20_mixed: (bra, ket) with chi_bra = chi_ket = 128, and both 256
N20_PAIRS = None  # filled from the workload's chi draw by n20_pairs()


def _cut_stats(trace, chi_rot, cutoff):
    gap, margin = np.inf, np.inf
    for k, sig, _rows in trace:
        if sig.size == 0 or sig[0] == 0.0:
            continue
        thr = cutoff * sig[0]
        above = sig[sig > thr]
        if above.size > 0:
            margin = min(margin, float(np.min(above - thr) / sig[0]))
        below = sig[sig <= thr]
        if below.size > 0:
            margin = min(margin, float(np.min(thr - below) / sig[0]))
        if k == chi_rot and sig.size > k and sig[k] > thr:
            gap = min(gap, float((sig[k - 1] - sig[k]) / sig[0]))
    return gap, margin


def _work(args):
    name, group = args
    sys.path.insert(0, ROOT)
    from oracle import mps as om
    from paper_2404_10223_gb300 import inputs
    w = inputs.workload(name)
    o = om.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff)
    for m in w.mps:
        o.add_mps(m.tensors, m.U)
    out = []
    for i, j in group:
        t0 = time.time()
        trace = []
        ket, disc = o.rotate(i, j, trace)
        H, S = om.contract(o.states[i], o.mpo(i), ket)
        chi_rot = o.chi_of(j)
        gap, margin = _cut_stats(trace, chi_rot, w.cutoff)
        out.append((i, j, H, S, disc, gap, margin))
        print(f"{name} ({i},{j}) H={H:.12e} S={S:.6e} disc={disc:.3e} gap={gap:.2e} "
              f"margin={margin:.2e} {time.time() - t0:.1f}s", flush=True)
    return out


def _groups(pairs, nproc):
    """Pairs grouped by bra (one MPO per group), groups spread longest first."""
    by_bra = {}
    for i, j in pairs:
        by_bra.setdefault(i, []).append((i, j))
    groups = sorted(by_bra.values(), key=len, reverse=True)
    # split the bigger groups so that every worker gets a share
    target = max(1, (len(pairs) + 2 * nproc - 1) // (2 * nproc))
    out = []
    for g in groups:
        for k in range(0, len(g), target):
            out.append(g[k:k + target])
    return sorted(out, key=len, reverse=True)


def run(name, pairs, path, nproc):
    sys.path.insert(0, ROOT)
    from oracle import mps as om
    from paper_2404_10223_gb300 import inputs
    w = inputs.workload(name)
    ctx = mp.get_context("spawn")
    with ctx.Pool(nproc) as pool:
        res = pool.map(_work, [(name, g) for g in _groups(pairs, nproc)], chunksize=1)
    rows = {(r[0], r[1]): r for part in res for r in part}
    rows = [rows[p] for p in pairs]
    arr = {
        "pairs": np.array(pairs, dtype=np.int64),
        "H": np.array([r[2] for r in rows]),
        "S": np.array([r[3] for r in rows]),
        "discarded": np.array([r[4] for r in rows]),
        "gap": np.array([r[5] for r in rows]),
        "margin": np.array([r[6] for r in rows]),
    }
    if len(pairs) == w.M * (w.M + 1) // 2:
        H = np.zeros((w.M, w.M))
        S = np.zeros((w.M, w.M))
        for (i, j), h, s in zip(pairs, arr["H"], arr["S"]):
            H[i, j] = H[j, i] = h
            S[i, j] = S[j, i] = s
        E, C, rank, kappa = om.solve(H, S)
        arr["E"] = E
        arr["rank"] = np.array(rank)
        arr["kappa1"] = np.array(kappa)
    np.savez(path, **arr)
    print("wrote", path)


def n20_pairs():
    sys.path.insert(0, ROOT)
    from paper_2404_10223_gb300 import inputs
    w = inputs.workload("n20_mixed")
    chis = [m.chi for m in w.mps]
    c128 = [k for k in range(w.M) if chis[k] == 128]
    c256 = [k for k in range(w.M) if chis[k] == 256]
    return [(c128[0], c128[1]), (c256[0], c256[1])]


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "n14"
    nproc = int(os.environ.get("GOLDEN_PROCS", "4"))
    os.environ.setdefault("OPENBLAS_NUM_THREADS", os.environ.get("GOLDEN_THREADS", "2"))
    os.environ.setdefault("OMP_NUM_THREADS", os.environ["OPENBLAS_NUM_THREADS"])
    if which == "n14":
        sys.path.insert(0, ROOT)
        from paper_2404_10223_gb300 import inputs
        w = inputs.workload("n14_chi128")
        run("n14_chi128", w.all_pairs(), os.path.join(HERE, "n14_chi128_oracle.npz"), nproc)
    elif which == "n20":
        run("n20_mixed", n20_pairs(), os.path.join(HERE, "n20_mixed_oracle.npz"), min(nproc, 2))
    else:
        raise SystemExit(f"unknown set {which!r}: n14 or n20")
