"""Write the algorithmic work of the rotations of a workload, counted from the oracle.

The roofline of the rotation kernel divides this work by the kernel's time.
It is counted here from the charge-block shapes the oracle's truncated
rotation goes through (Sec. II D, Eq. A5; the particle-number blocks of
Sec. IV A), with the same definition the kernel uses, so that the number the
benchmark reports can be reproduced without the GPU:

* per gate on sites (a, a+1), the two-site tensor in charge blocks:
  2 dL dM dR for every (left sector, k1, k2) whose middle and right sectors
  exist (dL, dM, dR the sector dimensions of bonds a, a+1, a+2);
* per charge block of the new middle bond (rows (l, k1), columns (k2, r) of
  that charge; m x n with m >= n): 8 m n (the gate) + 4 m n^2 + 8 n^3 (the
  operation count of a LAPACK-style SVD).

The oracle runs a dense SVD of the whole two-site matrix; the charge of each
kept singular vector is the charge of the row holding its largest entry
(each singular vector of a block-diagonal matrix lies in one block).  That
gives the sector dimensions of the new bond, gate by gate.

    python tests/golden/make_rotation_work.py [workload]     # default n14_chi128

Output: ``<workload>_rotation_work.json`` next to this script: per rotated
pair (i, j) of the workload (the rotation of state j into basis i) the work
in FLOPs, and their sum (one step of the benchmark rotates every pair i < j).
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
from collections import Counter

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

LQ = ((0, 0), (1, 0), (0, 1), (1, 1))        # local state k -> (n_alpha, n_beta)


def _add(q, d, sign=1):
    return (q[0] + sign * d[0], q[1] + sign * d[1])


def rotation_work(tensors, charges, V, chi_rot, cutoff):
    """FLOPs of one truncated rotation, counted from the oracle's block shapes."""
    from oracle import mps as om
    trace = []
    om.apply_rotation(tensors, V, chi_rot, cutoff, trace=trace)
    gates, _m, _neg = om.givens_plan(V)
    labels = [list(b) for b in charges]
    flops = 0
    for (a, _c, _s, _side), (_k, _sig, rows) in zip(gates, trace):
        L, M, R = labels[a], labels[a + 1], labels[a + 2]
        cL, cM, cR = Counter(L), Counter(M), Counter(R)
        for qL, dL in cL.items():
            for k1 in range(4):
                qM = _add(qL, LQ[k1])
                if qM not in cM:
                    continue
                for k2 in range(4):
                    qR = _add(qM, LQ[k2])
                    if qR in cR:
                        flops += 2 * dL * cM[qM] * cR[qR]
        rowq = [_add(L[l], LQ[x]) for l in range(len(L)) for x in range(4)]
        colq = [_add(R[r], LQ[y], -1) for y in range(4) for r in range(len(R))]
        nr, nc = Counter(rowq), Counter(colq)
        for q in nr:
            if q in nc:
                m, n = max(nr[q], nc[q]), min(nr[q], nc[q])
                flops += 4 * m * n * n + 8 * n ** 3 + 8 * m * n
        labels[a + 1] = [rowq[r] for r in rows]
    return flops


def _work(args):
    name, pairs = args
    sys.path.insert(0, ROOT)
    from paper_2404_10223_gb300 import inputs
    w = inputs.workload(name)
    out = []
    for i, j in pairs:
        m = w.mps[j]
        chi_rot = max(t.shape[2] for t in m.tensors[:-1]) if w.N > 1 else 1
        V = w.mps[i].U.T @ m.U
        f = rotation_work(m.tensors, m.charges, V, chi_rot, w.cutoff)
        print(f"{name} ({i},{j}) {f:.6e} FLOPs", flush=True)
        out.append((i, j, f))
    return out


def main(name, nproc):
    sys.path.insert(0, ROOT)
    from paper_2404_10223_gb300 import inputs
    w = inputs.workload(name)
    pairs = [(i, j) for i, j in w.all_pairs() if i != j]
    chunks = [pairs[k::nproc * 2] for k in range(nproc * 2)]
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.map(_work, [(name, c) for c in chunks if c], chunksize=1)
    got = {(i, j): f for part in res for i, j, f in part}
    rec = {"workload": name, "definition": "2 dL dM dR per two-site block + 8mn + 4mn^2 + 8n^3 per SVD block",
           "pairs": [[i, j] for i, j in pairs], "flops": [got[p] for p in pairs],
           "total": sum(got[p] for p in pairs)}
    path = os.path.join(HERE, f"{name}_rotation_work.json")
    with open(path, "w") as f:
        json.dump(rec, f)
    print("wrote", path, rec["total"])


if __name__ == "__main__":
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "2")
    main(sys.argv[1] if len(sys.argv) > 1 else "n14_chi128", int(os.environ.get("GOLDEN_PROCS", "4")))
