"""Local pairwise orbital co-optimisation at one bond of an MPS (Sec. II D).

Before a two-site tensor is split and truncated back to chi, a rotation of the
two orbitals p, p+1 can lower the truncation error without changing the state:
insert g(-theta) g(theta) = 1, let g(theta) act on the two-site tensor, and
merge g(-theta) into the state's orbital basis.  The paper picks
theta_opt = argmin xi(theta), xi = 1 - sum_{l <= chi} sigma_l^2 (the discarded
weight of the normalised two-site tensor), by a classical univariate search,
and in its permutation-only variant accepts an FSWAP (the theta = pi/2 Givens
gate up to a phase) when it lowers xi.

Each evaluation of xi(theta) is one call of tnqe_apply_gate_noalloc (the
library's gate + blocked Jacobi SVD + truncation on the GPU); the search is a
golden-section search (the paper names no optimiser) inside the best bracket
of a coarse scan of [-pi/2, pi/2], plus the two endpoints, which are the
FSWAP-like angles.
The rotation is kept only if it lowers xi.

Conventions (include/tnqe.h): the gate entry point applies G(J^T) with
J = [[c, -s], [s, c]] on orbitals (p, p+1), c = cos theta, s = sin theta.  For
psi = G(U) |MPS> and MPS' = G(J^T) |MPS>, psi = G(U J) |MPS'>, so the basis
becomes U J (J embedded at rows and columns p, p+1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Sequence, Tuple

import numpy as np

from . import tnqe

GOLDEN = (math.sqrt(5.0) - 1.0) / 2.0
GRID = 8            # coarse scan of [-pi/2, pi/2] before the golden-section refinement


def golden_section(f: Callable[[float], float], a: float, b: float, tol: float = 1e-7,
                   max_iter: int = 100) -> Tuple[float, float, int]:
    """Minimum of a unimodal f on [a, b] by golden-section search: (x, f(x), evaluations)."""
    c = b - GOLDEN * (b - a)
    d = a + GOLDEN * (b - a)
    fc, fd = f(c), f(d)
    n = 2
    while abs(b - a) > tol and n < max_iter:
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - GOLDEN * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + GOLDEN * (b - a)
            fd = f(d)
        n += 1
    return (c, fc, n) if fc < fd else (d, fd, n)


def embed(J: np.ndarray, N: int, p: int) -> np.ndarray:
    R = np.eye(N)
    R[p:p + 2, p:p + 2] = J
    return R


@dataclasses.dataclass
class BondResult:
    theta: float               # applied angle (0 if nothing improved)
    xi: float                  # truncation error after the step
    xi0: float                 # truncation error without rotation
    A: np.ndarray              # new site tensors [chi_l][4][k], [k][4][chi_r]
    B: np.ndarray
    q_mid: np.ndarray          # charges of the new bond (ascending)
    U: np.ndarray              # the state's new orbital basis
    evaluations: int


class BondOptimizer:
    """xi(theta) of one bond on the GPU through the allocation-free gate entry point.

    A [chi_l][4][chi_m] and B [chi_m][4][chi_r] hold the two-site tensor with the
    canonical centre on it; q_l, q_m, q_r are the bond charges (n_alpha * 16 + n_beta,
    ascending).  Device buffers come from PyTorch (memory only)."""

    def __init__(self, A, B, q_l, q_m, q_r, chi: int, cutoff: float = 0.0, max_sweeps: int = 60):
        import torch
        self.torch = torch
        self.A = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float64)).cuda()
        self.B = torch.from_numpy(np.ascontiguousarray(B, dtype=np.float64)).cuda()
        self.shape = (A.shape[0], A.shape[2], B.shape[2])
        self.q = (list(q_l), list(q_m), list(q_r))
        self.chi, self.cutoff, self.max_sweeps = chi, cutoff, max_sweeps
        chl, _, chr_ = self.shape
        self.Ao = torch.zeros(chl * 4 * chi, dtype=torch.float64, device="cuda")
        self.Bo = torch.zeros(chi * 4 * chr_, dtype=torch.float64, device="cuda")

    def apply(self, theta: float):
        """(xi, A_new, B_new, q_new) for the gate at angle theta; singular values go to A_new."""
        chl, chm, chr_ = self.shape
        self.torch.cuda.synchronize()
        k, q_new, disc = tnqe.tnqe_apply_gate_noalloc(
            self.A.data_ptr(), self.B.data_ptr(), chl, chm, chr_, *self.q, math.cos(theta), math.sin(theta), 0,
            self.chi, self.cutoff, self.max_sweeps, self.Ao.data_ptr(), self.Bo.data_ptr(), 0)
        An = self.Ao[: chl * 4 * k].cpu().numpy().reshape(chl, 4, k)
        Bn = self.Bo[: k * 4 * chr_].cpu().numpy().reshape(k, 4, chr_)
        kept = float(np.sum(An * An))           # B_new is right-orthonormal: |A_new|^2 = kept weight
        total = kept + disc
        return (disc / total if total > 0 else 0.0), An, Bn, q_new

    def xi(self, theta: float) -> float:
        return self.apply(theta)[0]


def optimize_bond(A, B, q_l, q_m, q_r, chi: int, U: np.ndarray, p: int, tol: float = 1e-8,
                  fswap: bool = True) -> BondResult:
    """theta_opt = argmin xi(theta) over [-pi/2, pi/2] at bond (p, p+1), kept only if it lowers xi."""
    opt = BondOptimizer(A, B, q_l, q_m, q_r, chi)
    xi0 = opt.xi(0.0)
    # xi(theta) need not be unimodal on the whole interval: a coarse scan picks the
    # bracket, golden-section search refines inside it
    grid = [-math.pi / 2 + k * math.pi / GRID for k in range(GRID + 1)]
    vals = [opt.xi(t) for t in grid]
    kb = min(range(1, GRID), key=lambda k: vals[k])
    th, xi_best, n = golden_section(opt.xi, grid[kb - 1], grid[kb + 1], tol=tol)
    n += GRID + 2
    if fswap:                                   # the FSWAP-like endpoints
        for t in (math.pi / 2, -math.pi / 2):
            x = opt.xi(t)
            n += 1
            if x < xi_best:
                th, xi_best = t, x
    if not xi_best < xi0:
        th = 0.0
    xi, An, Bn, q_new = opt.apply(th)
    c, s = math.cos(th), math.sin(th)
    U_new = U @ embed(np.array([[c, -s], [s, c]]), U.shape[0], p)
    return BondResult(th, xi, xi0, An, Bn, np.asarray(q_new), U_new, n + 1)


def optimize_mps_bonds(tensors: Sequence[np.ndarray], charges: Sequence[Sequence[int]], U: np.ndarray,
                       chi: int, tol: float = 1e-8) -> Tuple[List[np.ndarray], List[List[int]], np.ndarray,
                                                            List[BondResult]]:
    """One right-to-left pass over the bonds of an MPS whose centre is on its last site.

    At each bond (p, p+1) the best local rotation is found and applied; the
    singular values move left with the centre.  Returns the new tensors (centre
    on site 0), their bond charges, the new orbital basis and one record per bond."""
    ts = [np.asarray(t, dtype=np.float64) for t in tensors]
    qs = [list(q) for q in charges]
    out = []
    for p in range(len(ts) - 2, -1, -1):
        r = optimize_bond(ts[p], ts[p + 1], qs[p], qs[p + 1], qs[p + 2], chi, U, p, tol=tol)
        ts[p], ts[p + 1] = r.A, r.B
        qs[p + 1] = [int(x) for x in r.q_mid]
        U = r.U
        out.append(r)
    return ts, qs, U, out
