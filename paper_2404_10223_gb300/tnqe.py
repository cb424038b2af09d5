"""Thin ctypes binding of the C ABI in ``include/tnqe.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: arrays are made contiguous FP64 and passed as
pointers; device buffers (for example ``torch.Tensor.data_ptr()``) may be
passed as plain integers wherever the ABI accepts host or device memory.
The library must have been built (``build.py``); loading fails loudly
otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtnqe.so")

TNQE_PREC_FP64, TNQE_PREC_TF32X3, TNQE_PREC_BF16X3, TNQE_PREC_BF16X6, TNQE_PREC_BF16X10, TNQE_PREC_BF16X15 = range(6)
TNQE_FORM_BLOCKS, TNQE_FORM_DENSE = 0, 1
TNQE_PROFILE_LEN = 12
STATUS_NAMES = {0: "TNQE_OK", 1: "TNQE_ERR_ARG", 2: "TNQE_ERR_STATE", 3: "TNQE_ERR_NOMEM", 4: "TNQE_ERR_CUDA",
                5: "TNQE_ERR_NOCONV", 6: "TNQE_ERR_TIMEOUT", 7: "TNQE_ERR_NUMERIC"}


class TnqeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class tnqe_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("chi_rot", ctypes.c_int), ("cutoff", ctypes.c_double),
                ("solve_eps", ctypes.c_double), ("renormalize_rotated", ctypes.c_int),
                ("max_jacobi_sweeps", ctypes.c_int), ("max_spin", ctypes.c_longlong),
                ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("contraction_form", ctypes.c_int), ("autotune_cache", ctypes.c_char_p),
                ("workspace_limit", ctypes.c_longlong)]


EXPORTED = ["tnqe_default_options", "tnqe_mpo_host", "tnqe_check_mps", "tnqe_givens_host",
            "tnqe_rotate_integrals_host", "tnqe_gate_host", "tnqe_create", "tnqe_add_mps", "tnqe_reset_mps", "tnqe_rotate",
            "tnqe_get_rotated", "tnqe_matrix_elements", "tnqe_solve", "tnqe_set_precision", "tnqe_set_form", "tnqe_last_timing", "tnqe_last_profile", "tnqe_apply_gate_noalloc",
            "tnqe_solve_ex", "tnqe_dependence", "tnqe_autotune", "tnqe_set_tuning", "tnqe_set_block_tuning", "tnqe_clear_graphs", "tnqe_graph_count", "tnqe_last_error",
            "tnqe_destroy"]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtnqe.so not built at {path}; run paper_2404_10223_gb300/build.py")
    lib = ctypes.CDLL(path)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    lib.tnqe_default_options.argtypes = [ctypes.POINTER(tnqe_options)]
    lib.tnqe_default_options.restype = None
    lib.tnqe_create.argtypes = [P, P, I, I, I, ctypes.POINTER(tnqe_options), ctypes.POINTER(P)]
    lib.tnqe_mpo_host.argtypes = [P, P, I, P, P, P, P, P, LL]
    lib.tnqe_check_mps.argtypes = [I, I, I, P, P, P, ctypes.c_char_p, I]
    lib.tnqe_givens_host.argtypes = [P, I, P, P, P, P, I, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.tnqe_rotate_integrals_host.argtypes = [P, P, P, I, P, P]
    lib.tnqe_gate_host.argtypes = [D, D, P]
    lib.tnqe_add_mps.argtypes = [P, P, P, P, ctypes.POINTER(I)]
    lib.tnqe_reset_mps.argtypes = [P]
    lib.tnqe_rotate.argtypes = [P, I, I, ctypes.POINTER(D)]
    lib.tnqe_get_rotated.argtypes = [P, P, P, LL]
    lib.tnqe_matrix_elements.argtypes = [P, P, I, P, P]
    lib.tnqe_solve.argtypes = [P, P, P, I, P, P, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.tnqe_set_precision.argtypes = [P, I]
    lib.tnqe_set_form.argtypes = [P, I]
    lib.tnqe_last_timing.argtypes = [P, P, ctypes.POINTER(I)]
    lib.tnqe_last_profile.argtypes = [P, P, I]
    lib.tnqe_apply_gate_noalloc.argtypes = [P, P, I, I, I, P, P, P, D, D, I, I, D, I, P, P, P,
                                            ctypes.POINTER(I), ctypes.POINTER(D), P, ctypes.c_char_p, I]
    lib.tnqe_solve_ex.argtypes = [P, P, P, I, D, P, P, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.tnqe_dependence.argtypes = [P, P, I, D, P]
    lib.tnqe_autotune.argtypes = [P, P, I, P, P]
    lib.tnqe_set_tuning.argtypes = [P, I, I, I]
    lib.tnqe_set_block_tuning.argtypes = [P, I, I, I]
    lib.tnqe_clear_graphs.argtypes = [P]
    lib.tnqe_graph_count.argtypes = [P]
    lib.tnqe_last_error.argtypes = [P]
    lib.tnqe_last_error.restype = ctypes.c_char_p
    lib.tnqe_destroy.argtypes = [P]
    lib.tnqe_destroy.restype = None
    for name in EXPORTED:
        if name not in ("tnqe_default_options", "tnqe_last_error", "tnqe_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(ctx, st: int):
    if st != 0:
        msg = load().tnqe_last_error(ctx).decode() if ctx else ""
        raise TnqeError(st, msg)


def tnqe_default_options() -> tnqe_options:
    o = tnqe_options()
    load().tnqe_default_options(ctypes.byref(o))
    return o


def tnqe_givens_host(V):
    """The library's Givens plan of V: ([(site, c, s, side)], neg_site); side 0 = left, 1 = right."""
    lib = load()
    V = _f64(V)
    N = V.shape[0]
    cap = max(1, N * (N - 1) // 2)
    site = np.zeros(cap, dtype=np.int32)
    side = np.zeros(cap, dtype=np.int32)
    c = np.zeros(cap)
    s = np.zeros(cap)
    ng, neg = ctypes.c_int(0), ctypes.c_int(0)
    _check(None, lib.tnqe_givens_host(_ptr(V), N, _ptr(site), _ptr(side), _ptr(c), _ptr(s), cap,
                                      ctypes.byref(ng), ctypes.byref(neg)))
    return [(int(site[g]), float(c[g]), float(s[g]), int(side[g])) for g in range(ng.value)], neg.value


def tnqe_gate_host(c: float, s: float):
    """The library's 16 x 16 two-site gate, rows (k1', k2'), columns (k1, k2)."""
    G = np.zeros((16, 16))
    _check(None, load().tnqe_gate_host(float(c), float(s), _ptr(G)))
    return G


def tnqe_rotate_integrals_host(h1, eri, U):
    """(h', eri') in basis U as the library computes them."""
    lib = load()
    h1, eri, U = _f64(h1), _f64(eri), _f64(U)
    N = U.shape[0]
    ho = np.zeros((N, N))
    go = np.zeros((N, N, N, N))
    _check(None, lib.tnqe_rotate_integrals_host(_ptr(h1), _ptr(eri), _ptr(U), N, _ptr(ho), _ptr(go)))
    return ho, go


def tnqe_check_mps(tensors, U, n_alpha: int, n_beta: int):
    """Host-side checks of tnqe_add_mps on one state: (status, message); 0 = valid."""
    lib = load()
    ts = [_f64(t) for t in tensors]
    N = len(ts)
    dims = np.array([ts[0].shape[0]] + [t.shape[2] for t in ts], dtype=np.int32)
    ptrs = (ctypes.c_void_p * N)(*[t.ctypes.data for t in ts])
    U = _f64(U)
    buf = ctypes.create_string_buffer(256)
    st = lib.tnqe_check_mps(N, n_alpha, n_beta, ctypes.cast(ptrs, ctypes.c_void_p), _ptr(dims), _ptr(U), buf, 256)
    return st, buf.value.decode()


def tnqe_mpo_host(h1, eri, N: int):
    """The library's Hamiltonian MPO (host build): (dims, [(rowptr, col, val) per site]).

    Site t is a (4 D_{t+1}) x (4 D_t) CSR matrix, row k * D_{t+1} + w', column w * 4 + k'."""
    lib = load()
    h1, eri = _f64(h1), _f64(eri)
    dims = np.zeros(N + 1, dtype=np.int32)
    nnz = np.zeros(N, dtype=np.int64)
    _check(None, lib.tnqe_mpo_host(_ptr(h1), _ptr(eri), N, _ptr(dims), _ptr(nnz), None, None, None, 0))
    nrp = int(sum(4 * int(dims[t + 1]) + 1 for t in range(N)))
    tot = int(nnz.sum())
    rowptr = np.zeros(nrp, dtype=np.int32)
    col = np.zeros(max(tot, 1), dtype=np.int32)
    val = np.zeros(max(tot, 1), dtype=np.float64)
    _check(None, lib.tnqe_mpo_host(_ptr(h1), _ptr(eri), N, _ptr(dims), _ptr(nnz), _ptr(rowptr), _ptr(col),
                                   _ptr(val), tot))
    sites, ro, eo = [], 0, 0
    for t in range(N):
        n_r = 4 * int(dims[t + 1]) + 1
        k = int(nnz[t])
        sites.append((rowptr[ro:ro + n_r].copy(), col[eo:eo + k].copy(), val[eo:eo + k].copy()))
        ro += n_r
        eo += k
    return dims.astype(int).tolist(), sites


def tnqe_create(h1, eri, N: int, n_alpha: int, n_beta: int, options: Optional[tnqe_options] = None):
    lib = load()
    h1, eri = _f64(h1), _f64(eri)
    out = ctypes.c_void_p()
    st = lib.tnqe_create(_ptr(h1), _ptr(eri), N, n_alpha, n_beta,
                         ctypes.byref(options) if options is not None else None, ctypes.byref(out))
    if st != 0:
        raise TnqeError(st, "tnqe_create failed")
    return out


def tnqe_add_mps(ctx, tensors: Sequence[np.ndarray], U) -> int:
    ts = [_f64(t) for t in tensors]
    dims = np.array([1] + [t.shape[2] for t in ts], dtype=np.int32)
    arr = (ctypes.c_void_p * len(ts))(*[t.ctypes.data for t in ts])
    U = _f64(U)
    mid = ctypes.c_int()
    _check(ctx, load().tnqe_add_mps(ctx, arr, _ptr(dims), _ptr(U), ctypes.byref(mid)))
    return mid.value


def tnqe_reset_mps(ctx):
    _check(ctx, load().tnqe_reset_mps(ctx))


def tnqe_rotate(ctx, i: int, j: int) -> float:
    d = ctypes.c_double()
    _check(ctx, load().tnqe_rotate(ctx, i, j, ctypes.byref(d)))
    return d.value


def tnqe_get_rotated(ctx, N: int) -> List[np.ndarray]:
    dims = np.zeros(N + 1, dtype=np.int32)
    _check(ctx, load().tnqe_get_rotated(ctx, _ptr(dims), None, 0))
    total = int(sum(int(dims[s]) * 4 * int(dims[s + 1]) for s in range(N)))
    buf = np.zeros(max(total, 1))
    _check(ctx, load().tnqe_get_rotated(ctx, _ptr(dims), _ptr(buf), total))
    out, o = [], 0
    for s in range(N):
        n = int(dims[s]) * 4 * int(dims[s + 1])
        out.append(buf[o:o + n].reshape(int(dims[s]), 4, int(dims[s + 1])).copy())
        o += n
    return out


def tnqe_matrix_elements(ctx, pairs: Sequence[Tuple[int, int]], H_out=None, S_out=None):
    """H_out / S_out: None (host arrays returned) or device pointers as ints."""
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    n = pr.shape[0]
    host = H_out is None
    if host:
        H_out, S_out = np.zeros(n), np.zeros(n)
    _check(ctx, load().tnqe_matrix_elements(ctx, _ptr(pr), n, _ptr(H_out), _ptr(S_out)))
    return (H_out, S_out) if host else None


def tnqe_solve(ctx, H, S):
    H, S = _f64(H), _f64(S)
    M = H.shape[0]
    E, C = np.zeros(M), np.zeros((M, M))
    rank, k1 = ctypes.c_int(), ctypes.c_double()
    _check(ctx, load().tnqe_solve(ctx, _ptr(H), _ptr(S), M, _ptr(E), _ptr(C), ctypes.byref(rank), ctypes.byref(k1)))
    return E, C, rank.value, k1.value


def tnqe_solve_ex(ctx, H, S, eps: float):
    H, S = _f64(H), _f64(S)
    M = H.shape[0]
    E, C = np.zeros(M), np.zeros((M, M))
    rank, k1 = ctypes.c_int(), ctypes.c_double()
    _check(ctx, load().tnqe_solve_ex(ctx, _ptr(H), _ptr(S), M, eps, _ptr(E), _ptr(C), ctypes.byref(rank),
                                     ctypes.byref(k1)))
    return E, C, rank.value, k1.value


def tnqe_dependence(ctx, S, eps: float = 1e-12) -> np.ndarray:
    S = _f64(S)
    r = np.zeros(S.shape[0])
    _check(ctx, load().tnqe_dependence(ctx, _ptr(S), S.shape[0], eps, _ptr(r)))
    return r


def tnqe_set_precision(ctx, precision: int):
    _check(ctx, load().tnqe_set_precision(ctx, precision))


def tnqe_set_form(ctx, form: int):
    _check(ctx, load().tnqe_set_form(ctx, form))


def tnqe_last_timing(ctx):
    t = np.zeros(3)
    n = ctypes.c_int()
    _check(ctx, load().tnqe_last_timing(ctx, _ptr(t), ctypes.byref(n)))
    return t, n.value


def tnqe_last_profile(ctx) -> np.ndarray:
    p = np.zeros(TNQE_PROFILE_LEN)
    _check(ctx, load().tnqe_last_profile(ctx, _ptr(p), TNQE_PROFILE_LEN))
    return p


def tnqe_autotune(ctx, pairs):
    """Tune the contraction's launch shapes on `pairs` (charge-block CTA sizes, or the sliced-BF16
    tiles); returns (the three chosen shapes, 3x3 candidate times in ms, zeros from the cache)."""
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    cfg = np.zeros(3, dtype=np.int32)
    times = np.zeros(9)
    _check(ctx, load().tnqe_autotune(ctx, _ptr(pr), len(pr), _ptr(cfg), _ptr(times)))
    return tuple(int(x) for x in cfg), times.reshape(3, 3)


def tnqe_set_tuning(ctx, bn1: int, bn3: int, spmm_bw: int):
    _check(ctx, load().tnqe_set_tuning(ctx, bn1, bn3, spmm_bw))


def tnqe_set_block_tuning(ctx, t1: int, t2: int, t3: int):
    _check(ctx, load().tnqe_set_block_tuning(ctx, t1, t2, t3))


def tnqe_clear_graphs(ctx):
    _check(ctx, load().tnqe_clear_graphs(ctx))


def tnqe_graph_count(ctx) -> int:
    return int(load().tnqe_graph_count(ctx))


def tnqe_apply_gate_noalloc(A: int, B: int, chi_l: int, chi_m: int, chi_r: int, q_l, q_m, q_r, c: float,
                            s: float, sigma_side: int, chi_max: int, cutoff: float, max_sweeps: int,
                            A_out: int, B_out: int, stream: int = 0):
    """A, B, A_out, B_out: device pointers (ints).  Returns (k, q_out, discarded)."""
    ql, qm, qr = (np.ascontiguousarray(q, dtype=np.int32) for q in (q_l, q_m, q_r))
    q_out = np.zeros(chi_max, dtype=np.int32)
    k, disc = ctypes.c_int(), ctypes.c_double()
    err = ctypes.create_string_buffer(256)
    st = load().tnqe_apply_gate_noalloc(ctypes.c_void_p(A), ctypes.c_void_p(B), chi_l, chi_m, chi_r, _ptr(ql),
                                        _ptr(qm), _ptr(qr), c, s, sigma_side, chi_max, cutoff, max_sweeps,
                                        ctypes.c_void_p(A_out), ctypes.c_void_p(B_out), _ptr(q_out),
                                        ctypes.byref(k), ctypes.byref(disc), ctypes.c_void_p(stream), err, 256)
    if st != 0:
        raise TnqeError(st, err.value.decode())
    return k.value, q_out[:k.value].copy(), disc.value


def tnqe_last_error(ctx) -> str:
    return load().tnqe_last_error(ctx).decode()


def tnqe_destroy(ctx):
    if ctx:
        load().tnqe_destroy(ctx)


class Context:
    """Owning wrapper: a context plus the states added to it."""

    def __init__(self, h1, eri, N: int, n_alpha: int, n_beta: int, **opts):
        o = tnqe_default_options()
        for k, v in opts.items():
            if k == "autotune_cache" and isinstance(v, str):
                v = v.encode()
            setattr(o, k, v)
        self.N = N
        self.ctx = tnqe_create(h1, eri, N, n_alpha, n_beta, o)

    def add_mps(self, tensors, U) -> int:
        return tnqe_add_mps(self.ctx, tensors, U)

    def reset_mps(self):
        tnqe_reset_mps(self.ctx)

    def rotate(self, i: int, j: int) -> float:
        return tnqe_rotate(self.ctx, i, j)

    def get_rotated(self):
        return tnqe_get_rotated(self.ctx, self.N)

    def matrix_elements(self, pairs, H_out=None, S_out=None):
        return tnqe_matrix_elements(self.ctx, pairs, H_out, S_out)

    def solve(self, H, S):
        return tnqe_solve(self.ctx, H, S)

    def solve_ex(self, H, S, eps: float):
        return tnqe_solve_ex(self.ctx, H, S, eps)

    def dependence(self, S, eps: float = 1e-12):
        return tnqe_dependence(self.ctx, S, eps)

    def set_precision(self, p: int):
        tnqe_set_precision(self.ctx, p)

    def set_form(self, form: int):
        tnqe_set_form(self.ctx, form)

    def last_timing(self):
        return tnqe_last_timing(self.ctx)

    def last_profile(self):
        return tnqe_last_profile(self.ctx)

    def autotune(self, pairs):
        return tnqe_autotune(self.ctx, pairs)

    def set_tuning(self, bn1: int, bn3: int, spmm_bw: int):
        tnqe_set_tuning(self.ctx, bn1, bn3, spmm_bw)

    def set_block_tuning(self, t1: int, t2: int, t3: int):
        tnqe_set_block_tuning(self.ctx, t1, t2, t3)

    def clear_graphs(self):
        tnqe_clear_graphs(self.ctx)

    def graph_count(self) -> int:
        return tnqe_graph_count(self.ctx)

    def close(self):
        if self.ctx:
            tnqe_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
