"""Generalized sweep over a growing set of MPS in their own orbital bases, with
an optional learned proposal of the orbital-rotation generators.

The paper's generalized sweep (Sec. II C, App. A) grows the subspace one state
at a time; a new state starts in the orbitals of the previous one (App. A,
step "new MPS initialised in the previous basis"), and each sweep revisits
every state, proposes a change and keeps it only if the subspace energy of
H c = E S c (Eq. 9) goes down.  Here the tensors of each state are fixed
random draws and the proposals act on the rotation generator K_j of state j
(U_j = expm(K_j), Eq. 11): the plain proposal is K_j + sigma xi with xi a
random antisymmetric matrix, R candidates per step, the best one kept if it
lowers the energy by more than a tolerance.  Every matrix element and every
solve goes through the library (tnqe_matrix_elements, tnqe_solve).

The learned proposal adds the candidate K_j + f(x) to the R random ones, where f
is the proposal network (include/tnqe_mlp.h) and x holds the strictly-lower
entries of K_j and the padded subspace eigenvalues; the R random candidates
draw the same random numbers as in the plain run, so the plain proposal is
both the fallback and the yardstick.  A new state likewise starts from the
better of the previous state's orbitals and the network's proposal from there.
(learned_mode "replace" puts the network's step in place of the first random
candidate and takes its starting proposal unconditionally.)  The network is
trained on the (x, best accepted step, energy drop) records that plain sweeps
write (train_proposer).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

from . import inputs

N_EIG = 8   # subspace eigenvalues in the network input (zero-padded)


# ----------------------------------------------------------------------------- helpers
def k_vector(K: np.ndarray) -> np.ndarray:
    """Strictly-lower entries of an antisymmetric generator, row by row."""
    r, c = np.tril_indices(K.shape[0], -1)
    return K[r, c].copy()


def k_matrix(v: np.ndarray, N: int) -> np.ndarray:
    K = np.zeros((N, N))
    r, c = np.tril_indices(N, -1)
    K[r, c] = v
    return K - K.T


def features(K: np.ndarray, E: np.ndarray, E_ref: float, birth: float) -> np.ndarray:
    """Network input: K's strictly-lower entries, the subspace eigenvalues minus
    E_ref (zero-padded to N_EIG), and a flag: 1 when proposing a new state's
    starting generator, 0 for a step of an existing state."""
    e = np.zeros(N_EIG)
    m = min(N_EIG, len(E))
    e[:m] = np.asarray(E[:m]) - E_ref
    return np.concatenate([k_vector(K), e, [birth]])


def n_features(N: int) -> int:
    return N * (N - 1) // 2 + N_EIG + 1


class LibraryBackend:
    """Matrix elements and solves through the C ABI (tnqe.Context)."""

    def __init__(self, h1, eri, N, na, nb, **opts):
        from . import tnqe
        self.args = (h1, eri, N, na, nb)
        self.ctx = tnqe.Context(h1, eri, N, na, nb, **opts)

    def reset(self):
        self.ctx.reset_mps()

    def add_mps(self, tensors, U) -> int:
        return self.ctx.add_mps(tensors, U)

    def matrix_elements(self, pairs):
        return self.ctx.matrix_elements(pairs)

    def energies(self, H, S) -> np.ndarray:
        E, _, rank, _ = self.ctx.solve(H, S)
        return np.asarray(E[:rank])

    def close(self):
        self.ctx.close()


@dataclasses.dataclass
class SweepConfig:
    N: int = 12
    n_alpha: int = 6
    n_beta: int = 6
    L: int = 24
    chi: int = 64
    M_max: int = 8
    sweeps: int = 20
    grow_every: int = 2          # a new state joins at the start of sweeps 1, 1 + g, 1 + 2g, ...
    R: int = 4                   # candidates per step
    sigma: float = 0.05          # plain proposal: K + sigma * xi
    learned_scales: Tuple[float, ...] = (1.0,)   # learned candidates per step: K + scale * f(x)
    learned_mode: str = "extra"  # "extra": R random + the learned candidates; "replace": learned in place of random
    step_cap_sigmas: float = 5.0 # learned steps are clipped to this many random-step norms
    birth_cap: float = 3.0       # Frobenius-norm cap of a learned starting offset
    tol: float = 1e-8            # acceptance: E_new < E_old - tol
    ham_seed: int = 0            # the Hamiltonian (integrals) is fixed; sweep seeds vary the rest
    cutoff: float = 1e-14


@dataclasses.dataclass
class SweepResult:
    energies: List[float]                      # subspace ground energy after each sweep
    M: List[int]                               # subspace size after each sweep
    accepted: int
    proposals: int
    learned_accepted: int
    records: List[Tuple[np.ndarray, np.ndarray, float]]   # (features, best step dK, energy drop) per step
    learned_births: int = 0                    # new states that started from the network's proposal


def hamiltonian(cfg: SweepConfig):
    rng = np.random.default_rng(cfg.ham_seed)
    return inputs.draw_integrals(rng, cfg.N, cfg.L)


def rotation(K: np.ndarray) -> np.ndarray:
    """U = expm(K), re-orthonormalised (polar factor) so that large generators stay orthogonal to 1e-15."""
    u, _, vt = np.linalg.svd(scipy.linalg.expm(K))
    return u @ vt


def clip_step(d: np.ndarray, cap: float) -> np.ndarray:
    """Scale a proposed generator step down to Frobenius norm cap (a guard against wild network outputs)."""
    n = float(np.linalg.norm(d))
    return d * (cap / n) if n > cap else d


def random_step(rng: np.random.Generator, N: int, sigma: float) -> np.ndarray:
    Lo = np.tril(rng.normal(0.0, sigma, (N, N)), -1)
    return Lo - Lo.T


# ----------------------------------------------------------------------------- the sweep
def run_sweep(cfg: SweepConfig, seed: int, backend, proposer: Optional[Callable[[np.ndarray], np.ndarray]] = None,
              E_stop: Optional[float] = None) -> SweepResult:
    """One generalized sweep run.

    backend: LibraryBackend (or any object with reset / add_mps /
    matrix_elements / energies).  proposer: None for the plain method, else a
    function from a batch of network inputs (B x n_in) to generator steps
    (B x N(N-1)/2); it then proposes the first candidate of every step, at the
    scales cfg.learned_scales, and the starting generator of every new state
    (K_prev + f).  E_stop: stop after the first sweep whose energy is at or
    below it (used to count sweeps to a target).

    The stored H and S always put the state earlier in the list in the bra:
    with truncated rotations H_ab and H_ba differ slightly, so every recomputed
    entry keeps that orientation.
    """
    N = cfg.N
    rng = np.random.default_rng(1_000_003 * seed + 17)
    tensors: List[List[np.ndarray]] = []
    Ks: List[np.ndarray] = []
    ids: List[int] = []
    H = np.zeros((0, 0))
    S = np.zeros((0, 0))
    E_cur = math.inf
    Evec = np.zeros(0)
    E_ref = 0.0
    res = SweepResult([], [], 0, 0, 0, [], 0)
    births: List[Tuple[int, np.ndarray, np.ndarray]] = []   # (state, features at birth, K at birth)

    def rebuild():
        backend.reset()
        ids[:] = [backend.add_mps(t, rotation(K)) for t, K in zip(tensors, Ks)]

    def energy(Hm, Sm) -> Tuple[float, np.ndarray]:
        E = backend.energies(Hm, Sm)
        return float(E[0]), E

    def pair(a_pos: int, a_id: int, b_pos: int, b_id: int):
        return (a_id, b_id) if a_pos <= b_pos else (b_id, a_id)

    for sweep in range(cfg.sweeps):
        rebuild()
        # grow: the new state starts in the orbitals of the last one (or the network's proposal from there)
        if len(Ks) < cfg.M_max and sweep % cfg.grow_every == 0:
            t_new, _ = inputs.draw_mps(rng, N, cfg.n_alpha, cfg.n_beta, cfg.chi)
            K_new = Ks[-1].copy() if Ks else np.zeros((N, N))
            x_birth = features(K_new, Evec, E_ref, 1.0)
            starts = [K_new]
            if proposer is not None and Ks:
                d = k_matrix(np.asarray(proposer(x_birth[None, :]), dtype=np.float64)[0], N)
                K_l = K_new + clip_step(d, cfg.birth_cap)
                starts = [K_l] if cfg.learned_mode == "replace" else [K_new, K_l]
            M = len(Ks) + 1
            cids = [backend.add_mps(t_new, rotation(K0)) for K0 in starts]
            rows = backend.matrix_elements([(ids[i], c) for c in cids for i in range(M - 1)] + [(c, c) for c in cids])
            best_c = 0
            if len(cids) > 1:                      # keep the start with the lower subspace energy
                e_c = []
                for q in range(len(cids)):
                    Hc = np.zeros((M, M))
                    Sc = np.zeros((M, M))
                    Hc[:M - 1, :M - 1] = H
                    Sc[:M - 1, :M - 1] = S
                    hv = np.append(rows[0][q * (M - 1):(q + 1) * (M - 1)], rows[0][len(cids) * (M - 1) + q])
                    sv = np.append(rows[1][q * (M - 1):(q + 1) * (M - 1)], rows[1][len(cids) * (M - 1) + q])
                    Hc[:, M - 1] = Hc[M - 1, :] = hv
                    Sc[:, M - 1] = Sc[M - 1, :] = sv
                    e_c.append(energy(Hc, Sc)[0])
                best_c = int(np.argmin(e_c))
                if best_c > 0:
                    res.learned_births += 1
            K_new = starts[best_c]
            births.append((len(Ks), x_birth, K_new.copy()))
            tensors.append(t_new)
            Ks.append(K_new)
            ids.append(cids[best_c])
            nc = len(cids)
            Hn = np.append(rows[0][best_c * (M - 1):(best_c + 1) * (M - 1)], rows[0][nc * (M - 1) + best_c])
            Sn = np.append(rows[1][best_c * (M - 1):(best_c + 1) * (M - 1)], rows[1][nc * (M - 1) + best_c])
            H2 = np.zeros((M, M))
            S2 = np.zeros((M, M))
            H2[:M - 1, :M - 1] = H
            S2[:M - 1, :M - 1] = S
            H2[:, M - 1] = H2[M - 1, :] = Hn
            S2[:, M - 1] = S2[M - 1, :] = Sn
            H, S = H2, S2
            E_cur, Evec = energy(H, S)
            if M == 1:
                E_ref = E_cur
        M = len(Ks)
        for j in range(M):
            x = features(Ks[j], Evec, E_ref, 0.0)
            steps = [random_step(rng, N, cfg.sigma) for _ in range(cfg.R)]
            learned = proposer is not None
            learned_idx = set()
            if learned:
                d = k_matrix(np.asarray(proposer(x[None, :]), dtype=np.float64)[0], N)
                d = clip_step(d, cfg.step_cap_sigmas * cfg.sigma * math.sqrt(N * (N - 1) / 2))
                if cfg.learned_mode == "replace":
                    n_learned = min(len(cfg.learned_scales), cfg.R)
                    for q in range(n_learned):
                        steps[q] = cfg.learned_scales[q] * d
                    learned_idx = set(range(n_learned))
                else:
                    learned_idx = set(range(len(steps), len(steps) + len(cfg.learned_scales)))
                    steps += [sc * d for sc in cfg.learned_scales]
            cand_ids = [backend.add_mps(tensors[j], rotation(Ks[j] + dK)) for dK in steps]
            others = [i for i in range(M) if i != j]
            pairs = [pair(i, ids[i], j, c) for c in cand_ids for i in others] + [(c, c) for c in cand_ids]
            Hv, Sv = backend.matrix_elements(pairs)
            off = (M - 1) * len(cand_ids)
            best, best_E, best_H, best_S, best_Ev = -1, E_cur, None, None, None
            for r in range(len(cand_ids)):
                Hc, Sc = H.copy(), S.copy()
                for q, i in enumerate(others):
                    Hc[i, j] = Hc[j, i] = Hv[r * (M - 1) + q]
                    Sc[i, j] = Sc[j, i] = Sv[r * (M - 1) + q]
                Hc[j, j] = Hv[off + r]
                Sc[j, j] = Sv[off + r]
                Ec, Ev = energy(Hc, Sc)
                if Ec < best_E - cfg.tol:
                    best, best_E, best_H, best_S, best_Ev = r, Ec, Hc, Sc, Ev
            res.proposals += len(cand_ids)
            if best >= 0:
                res.records.append((x, k_vector(steps[best]), E_cur - best_E))
                Ks[j] = Ks[j] + steps[best]
                ids[j] = cand_ids[best]
                H, S, E_cur, Evec = best_H, best_S, best_E, best_Ev
                res.accepted += 1
                if best in learned_idx:
                    res.learned_accepted += 1
        res.energies.append(E_cur)
        res.M.append(len(Ks))
        if E_stop is not None and E_cur <= E_stop:
            break
    # birth records: where each new state's generator ended up, weighted by the energy it gained since
    drop_total = max(res.energies[0] - res.energies[-1], 0.0) if res.energies else 0.0
    for j, x_b, K_b in births:
        if j > 0 and drop_total > 0:
            res.records.append((x_b, k_vector(Ks[j] - K_b), drop_total / max(len(births) - 1, 1)))
    return res


def sweeps_to_reach(res: SweepResult, target: float, slack: float = 1e-9) -> int:
    """1-based index of the first sweep at or below target (len + 1 if never)."""
    for t, e in enumerate(res.energies):
        if e <= target + slack:
            return t + 1
    return len(res.energies) + 1


# ----------------------------------------------------------------------------- learning
def training_set(records: Sequence[Tuple[np.ndarray, np.ndarray, float]]):
    """Rows (features, accepted step, weight); the weight is the energy drop over its mean."""
    X = np.array([r[0] for r in records], dtype=np.float32)
    T = np.array([r[1] for r in records], dtype=np.float32)
    w = np.array([r[2] for r in records], dtype=np.float64)
    w = (w / max(w.mean(), 1e-300)).astype(np.float32)
    return X, T, w


def train_proposer(records, n_in: int, n_out: int, n_hidden: int = 256, epochs: int = 200, batch: int = 512,
                   lr: float = 1e-3, seed: int = 0):
    """Fit the proposal network (weighted MSE toward the accepted steps) with the library's Adam kernels.

    Returns (network, loss history)."""
    from . import mlp
    X, T, w = training_set(records)
    rng = np.random.default_rng(seed)
    net = mlp.Mlp(n_in, n_hidden, n_out, max_batch=max(batch, 1))
    net.set_params(inputs.draw_mlp_params(rng, n_in, n_hidden, n_out))
    hist = []
    n = len(X)
    for ep in range(epochs):
        order = rng.permutation(n)
        tot = 0.0
        for b0 in range(0, n, batch):
            idx = order[b0:b0 + batch]
            tot += net.adam_step(X[idx], T[idx], w[idx], lr=lr) * len(idx)
        hist.append(tot / n)
    return net, hist


def network_proposer(net) -> Callable[[np.ndarray], np.ndarray]:
    return lambda x: net.forward(x)


# ----------------------------------------------------------------------------- the learned-vs-plain experiment
def experiment(cfg: SweepConfig, train_seeds: Sequence[int], eval_seeds: Sequence[int], epochs: int = 200,
               lr: float = 1e-3, n_hidden: int = 256, backend=None, log=print) -> dict:
    """Train the proposer on plain sweeps of train_seeds, then on each eval seed
    count the sweeps the plain and the learned proposal need to reach the plain
    run's final energy.  Both runs of a seed draw the same random numbers; only
    candidate 0 of each step differs (random vs network)."""
    import time
    h1, eri = hamiltonian(cfg)
    own = backend is None
    if own:
        backend = LibraryBackend(h1, eri, cfg.N, cfg.n_alpha, cfg.n_beta, cutoff=cfg.cutoff, use_graphs=0)
    n_k = cfg.N * (cfg.N - 1) // 2
    t0 = time.time()
    records = []
    for s in train_seeds:
        r = run_sweep(cfg, s, backend)
        records += r.records
        log(f"train seed {s}: E {r.energies[-1]:.8f} accepted {r.accepted}/{r.proposals}")
    t_gen = time.time() - t0
    t0 = time.time()
    net, hist = train_proposer(records, n_features(cfg.N), n_k, n_hidden=n_hidden, epochs=epochs, lr=lr)
    t_train = time.time() - t0
    rows = []
    t0 = time.time()
    for s in eval_seeds:
        plain = run_sweep(cfg, s, backend)
        target = plain.energies[-1]
        learned = run_sweep(cfg, s, backend, proposer=network_proposer(net))
        sp, sl = sweeps_to_reach(plain, target), sweeps_to_reach(learned, target)
        rows.append({"seed": s, "E_plain": target, "E_learned": learned.energies[-1],
                     "dE_final": learned.energies[-1] - target, "sweeps_plain": sp, "sweeps_learned": sl,
                     "outcome": "win" if sl < sp else ("tie" if sl == sp else "loss"),
                     "learned_accepted": learned.learned_accepted, "accepted": learned.accepted,
                     "learned_births": learned.learned_births})
        log(f"eval seed {s}: plain {sp} sweeps, learned {sl}, final dE {rows[-1]['dE_final']:+.3e} "
            f"(network candidates accepted {learned.learned_accepted}/{learned.accepted}, "
            f"births {learned.learned_births})")
    t_eval = time.time() - t0
    net.close()
    if own:
        backend.close()
    return {"config": dataclasses.asdict(cfg), "train_seeds": list(train_seeds), "eval_seeds": list(eval_seeds),
            "samples": len(records), "loss_first": hist[0] if hist else None, "loss_last": hist[-1] if hist else None,
            **paired_summary(rows), "rows": rows, "seconds": {"generate": t_gen, "train": t_train, "evaluate": t_eval}}


def paired_summary(rows) -> dict:
    """Paired comparison over evaluation seeds: sweeps to reach the plain run's final energy (win =
    fewer), the final-energy difference, and a two-sided sign test on wins against losses."""
    sp = np.array([r["sweeps_plain"] for r in rows], dtype=float)
    sl = np.array([r["sweeps_learned"] for r in rows], dtype=float)
    de = np.array([r["dE_final"] for r in rows], dtype=float)
    wins = int(np.sum(sl < sp))
    losses = int(np.sum(sl > sp))
    n = wins + losses
    k = min(wins, losses)
    p = min(1.0, 2.0 * sum(math.comb(n, i) for i in range(k + 1)) / 2.0 ** n) if n else 1.0
    return {"mean_sweeps_plain": float(sp.mean()), "mean_sweeps_learned": float(sl.mean()),
            "mean_sweep_difference": float((sl - sp).mean()), "wins": wins, "ties": len(rows) - n,
            "losses": losses, "sign_test_p": p, "mean_dE_final": float(de.mean()),
            "learned_lower_or_equal_final": int(np.sum(de <= 1e-9))}


def _seeds(spec: str) -> List[int]:
    out: List[int] = []
    for part in spec.split(","):
        if "-" in part:
            a, b = part.split("-")
            out += list(range(int(a), int(b) + 1))
        elif part:
            out.append(int(part))
    return out


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="plain vs learned rotation proposals in the generalized sweep")
    ap.add_argument("--N", type=int, default=12)
    ap.add_argument("--electrons", type=int, default=6, help="alpha = beta electrons")
    ap.add_argument("--chi", type=int, default=64)
    ap.add_argument("--M-max", type=int, default=8)
    ap.add_argument("--sweeps", type=int, default=20)
    ap.add_argument("--R", type=int, default=4)
    ap.add_argument("--sigma", type=float, default=0.05)
    ap.add_argument("--train", default="1-100")
    ap.add_argument("--eval", default="101-120")
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--out", default=None, help="write the JSON result here")
    a = ap.parse_args(argv)
    cfg = SweepConfig(N=a.N, n_alpha=a.electrons, n_beta=a.electrons, L=2 * a.N, chi=a.chi, M_max=a.M_max,
                      sweeps=a.sweeps, R=a.R, sigma=a.sigma)
    res = experiment(cfg, _seeds(a.train), _seeds(a.eval), epochs=a.epochs)
    txt = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt + "\n")
    print(json.dumps({k: v for k, v in res.items() if k != "rows"}))


if __name__ == "__main__":
    main()
