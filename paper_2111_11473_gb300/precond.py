"""Learned-preconditioner protocol: record pairs, train on the GPU, compare.

Every step runs in the library: thc_solve records the training pairs
(features of the residual at iteration k -> step to the converged core),
thc_mlp_train fits the network with its own forward/backward/Adam kernels,
and thc_solve with use_mlp = 1 applies it under the accept/reject rule.
This module only sequences those calls and summarises the outcome.

The time to an energy tolerance is measured against a reference energy
(normally the float64 converged energy of the same system): the wall time,
from the start of the solve, of the first iteration whose energy is within
the tolerance of it.
"""
from __future__ import annotations

import numpy as np

from .binding import Context, Mlp

PAIRS_PER_ITER = 2048


def collect_pairs(ctx: Context, r_tol=1e-6, max_iter=80, per_iter=PAIRS_PER_ITER, seed=0):
    """Solve with pair recording.  Returns (X, j, t, report); empty arrays if
    the solve did not converge (the targets need the converged core)."""
    _, _, rep = ctx.solve(r_tol=r_tol, max_iter=max_iter, record_pairs=per_iter,
                          record_seed=seed, raise_on_failure=False)
    X, j, t = ctx.solve_pairs()
    return X, j, t, rep


def train(X, j, t, hidden=256, bf16=True, epochs=20, batch=2048, lr=1e-3, seed=1):
    """A fresh network trained on the pairs; returns (mlp, final loss, loss of
    the plain Jacobi step on the same pairs)."""
    net = Mlp(hidden=hidden, seed=seed, bf16=bf16)
    loss = net.train(X, j, t, epochs=epochs, batch=batch, lr=lr, seed=seed)
    jacobi = float(np.mean((j.astype(np.float64) - t.astype(np.float64)) ** 2))
    return net, loss, jacobi


def time_to(history, e_ref, tol=1e-6):
    """(iteration, seconds) of the first history entry with |E - e_ref| < tol."""
    for k, (e, _, sec) in enumerate(history):
        if abs(e - e_ref) < tol:
            return k + 1, sec
    return None, None


def run_solve(ctx: Context, e_ref=None, mlp=None, r_tol=1e-6, max_iter=80, e_tol=1e-6,
              stop_de=0.0):
    """One solve from zero; returns a summary dict.  With e_ref None the
    solve's own final energy is the reference.  stop_de > 0 also requires the
    energy change of the last iteration to be below it before stopping."""
    hist = []
    _, _, rep = ctx.solve(r_tol=r_tol, e_tol=stop_de, max_iter=max_iter,
                          use_mlp=mlp is not None, mlp=mlp, history=hist,
                          raise_on_failure=False)
    ref = rep.energy if e_ref is None else e_ref
    it_e, t_e = time_to(hist, ref, e_tol)
    return {"status": rep.status, "iters": rep.iters, "energy": rep.energy,
            "r_norm": rep.r_norm, "wall_s": rep.wall_s, "iters_to_e_tol": it_e,
            "time_to_e_tol_s": t_e, "mlp_accepted": rep.mlp_accepted,
            "mlp_rejected": rep.mlp_rejected}


def compare(ctx: Context, mlp: Mlp, e_ref=None, r_tol=1e-6, max_iter=80, e_tol=1e-6):
    """Plain Jacobi + DIIS against the same solve with the network's proposals.

    The plain solve decides: its converged energy is the reference when
    e_ref is None, and ``energy_diff`` reports how far the learned solve's
    converged energy lies from it."""
    plain = run_solve(ctx, e_ref, None, r_tol, max_iter, e_tol)
    ref = plain["energy"] if e_ref is None else e_ref
    learned = run_solve(ctx, ref, mlp, r_tol, max_iter, e_tol)
    return {"plain": plain, "learned": learned,
            "energy_diff": learned["energy"] - plain["energy"],
            "iter_gain": plain["iters"] - learned["iters"]}


def family_sizes(o):
    """(o, v, P, G, K) of the learned-preconditioner family: v = 5o, P = 10o,
    G = 30o, K = 15o (the bench system's ratios)."""
    return o, 5 * o, 10 * o, 30 * o, 15 * o


def protocol(n_train=50, n_heldout=10, o_lo=20, o_hi=80, o_heldout=60, epochs=20,
             r_tol=1e-6, log=print):
    """Train on n_train systems with o drawn uniformly from [o_lo, o_hi] (seed 99;
    system seeds 100+k), evaluate on n_heldout systems with o = o_heldout
    (seeds 200+k), all in mixed precision.  Returns a summary dict."""
    import time

    from synth import make_system

    from .binding import THC_PREC_MIXED
    rng = np.random.default_rng(99)
    orders = rng.integers(o_lo, o_hi + 1, n_train)
    Xs, js, ts = [], [], []
    t0 = time.perf_counter()
    for k, o in enumerate(orders):
        s = make_system(*family_sizes(int(o)), 100 + k)
        with Context(s.eps_o, s.eps_v, s.Y, s.L, s.x, s.z, precision=THC_PREC_MIXED) as ctx:
            X, j, t, rep = collect_pairs(ctx, r_tol=r_tol, seed=k)
        log(f"train {k}: o={o} {rep.status} iters={rep.iters} pairs={len(j)}")
        Xs.append(X)
        js.append(j)
        ts.append(t)
    X, j, t = (np.concatenate(a) for a in (Xs, js, ts))
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, loss, jacobi = train(X, j, t, epochs=epochs)
    train_s = time.perf_counter() - t0
    log(f"trained on {len(j)} pairs in {train_s:.1f} s: loss {loss:.4f} "
        f"(plain Jacobi step {jacobi:.4f})")
    results = []
    for k in range(n_heldout):
        s = make_system(*family_sizes(o_heldout), 200 + k)
        with Context(s.eps_o, s.eps_v, s.Y, s.L, s.x, s.z, precision=THC_PREC_MIXED) as ctx:
            c = compare(ctx, net, r_tol=r_tol)
        p, l = c["plain"], c["learned"]
        log(f"held-out {k}: plain {p['iters']} iters {p['wall_s']:.2f} s "
            f"({p['iters_to_e_tol']} to 1e-6 Eh); learned {l['iters']} iters {l['wall_s']:.2f} s "
            f"({l['iters_to_e_tol']} to 1e-6 Eh), accepted {l['mlp_accepted']} "
            f"rejected {l['mlp_rejected']}, dE {c['energy_diff']:.1e}")
        results.append(c)
    net.close()
    mean = lambda key, side: float(np.mean([r[side][key] for r in results]))
    return {"train_systems": n_train, "pairs": int(len(j)), "pair_seconds": gen_s,
            "train_seconds": train_s, "loss": loss, "loss_plain_jacobi": jacobi,
            "heldout": results,
            "mean_iters": {"plain": mean("iters", "plain"), "learned": mean("iters", "learned")},
            "mean_wall_s": {"plain": mean("wall_s", "plain"),
                            "learned": mean("wall_s", "learned")}}


if __name__ == "__main__":
    import argparse
    import json
    import sys
    ap = argparse.ArgumentParser(description=protocol.__doc__)
    ap.add_argument("--train", type=int, default=50)
    ap.add_argument("--heldout", type=int, default=10)
    ap.add_argument("--o-lo", type=int, default=20)
    ap.add_argument("--o-hi", type=int, default=80)
    ap.add_argument("--o-heldout", type=int, default=60)
    ap.add_argument("--epochs", type=int, default=20)
    a = ap.parse_args()
    out = protocol(a.train, a.heldout, a.o_lo, a.o_hi, a.o_heldout, a.epochs,
                   log=lambda m: print(m, file=sys.stderr, flush=True))
    print(json.dumps(out))
