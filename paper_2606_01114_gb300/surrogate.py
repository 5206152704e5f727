"""Training data, training and the gain measurement for the FNO demag
surrogate on 2-D films, all on the GPU through the C ABI.

* ``generate_pairs``: (m, H_demag / Ms) pairs taken along relaxation
  trajectories (RKF45, Eq. 1 with the field of Eqs. 2 and 4) started from
  seeded film textures: random, vortex, domain wall, smooth random.
* ``train``: Adam on the relative-L2 loss with the library's own forward
  and backward kernels.
* ``gain``: relax() of held-out states with the plain FP32 solver and with
  the surrogate (exact field every k steps, fallback above the residual
  bound, exact final approach), timed on the device, with the relaxed
  energies compared.

Run as ``python -m paper_2606_01114_gb300.surrogate --out result.json``; the
defaults are the 256 x 256 x 1 film with 4 nm cells, 20,000 training pairs,
a 4-layer network of width 32 with 16 modes per axis and 64 test states.
"""

import argparse
import json
import math
import time

import numpy as np
import torch

from . import (MM_F32, mm_demag_field, mm_destroy, mm_energy, mm_fno_adam_step, mm_fno_backward, mm_fno_create,
               mm_fno_destroy, mm_fno_forward, mm_fno_loss, mm_fno_params, mm_fno_zero_grad, mm_init_mesh,
               mm_max_torque, mm_relax, mm_relax_surrogate, mm_set_material)

FILM = dict(n=(256, 256, 1), d=(4e-9, 4e-9, 4e-9), Ms=8.0e5, A=1.3e-11, alpha=0.5)


def film_context(film=FILM):
    ctx = mm_init_mesh(*film["n"], *film["d"], precision=MM_F32)
    mm_set_material(ctx, film["Ms"], film["A"], film["alpha"], 0.0, (0.0, 0.0, 1.0))
    return ctx


def initial_state(film, seed):
    import workloads
    m = workloads.film_state(film["n"], film["d"], seed)
    return torch.tensor(m, dtype=torch.float32, device="cuda")


def generate_pairs(ctx, film, n_traj, per_traj, seed0, t_first=1e-12, growth=1.15):
    """n_traj trajectories x per_traj snapshots at t = 0 and after windows of
    t_first * growth^k seconds; returns device tensors m, h [N][3][ny][nx]."""
    nx, ny, _ = film["n"]
    N = n_traj * per_traj
    ms = torch.empty((N, 3, ny, nx), dtype=torch.float32, device="cuda")
    hs = torch.empty_like(ms)
    H = torch.empty((3, 1, ny, nx), dtype=torch.float32, device="cuda")
    i = 0
    for t in range(n_traj):
        m = initial_state(film, seed0 + t)
        for k in range(per_traj):
            if k:
                mm_relax(ctx, m, t_first * growth ** (k - 1), torque_tol=0.0)
            mm_demag_field(ctx, m, H)
            ms[i] = m[:, 0]
            hs[i] = H[:, 0] / film["Ms"]
            i += 1
    return ms, hs


def train(f, ms, hs, steps, batch, lr, seed=0, log_every=0):
    """Adam with cosine decay over `steps`, batches drawn without
    replacement per epoch; returns the loss history (one float per step)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    N = ms.shape[0]
    perm, pos = torch.randperm(N, generator=g), 0
    out = torch.empty((batch,) + tuple(ms.shape[1:]), dtype=torch.float32, device="cuda")
    dh = torch.empty_like(out)
    losses = []
    for s in range(1, steps + 1):
        if pos + batch > N:
            perm, pos = torch.randperm(N, generator=g), 0
        idx = perm[pos:pos + batch].to("cuda")
        pos += batch
        mb, hb = ms.index_select(0, idx), hs.index_select(0, idx)
        mm_fno_forward(f, mb, out)
        losses.append(mm_fno_loss(f, out, hb, dh))
        mm_fno_zero_grad(f)
        mm_fno_backward(f, mb, dh)
        mm_fno_adam_step(f, lr * 0.5 * (1 + math.cos(math.pi * (s - 1) / steps)), step=s)
        if log_every and s % log_every == 0:
            print(f"step {s}: loss {np.mean(losses[-log_every:]):.4e}", flush=True)
    return losses


def evaluate(f, ms, hs, batch):
    """Mean relative-L2 error of the surrogate on held pairs."""
    errs = []
    out = torch.empty((batch,) + tuple(ms.shape[1:]), dtype=torch.float32, device="cuda")
    for i in range(0, ms.shape[0] - batch + 1, batch):
        mm_fno_forward(f, ms[i:i + batch], out)
        d = (out - hs[i:i + batch]).flatten(1).norm(dim=1) / hs[i:i + batch].flatten(1).norm(dim=1)
        errs += d.tolist()
    return float(np.mean(errs)), float(np.max(errs))


def per_eval_ms(fn, reps=200):
    for _ in range(5):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def gain(ctx, f, film, seeds, t_max, torque_tol, k_exact, bound, torque_exact, log=None):
    """Relax each seeded state with the plain solver and with the surrogate;
    device-synchronised wall time and relaxed energies per state (each row
    is also printed as it completes, when `log` is given)."""
    rows = []
    for seed in seeds:
        m0 = initial_state(film, seed)
        row = {"seed": int(seed)}
        for mode in ("plain", "surrogate"):
            m = m0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode == "plain":
                t, steps = mm_relax(ctx, m, t_max, torque_tol)
                stats = None
            else:
                t, steps, ex, su, fb = mm_relax_surrogate(ctx, f, m, t_max, torque_tol, k_exact=k_exact, bound=bound,
                                                          torque_exact=torque_exact)
                stats = {"exact_evals": ex, "surrogate_evals": su, "fallbacks": fb}
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            E = mm_energy(ctx, m)
            row[mode] = {"seconds": wall, "t": t, "steps": steps, "energy": float(np.sum(E)),
                         "torque": mm_max_torque(ctx, m), **(stats or {})}
        if torque_exact > torque_tol:
            m = m0.clone()
            row["plain_steps_to_torque_exact"] = mm_relax(ctx, m, t_max, torque_exact)[1]
        else:
            row["plain_steps_to_torque_exact"] = row["plain"]["steps"]
        row["energy_rel_err"] = abs(row["surrogate"]["energy"] - row["plain"]["energy"]) / abs(row["plain"]["energy"])
        rows.append(row)
        if log:
            print(json.dumps(row), file=log, flush=True)
    return rows


def timing(film, width, modes, layers, batch, bf16=True):
    """Kernel timing of the network alone: a batch-1 evaluation and one
    training step (forward, loss, backward, Adam) at `batch`, random data."""
    nx, ny = film["n"][0], film["n"][1]
    f = mm_fno_create(nx, ny, width=width, modes=modes, layers=layers, store_bf16=bf16, max_batch=batch, seed=1)
    m = torch.randn(1, 3, ny, nx, device="cuda")
    h = torch.empty_like(m)
    fwd_ms = per_eval_ms(lambda: mm_fno_forward(f, m, h), reps=100)
    mb = torch.randn(batch, 3, ny, nx, device="cuda")
    hb, dh = torch.empty_like(mb), torch.empty_like(mb)
    state = {"s": 0}

    def step():
        state["s"] += 1
        mm_fno_forward(f, mb, hb)
        mm_fno_loss(f, hb, mb, dh)
        mm_fno_zero_grad(f)
        mm_fno_backward(f, mb, dh)
        mm_fno_adam_step(f, 1e-3, step=state["s"])
    step_ms = per_eval_ms(step, reps=20)
    mm_fno_destroy(f)
    return {"forward_batch1_ms": fwd_ms, f"train_step_batch{batch}_ms": step_ms}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--trajectories", type=int, default=400)
    ap.add_argument("--per-trajectory", type=int, default=50)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--modes", type=int, default=16)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--fp32-storage", action="store_true", help="FP32 activations instead of BF16")
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--test-states", type=int, default=64)
    ap.add_argument("--t-max", type=float, default=5e-9)
    ap.add_argument("--torque-tol", type=float, default=1e-4)
    ap.add_argument("--k-exact", type=int, default=10)
    ap.add_argument("--bound", type=float, default=1e-3)
    ap.add_argument("--torque-exact", type=float, default=1e-2)
    ap.add_argument("--out", default=None)
    ap.add_argument("--params-out", default=None, help="save the trained parameters (numpy .npy) here")
    ap.add_argument("--params-in", default=None,
                    help="load trained parameters from this .npy and skip data generation and training")
    ap.add_argument("--rows-log", default=None, help="append each test state's result (JSON line) as it completes")
    ap.add_argument("--timing", action="store_true", help="time the network's kernels only and exit")
    a = ap.parse_args(argv)
    film = FILM
    if a.timing:
        res = timing(film, a.width, a.modes, a.layers, a.batch, bf16=not a.fp32_storage)
        print(json.dumps(res), flush=True)
        return res
    ctx = film_context(film)
    res = {"film": {k: list(v) if isinstance(v, tuple) else v for k, v in film.items()}, "args": vars(a)}

    vm, vh = generate_pairs(ctx, film, 8, 8, seed0=20000)
    f = mm_fno_create(film["n"][0], film["n"][1], width=a.width, modes=a.modes, layers=a.layers,
                      store_bf16=not a.fp32_storage, max_batch=max(a.batch, 16), seed=7)
    if a.params_in:
        mm_fno_params(f, set_params=np.load(a.params_in).astype(np.float32))
        res["params_in"] = a.params_in
    else:
        t0 = time.perf_counter()
        ms, hs = generate_pairs(ctx, film, a.trajectories, a.per_trajectory, seed0=100)
        torch.cuda.synchronize()
        res["pairs"] = int(ms.shape[0])
        res["generate_seconds"] = time.perf_counter() - t0
        print(f"{ms.shape[0]} pairs in {res['generate_seconds']:.1f} s", flush=True)
        t0 = time.perf_counter()
        losses = train(f, ms, hs, a.train_steps, a.batch, a.lr, log_every=max(a.train_steps // 20, 1))
        torch.cuda.synchronize()
        res["train_seconds"] = time.perf_counter() - t0
        res["train_loss_first"] = float(np.mean(losses[:10]))
        res["train_loss_last"] = float(np.mean(losses[-50:]))
        del ms, hs
        if a.params_out:
            np.save(a.params_out, mm_fno_params(f)[0])
    res["val_rel_l2_mean"], res["val_rel_l2_max"] = evaluate(f, vm, vh, 16)
    print(f"validation rel-L2 mean {res['val_rel_l2_mean']:.3e} max {res['val_rel_l2_max']:.3e}", flush=True)
    if a.test_states == 0:
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(res, fh, indent=1)
        return res

    m1 = initial_state(film, 30000)
    H1 = torch.empty_like(m1)
    h1 = torch.empty((1, 3, film["n"][1], film["n"][0]), dtype=torch.float32, device="cuda")
    res["exact_demag_ms"] = per_eval_ms(lambda: mm_demag_field(ctx, m1, H1))
    res["surrogate_eval_ms"] = per_eval_ms(lambda: mm_fno_forward(f, m1.view(1, 3, *m1.shape[2:]), h1))
    print(f"per evaluation: exact demag {res['exact_demag_ms']:.4f} ms, surrogate {res['surrogate_eval_ms']:.4f} ms",
          flush=True)

    log = open(a.rows_log, "a") if a.rows_log else None
    rows = gain(ctx, f, film, range(10000, 10000 + a.test_states), a.t_max, a.torque_tol, a.k_exact, a.bound,
                a.torque_exact, log=log)
    if log:
        log.close()
    tp = sum(r["plain"]["seconds"] for r in rows)
    ts = sum(r["surrogate"]["seconds"] for r in rows)
    errs = np.array([r["energy_rel_err"] for r in rows])
    res["gain"] = {
        "plain_seconds": tp, "surrogate_seconds": ts, "speedup": tp / ts,
        "energy_rel_err_median": float(np.median(errs)), "energy_rel_err_max": float(errs.max()),
        "states_within_1e-6": int(np.sum(errs <= 1e-6)), "states": len(rows),
        "fallbacks": int(sum(r["surrogate"]["fallbacks"] for r in rows)),
        "exact_evals": int(sum(r["surrogate"]["exact_evals"] for r in rows)),
        "surrogate_evals": int(sum(r["surrogate"]["surrogate_evals"] for r in rows)),
        "plain_steps": int(sum(r["plain"]["steps"] for r in rows)),
        "plain_steps_above_torque_exact": int(sum(r["plain_steps_to_torque_exact"] for r in rows)),
    }
    res["rows"] = rows
    print(json.dumps(res["gain"]), flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    mm_fno_destroy(f)
    mm_destroy(ctx)
    return res


if __name__ == "__main__":
    main()
