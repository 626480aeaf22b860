"""Training and evaluation of the learned preconditioner.

Data: seeded hull-in-waves samples (hull offset, wave amplitude/wavelength/phase and velocities
drawn per seed) whose pressure the plain PCG solver computes on the GPU; each sample is stored on
the device as its geometry channels (BF16), unknown mask, scaled right-hand side S b_hat and scaled
solution S^-1 x (FP32).  Training: the library's forward/backward/Adam kernels (vofp_nn_train_step)
on one sample per step.  Evaluation: flexible CG with the network against plain and mixed PCG on
held-out seeds.  Checkpoints are .npz files of the FP32 master weights.

    python -m paper_1410_1937_gb300.learned --samples 2000 --epochs 8 --out weights.npz
    python -m paper_1410_1937_gb300.learned --samples 0 --init weights.npz   # evaluate only
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import time

import numpy as np

TRAIN_SEED0 = 100000
HELD_OUT_SEED0 = 200000
TRAIN_SHAPE = (256, 128, 64)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_hull_256x128x64.npz")


def _geometry_worker(args):
    """Inputs of one sample, computed in a worker process (numpy only, FP32 for transfer)."""
    from paper_1410_1937_gb300 import inputs as I
    seed, shape = args
    p = I.config3_sample(seed, shape)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32).ravel()
    return seed, (p.dx, p.dy, p.dz), {k: f32(getattr(p, k)) for k in ("F", "vf", "ax", "ay", "az", "u", "v", "w")}


def generate(seeds, shape=TRAIN_SHAPE, workers=None, rtol=1e-9, stages=(0,), log=print):
    """Solve every seed's sample with the mixed-precision PCG and keep the training tensors on the GPU.
    Geometry is built by a spawned process pool (started before this process touches CUDA).

    A preconditioner is applied to residuals, so each sample gives one input/target pair per CG
    stage k in `stages`: the scaled residual S (b_hat - A_hat x_k) of the FP64 Jacobi-PCG iterate
    after k iterations and the scaled error S^-1 (x - x_k) (k = 0: the right-hand side and the
    solution).  Pairs share their sample's geometry channels."""
    ctxmp = mp.get_context("spawn")
    workers = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
    pool = ctxmp.Pool(workers)
    import torch
    from paper_1410_1937_gb300 import vofp
    data = {"geo": [], "pairs": []}
    t0 = time.perf_counter()
    net = vofp.Network(seed=0)
    try:
        for i, (seed, (dx, dy, dz), arr) in enumerate(pool.imap(_geometry_worker, [(s, shape) for s in seeds],
                                                                chunksize=1)):
            d = {k: torch.from_numpy(v).cuda().double() for k, v in arr.items()}
            ctx = vofp.Context(dx, dy, dz)
            ctx.vofp_build_operator(d["F"], d["ax"], d["ay"], d["az"], d["vf"],
                                    (0, 1, 0, 0, 0, 0), 1000.0, 1.2, 0.1, 0, 1.0)
            b = ctx.vofp_rhs_from_face_velocity(d["u"], d["v"], d["w"])
            x, info = ctx.vofp_solve(b, rtol=rtol, mode=vofp.MODE_MIXED, precond=vofp.PRECOND_RBSGS)
            net.bind(ctx, d["F"])
            geo, mask = net.export_geometry()
            g = len(data["geo"])
            data["geo"].append((geo, mask))
            for k in stages:
                if k == 0:
                    r, e = ctx.vofp_scaled_pair(b, x)
                else:
                    xk, _ = ctx.vofp_solve(b, rtol=1e-30, max_iter=k, mode=vofp.MODE_FP64, check_every=2,
                                           raise_on_error=False)
                    r, e = ctx.vofp_scaled_pair(b - ctx.vofp_apply(xk), x - xk)
                data["pairs"].append({"seed": seed, "geo": g, "stage": k, "r": r, "x": e})
            ctx.close()
            if (i + 1) % 100 == 0 or i + 1 == len(seeds):
                log(f"generated {i + 1}/{len(seeds)} samples ({len(data['pairs'])} pairs) in "
                    f"{time.perf_counter() - t0:.1f} s")
    finally:
        pool.close()
        pool.join()
    return data


def train(net, data, shape=TRAIN_SHAPE, epochs=4, lr=1e-3, seed=0, log=print):
    """One input/target pair per Adam step, pairs shuffled every epoch, cosine learning-rate decay."""
    rng = np.random.default_rng(seed)
    nz_ny_nx = (shape[2], shape[1], shape[0])
    pairs = data["pairs"]
    total = epochs * len(pairs)
    step = 0
    hist = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        losses = []
        for i in rng.permutation(len(pairs)):
            s = pairs[i]
            geo, mask = data["geo"][s["geo"]]
            net.set_geometry(nz_ny_nx, geo, mask)
            lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / max(total, 1)))
            losses.append(net.train_step(s["r"], s["x"], lr=lr_t))
            step += 1
        hist.append(float(np.mean(losses)))
        log(f"epoch {ep + 1}/{epochs}: mean loss {hist[-1]:.4e} ({time.perf_counter() - t0:.1f} s)")
    return hist


def _bounded_imap(pool, args, batch=64):
    """pool.imap over `args` in batches: the workers build inputs faster than the GPU trains on
    them, and an unbounded imap would queue every sample's arrays (~70 MB at 256x128x64) in host
    memory."""
    for i in range(0, len(args), batch):
        yield from pool.imap(_geometry_worker, args[i:i + batch], chunksize=1)


def train_anorm(net, seeds, shape=TRAIN_SHAPE, epochs=2, lr=1e-3, stages=(0, 16, 64, 256), workers=None,
                log=print):
    """Online training as a preconditioner: per sample (seeded geometry, waves and velocities) the
    plain FP64 Jacobi-PCG solves to 1e-10 on the GPU, and each CG stage k in `stages` gives a
    scaled residual r_k = S (b_hat - A_hat x_k) with its exact error e_k = S^-1 (x - x_k); one Adam
    step per pair on the relative A-norm error of the network's output against e_k under the
    sample's own operator (vofp_nn_train_step_anorm).  The loss is 1 for a zero output and 0 for the
    exact error, whatever the scale of r_k, so early and late residuals weigh alike.  Inputs are
    built by a spawned process pool (started before this process touches CUDA); cosine decay."""
    ctxmp = mp.get_context("spawn")
    workers = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
    pool = ctxmp.Pool(workers)
    import torch
    from paper_1410_1937_gb300 import vofp
    total = epochs * len(seeds) * len(stages)
    step, hist = 0, []
    t0 = time.perf_counter()
    try:
        for ep in range(epochs):
            losses, by_stage = [], {k: [] for k in stages}
            for i, (seed, (dx, dy, dz), arr) in enumerate(_bounded_imap(pool, [(s, shape) for s in seeds])):
                d = {k: torch.from_numpy(v).cuda().double() for k, v in arr.items()}
                ctx = vofp.Context(dx, dy, dz)
                ctx.vofp_build_operator(d["F"], d["ax"], d["ay"], d["az"], d["vf"],
                                        (0, 1, 0, 0, 0, 0), 1000.0, 1.2, 0.1, 0, 1.0)
                b = ctx.vofp_rhs_from_face_velocity(d["u"], d["v"], d["w"])
                x, info = ctx.vofp_solve(b, rtol=1e-10, mode=vofp.MODE_FP64, raise_on_error=False)
                net.bind(ctx, d["F"])
                for k in stages:
                    if k == 0:
                        r, e = ctx.vofp_scaled_pair(b, x)
                    else:
                        xk, _ = ctx.vofp_solve(b, rtol=1e-30, max_iter=k, mode=vofp.MODE_FP64, check_every=2,
                                               raise_on_error=False)
                        r, e = ctx.vofp_scaled_pair(b - ctx.vofp_apply(xk), x - xk)
                    lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / max(total, 1)))
                    loss = net.train_step_anorm(ctx, r, e, lr=lr_t)
                    losses.append(loss)
                    by_stage[k].append(loss)
                    step += 1
                ctx.close()
                if (i + 1) % 200 == 0:
                    log(f"epoch {ep + 1}: {i + 1}/{len(seeds)} samples, mean loss of the last 200 "
                        f"{np.mean(losses[-200 * len(stages):]):.4f} ({time.perf_counter() - t0:.0f} s)")
            hist.append({"loss": float(np.mean(losses)), "by_stage": {k: float(np.mean(v)) for k, v in by_stage.items()}})
            log(f"epoch {ep + 1}/{epochs}: mean relative A-norm error {hist[-1]}")
    finally:
        pool.close()
        pool.join()
    return hist


def save(net, path):
    np.savez_compressed(path, params=net.get_params(), layers=np.array([27, 16, 32, 64]))


def load(net, path):
    net.set_params(np.load(path)["params"])


def evaluate(net, seeds, shape, rtol=1e-8, log=print):
    """Per seed: iterations and device time to rtol for flexible CG with the network, and for
    mixed-precision PCG (Jacobi and red-black) and plain FP64 PCG on the same input."""
    import torch
    from paper_1410_1937_gb300 import inputs as I
    from paper_1410_1937_gb300 import vofp
    rows = []
    for seed in seeds:
        p = I.config3_sample(seed, shape)
        ctx, t = vofp.context_for(p)
        b = ctx.vofp_rhs_from_face_velocity(t["u"], t["v"], t["w"])
        net.bind(ctx, t["F"])
        row = {"seed": seed}
        for name, kw in (("fcg_nn", dict(mode=vofp.MODE_FCG_NN, nn=net)),
                         ("mixed_rbsgs", dict(mode=vofp.MODE_MIXED, precond=vofp.PRECOND_RBSGS)),
                         ("mixed_jacobi", dict(mode=vofp.MODE_MIXED)),
                         ("fp64_jacobi", dict(mode=vofp.MODE_FP64))):
            ctx.vofp_solve(b, rtol=rtol, raise_on_error=False, **kw)       # warm-up
            _, info = ctx.vofp_solve(b, rtol=rtol, raise_on_error=False, **kw)
            row[name] = {k: info[k] for k in ("iterations", "seconds", "rel_residual", "status_name",
                                              "nn_applications", "fell_back")}
        # what the network gains per iteration: relative residual after k iterations
        early = {}
        for k in (2, 6, 10, 20, 40):
            _, a = ctx.vofp_solve(b, rtol=rtol, max_iter=k, mode=vofp.MODE_FCG_NN, nn=net, stag_window=10 ** 6,
                                  raise_on_error=False)
            _, c = ctx.vofp_solve(b, rtol=rtol, max_iter=k, mode=vofp.MODE_MIXED, check_every=2,
                                  raise_on_error=False)
            _, d = ctx.vofp_solve(b, rtol=rtol, max_iter=k, mode=vofp.MODE_MIXED, check_every=2,
                                  precond=vofp.PRECOND_RBSGS, raise_on_error=False)
            early[k] = {"fcg_nn": a["rel_residual"], "cg_jacobi": c["rel_residual"], "cg_rbsgs": d["rel_residual"]}
        row["residual_after_k_iterations"] = early
        rows.append(row)
        log(json.dumps(row))
        ctx.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--shape", type=int, nargs=3, default=list(TRAIN_SHAPE))
    ap.add_argument("--eval-seeds", type=int, default=4)
    ap.add_argument("--eval-shape", type=int, nargs=3, default=list(TRAIN_SHAPE))
    ap.add_argument("--out", default="weights.npz")
    ap.add_argument("--init", default=None)
    ap.add_argument("--workers", type=int, default=0)
    ap.add_argument("--report", default=None)
    ap.add_argument("--stages", default="0", help="CG stages of the training pairs, e.g. 0,16,64,256")
    ap.add_argument("--loss", default="mse", choices=["mse", "anorm"],
                    help="mse: scaled solution error of stored pairs; anorm: relative A-norm error, online")
    args = ap.parse_args()
    shape = tuple(args.shape)
    stages = tuple(int(v) for v in args.stages.split(","))
    hist = []
    seeds = range(TRAIN_SEED0, TRAIN_SEED0 + args.samples)
    if args.samples > 0 and args.loss == "mse":
        data = generate(seeds, shape, workers=args.workers or None, stages=stages)
    from paper_1410_1937_gb300 import vofp
    net = vofp.Network(seed=1)
    if args.init:
        load(net, args.init)
    if args.samples > 0 and args.loss == "mse":
        hist = train(net, data, shape, args.epochs, args.lr)
        save(net, args.out)
        del data
    elif args.samples > 0:
        hist = train_anorm(net, seeds, shape, args.epochs, args.lr, stages, workers=args.workers or None)
        save(net, args.out)
    rows = evaluate(net, range(HELD_OUT_SEED0, HELD_OUT_SEED0 + args.eval_seeds), tuple(args.eval_shape))
    if args.report:
        with open(args.report, "w") as f:
            json.dump({"samples": args.samples, "stages": stages, "epochs": args.epochs, "loss": hist, "eval": rows},
                  f, indent=1)


if __name__ == "__main__":
    main()
