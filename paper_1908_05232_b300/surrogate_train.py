"""Training data and training of the learned flood surrogate (build-added; the
paper has no surrogate).

Data: trajectories of the plain coupled step at a fixed time step on seeded
shopping-centre scenarios (the stand-in for the paper's shopping centre):
512x512 centres with 10,000 evacuees and 2048x2048 centres with 100,000
pedestrians building a sandbag barrier, flooded from t = 900 s (pairs taken
from mid-flood on).  A
sample pairs the state U = (h, hu, hv) and bed z at some step with the change
of U over the next FP_SUR_WINDOW steps.  Training crops are 32 x 32 cells of
that change with the 5-cell halo of (h, hu, hv, z) around them; cells past the
domain edge repeat the edge cell, as in the simulation's surrogate window.
Training itself runs on the library's CUDA kernels (fp_surrogate_train_step:
tensor-core forward, FP32 backward, Adam); PyTorch only holds and slices the
device buffers.

    python -m paper_1908_05232_b300.surrogate_train --out weights.npy

writes FP32 parameters that Surrogate.set_params loads.
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import _native as N

WINDOW = 8
HALO = 5
DT_DEFAULT = 2.0 ** -5  # s; Courant number <= 0.5 at the depths of these floods at dx = 0.5 m


def _torch():
    import torch
    return torch


def trajectory_pairs(sc, dt=DT_DEFAULT, every=256, n_pairs=64, skip_steps=0, device="cuda", cfl_until=None):
    """Run the plain coupled step on scenario ``sc`` at a fixed step dt and return
    a list of (x, d) device tensors: x = (h, hu, hv, z) [ny+10, nx+10, 4] with
    edge-repeating halo, d = change of (h, hu, hv) over WINDOW steps [ny, nx, 3].
    cfl_until: first advance with the CFL step to this simulated time (s)."""
    torch = _torch()
    if cfl_until is not None:
        sc.dt_fixed_ticks = 0
        sim = N.from_scenario(sc)
        while sim.counters()["t_ticks"] < int(cfl_until * N.TICKS):
            sim.step(256)
        sim.set_fixed_dt(dt)
    else:
        sc.dt_fixed_ticks = int(round(dt * N.TICKS))
        sim = N.from_scenario(sc)
    out = []

    def read():
        planes = []
        for k in (N.FP_FIELD_H, N.FP_FIELD_HU, N.FP_FIELD_HV):
            t = torch.empty((sc.ny, sc.nx), dtype=torch.float32, device=device)
            N.fp_read_state(sim.h, k, t)
            planes.append(t)
        return torch.stack(planes, dim=-1)

    if skip_steps:
        sim.step(skip_steps)
    for _ in range(n_pairs):
        if every > WINDOW:
            sim.step(every - WINDOW)
        u0 = read()
        sim.step(WINDOW)
        u1 = read()
        z = torch.empty((sc.ny, sc.nx), dtype=torch.float32, device=device)
        N.fp_read_state(sim.h, N.FP_FIELD_Z, z)  # barrier layers included
        x = torch.cat([u0, z[..., None]], dim=-1).permute(2, 0, 1)[None]
        x = torch.nn.functional.pad(x, (HALO, HALO, HALO, HALO), mode="replicate")[0].permute(1, 2, 0).contiguous()
        out.append((x, (u1 - u0).contiguous()))
    c = sim.counters()
    sim.close()
    return out, c


class CropSampler:
    """Random 32 x 32 training crops from trajectory pairs: a share ``active_frac``
    where the depth changes by more than 1 mm somewhere in the crop (the flood
    front and the flowing water), a share ``wet_frac`` holding water anywhere in
    the input, the rest anywhere."""

    def __init__(self, pairs, crop=32, wet_frac=0.4, active_frac=0.5, seed=0):
        torch = _torch()
        self.pairs = pairs
        self.crop = crop
        self.rng = np.random.default_rng(seed)
        self.wet_frac = wet_frac
        self.active_frac = active_frac
        k = crop + 2 * HALO
        self.wet_origins, self.active_origins = [], []
        for x, d in pairs:
            h = x[..., 0][None, None]
            m = torch.nn.functional.max_pool2d((h > 0).float(), kernel_size=k, stride=1)[0, 0]
            self.wet_origins.append(torch.nonzero(m > 0).cpu().numpy())
            a = torch.nn.functional.max_pool2d(d[..., 0].abs()[None, None], kernel_size=crop, stride=1)[0, 0]
            self.active_origins.append(torch.nonzero(a > 1e-3).cpu().numpy())

    def batch(self, B):
        torch = _torch()
        xs, ts = [], []
        k = self.crop + 2 * HALO
        for _ in range(B):
            p = int(self.rng.integers(len(self.pairs)))
            x, d = self.pairs[p]
            wo, ao = self.wet_origins[p], self.active_origins[p]
            r = self.rng.random()
            if len(ao) and r < self.active_frac:
                oy, ox = ao[int(self.rng.integers(len(ao)))]
            elif len(wo) and r < self.active_frac + self.wet_frac:
                oy, ox = wo[int(self.rng.integers(len(wo)))]
            else:
                oy = int(self.rng.integers(x.shape[0] - k + 1))
                ox = int(self.rng.integers(x.shape[1] - k + 1))
            xs.append(x[oy:oy + k, ox:ox + k])
            ts.append(d[oy:oy + self.crop, ox:ox + self.crop])
        return torch.stack(xs).contiguous(), torch.stack(ts).contiguous()


def train(sur, sampler, steps=2000, batch=64, lr=1e-3, lr_end=1e-4, log_every=0):
    """Adam on the sampler's crops with an exponential learning-rate decay; returns the losses."""
    losses = []
    for s in range(steps):
        a = s / max(1, steps - 1)
        x, t = sampler.batch(batch)
        losses.append(sur.train_step(x, t, lr * (lr_end / lr) ** a))
        if log_every and (s % log_every == 0 or s == steps - 1):
            print("step %5d  loss %.3e" % (s, losses[-1]), flush=True)
    return losses


def window_errors(sur, pairs):
    """Per pair: largest |dh| error of the net and of persistence (dU = 0) over the
    cells, and the mean |dh| errors, on full fields."""
    torch = _torch()
    res = []
    for x, d in pairs:
        H, W = x.shape[0], x.shape[1]
        y = torch.empty((1, H - 2 * HALO, W - 2 * HALO, 3), dtype=torch.float32, device=x.device)
        sur.forward(x[None].contiguous(), y)
        e = (y[0, ..., 0] - d[..., 0]).abs()
        p = d[..., 0].abs()
        res.append(dict(net_max=float(e.max()), net_mean=float(e.mean()), persist_max=float(p.max()),
                        persist_mean=float(p.mean()), net_over_1cm=float((e > 0.01).float().mean()),
                        persist_over_1cm=float((p > 0.01).float().mean())))
    return res


def main(argv=None):
    import scenarios as S

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--n", type=int, default=512, help="grid side of the training scenarios")
    ap.add_argument("--seeds", default="2,3,4,5")
    ap.add_argument("--peaks", default="0.6,1.0,1.4,1.0")
    ap.add_argument("--pairs", type=int, default=100)
    ap.add_argument("--every", type=int, default=512)
    ap.add_argument("--dt", type=float, default=DT_DEFAULT)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--barrier-seeds", default="4,5", help="2048x2048 barrier scenarios (empty: none)")
    ap.add_argument("--barrier-pairs", type=int, default=24)
    ap.add_argument("--barrier-start", type=float, default=1000.0)
    ap.add_argument("--barrier-every", type=int, default=1536)
    args = ap.parse_args(argv)
    t0 = time.time()
    pairs = []
    for seed, peak in zip([int(s) for s in args.seeds.split(",")], [float(p) for p in args.peaks.split(",")]):
        sc = S.shopping_centre(args.n, 0.5, 10_000 * args.n * args.n // (512 * 512), 0, seed, 1800.0,
                               peak_depth=peak)
        pr, c = trajectory_pairs(sc, args.dt, args.every, args.pairs)
        print("seed %d peak %.1f: %d pairs, %d steps over the Courant limit" % (seed, peak, len(pr),
                                                                              c["cfl_exceeded"]), flush=True)
        pairs += pr
    for seed in [int(v) for v in args.barrier_seeds.split(",") if v]:
        pr, c = trajectory_pairs(S.config_barrier(seed), args.dt, args.barrier_every, args.barrier_pairs,
                                 cfl_until=args.barrier_start)
        print("barrier 2048 seed %d: %d pairs from t = %.0f s, %d steps over the Courant limit"
              % (seed, len(pr), args.barrier_start, c["cfl_exceeded"]), flush=True)
        pairs += pr
    print("data %.1f s" % (time.time() - t0), flush=True)
    sur = N.Surrogate(seed=args.init_seed)
    sampler = CropSampler(pairs, seed=args.init_seed)
    t1 = time.time()
    train(sur, sampler, steps=args.steps, batch=args.batch, lr=args.lr, lr_end=args.lr * 1e-2,
          log_every=max(1, args.steps // 20))
    print("training %.1f s" % (time.time() - t1), flush=True)
    np.save(args.out, sur.params())
    held, _ = trajectory_pairs(S.shopping_centre(args.n, 0.5, 10_000 * args.n * args.n // (512 * 512), 0, 7,
                                                 1800.0, peak_depth=1.2), args.dt, args.every, 20)
    errs = window_errors(sur, held)
    for k in ("net_max", "persist_max", "net_mean", "persist_mean", "net_over_1cm", "persist_over_1cm"):
        print("held-out %-12s %.3e" % (k, np.mean([e[k] for e in errs])))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
