"""Learned warm start of the constant-density solve: data from the solver's own runs,
training on the GPU, and the comparison with the zero and previous-step warm starts.

Every numerical step runs in libsph.so (the DFSPH steps, the feature sweep, the network's
training and inference kernels); this module only orchestrates the calls and moves data
between them.  Samples: seeded dam breaks of 0.5M-1.2M fluid particles (tank aspect
U[1, 3], fluid fill U[20 %, 60 %]) stepped with the previous-step warm start; after each
step a uniform random subset of particles contributes (features recorded at the warm
start, converged total density stiffness / (9.81 h)).
"""
from __future__ import annotations

import time

import numpy as np

from paper_2403_11156_gb300 import build, scenes, sph


def generate_dataset(n_samples=200_000, total_steps=500, n_scenes=5, seed=4, size_range=(5e5, 1.2e6)):
    """Returns (features [n][4], labels [n]) as float32 CUDA tensors."""
    import torch
    build.build()
    rng = np.random.default_rng(seed)
    per_step = int(np.ceil(n_samples / total_steps))
    steps_per_scene = int(np.ceil(total_steps / n_scenes))
    feats, labels = [], []
    taken = 0
    for k in range(n_scenes):
        n_target = int(rng.uniform(*size_range))
        d = scenes.dam_break_random(seed * 100 + k, n_target, warm_start=scenes.WARM_PREVIOUS)
        n = len(d["fluid_x"])
        kref = 9.81 * 4.0 * d["radius"]
        with sph.Context(d) as g:
            f_buf = torch.empty((n, 4), dtype=torch.float32, device="cuda")
            k_buf = torch.empty(n, dtype=torch.float32, device="cuda")
            for _ in range(steps_per_scene):
                if taken >= n_samples:
                    break
                g.sph_step(0.0)
                g.sph_read_field_device(sph.FIELD_FEATURES, f_buf)
                g.sph_read_field_device(sph.FIELD_KAPPA, k_buf)
                m = min(per_step, n_samples - taken)
                idx = torch.from_numpy(rng.choice(n, size=m, replace=False)).cuda()
                feats.append(f_buf[idx].clone())
                labels.append(k_buf[idx] / kref)
                taken += m
            g.sph_synchronize(raise_on_error=False)
    return torch.cat(feats), torch.cat(labels)


def init_params(seed=4, scale=None):
    """Seeded initial weights (Glorot-style normal), zero biases, unit statistics."""
    rng = np.random.default_rng(seed)
    p = np.zeros(sph.MLP_PARAMS, np.float32)
    H, F = 64, 4
    p[0:H * F] = rng.normal(scale=np.sqrt(2.0 / (F + H)) if scale is None else scale, size=H * F)
    p[H * F + H:H * F + H + H * H] = rng.normal(scale=np.sqrt(2.0 / (2 * H)) if scale is None else scale,
                                                size=H * H)
    o = H * F + H + H * H + H
    p[o:o + H] = rng.normal(scale=np.sqrt(2.0 / (H + 1)) if scale is None else scale, size=H)
    p[sph.MLP_WEIGHTS + 4:sph.MLP_WEIGHTS + 8] = 1.0
    p[-1] = 1.0
    return p


def train(features, labels, epochs=30, batch=4096, lr=1e-3, seed=4):
    """Train on the GPU; returns (params as float32 numpy, per-epoch loss numpy)."""
    import torch
    n = int(features.shape[0])
    params = torch.tensor(init_params(seed), device="cuda")
    adam = torch.zeros(2 * sph.MLP_WEIGHTS, dtype=torch.float32, device="cuda")
    hist = torch.zeros(epochs, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = sph.sph_mlp_train(features.contiguous(), labels.contiguous(), n, params, adam, epochs, batch, lr,
                           seed, hist, err)
    if st != sph.SPH_OK:
        raise sph.SphError(st, "sph_mlp_train failed")
    torch.cuda.synchronize()
    if int(err.item()) != 0:
        raise sph.SphError(sph.SPH_ETIMEOUT, "a tensor-core wait gave up during training")
    return params.cpu().numpy(), hist.cpu().numpy()


def compare_warm_starts(desc, params, steps=100, warmup=0, dt=0.0, gate=0):
    """Step the same scene with the zero, previous-step and learned warm starts (and, with
    gate > 0, the learned start held back while the previous density solve took at most
    `gate` iterations); returns per mode: mean density iterations per step, mean
    first-iteration density error, mean final error, and GPU milliseconds per step (CUDA
    events, graph replay)."""
    import torch
    out = {}
    modes = [("zero", scenes.WARM_ZERO, 0), ("previous", scenes.WARM_PREVIOUS, 0),
             ("learned", scenes.WARM_LEARNED, 0)]
    if gate > 0:
        modes.append(("learned_gated", scenes.WARM_LEARNED, gate))
    for name, mode, g_it in modes:
        d = dict(desc)
        d["warm_start"] = mode
        d["learned_gate"] = g_it
        stream = torch.cuda.Stream()
        with sph.Context(d, stream=stream) as g:
            if mode == scenes.WARM_LEARNED:
                g.sph_set_mlp(params)
            g.sph_steps(warmup, dt)
            g.sph_synchronize(raise_on_error=False)
            s0 = g.sph_get_stats()
            iters, err0, err = [], [], []
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            total_ms = 0.0
            for _ in range(steps):
                a.record(stream)
                g.sph_step(dt)
                b.record(stream)
                st = g.sph_get_stats()          # synchronises
                total_ms += a.elapsed_time(b)
                iters.append(st["dens_iters"])
                err0.append(st["dens_err0"])
                err.append(st["dens_err"])
            s1 = g.sph_get_stats()
        out[name] = {"density_iters_per_step": float(np.mean(iters)),
                     "divergence_iters_per_step": (s1["total_div_iters"] - s0["total_div_iters"]) / steps,
                     "first_iteration_error": float(np.mean(err0)), "final_error": float(np.mean(err)),
                     "ms_per_step": total_ms / steps}
    return out


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--samples", type=int, default=200_000)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--eval-steps", type=int, default=100)
    ap.add_argument("--out", default=None, help="write the trained parameter block (.npy)")
    args = ap.parse_args()
    t = time.perf_counter()
    f, y = generate_dataset(args.samples, args.steps)
    t_data = time.perf_counter() - t
    t = time.perf_counter()
    params, hist = train(f, y, epochs=args.epochs)
    t_train = time.perf_counter() - t
    if args.out:
        np.save(args.out, params)
    res = compare_warm_starts(scenes.dam_break_small(), params, steps=args.eval_steps)
    print(json.dumps({"samples": int(f.shape[0]), "data_s": t_data, "train_s": t_train,
                      "loss_first": float(hist[0]), "loss_last": float(hist[-1]), "compare": res}))


if __name__ == "__main__":
    main()
