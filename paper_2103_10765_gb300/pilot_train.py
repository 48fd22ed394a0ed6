"""Training of the learned pilot on the GPU with the library's own kernels.

  python -m paper_2103_10765_gb300.pilot_train --out pilot_theta.f32

The training set is the method's own output: seeded synthetic 1024 x 1024
noisy scenes with sigma uniform in [5, 50] / 255 (synth.pilot_training_specs),
their stage-1 estimates Y1 computed by gbm3d_denoise with stages = 1 on the
whole scene, and both cut into 256 x 256 crops (so that the crops keep the
scale of the images the network serves and every target saw its full search
windows).  Training runs Adam (gbm3d_pilot_train_step) over shuffled
mini-batches with a cosine learning-rate decay; every kernel is the
library's.  The result is the flat FP32 parameter vector, written raw.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np
import torch

from . import gbm3d, synth

MID_LAYERS = 14  # 32 -> 32 layers between the 2 -> 32 and 32 -> 1 ones


def training_set(n: int, size: int = 256, seed: int = 21, device="cuda", p: gbm3d.Params | None = None,
                 full: int = 1024):
    """(Z [n, size, size], Y1 [n, size, size], sigmas): the first n crops,
    scene by scene and row-major within a scene, of full x full scenes and
    their stage-1 estimates, on the device."""
    if full % size:
        raise ValueError("the scene side must be a multiple of the crop side")
    p = (p or gbm3d.params_default()).replace(stages=1)
    per_side = full // size
    per = per_side * per_side
    specs = synth.pilot_training_specs((n + per - 1) // per, seed, full)
    Z = torch.empty((n, size, size), dtype=torch.float32, device=device)
    Y1 = torch.empty_like(Z)
    sig = []
    ws = gbm3d.workspace(full, full, p, device)
    zf = torch.empty((full, full), dtype=torch.float32, device=device)
    yf = torch.empty_like(zf)
    k = 0
    for H, W, sigma, scene in specs:
        _, noisy = synth.make_pair(H, W, sigma, scene)
        zf.copy_(torch.from_numpy(noisy))
        gbm3d.denoise(zf, sigma, p, ws, yf)
        for a in range(per_side):
            for b in range(per_side):
                if k == n:
                    break
                rows, cols = slice(a * size, (a + 1) * size), slice(b * size, (b + 1) * size)
                Z[k].copy_(zf[rows, cols])
                Y1[k].copy_(yf[rows, cols])
                sig.append(sigma)
                k += 1
    torch.cuda.synchronize()
    return Z, Y1, sig


def initial_theta(seed: int = 11) -> np.ndarray:
    """He-normal start for the network's layer shapes (9 ci inputs per output)."""
    shapes = [(9 * 2, 32)] + [(9 * 32, 32)] * MID_LAYERS + [(9 * 32, 1)]
    return synth.he_normal_params(seed, shapes).astype(np.float32)


def train(Z, Y1, sigmas, epochs: int = 240, batch: int = 16, lr: float = 3e-4, lr_min: float = 1e-5,
          seed: int = 5, theta0=None, log=None):
    """Adam over shuffled mini-batches (the order drawn from a SplitMix64
    stream); returns the trained PilotNet and the per-epoch mean losses."""
    n = Z.shape[0]
    net = gbm3d.PilotNet(initial_theta() if theta0 is None else theta0, Z.device)
    sig = torch.tensor(sigmas, dtype=torch.float32)
    steps_per_epoch = n // batch
    total = epochs * steps_per_epoch
    losses = []
    step = 0
    for ep in range(epochs):
        order = np.argsort(synth.uniforms(seed + ep, n))
        acc = torch.zeros(1, device=Z.device)
        for b in range(steps_per_epoch):
            idx = torch.from_numpy(order[b * batch:(b + 1) * batch].copy()).to(Z.device)
            rate = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / max(total, 1)))
            acc += net.train_step(Z.index_select(0, idx).contiguous(), Y1.index_select(0, idx).contiguous(),
                                  sig[idx.cpu()].tolist(), rate)
            step += 1
        losses.append(float(acc) / steps_per_epoch)
        if log:
            log(f"epoch {ep + 1}/{epochs} loss {losses[-1]:.3e}")
    return net, losses


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--n", type=int, default=2000, help="training crops (16 per 1024 x 1024 scene)")
    ap.add_argument("--epochs", type=int, default=240)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=3e-4)
    a = ap.parse_args()
    t0 = time.perf_counter()
    Z, Y1, sig = training_set(a.n)
    t1 = time.perf_counter()
    print(f"training set: {a.n} crops in {t1 - t0:.1f} s", flush=True)
    net, losses = train(Z, Y1, sig, a.epochs, a.batch, a.lr, log=lambda s: print(s, flush=True))
    torch.cuda.synchronize()
    print(f"training: {time.perf_counter() - t1:.1f} s, final loss {losses[-1]:.3e}", flush=True)
    net.theta.cpu().numpy().astype("<f4").tofile(a.out)


if __name__ == "__main__":
    main()
