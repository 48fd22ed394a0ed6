"""Runs one G-BM3D entry point on a seeded synthetic image, for profilers.

  python -m paper_2103_10765_gb300.profile_case --op match --size 1024 --reps 2

Every op first runs one whole denoise (warm-up, and to make the stage-1
estimate for stage-2 ops), then `reps` launches of the chosen entry point:
  match1 / match2   gbm3d_match on the noisy image (K1) / stage-1 estimate (K2)
  ht                gbm3d_filter_ht        wiener   gbm3d_filter_wiener
  agg1 / agg2       gbm3d_aggregate of the stage-1 / stage-2 groups
  denoise           gbm3d_denoise
  match3            gbm3d_match with the box-sum engine (K1)
  pilot             the learned pilot's forward pass (committed parameters)
  pilotgrad         its loss gradient (forward + backward) on a batch of 8
                    images of size x size (the training step's kernels)
  pnp               one plug-and-play iteration of a 4-image batch (no graph)
"""
import argparse

import torch

from paper_2103_10765_gb300 import gbm3d, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="match2")
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--sigma", type=float, default=25 / 255)
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args()
    H = W = a.size
    p = gbm3d.params_default()
    _, noisy = synth.make_pair(H, W, a.sigma, 1)
    z = torch.from_numpy(noisy).cuda()
    ws = gbm3d.workspace(H, W, p)
    y1 = gbm3d.denoise(z, a.sigma, p.replace(stages=1), ws)
    idx1, _ = gbm3d.match(z, p.k1, p)
    idx2, _ = gbm3d.match(y1, p.k2, p)
    g1, w1 = gbm3d.filter_ht(z, idx1, a.sigma, p, ws)
    g2, w2 = gbm3d.filter_wiener(z, y1, idx2, a.sigma, p)
    torch.cuda.synchronize()
    ops = {
        "match1": lambda: gbm3d.match(z, p.k1, p),
        "match2": lambda: gbm3d.match(y1, p.k2, p),
        "ht": lambda: gbm3d.filter_ht(z, idx1, a.sigma, p, ws),
        "wiener": lambda: gbm3d.filter_wiener(z, y1, idx2, a.sigma, p),
        "agg1": lambda: gbm3d.aggregate(g1, w1, idx1, H, W, p, 0.0, ws),
        "agg2": lambda: gbm3d.aggregate(g2, w2, idx2, H, W, p, p.kaiser_beta, ws),
        "denoise": lambda: gbm3d.denoise(z, a.sigma, p, ws),
        "match3": lambda: gbm3d.match(z, p.k1, p.replace(match_engine=3)),
    }
    if a.op == "pilot":
        import os

        import numpy as np
        theta = np.fromfile(os.path.join(os.path.dirname(gbm3d.__file__), "pilot_theta.f32"), dtype="<f4")
        net = gbm3d.PilotNet(theta, z.device)
        zb = z[None].contiguous()
        ops["pilot"] = lambda: net.forward(zb, [a.sigma])
    if a.op == "pilotgrad":
        import os

        import numpy as np
        theta = np.fromfile(os.path.join(os.path.dirname(gbm3d.__file__), "pilot_theta.f32"), dtype="<f4")
        net = gbm3d.PilotNet(theta, z.device)
        zb = torch.stack([torch.from_numpy(synth.make_pair(H, W, a.sigma, 20 + i)[1]) for i in range(8)]).cuda()
        yb = zb.clone()
        ops["pilotgrad"] = lambda: net.loss_grad(zb, yb, [a.sigma] * 8)
    if a.op == "pnp":
        import numpy as np
        t = np.arange(9) - 4.0
        g = np.exp(-0.5 * (t / 1.6) ** 2)
        g = (g / g.sum()).astype(np.float32)
        ys = [torch.from_numpy(synth.make_blur_pair(h, w, 0.1, 7)[1]).cuda() for h, w in ((H, W), (H // 2, W), (H, W // 2), (H // 2, W // 2))]
        plan = gbm3d.PnpPlan(ys, [0.1] * 4, g, p, gbm3d.PnpParams(iters=1, use_graph=0, autotune=0))
        ops["pnp"] = plan.run
    for _ in range(a.reps):
        ops[a.op]()
    torch.cuda.synchronize()
    print(f"profile_case {a.op} {H}x{W} reps={a.reps} ok")


if __name__ == "__main__":
    main()
