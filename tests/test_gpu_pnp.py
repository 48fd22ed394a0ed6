"""GPU: plug-and-play ADMM deconvolution (gbm3d_pnp_*) against the FP64 oracle
(oracle/pnp.py, readings P1-P6).

  * x-update: with sigma_n = 0 the denoiser is the identity up to FP32
    rounding, so the loop is the exact proximal least-squares iteration;
    compared element by element with the oracle's DFT solve.  Tolerance: the
    FP32 transforms carry about 1e-6 relative rounding (sums of up to 2 x 1024
    products), which the division by lam^2 + rho >= rho amplifies by up to
    1 / rho in every iteration: max-abs <= 5e-6 * iters * (1 + 1/rho);
  * with G-BM3D: PSNR within 0.05 dB of the oracle after a few iterations
    and after the full 50-iteration loop;
  * the graph-captured batch equals the plain per-image launches, and every
    autotuned tile shape, bit for bit.
"""
import os

import numpy as np
import pytest

from paper_2103_10765_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2103_10765_gb300 import gbm3d  # noqa: E402

NT = os.cpu_count() or 4
DEV = torch.device("cuda:0")


def psf1d(size=9, std=1.6):
    t = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-0.5 * (t / std) ** 2)
    return (g / g.sum()).astype(np.float32)


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def run_plan(ys, sigmas, q, p=None, g=None):
    plan = gbm3d.PnpPlan([gpu(y) for y in ys], sigmas, psf1d() if g is None else g, p, q)
    outs = [o.cpu().numpy() for o in plan.run()]
    torch.cuda.synchronize()
    plan.close()
    return outs


def oracle_psf(g):
    return np.outer(g.astype(np.float64), g.astype(np.float64))


@pytest.mark.parametrize("shape,rho,iters", [((64, 72), 0.1, 1), ((96, 136), 0.05, 3), ((120, 64), 1.0, 2)])
def test_x_update_exact_with_identity_denoiser(pnp_orc, shape, rho, iters):
    clean, y = synth.make_blur_pair(*shape, 0.05, 4)
    out = run_plan([y], [0.0], gbm3d.PnpParams(iters=iters, rho=rho))[0]
    g = psf1d()
    h = oracle_psf(g)  # the same FP32 taps the library received, in FP64

    def ident(img, s):
        return img
    ref = y.astype(np.float64)
    hty = pnp_orc.blur_adjoint(ref, h)
    v, u = ref.copy(), np.zeros_like(ref)
    for _ in range(iters):
        x = pnp_orc.x_update(hty + rho * (v - u), h, rho)
        v = ident(x + u, 0.0)
        u = u + x - v
    assert np.abs(out - v).max() <= 5e-6 * iters * (1 + 1 / rho)


def test_gbm3d_denoiser_psnr_parity(pnp_orc, orc):
    specs = [(64, 72, 10 / 255, 11), (96, 64, 25 / 255, 12), (80, 80, 40 / 255, 13)]
    pairs = [synth.make_blur_pair(h, w, s, seed) for h, w, s, seed in specs]
    q = gbm3d.PnpParams(iters=3)
    outs = run_plan([y for _, y in pairs], [s for _, _, s, _ in specs], q)
    for (clean, y), (h, w, s, _), out in zip(pairs, specs, outs):
        ref = pnp_orc.pnp_admm(y, s, pnp_orc.PnpParams(iters=3, rho=0.1), nthreads=NT)
        pg, po = orc.psnr(out, clean), orc.psnr(ref, clean)
        assert abs(pg - po) <= 0.05, (h, w, pg, po)
        assert pg > orc.psnr(y, clean) + 1.0


def test_full_length_loop_psnr_parity(pnp_orc, orc):
    """The benchmark's 50-iteration loop (rho 0.1, the graph-captured batch)
    against the oracle's loop on two images of 128-160 pixels: PSNR within
    0.05 dB after every one of the 50 denoiser calls has fed the next
    x-update."""
    specs = [(128, 136, 12 / 255, 21), (160, 152, 40 / 255, 23)]
    pairs = [synth.make_blur_pair(h, w, s, seed) for h, w, s, seed in specs]
    q = gbm3d.PnpParams(iters=50)
    outs = run_plan([y for _, y in pairs], [s for _, _, s, _ in specs], q)
    for (clean, y), (h, w, s, _), out in zip(pairs, specs, outs):
        ref = pnp_orc.pnp_admm(y, s, pnp_orc.PnpParams(iters=50, rho=0.1), nthreads=NT)
        pg, po = orc.psnr(out, clean), orc.psnr(ref, clean)
        print(f"{h}x{w} sigma {s * 255:.0f}: GPU {pg:.4f} dB, oracle {po:.4f} dB, blurred {orc.psnr(y, clean):.4f}")
        assert abs(pg - po) <= 0.05, (h, w, pg, po)
        assert pg > orc.psnr(y, clean) + 1.0


def test_graph_equals_plain_and_every_tile_shape():
    specs = synth.pnp_batch_specs(6, seed=9, lo=128, hi=264)
    pairs = [synth.make_blur_pair(h, w, s, seed) for h, w, s, seed in specs]
    ys, sig = [y for _, y in pairs], [s for _, _, s, _ in specs]
    a = run_plan(ys, sig, gbm3d.PnpParams(iters=2, use_graph=1, autotune=1))
    b = run_plan(ys, sig, gbm3d.PnpParams(iters=2, use_graph=0, autotune=0))
    for x, z in zip(a, b):
        assert np.array_equal(x, z)


def test_rerun_is_deterministic_and_tiles_are_recorded():
    specs = synth.pnp_batch_specs(3, seed=5, lo=128, hi=200)
    ys = [gpu(synth.make_blur_pair(h, w, s, seed)[1]) for h, w, s, seed in specs]
    plan = gbm3d.PnpPlan(ys, [s for _, _, s, _ in specs], psf1d(), q=gbm3d.PnpParams(iters=2))
    first = [o.clone() for o in plan.run()]
    second = plan.run()
    torch.cuda.synchronize()
    for x, z in zip(first, second):
        assert torch.equal(x, z)
    for i in range(3):
        a, b = plan.gemm_configs(i)
        assert 0 <= a < 2 and 0 <= b < 2
    plan.close()


def test_full_batch_runs_and_restores():
    """The 64-image batch of uneven sizes 128..1024 (seed 7), a few iterations:
    finite results, every image better than its blurred noisy input."""
    specs = synth.pnp_batch_specs()
    pairs = [synth.make_blur_pair(h, w, s, seed) for h, w, s, seed in specs]
    outs = run_plan([y for _, y in pairs], [s for _, _, s, _ in specs], gbm3d.PnpParams(iters=3))
    for (clean, y), out in zip(pairs, outs):
        assert np.isfinite(out).all()
        mse_y = np.mean((y.astype(np.float64) - clean) ** 2)
        mse_o = np.mean((out.astype(np.float64) - clean) ** 2)
        assert mse_o < mse_y
