"""Runs the ADMM iteration on one synthetic cube (for profiling and quick checks).

  python -m paper_1504_06847_gb300.run_case --N 1024 --L 8 --iters 2 [--precision fp32|splitbf16]
      [--tile 64|32] [--J 3] [--resid]
  python -m paper_1504_06847_gb300.run_case --batch 16 --iters 100      # batched form, timed
  python -m paper_1504_06847_gb300.run_case --N 256 --L 32 --iters 20 --backward   # differentiable form, timed
  python -m paper_1504_06847_gb300.run_case --N 1024 --L 64 --xstep    # step I: ours vs cuFFT (reference point)

Prints the plan's report (or, for --batch / --backward, the measured times as
JSON).  The cubes follow the synthetic recipe of paper_1504_06847_gb300.synth
(seeded sources, disk-array PSF, 20 dB noise).
"""

from __future__ import annotations

import argparse
import json

import torch

from . import MF_FP32, MF_FP32_DCT_SPLITBF16, MF_OPT_WAV_TILE, Plan, synth


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--L", type=int, default=8)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--J", type=int, default=3)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "splitbf16"])
    ap.add_argument("--tile", type=int, default=64, choices=[64, 32])
    ap.add_argument("--resid", action="store_true")
    ap.add_argument("--seed", type=int, default=9)
    ap.add_argument("--batch", type=int, default=0, help="time the batched form on this many uneven cubes")
    ap.add_argument("--backward", action="store_true", help="time forward and reverse pass of --iters iterations")
    ap.add_argument("--xstep", action="store_true", help="time step I against a cuFFT (torch.fft) reference point")
    a = ap.parse_args(argv)
    if a.xstep:
        return run_xstep(a)
    if a.batch:
        return run_batch(a)
    if a.backward:
        return run_backward(a)
    c = synth.make_cube(a.N, a.L, n_sources=max(2, int(40 * (a.N / 256) ** 2)), n_antennas=128, seed=a.seed)
    plan = Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    plan.set_option(MF_OPT_WAV_TILE, a.tile)
    prec = MF_FP32_DCT_SPLITBF16 if a.precision == "splitbf16" else MF_FP32
    plan.iterate(torch.tensor(c.y, dtype=torch.float32, device="cuda"), a.iters, wavelet_levels=a.J,
                 precision=prec, resid_every=1 if a.resid else 0, **synth.WORKLOAD_PARAMS)
    print(json.dumps(plan.report()))


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_batch(a):
    """Batched form: every cube's iterations in one graph launch, against the
    same cubes iterated one plan after the other."""
    from . import batch_iterate

    cubes = synth.batch_workload(a.batch)
    plans = [Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda")) for c in cubes]
    ys = [torch.tensor(c.y, dtype=torch.float32, device="cuda") for c in cubes]
    prm = synth.WORKLOAD_PARAMS
    vox = sum(c.y.size for c in cubes)
    batch_iterate(plans, ys, 2, **prm)
    s, e = _events()
    s.record()
    batch_iterate(plans, ys, a.iters, **prm)
    e.record()
    torch.cuda.synchronize()
    t_batch = s.elapsed_time(e)
    for p, y in zip(plans, ys):
        p.iterate(y, 2, **prm)
    s.record()
    for p, y in zip(plans, ys):
        p.iterate(y, a.iters, **prm)
    e.record()
    torch.cuda.synchronize()
    t_solo = s.elapsed_time(e)
    print(json.dumps({"form": "batched", "cubes": a.batch, "shapes": synth.batch_shapes(a.batch), "iters": a.iters,
                      "voxels": vox, "batch_ms": t_batch, "batch_voxel_it_per_s": vox * a.iters / (t_batch * 1e-3),
                      "sequential_ms": t_solo, "sequential_voxel_it_per_s": vox * a.iters / (t_solo * 1e-3)}))


def run_backward(a):
    """Differentiable form: forward of --iters iterations from the zero state and
    the reverse pass (tied rho) for L = ||X_K - X_true||^2."""
    c = synth.make_cube(a.N, a.L, n_sources=max(2, int(40 * (a.N / 256) ** 2)), n_antennas=256, seed=a.seed)
    plan = Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
    truth = torch.tensor(c.sky, dtype=torch.float32, device="cuda")
    prm = synth.WORKLOAD_PARAMS
    kw = dict(mu_eps=prm["mu_eps"], mu_s=prm["mu_s"], mu_nu=prm["mu_nu"])
    plan.iterate(y, a.iters, rho_P=1.0, rho_T=1.0, rho_V=1.0, rho_S=1.0, **kw)
    g = 2 * (plan.x() - truth)
    plan.backward(y, a.iters, g, rho=1.0, **kw)
    s, e = _events()
    s.record()
    plan.iterate(y, a.iters, rho_P=1.0, rho_T=1.0, rho_V=1.0, rho_S=1.0, **kw)
    e.record()
    torch.cuda.synchronize()
    t_fwd = s.elapsed_time(e)
    s.record()
    _, dms, dmn, dr = plan.backward(y, a.iters, g, rho=1.0, **kw)
    e.record()
    torch.cuda.synchronize()
    t_bwd = s.elapsed_time(e)
    vox = c.y.size
    print(json.dumps({"form": "differentiable", "N": a.N, "L": a.L, "iters": a.iters, "forward_ms": t_fwd,
                      "backward_ms": t_bwd, "backward_over_forward": t_bwd / t_fwd,
                      "forward_voxel_it_per_s": vox * a.iters / (t_fwd * 1e-3),
                      "dL_dmu_s": dms, "dL_dmu_nu": dmn, "dL_drho": dr}))


def run_xstep(a):
    """Step I (X = c + g F(b), inverse FFT) of this library's kernels, against the
    same filter applied with cuFFT through torch.fft (a reference point only: it
    is not on this library's path)."""
    c = synth.make_cube(a.N, a.L, n_sources=max(2, int(40 * (a.N / 256) ** 2)), n_antennas=128, seed=a.seed)
    prm = synth.WORKLOAD_PARAMS
    psf = torch.tensor(c.psf, dtype=torch.float32, device="cuda")
    y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
    plan = Plan(psf)
    plan.iterate(y, 3, **prm)
    plan.set_timing(True)
    plan.iterate(y, 10, warm_start=1, **prm)
    t = plan.timing()
    plan.set_timing(False)
    ours = sum(t[k][0] / max(t[k][1], 1) for k in ("rows_fwd", "cols_solve", "rows_inv"))
    # reference: rfft2 / filter / irfft2 on the same shapes (FP32 complex)
    rho_bar = prm["mu_eps"] + prm["rho_P"] + prm["rho_S"] + 9 * prm["rho_T"]
    hh = torch.fft.rfft2(torch.fft.ifftshift(psf, dim=(-2, -1)))
    g = 1.0 / (hh.abs() ** 2 + rho_bar)
    cc = torch.conj(hh) * torch.fft.rfft2(y) * g
    b = torch.randn_like(y)
    xs = torch.empty_like(y)

    def ref():
        xs.copy_(torch.fft.irfft2(cc + g * torch.fft.rfft2(b), s=(a.N, a.N)))

    for _ in range(3):
        ref()
    s, e = _events()
    s.record()
    for _ in range(10):
        ref()
    e.record()
    torch.cuda.synchronize()
    cufft = s.elapsed_time(e) / 10
    vox = c.y.size
    print(json.dumps({"form": "step I", "N": a.N, "L": a.L, "ours_ms": ours, "cufft_torch_ms": cufft,
                      "ours_voxels_per_s": vox / (ours * 1e-3), "cufft_voxels_per_s": vox / (cufft * 1e-3),
                      "kernels": {k: t[k][0] / max(t[k][1], 1) for k in ("rows_fwd", "cols_solve", "rows_inv")}}))


if __name__ == "__main__":
    main()
