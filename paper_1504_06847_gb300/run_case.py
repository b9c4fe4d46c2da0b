"""Runs the ADMM iteration on one synthetic cube (for profiling and quick checks).

  python -m paper_1504_06847_gb300.run_case --N 1024 --L 8 --iters 2 [--precision fp32|splitbf16]
      [--tile 64|32] [--J 3] [--resid]

Prints the plan's report.  The cube follows the synthetic recipe of
paper_1504_06847_gb300.synth (seeded sources, disk-array PSF, 20 dB noise).
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
    a = ap.parse_args(argv)
    c = synth.make_cube(a.N, a.L, n_sources=max(2, int(40 * (a.N / 256) ** 2)), n_antennas=128, seed=a.seed)
    plan = Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
    plan.set_option(MF_OPT_WAV_TILE, a.tile)
    prec = MF_FP32_DCT_SPLITBF16 if a.precision == "splitbf16" else MF_FP32
    plan.iterate(torch.tensor(c.y, dtype=torch.float32, device="cuda"), a.iters, wavelet_levels=a.J,
                 precision=prec, resid_every=1 if a.resid else 0, **synth.WORKLOAD_PARAMS)
    print(json.dumps(plan.report()))


if __name__ == "__main__":
    main()
