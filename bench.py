#!/usr/bin/env python
"""Benchmark of the spatio-spectral ADMM iteration (arXiv:1504.06847, Algorithm 1).

One step = one full ADMM iteration (steps I-VI: FFT X-solve, positivity,
wavelet and DCT soft-thresholds, S update, duals) over the 1024 x 1024 x 64
synthetic cube, through the C ABI.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Besides the contract's fields the line carries the batched form (16 uneven
cubes, 100 iterations each, one graph launch), the differentiable form
(20 unrolled iterations at 256 x 256 x 32, forward and reverse pass), step I
against a cuFFT reference point, and the FP64 oracle on the host cores
(3 iterations of the full workload, a 1-thread run, the paper's settings at
256 x 256 x 15).

Multi-GPU runs (torchrun, one rank per GPU) solve one independent replica of
the cube per rank (the path has no exchange between cubes): weak scaling.
The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores instead, one Algorithm-1 iteration of the workload per step.

Single cases for profiling (no JSON contract line):
  python bench.py --case plain --N 1024 --L 8 --iters 2 [--precision fp32|splitbf16] [--tile 64|32] [--resid]
                   [--spectral-mask 1|2|3]
  python bench.py --case linear|vis --N 512 --L 32 --iters 2 [--cg-iters 10] [--resid]
  python bench.py --case batch [--batch 16] [--iters 100]
  python bench.py --case backward --N 256 --L 32 --iters 20
  python bench.py --case xstep --N 1024 --L 64
  python bench.py --case configs        (64x64x8 FP64/FP32 and 256x256x32 FP32 in full, with the oracle)
"""

from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("ADMM voxel-iterations/sec at 1024²×64 bands and % HBM roofline, "
          "FP32/split-BF16 vs FP64")
UNIT = "voxel-it/s"
WORKLOAD = "1024x1024x64"
SAMPLE = dict(N=256, L=64, n_sources=19, n_antennas=512, seed=3, point_frac=0.2)
SAMPLE_NAME = "256x256x64 cube from the same recipe (seed 3, 19 sources, 512 antennas)"
FALLBACK_HBM_GBS = 6800.0
# Minimum HBM bytes per voxel-iteration of the whole step (FP32, 8 distinct bases):
# 12 persistent arrays read+written (96 B), X (12 B), b (16 B), FFT intermediates (16 B),
# Fourier constants (6 B).
STEP_ALG_BYTES_PER_VOXEL = 146.0
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of each kernel at the
# benchmark workload (None where no capture of the current kernel exists).  Level 1:
# captured at 1024 x 1024 x 8 (541.3 MB per launch) and scaled by the 8x bands.
NCU_TRAFFIC_PER_LAUNCH = {"wav_level1": 8 * 539.6e6}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def alg_bytes_per_iteration(N, L, nd=8, J=3, esz=4):
    """Algorithmic HBM bytes of each kernel class over one iteration (sum of its launches)."""
    V = N * N * L
    out = {
        "rows_fwd": 2 * V * esz,                      # b in, packed half spectrum out
        "cols_solve": 3.5 * V * esz,                  # spectrum in/out, c (complex), g (real)
        "rows_inv": 2 * V * esz,                      # spectrum in, X out
        "spectral": 10 * V * esz,                     # X; Gamma_P, S, Gamma_V, Gamma_S in/out; b out
    }
    ll = 0.0
    for j in range(1, J):
        src = V if j == 1 else nd * V / 4 ** (j - 1)
        ll += (src + nd * V / 4 ** j) * esz
    out["wav_ll"] = ll
    lvl1 = (V + 2 * V + 2 * nd * (0.75 if J > 1 else 1.0) * V + (nd * V / 4 if J > 1 else 0)) * esz
    out["wav_level1"] = lvl1
    lj = 0.0
    for j in range(2, J + 1):
        size = V / 4 ** (j - 1)
        coarsest = j == J
        lj += (nd * size + 2 * nd * (1.0 if coarsest else 0.75) * size + (0 if coarsest else nd * size / 4)
               + nd * size) * esz
    out["wav_levelj"] = lj
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        if shutil.which("nvidia-smi") is None:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits", "-lms", "200"],
                                     stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


PAPER_SAMPLE = dict(N=256, L=15, n_sources=40, n_antennas=256, seed=15)
PAPER_SAMPLE_NAME = "256x256x15 cube from the same recipe (seed 15, 40 sources, 256 antennas), the paper's Section 4 settings"
ORACLE_SAMPLES = {"256x256x64": (SAMPLE, "WORKLOAD_PARAMS"), "256x256x15-paper": (PAPER_SAMPLE, "PAPER_PARAMS"),
                  "64x64x8": (None, "WORKLOAD_PARAMS"), "256x256x32": (None, "WORKLOAD_PARAMS")}


def _oracle_rate(pb, n_iter):
    """voxel-it/s of n_iter oracle iterations after one untimed one, and the seconds taken."""
    st = pb.zero_state()
    pb.iterate(st, 1)
    t0 = time.perf_counter()
    pb.iterate(st, n_iter)
    el = time.perf_counter() - t0
    return pb.N * pb.N * pb.L * n_iter / el, el


def oracle_case(name, n_iter):
    """The oracle on one of the small samples (the 1-thread leg runs this in a child process)."""
    import oracle
    from paper_1504_06847_gb300 import synth

    kw, params = ORACLE_SAMPLES[name]
    c = synth.make_cube(**kw) if kw is not None else synth.workload(name)
    v, el = _oracle_rate(oracle.Problem(c.psf, c.y, getattr(synth, params)), n_iter)
    return {"value": v, "seconds": el, "iters": n_iter}


def cpu_baseline(cube):
    """The FP64 oracle as it stands on the host cores: the benchmarked workload
    itself over 3 iterations (the line's value), the 256 x 256 x 64 sample of
    the same recipe on every core and on one, and the paper's own settings at
    256 x 256 x 15 (the shape class of its Section 4 timing)."""
    cores = len(os.sched_getaffinity(0))
    os.environ["OMP_NUM_THREADS"] = str(cores)
    import oracle
    from paper_1504_06847_gb300 import synth

    V = cube.y.size
    full, full_s = _oracle_rate(oracle.Problem(cube.psf, cube.y, synth.WORKLOAD_PARAMS), 3)
    sample = oracle_case("256x256x64", 20)
    paper = oracle_case("256x256x15-paper", 40)
    one = None
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--case", "oracle", "--sample",
                              "256x256x64", "--iters", "2"], env=env, capture_output=True, text=True, timeout=300)
        one = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal
        one = {"error": str(e)[:200]}
    return {"value": full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"3 FP64 Algorithm-1 iterations of the {WORKLOAD} workload itself ({full_s:.1f} s, "
                      f"after one untimed iteration); value = {V} voxels x 3 / time",
            "sample_256x256x64": {"value": sample["value"], "cores": cores, "iters": sample["iters"],
                                  "note": SAMPLE_NAME},
            "one_thread_256x256x64": dict(one, cores=1, note=SAMPLE_NAME),
            "paper_settings_256x256x15": {"value": paper["value"], "cores": cores, "iters": paper["iters"],
                                          "note": PAPER_SAMPLE_NAME}}


def max_over_ranks(seconds, dist=None, device="cpu"):
    """The slowest rank's time (every rank gets it); the rank's own time without a group."""
    if dist is None:
        return float(seconds)
    import torch

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds, world):
    """Units all ranks processed (each rank solves its own replica) per second of the slowest rank."""
    return world * units_per_rank / seconds


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, one Algorithm-1
    iteration per step of the benchmarked workload itself when the run stays
    within a few minutes (K + W <= 40 steps of ~4 s), else of the 256 x 256 x 64
    sample of the same recipe."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    os.environ["OMP_NUM_THREADS"] = str(cores)
    import oracle
    from paper_1504_06847_gb300 import synth

    full = args.steps + args.warmup <= 40
    c = synth.workload(WORKLOAD) if full else synth.make_cube(**SAMPLE)
    name = f"the {WORKLOAD} workload" if full else f"the {SAMPLE_NAME}"
    pb = oracle.Problem(c.psf, c.y, synth.WORKLOAD_PARAMS)
    st = pb.zero_state()
    for _ in range(args.warmup):
        pb.iterate(st, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pb.iterate(st, 1)
    el = time.perf_counter() - t0
    V = c.y.size
    value = V * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": name, "n_iter_per_step": 1,
                                            "same_config": full},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one FP64 Algorithm-1 iteration of {name} per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure_forms(stream, xstep_ms=None):
    """The batched and differentiable forms (and step I against cuFFT), timed
    with CUDA events on `stream`."""
    import torch

    import paper_1504_06847_gb300 as mf
    from paper_1504_06847_gb300 import autotune, synth

    prm = synth.WORKLOAD_PARAMS
    out = {}
    with torch.cuda.stream(stream):
        # batched form: 16 uneven cubes, 100 iterations each, one graph launch
        cubes = synth.batch_workload(16)
        plans = [mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda")) for c in cubes]
        ys = [torch.tensor(c.y, dtype=torch.float32, device="cuda") for c in cubes]
        vox = sum(c.y.size for c in cubes)
        n_it = 100
        kw = dict(prm, stream=stream.cuda_stream)
        # each cube's wavelet tile picked by the autotuner (timed trials, state restored)
        tiles = [autotune.tune(p_, y, cache=None, **kw)["wav_tile"] for p_, y in zip(plans, ys)]
        s, e = _events(torch)
        # first call: capture and instantiation of the graph, then its launch
        s.record(stream)
        mf.batch_iterate(plans, ys, n_it, **kw)
        e.record(stream)
        stream.synchronize()
        t_first = s.elapsed_time(e)
        # the same call again relaunches the captured graph
        s.record(stream)
        mf.batch_iterate(plans, ys, n_it, **kw)
        e.record(stream)
        stream.synchronize()
        t_batch = s.elapsed_time(e)
        s.record(stream)
        for p_, y in zip(plans, ys):
            p_.iterate(y, n_it, **kw)
        e.record(stream)
        stream.synchronize()
        t_seq = s.elapsed_time(e)
        out["batched"] = {"cubes": len(cubes), "shapes": synth.batch_shapes(16), "iters_each": n_it, "voxels": vox,
                          "ms": t_batch, "voxel_it_per_s": vox * n_it / (t_batch * 1e-3),
                          "first_call_ms": t_first, "wav_tiles": tiles,
                          "note": "ms: a repeated identical call (the captured graph relaunched); first_call_ms "
                                  "includes capturing and instantiating the graph",
                          "sequential_ms": t_seq, "sequential_voxel_it_per_s": vox * n_it / (t_seq * 1e-3),
                          "dtype": "f32"}
        for p_ in plans:
            p_.close()
        del plans, ys
        # differentiable form: 20 unrolled iterations at 256 x 256 x 32, forward + reverse
        c = synth.workload("256x256x32")
        K = 20
        plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
        y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
        truth = torch.tensor(c.sky, dtype=torch.float32, device="cuda")
        tied = dict(mu_eps=prm["mu_eps"], mu_s=prm["mu_s"], mu_nu=prm["mu_nu"])
        rho = dict(rho_P=1.0, rho_T=1.0, rho_V=1.0, rho_S=1.0)
        plan.iterate(y, K, stream=stream.cuda_stream, **tied, **rho)
        g = 2 * (plan.x() - truth)
        plan.backward(y, K, g, rho=1.0, stream=stream.cuda_stream, **tied)  # allocates the checkpoints
        s.record(stream)
        plan.iterate(y, K, stream=stream.cuda_stream, **tied, **rho)
        e.record(stream)
        stream.synchronize()
        t_fwd = s.elapsed_time(e)
        s.record(stream)
        plan.backward(y, K, g, rho=1.0, stream=stream.cuda_stream, **tied)
        e.record(stream)
        stream.synchronize()
        t_bwd = s.elapsed_time(e)
        out["differentiable"] = {"N": 256, "L": 32, "unrolled_iters": K, "forward_ms": t_fwd,
                                 "forward_and_reverse_ms": t_bwd,
                                 "note": "the reverse pass re-runs the forward with per-iteration checkpoints",
                                 "voxel_it_per_s_forward_and_reverse": c.y.size * K / (t_bwd * 1e-3),
                                 "dtype": "f32"}
        plan.close()
        # the paper's first simulation: 256 x 256 x 15, its settings, its 350 iterations
        c = synth.two_gaussians()
        plan_e1 = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
        y_e1 = torch.tensor(c.y, dtype=torch.float32, device="cuda")
        kw_e1 = dict(synth.PAPER_PARAMS, stream=stream.cuda_stream)
        plan_e1.iterate(y_e1, 3, **kw_e1)
        s.record(stream)
        plan_e1.iterate(y_e1, synth.PAPER_ITERS, **kw_e1)
        e.record(stream)
        stream.synchronize()
        t_e1 = s.elapsed_time(e)
        out["paper_e1_256x256x15"] = {"iters": synth.PAPER_ITERS, "ms": t_e1,
                                      "voxel_it_per_s": c.y.size * synth.PAPER_ITERS / (t_e1 * 1e-3),
                                      "params": "Section 4 settings", "dtype": "f32",
                                      "note": "the paper reports about 1.5 h on 15 CPU cores for a 256x256x15 run "
                                              "of 350 iterations"}
        plan_e1.close()
    if xstep_ms is not None:
        out["xstep_vs_cufft"] = xstep_reference(stream, xstep_ms)
    return out


# Bytes per voxel of the N x N cube moved by one conjugate-gradient iteration of
# step I (FP32).  One zero-padded 2N convolution with its known zeros and
# discarded outputs skipped: row transform 4 in (the N x N image) + 8 out (the
# first N rows' half spectra), column pass 8 in + 16 (the 2N x N complex
# transfer function) + 8 out (first N rows), inverse rows 8 in + 4 out
# ([0,N)^2): 56.  The CG vector updates (q; X and r; p) move 48.  Linear
# convolution: two convolutions per operator application; visibilities: one.
CG_BYTES = {"linear": 2 * 56 + 48, "vis": 56 + 48}
# the spectral step with the Chebyshev basis added: X in; Gamma_P, S, Gamma_V,
# Gamma_V2, Gamma_S and S in the Chebyshev basis in and out; b out
SPECTRAL_B2_BYTES = 4 + 6 * 8 + 4


def measure_widened_rows(stream, plan, y, peak):
    """The rows beyond the benchmark's path, each timed with CUDA events (per-kernel
    events inside the library) on `stream`: the Chebyshev spectral dictionary and
    the spectral-index fit on the benchmark cube, step I by conjugate gradients for
    a linear convolution and for visibilities at 512 x 512 x 32."""
    import torch

    import paper_1504_06847_gb300 as mf
    from paper_1504_06847_gb300 import synth

    prm = synth.WORKLOAD_PARAMS
    out = {}
    N, L = plan.N, plan.L
    V = N * N * L
    with torch.cuda.stream(stream):
        # DCT alone (FP32) and DCT + Chebyshev, 10 iterations each, same cube
        rows = {}
        for mask in (1, 3):
            kw = dict(prm, stream=stream.cuda_stream, precision=mf.MF_FP32, spectral_mask=mask)
            plan.iterate(y, 2, **kw)
            plan.set_timing(True)
            s, e = _events(torch)
            s.record(stream)
            plan.iterate(y, 10, **dict(kw, warm_start=1))
            e.record(stream)
            stream.synchronize()
            t = plan.timing()
            plan.set_timing(False)
            sp_ms, sp_n = t["spectral"]
            b = (SPECTRAL_B2_BYTES if mask == 3 else 40) * V
            rows[mask] = {"ms_per_iteration": s.elapsed_time(e) / 10, "spectral_ms_per_launch": sp_ms / sp_n,
                          "spectral_alg_bytes_per_launch": b,
                          "spectral_achieved_gbs": b / (sp_ms / sp_n * 1e-3) / 1e9,
                          "spectral_frac": b / (sp_ms / sp_n * 1e-3) / 1e9 / peak}
        out["chebyshev_dictionary"] = {"workload": f"{N}x{N}x{L}", "dct_only_fp32": rows[1],
                                       "dct_and_chebyshev_fp32": rows[3], "dtype": "f32"}
        # spectral-index fit of the reconstructed cube
        x = plan.x()
        nu = 1.0 + np.arange(L) / (L - 1)
        mf.spectral_index(x, nu, stream=stream.cuda_stream)
        s, e = _events(torch)
        s.record(stream)
        for _ in range(10):
            mf.spectral_index(x, nu, stream=stream.cuda_stream)
        e.record(stream)
        stream.synchronize()
        t_si = s.elapsed_time(e) / 10
        b = (L + 3) * N * N * 4
        out["spectral_index"] = {"workload": f"{N}x{N}x{L}", "ms": t_si, "alg_bytes": b,
                                 "achieved_gbs": b / (t_si * 1e-3) / 1e9, "frac": b / (t_si * 1e-3) / 1e9 / peak}
        # step I by conjugate gradients: linear convolution and visibilities
        n2, l2, cg, n_it = 512, 32, 10, 5
        c = synth.make_cube(n2, l2, n_sources=40, n_antennas=128, seed=12)
        lin = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"), linear=True)
        yl = torch.tensor(c.y, dtype=torch.float32, device="cuda")
        cv = synth.make_visibilities(n2, l2, n_sources=40, n_antennas=128, seed=13, random_weights=True)
        t0 = time.perf_counter()
        vis = mf.Plan.from_visibilities(n2, [torch.tensor(q, dtype=torch.float32, device="cuda") for q in cv.uv],
                                        [torch.tensor(w, dtype=torch.float32, device="cuda") for w in cv.weights])
        torch.cuda.synchronize()
        t_create = (time.perf_counter() - t0) * 1e3
        yv = torch.tensor(np.concatenate(cv.vis).astype(np.complex64), device="cuda")
        for name, p_, yy in (("linear", lin, yl), ("vis", vis, yv)):
            kw = dict(prm, stream=stream.cuda_stream, cg_iters=cg)
            p_.iterate(yy, 2, **kw)
            p_.set_timing(True)
            s, e = _events(torch)
            s.record(stream)
            p_.iterate(yy, n_it, **kw)
            e.record(stream)
            stream.synchronize()
            t = p_.timing()
            p_.set_timing(False)
            v2 = n2 * n2 * l2
            cg_ms = t["cg"][0] / n_it
            b = (cg + 1) * CG_BYTES[name] * v2
            row = {"workload": f"{n2}x{n2}x{l2}", "cg_iters": cg, "ms_per_iteration": s.elapsed_time(e) / n_it,
                   "step_I_ms": cg_ms, "step_I_alg_bytes": b, "step_I_achieved_gbs": b / (cg_ms * 1e-3) / 1e9,
                   "step_I_frac": b / (cg_ms * 1e-3) / 1e9 / peak,
                   "per_call_setup_ms": t["setup"][0] / max(1, t["setup"][1]),
                   "voxel_it_per_s": v2 * n_it / (s.elapsed_time(e) * 1e-3), "dtype": "f32"}
            if name == "vis":
                row.update({"visibilities": int(yv.shape[0]), "plan_create_ms": t_create,
                            "note": "per_call_setup_ms is the gridded dirty image Re(Phi^H W y)"})
            out[f"{name}_cg"] = row
        lin.close()
        vis.close()
    return out


def xstep_reference(stream, ours_ms):
    """Step I of the benchmarked cube with cuFFT (torch.fft: rfft2, the filter,
    irfft2), a reference point only: it is not on this library's path."""
    import torch

    from paper_1504_06847_gb300 import synth

    c = synth.workload(WORKLOAD)
    prm = synth.WORKLOAD_PARAMS
    N = c.y.shape[-1]
    with torch.cuda.stream(stream):
        psf = torch.tensor(c.psf, dtype=torch.float32, device="cuda")
        y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
        rho_bar = prm["mu_eps"] + prm["rho_P"] + prm["rho_S"] + 9 * prm["rho_T"]
        hh = torch.fft.rfft2(torch.fft.ifftshift(psf, dim=(-2, -1)))
        g = 1.0 / (hh.abs() ** 2 + rho_bar)
        cc = torch.conj(hh) * torch.fft.rfft2(y) * g
        b = torch.randn_like(y)
        xs = torch.empty_like(y)

        def ref():
            xs.copy_(torch.fft.irfft2(cc + g * torch.fft.rfft2(b), s=(N, N)))

        for _ in range(3):
            ref()
        s, e = _events(torch)
        s.record(stream)
        for _ in range(10):
            ref()
        e.record(stream)
        stream.synchronize()
    cufft = s.elapsed_time(e) / 10
    return {"ours_ms": ours_ms, "cufft_torch_ms": cufft, "ours_over_cufft": ours_ms / cufft}


def _oracle_one_thread(name, n_iter):
    """The oracle on one core, in a child process (OpenMP reads its thread count at start)."""
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--case", "oracle", "--sample", name,
                              "--iters", str(n_iter)], env=env, capture_output=True, text=True, timeout=600)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal
        return {"error": str(e)[:200]}


def measure_configs(stream):
    """The small configurations in full: 64 x 64 x 8 (50 iterations, FP64 and FP32
    plans) and 256 x 256 x 32 (100 iterations, FP32), each timed with CUDA events
    after 3 warm-up iterations, X compared with the FP64 oracle's after the same
    iterations, and the oracle timed on every core and on one."""
    import torch

    import oracle
    import paper_1504_06847_gb300 as mf
    from paper_1504_06847_gb300 import autotune, synth

    cores = len(os.sched_getaffinity(0))
    os.environ["OMP_NUM_THREADS"] = str(cores)
    peak, _ = measured_peak()
    prm = synth.WORKLOAD_PARAMS
    out = []
    for name, dtype, n_iter, one_iters in (("64x64x8", torch.float64, 50, 50), ("64x64x8", torch.float32, 50, None),
                                           ("256x256x32", torch.float32, 100, 3)):
        c = synth.workload(name)
        V = c.y.size
        with torch.cuda.stream(stream):
            plan = mf.Plan(torch.tensor(c.psf, dtype=dtype, device="cuda"))
            y = torch.tensor(c.y, dtype=dtype, device="cuda")
            kw = dict(prm, stream=stream.cuda_stream)
            tile = autotune.tune(plan, y, cache=None, **kw)["wav_tile"]
            plan.iterate(y, 3, **kw)
            s, e = _events(torch)
            s.record(stream)
            plan.iterate(y, n_iter, **kw)
            e.record(stream)
            stream.synchronize()
            ms = s.elapsed_time(e)
            x = plan.x().double().cpu().numpy()
            plan.close()
        pb = oracle.Problem(c.psf, c.y, prm)
        st = pb.zero_state()
        t0 = time.perf_counter()
        pb.iterate(st, n_iter)
        o_s = time.perf_counter() - t0
        err = float(np.abs(x - st["X"]).max() / np.abs(st["X"]).max())
        esz = 8 if dtype == torch.float64 else 4
        ach = STEP_ALG_BYTES_PER_VOXEL * esz / 4 * V * n_iter / (ms * 1e-3) / 1e9
        row = {"workload": name, "dtype": "f64" if esz == 8 else "f32", "iters": n_iter, "ms": ms, "wav_tile": tile,
               "voxel_it_per_s": V * n_iter / (ms * 1e-3), "step_alg_gbs": ach, "step_frac": ach / peak,
               "x_max_rel_err_vs_oracle": err,
               "oracle": {"voxel_it_per_s": V * n_iter / o_s, "cores": cores, "iters": n_iter, "seconds": o_s}}
        if one_iters:
            row["oracle_one_thread"] = _oracle_one_thread(name, one_iters)
        out.append(row)
    return out


def run_case(args):
    """Single runs for profiling and quick checks (no contract line)."""
    import torch

    import paper_1504_06847_gb300 as mf
    from paper_1504_06847_gb300 import synth

    if args.case == "oracle":
        print(json.dumps(oracle_case(args.sample, args.iters)))
        return 0
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    if args.case == "batch":
        print(json.dumps(measure_forms(stream)["batched"]))
        return 0
    if args.case == "backward":
        print(json.dumps(measure_forms(stream)["differentiable"]))
        return 0
    if args.case == "configs":
        print(json.dumps(measure_configs(stream)))
        return 0
    prm = synth.WORKLOAD_PARAMS
    if args.case in ("linear", "vis"):
        # step I by conjugate gradients, the cubes of the widened-rows measurement
        with torch.cuda.stream(stream):
            if args.case == "linear":
                c = synth.make_cube(args.N, args.L, n_sources=40, n_antennas=128, seed=12)
                plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"), linear=True)
                y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
            else:
                cv = synth.make_visibilities(args.N, args.L, n_sources=40, n_antennas=128, seed=13,
                                             random_weights=True)
                plan = mf.Plan.from_visibilities(
                    args.N, [torch.tensor(q, dtype=torch.float32, device="cuda") for q in cv.uv],
                    [torch.tensor(w, dtype=torch.float32, device="cuda") for w in cv.weights])
                y = torch.tensor(np.concatenate(cv.vis).astype(np.complex64), device="cuda")
            plan.iterate(y, args.iters, cg_iters=args.cg_iters, wavelet_levels=args.J,
                         resid_every=1 if args.resid else 0, **prm)
            print(json.dumps(plan.report()))
            plan.close()
        return 0
    c = synth.make_cube(args.N, args.L, n_sources=max(2, int(40 * (args.N / 256) ** 2)), n_antennas=128,
                        seed=args.seed)
    prec = mf.MF_FP32_DCT_SPLITBF16 if args.precision == "splitbf16" else mf.MF_FP32
    with torch.cuda.stream(stream):
        plan = mf.Plan(torch.tensor(c.psf, dtype=torch.float32, device="cuda"))
        plan.set_option(mf.MF_OPT_WAV_TILE, args.tile)
        y = torch.tensor(c.y, dtype=torch.float32, device="cuda")
        if args.case == "xstep":
            plan.iterate(y, 3, precision=prec, **prm)
            plan.set_timing(True)
            plan.iterate(y, 10, warm_start=1, precision=prec, **prm)
            t = plan.timing()
            plan.set_timing(False)
            ours = sum(t[k][0] / max(t[k][1], 1) for k in ("rows_fwd", "cols_solve", "rows_inv"))
            print(json.dumps(dict(xstep_reference(stream, ours), N=args.N, L=args.L)))
            return 0
        plan.iterate(y, args.iters, wavelet_levels=args.J, precision=prec, resid_every=1 if args.resid else 0,
                     spectral_mask=args.spectral_mask, **prm)
        print(json.dumps(plan.report()))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="leave out the batched and differentiable forms")
    ap.add_argument("--precision", default="splitbf16", choices=["splitbf16", "fp32"],
                    help="DCT arithmetic of the spectral step (the cube is FP32 either way)")
    ap.add_argument("--case", default=None,
                    choices=["plain", "linear", "vis", "batch", "backward", "xstep", "oracle", "configs"],
                    help="a single run for profiling instead of the benchmark line")
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--L", type=int, default=8)
    ap.add_argument("--J", type=int, default=3)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--tile", type=int, default=64, choices=[64, 32])
    ap.add_argument("--cg-iters", type=int, default=10, help="CG iterations of step I (--case linear|vis)")
    ap.add_argument("--resid", action="store_true")
    ap.add_argument("--spectral-mask", type=int, default=1, choices=[1, 2, 3],
                    help="spectral dictionary of --case plain: 1 DCT, 2 Chebyshev, 3 both (FP32 DCT)")
    ap.add_argument("--seed", type=int, default=9)
    ap.add_argument("--sample", default="256x256x64", choices=sorted(ORACLE_SAMPLES))
    args = ap.parse_args()
    if args.case is not None:
        return run_case(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_1504_06847_gb300 as mf
    from paper_1504_06847_gb300 import synth

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    cube = synth.workload(WORKLOAD)
    N, L = cube.y.shape[-1], cube.y.shape[0]
    V = N * N * L
    prm = synth.WORKLOAD_PARAMS
    precision = mf.MF_FP32_DCT_SPLITBF16 if args.precision == "splitbf16" else mf.MF_FP32
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        psf = torch.tensor(cube.psf, dtype=torch.float32, device="cuda")
        y = torch.tensor(cube.y, dtype=torch.float32, device="cuda")
        plan = mf.Plan(psf)
        params = plan.params(stream=stream.cuda_stream, precision=precision, **prm)
        params_warm = plan.params(stream=stream.cuda_stream, warm_start=1, precision=precision, **prm)
        plan.iterate(y, args.warmup, params)
    stream.synchronize()

    # --- device-timed region: K iterations, inputs resident in HBM (working set >> L2) ---
    plan.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        plan.iterate(y, args.steps, params_warm)
        ev1.record(stream)
        stream.synchronize()
    barrier()
    timing = plan.timing()
    plan.set_timing(False)
    ms = 1e3 * max_over_ranks(ev0.elapsed_time(ev1) * 1e-3, dist, "cuda")
    value = whole_job_rate(V * args.steps, ms * 1e-3, world)
    launches = sum(n for _, n in timing.values())

    # --- end to end through the public API with host buffers: each step copies y
    # from pinned host memory, runs one iteration with the FP64 residual report
    # (primal and dual residuals, objective), reads the report and copies X back
    # into pinned host memory.  The copies run on a second stream, double
    # buffered, so that step k+1's upload and step k's download overlap the
    # iterations (every copy is inside the timed region) ---
    y_host = torch.tensor(cube.y, dtype=torch.float32).pin_memory()
    x_host = [torch.empty(cube.y.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    y_dev = [torch.empty_like(y) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    uploaded = [torch.cuda.Event() for _ in range(2)]
    stepped = [torch.cuda.Event() for _ in range(2)]
    params_e2e = plan.params(stream=stream.cuda_stream, warm_start=1, resid_every=1, precision=precision, **prm)
    with torch.cuda.stream(stream):  # the dual residual's work cubes are allocated by the first such call
        plan.iterate(y, 1, params_e2e)
        plan.report()
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(copy_stream):
        y_dev[0].copy_(y_host, non_blocking=True)
        uploaded[0].record(copy_stream)
    for k in range(e2e_steps):
        b = k % 2
        stream.wait_event(uploaded[b])
        with torch.cuda.stream(stream):
            plan.iterate(y_dev[b], 1, params_e2e)
        if k + 1 < e2e_steps:  # y_dev[1 - b] was read by step k - 1, complete since its report
            with torch.cuda.stream(copy_stream):
                y_dev[1 - b].copy_(y_host, non_blocking=True)
                uploaded[1 - b].record(copy_stream)
        rep = plan.report()  # waits for step k
        with torch.cuda.stream(stream):
            x_dev = plan.x()
            stepped[b].record(stream)
        copy_stream.wait_event(stepped[b])
        with torch.cuda.stream(copy_stream):
            x_host[b].copy_(x_dev, non_blocking=True)
        x_dev.record_stream(copy_stream)
    copy_stream.synchronize()
    stream.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = whole_job_rate(V * e2e_steps, e2e_s, world)
    if rep["status"] != mf.MF_OK:
        raise RuntimeError(f"e2e report status {rep['status']}")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # --- roofline of the dominant kernel (device time from the live CUDA events) ---
    peak, peak_kind = measured_peak()
    alg = alg_bytes_per_iteration(N, L)
    per_kernel = {}
    for name, (kms, n) in timing.items():
        if n == 0:
            continue
        d = {"ms_total": kms, "launches": n, "ms_per_launch": kms / n}
        if name in alg and kms > 0:
            d["achieved_gbs"] = alg[name] * args.steps / (kms * 1e-3) / 1e9
        per_kernel[name] = d
    dom = max((k for k in per_kernel if k in alg), key=lambda k: per_kernel[k]["ms_total"])
    dk = per_kernel[dom]
    launches_per_iter = dk["launches"] / args.steps
    ach = dk["achieved_gbs"]
    traffic = NCU_TRAFFIC_PER_LAUNCH.get(dom)
    roofline = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": traffic, "kernel": dom, "peak_kind": f"{peak_kind} copy bandwidth",
                "alg_bytes_per_launch": alg[dom] / launches_per_iter,
                "ms_per_launch": dk["ms_per_launch"]}
    step_ach = STEP_ALG_BYTES_PER_VOXEL * V / (ms / args.steps * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f32+bf16x3", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "L": L, "wavelet_levels": 3, "bases": "Db1-Db8+Haar",
                   "dct": "split-BF16 tcgen05, FP32 accumulate" if args.precision == "splitbf16" else "FP32",
                   "n_iter_per_step": 1, "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"inputs larger than L2 (plan working set {plan.device_bytes / 1e9:.1f} GB)",
                   "resid_every": 0, "e2e_resid_every": 1, "params": prm},
        "roofline": roofline,
        "step_roofline": {"bound": "hbm", "alg_bytes_per_voxel": STEP_ALG_BYTES_PER_VOXEL, "achieved": step_ach,
                          "peak": peak, "unit": "GB/s", "frac": step_ach / peak},
        "kernels": per_kernel,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(y_host.numel() * 4),
                "d2h_bytes_per_step": int(x_host[0].numel() * 4) + 16 * 8 + 4, "steps": e2e_steps,
                "note": "per step: pinned y upload, one iteration with the FP64 primal/dual residuals and "
                        "objective, report read-back, X copied back into pinned host memory; the copies run "
                        "on a second stream (double buffers) and overlap the neighbouring steps' iterations"},
    }
    line["clocks"] = clk.summary()
    if not args.no_forms:
        xs = sum(per_kernel[k]["ms_per_launch"] for k in ("rows_fwd", "cols_solve", "rows_inv"))
        line["forms"] = measure_forms(stream, xs)
        line["widened_rows"] = measure_widened_rows(stream, plan, y, peak)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cube)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
