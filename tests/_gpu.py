"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and map its state onto the oracle's (the CUDA path keeps S and Gamma_S in the
DCT domain and stores one Gamma_T for Db1 and Haar)."""

import json
import os

import numpy as np
import torch

import oracle
import paper_1504_06847_gb300 as mf


def rel_err(a, b):
    """max_i |a_i - b_i| / max_i |b_i| (the error measure of the parity tests)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def run_gpu(cube, params, n_iter, J=3, mask=0x1FF, dtype=torch.float32, resid_every=0):
    plan = mf.Plan(torch.tensor(cube.psf, dtype=dtype, device="cuda"))
    plan.iterate(torch.tensor(cube.y, dtype=dtype, device="cuda"), n_iter, wavelet_levels=J, wavelet_mask=mask,
                 resid_every=resid_every, **params)
    return plan


def gpu_state(plan):
    g = lambda w: plan.get(w).double().cpu().numpy()
    return {"X": g(mf.ARR_X), "GP": g(mf.ARR_GAMMA_P), "Sd": g(mf.ARR_S_DCT), "GV": g(mf.ARR_GAMMA_V),
            "GSd": g(mf.ARR_GAMMA_S_DCT), "b": g(mf.ARR_B), "GT": g(mf.ARR_GAMMA_T)}


def oracle_view(pb, st):
    """The oracle's state in the CUDA path's representation."""
    C = oracle.dct_matrix(pb.L)
    dct = lambda a: np.einsum("kl,lij->kij", C, a)
    names = [n for n, _ in pb.bases]
    slots = []
    for K in range(1, 9):
        if f"db{K}" in names:
            slots.append(names.index(f"db{K}"))
        elif K == 1 and "haar" in names:
            slots.append(names.index("haar"))
    return {"X": st["X"], "GP": st["GP"], "Sd": dct(st["S"]), "GV": st["GV"], "GSd": dct(st["GS"]),
            "b": pb.make_b(st) - pb.HtY, "GT": st["GT"][slots]}


def scales(pb, st):
    """Error scale of each compared array.  X, S W_nu and b: their own max.
    A multiplier is updated by rho_c times a constraint residual (step VI), so
    its rounding floor is set by rho_c times the primal operand of its
    constraint, in the domain the multiplier is compared in: Gamma_P by
    rho_P |X|; Gamma_S, compared as Gamma_S W_nu, by rho_S |X W_nu|; Gamma_V
    (DCT domain) by rho_V |S W_nu|; Gamma_T by rho_T |W_s X|."""
    p = pb.params
    C = oracle.dct_matrix(pb.L)
    xm = np.abs(st["X"]).max()
    xdm = np.abs(np.einsum("kl,lij->kij", C, st["X"])).max()
    sm = np.abs(np.einsum("kl,lij->kij", C, st["S"])).max()
    zm = max(np.abs(oracle.dwt2(st["X"], h, pb.J)).max() for _, h in pb.bases)
    bm = np.abs(pb.make_b(st) - pb.HtY).max()
    return {"X": xm, "Sd": sm, "b": bm, "GP": p["rho_P"] * xm, "GSd": p["rho_S"] * xdm,
            "GV": p["rho_V"] * sm, "GT": p["rho_T"] * zm}


def compare(gs, os_, sc=None, keys=("X", "GP", "Sd", "GV", "GSd", "b", "GT")):
    """max |gpu - oracle| over each array, divided by its scale (default: max |oracle|).
    With MF_PARITY_LOG set, each comparison is appended to that file as one JSON line."""
    out = {}
    for k in keys:
        den = sc[k] if sc is not None else np.abs(os_[k]).max()
        out[k] = float(np.abs(np.asarray(gs[k]) - np.asarray(os_[k])).max() / (den if den > 0 else 1.0))
    log_errors(out)
    return out


def log_errors(errs):
    """Appends errs to the file named by MF_PARITY_LOG (if set), one JSON line per call."""
    log = os.environ.get("MF_PARITY_LOG")
    if log:
        with open(log, "a") as f:
            f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", ""), "errors": errs}) + "\n")
