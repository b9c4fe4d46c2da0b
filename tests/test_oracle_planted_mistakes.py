"""Planted mistakes: the oracle's pins must catch a plausible error anywhere
in it.  Each case copies the oracle's C source, plants one mistake (a dropped
term, a wrong sign, a shifted index, a transposed operand), builds that copy
as a separate library with the oracle's flags, and runs the pins that must
catch it against the copy (MF_ORACLE_LIB) in a child pytest, which has to
fail on an assertion.  The unchanged source, built the same way, passes the
same pins.  CPU only; the committed oracle is never modified."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mf_oracle.c")
FLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

# (id, what the mistake is, text of the source, its replacement, pin file, -k selection)
CASES = [
    ("rho_bar_without_ns", "Eq. Qlsimp: rho = mu_eps + rho_S + rho_P + rho_T, the n_s factor dropped",
     "return pb->mu_eps + pb->rho_S + pb->rho_P + pb->nb * pb->rho_T;",
     "return pb->mu_eps + pb->rho_S + pb->rho_P + pb->rho_T;",
     "test_oracle_steps.py", "step_I"),
    ("hty_without_conjugate", "set-up: H y formed in place of H^T y (the conjugate filter dropped)",
     "ti[i] = hre[i] * yim[i] - him[i] * yre[i];",
     "ti[i] = hre[i] * yim[i] + him[i] * yre[i];",
     "test_oracle_steps.py", "asymmetric"),
    ("make_b_without_gamma_S", "Eq. matB: the Gamma_S term of b dropped",
     "bl[i] = HtY[q] + GP[q] + pb->rho_P * P[q] + GS[q] + pb->rho_S * S[q];",
     "bl[i] = HtY[q] + GP[q] + pb->rho_P * P[q] + pb->rho_S * S[q];",
     "test_oracle_steps.py", "step_I"),
    ("fft_direction", "the 2-D FFT run in the inverse direction",
     "fft2_image(re + (long)i * N * N, im + (long)i * N * N, N, sign > 0, twr, twi, lr, li);",
     "fft2_image(re + (long)i * N * N, im + (long)i * N * N, N, sign < 0, twr, twi, lr, li);",
     "test_oracle_transforms.py", "fft"),
    ("dct_index_swap", "DCT-II matrix with the frequency and sample indices swapped (its transpose)",
     "C[k * L + l] = a * cos(M_PI * (2.0 * l + 1.0) * k / (2.0 * L));",
     "C[k * L + l] = a * cos(M_PI * (2.0 * k + 1.0) * l / (2.0 * L));",
     "test_oracle_transforms.py", "dct"),
    ("primal_residual_without_T", "primal residual: the ||T - W_s X||^2 term dropped",
     "double r2 = sumsq_diff(P, X, V_) + sumsq_diff(T, Z, VT) + sumsq_diff(S, X, V_);",
     "double r2 = sumsq_diff(P, X, V_) + sumsq_diff(S, X, V_);",
     "test_oracle_reductions.py", "history_matches"),
    ("dwt_index_shift", "DWT analysis reads x[(2i + n + 1) mod M] instead of x[(2i + n) mod M]",
     "double v = x[(2 * i + n) % M];",
     "double v = x[(2 * i + n + 1) % M];",
     "test_oracle_transforms.py", "dwt or haar"),
    ("gamma_P_sign", "step VI: Gamma_P -= rho_P (P - X)",
     "GP[i] += pb->rho_P * (P[i] - X[i]);",
     "GP[i] -= pb->rho_P * (P[i] - X[i]);",
     "test_oracle_steps.py", "VI"),
    ("threshold_without_rho_T", "step III: threshold mu_s instead of mu_s / rho_T",
     "double tauT = pb->mu_s / pb->rho_T;",
     "double tauT = pb->mu_s;",
     "test_oracle_steps.py", "II_to_V"),
    ("step_IV_multiplier_sign", "step IV: S W_nu + Gamma_V / rho_V inside the threshold",
     "v[k] = soft(sw - GVj[k * NN + p] / pb->rho_V, tauV);",
     "v[k] = soft(sw + GVj[k * NN + p] / pb->rho_V, tauV);",
     "test_oracle_steps.py", "II_to_V"),
    ("step_IV_transposed_basis", "step IV: S W_nu formed with the transposed spectral basis",
     "for (int l = 0; l < L; l++) sw += C[k * L + l] * S[l * NN + p];\n        v[k] = soft(",
     "for (int l = 0; l < L; l++) sw += C[l * L + k] * S[l * NN + p];\n        v[k] = soft(",
     "test_oracle_steps.py", "II_to_V"),
    ("step_V_divisor_without_m_nu", "step V: divisor rho_V + rho_S instead of m_nu rho_V + rho_S",
     "/ ((double)mnu * pb->rho_V + pb->rho_S);",
     "/ (pb->rho_V + pb->rho_S);",
     "test_oracle_spectral_dict.py", "steps_IV_and_V"),
    ("dual_residual_without_rho_V_term", "dual residual: the rho_V^2 ||dS W_nu||^2 term dropped",
     "s2 += pb.mnu * pb.rho_V * pb.rho_V * dS2;",
     "s2 += 0.0 * dS2;",
     "test_oracle_reductions.py", "history_matches"),
    ("objective_without_mu_nu", "objective: the mu_nu ||X W_nu||_1 term dropped",
     "hh[3] = fit + 0.5 * pb.mu_eps * x2 + pb.mu_s * l1s + pb.mu_nu * l1n;",
     "hh[3] = fit + 0.5 * pb.mu_eps * x2 + pb.mu_s * l1s;",
     "test_oracle_reductions.py", "history_matches"),
    ("cg_beta_inverted", "conjugate gradients: beta = |r_k|^2 / |r_k+1|^2",
     "double beta = g2 / g;",
     "double beta = g / g2;",
     "test_oracle_linear.py", "textbook or dense_solve"),
    ("linear_psf_off_by_one", "linear H: the PSF embedded one row off its centre",
     "int r = ((u - N / 2) % M + M) % M, c = ((v - N / 2) % M + M) % M;",
     "int r = ((u - N / 2 + 1) % M + M) % M, c = ((v - N / 2) % M + M) % M;",
     "test_oracle_linear.py", "dense_linear_convolution or delta_psf"),
    ("linear_adjoint_without_conjugate", "linear H: H^T applied with the transfer function itself",
     "double hr = h2re[i], hi = adjoint ? -h2im[i] : h2im[i];",
     "double hr = h2re[i], hi = h2im[i];",
     "test_oracle_linear.py", "dense_linear_convolution"),
    ("visibility_phase_sign", "visibility operator: exp(+2 pi i ...) instead of exp(-2 pi i ...)",
     "double a = -2.0 * M_PI * f * (double)(n - N / 2) / (double)N;",
     "double a = 2.0 * M_PI * f * (double)(n - N / 2) / (double)N;",
     "test_oracle_vis.py", "integer_coordinates or pixel_shift"),
]

_control = {}


def _build(src_text, path):
    c_path = path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", *FLAGS, "-o", path + ".so", c_path, "-lm"])
    return path + ".so"


def _pins(lib, pin_file, kexpr):
    env = dict(os.environ, MF_ORACLE_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pin_file), "-q", "-x", "-m", "not gpu",
           "-p", "no:cacheprovider", "-k", kexpr]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def sources(tmp_path_factory):
    with open(SRC) as f:
        src = f.read()
    d = tmp_path_factory.mktemp("planted")
    return src, str(d), _build(src, os.path.join(str(d), "control"))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pins_catch_planted_mistake(sources, case):
    name, what, find, repl, pin_file, kexpr = case
    src, tmp, control = sources
    assert src.count(find) == 1, f"{name}: the planted site must be unique in the source"
    key = (pin_file, kexpr)
    if key not in _control:
        _control[key] = _pins(control, pin_file, kexpr)
    good = _control[key]
    assert good.returncode == 0, f"the unchanged oracle fails its pins:\n{good.stdout[-3000:]}"
    mutant = _build(src.replace(find, repl), os.path.join(tmp, name))
    bad = _pins(mutant, pin_file, kexpr)
    # 1: tests ran and failed (not a crash, a collection error or no tests selected)
    assert bad.returncode == 1, f"{name} ({what}) was not caught:\n{bad.stdout[-3000:]}"
    assert "assert" in bad.stdout.lower(), bad.stdout[-3000:]
