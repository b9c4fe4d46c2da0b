"""The benchmark's byte model (host logic, no GPU).

Per voxel of the cube, FP32, 8 distinct bases, J = 3: the kernels move
8 (rows_fwd) + 14 (cols) + 8 (rows_inv) + 40 (spectral) + 22 (low-low) +
68 (level 1) + 38 (levels 2-3) = 198 bytes, against the 146-byte minimum of
the whole step; the roofline of the dominant kernel divides level 1's 68 B.
"""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("N,L", [(1024, 64), (256, 32)])
def test_kernel_bytes_per_voxel(N, L):
    V = N * N * L
    per_voxel = {k: v / V for k, v in bench.alg_bytes_per_iteration(N, L).items()}
    expect = {"rows_fwd": 8, "cols_solve": 14, "rows_inv": 8, "spectral": 40, "wav_ll": 22,
              "wav_level1": 68, "wav_levelj": 38}
    for k, v in expect.items():
        assert per_voxel[k] == pytest.approx(v), k
    assert sum(per_voxel.values()) == pytest.approx(198)
    assert bench.STEP_ALG_BYTES_PER_VOXEL == 146.0


def test_single_level_dictionary_moves_no_coarse_bands():
    # J = 1: no low-low pass and no coarser level; level 1 thresholds every coefficient
    b = bench.alg_bytes_per_iteration(256, 8, J=1)
    V = 256 * 256 * 8
    assert b["wav_ll"] == 0 and b["wav_levelj"] == 0
    assert b["wav_level1"] / V == pytest.approx(4 + 8 + 2 * 8 * 4)


def test_clock_samples_summary(tmp_path):
    # nvidia-smi --format=csv,noheader,nounits lines: index, sm, max sm, power, active mask,
    # hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1995, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
                    "0, 2040, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage line\n")
    c = bench.ClockSampler(0)
    c.path = str(path)
    s = c.summary()
    assert s["sm_mhz"] == 2040 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert not path.exists()  # the sample file is removed


def test_clock_samples_missing():
    c = bench.ClockSampler(0)
    assert c.summary() is None
