"""Host logic of the wavelet-tile autotuner, with a stand-in plan (no GPU).

The tuner must keep the tile whose level kernels were faster, restore the
plan's state after its trials, write its choice to the cache file atomically,
answer later calls from the cache without timing again, and treat an
unreadable cache as empty.
"""

import json

import pytest

pytest.importorskip("torch")

from paper_1504_06847_gb300 import MF_OPT_WAV_TILE, autotune  # noqa: E402


class _State:
    def __init__(self, tag):
        self.tag = tag

    def clone(self):
        return _State(self.tag)


class FakePlan:
    """Records calls; level kernels take ms_by_tile[tile] per iteration."""

    def __init__(self, ms_by_tile, N=256, L=32):
        self.N, self.L = N, L
        self.ms_by_tile = ms_by_tile
        self.tile = 64
        self.timing_on = False
        self.acc = 0.0
        self.n = 0
        self.iterations = 0
        self.state = _State("initial")

    def set_option(self, opt, value):
        assert opt == MF_OPT_WAV_TILE
        self.tile = value

    def get_state(self):
        return self.state

    def set_state(self, st):
        self.state = st

    def iterate(self, y, n, **kw):
        self.iterations += n
        self.state = _State("iterated")
        if self.timing_on:
            self.acc += n * self.ms_by_tile[self.tile]
            self.n += n

    def set_timing(self, on):
        self.timing_on = on
        if on:
            self.acc, self.n = 0.0, 0

    def timing(self):
        return {"wav_level1": (0.75 * self.acc, self.n), "wav_levelj": (0.25 * self.acc, 2 * self.n)}


@pytest.fixture(autouse=True)
def _no_cuda_key(monkeypatch):
    monkeypatch.setattr(autotune, "_key", lambda N, L, p: f"fake|N={N}|L={L}|prec={p}")


@pytest.mark.parametrize("ms,best", [({64: 2.0, 32: 3.0}, 64), ({64: 3.0, 32: 1.5}, 32)])
def test_picks_faster_tile_and_restores_state(tmp_path, ms, best):
    p = FakePlan(ms)
    rec = autotune.tune(p, None, iters=3, cache=str(tmp_path / "t.json"))
    assert rec["wav_tile"] == best and p.tile == best
    assert p.state.tag == "initial"  # the trials do not leave their state behind
    assert rec["ms"]["64"] == pytest.approx(ms[64]) and rec["ms"]["32"] == pytest.approx(ms[32])


def test_cache_is_written_and_reused(tmp_path):
    path = tmp_path / "sub" / "t.json"
    p = FakePlan({64: 1.0, 32: 2.0})
    autotune.tune(p, None, cache=str(path))
    db = json.loads(path.read_text())
    assert list(db.values())[0]["wav_tile"] == 64
    q = FakePlan({64: 9.0, 32: 1.0})  # would now prefer 32, but the cache answers
    q.tile = 32
    rec = autotune.tune(q, None, cache=str(path))
    assert rec["wav_tile"] == 64 and q.tile == 64 and q.iterations == 0
    assert not list(path.parent.glob("*.tmp"))


def test_unreadable_cache_is_ignored(tmp_path):
    path = tmp_path / "t.json"
    path.write_text("{not json")
    p = FakePlan({64: 2.0, 32: 1.0})
    rec = autotune.tune(p, None, cache=str(path))
    assert rec["wav_tile"] == 32
    assert json.loads(path.read_text())  # replaced by a valid file


def test_no_cache(tmp_path):
    p = FakePlan({64: 1.0, 32: 2.0})
    assert autotune.tune(p, None, cache=None)["wav_tile"] == 64
