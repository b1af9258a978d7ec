"""Host logic of the measuring autotuner and the batch's subdomain counts, with
the timings faked (no GPU): the schedule search skips candidates the library
refuses, picks the fastest, leaves the handle on it and fails loudly when no
candidate is valid; parts_for splits each axis into round(n / box) boxes, at
least one and at most n."""
import os
from types import SimpleNamespace

import pytest


@pytest.fixture(scope="module")
def mods():
    from paper_2007_13966_gb300 import build_lib, ras
    if not os.path.exists(ras.LIB_PATH):
        build_lib.build()
    ras.lib()
    from paper_2007_13966_gb300 import autotune, batch
    return ras, autotune, batch


class FakePrecond:
    def __init__(self, ras, refused):
        self.ras, self.refused, self.cur, self.calls = ras, refused, None, []

    def set_schedule(self, chunk, threads):
        self.calls.append((chunk, threads))
        if chunk in self.refused:
            raise self.ras.RasError(self.ras.RAS_EINVAL, "ras_set_apply_schedule")
        self.cur = (chunk, threads or 64)

    def schedule(self):
        return self.cur

    def apply(self, r, z):
        pass


def test_schedule_search_picks_the_fastest_valid(mods, monkeypatch):
    ras, autotune, _ = mods
    pc = FakePrecond(ras, refused={1536})
    secs = {256: 3e-5, 384: 2e-5, 512: 1.5e-5, 768: 1.7e-5, 1024: 1.9e-5}
    monkeypatch.setattr(autotune, "_time", lambda fn, reps, warmup=2: secs[pc.cur[0]])
    best, table = autotune.tune_schedule(pc, None, None)
    assert best == (512, 64)
    assert pc.schedule() == (512, 64)
    assert [d["schedule"][0] for d in table] == [256, 384, 512, 768, 1024]


def test_schedule_search_without_a_valid_candidate_raises(mods, monkeypatch):
    ras, autotune, _ = mods
    pc = FakePrecond(ras, refused=set(autotune.CHUNKS))
    monkeypatch.setattr(autotune, "_time", lambda fn, reps, warmup=2: 1.0)
    with pytest.raises(RuntimeError):
        autotune.tune_schedule(pc, None, None)


def test_parts_for_rounds_and_clamps(mods):
    _, _, batch = mods
    res = SimpleNamespace(grid=SimpleNamespace(nx=96, ny=40, nz=5))
    assert batch.parts_for(res, 16) == (6, 2, 1)      # 96/16, round(2.5) = 2, at least one
    assert batch.parts_for(res, 1) == (96, 40, 5)     # at most n
    assert batch.parts_for(SimpleNamespace(grid=SimpleNamespace(nx=33, ny=31, nz=1)), 16) == (2, 2, 1)
