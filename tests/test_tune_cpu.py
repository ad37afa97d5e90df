"""The autotuner's search and cache, on the CPU with a stand-in system whose step time is a known
function of the launch shape (the GPU test times real steps)."""
import json

import pytest

from paper_2003_14061_gb300 import binding as B
from paper_2003_14061_gb300 import tune


class FakeParams:
    def __init__(self, precision):
        self.precision = precision


class FakeSystem:
    def __init__(self, precision=B.MD_MIXED):
        self.params = FakeParams(precision)
        self.t = {"ctas_per_sm": 8, "nbr_batch": 2, "build_batch": 2, "use_graph": 1, "step_kernel": 1,
                  "build_stage": 2, "reorder_every": 100}
        self.set_calls = []
        self.steps = 0

    def tuning(self):
        return dict(self.t)

    def set_tuning(self, **kw):
        self.set_calls.append(dict(kw))
        self.t.update({k: v for k, v in kw.items() if v})

    def integrate(self, n):
        self.steps += n


def cost(t):
    # a unique minimum at step kernel 1, 12 CTAs/SM, 4 entries per batch, build batch 4
    c = 1.0 + 0.1 * abs(t["ctas_per_sm"] - 12) + 0.05 * abs(t["nbr_batch"] - 4)
    c += {1: 0.0, 2: 0.5, 3: 0.7, 4: 0.9, 5: 0.6}[t["step_kernel"]] + {1: 0.1, 2: 0.02, 4: 0.0, 32: 0.3}[t["build_batch"]]
    c += {1: 0.0, 2: 0.01}[t["build_stage"]] + {100: 0.0, -1: 0.02}[t["reorder_every"]]
    return c


@pytest.fixture
def fake_timing(monkeypatch):
    monkeypatch.setattr(tune, "_time_steps", lambda system, steps, rate=None: cost(system.tuning()))
    monkeypatch.setattr(tune, "signature", lambda system: f"fake|prec{system.params.precision}")


def test_search_finds_the_fastest_shape(fake_timing):
    s = FakeSystem()
    res = tune.tune(s, steps=64)
    assert res["best"] == {"ctas_per_sm": 12, "nbr_batch": 4, "build_batch": 4, "step_kernel": 1, "build_stage": 1,
                           "reorder_every": 100}
    assert {json.loads(k)["reorder_every"] for k in res["trials"]} == {100, -1}
    assert res["ms_per_step"] == pytest.approx(1.0)
    assert res["ms_per_step"] == min(res["trials"].values())
    tried = [json.loads(k) for k in res["trials"]]
    assert {t["step_kernel"] for t in tried} == {1, 4, 5}            # 2 and 3 only on request
    assert {t["ctas_per_sm"] for t in tried if t["step_kernel"] == 1} == set(tune.CTAS)
    assert {t["ctas_per_sm"] for t in tried if t["step_kernel"] == 4} == set(tune.CTAS_CELLS)
    assert {t["ctas_per_sm"] for t in tried if t["step_kernel"] == 5} == set(tune.CTAS_CELLS)
    assert {t["nbr_batch"] for t in tried if t["step_kernel"] in (4, 5)} == {2}
    assert {t["build_batch"] for t in tried} == set(tune.BUILD_BATCH)
    assert s.tuning()["ctas_per_sm"] == 12 and s.tuning()["build_batch"] == 4
    assert s.tuning()["use_graph"] == 1                # trials run direct launches; graphs come back
    assert s.steps % 16 == 0                       # whole 16-step graph replays only


def test_fp64_searches_the_per_thread_kernel_only(fake_timing):
    res = tune.tune(FakeSystem(B.MD_FP64), steps=32)
    assert {json.loads(k)["step_kernel"] for k in res["trials"]} == {1}


def test_step_kernels_can_be_restricted(fake_timing):
    # the adjoint reads the neighbour matrix: its tuning leaves the list-free kernel out
    res = tune.tune(FakeSystem(), steps=32, step_kernels=(1, 2, 3))
    tried = [json.loads(k) for k in res["trials"]]
    assert {t["step_kernel"] for t in tried} == {1, 2, 3}
    assert {t["ctas_per_sm"] for t in tried if t["step_kernel"] == 2} == set(tune.CTAS_RING)
    assert {t["ctas_per_sm"] for t in tried if t["step_kernel"] == 3} == set(tune.CTAS_STAGED)


def test_cache_round_trip(fake_timing, tmp_path):
    cache = str(tmp_path / "sub" / "tune.json")
    first = tune.tune(FakeSystem(), steps=32, cache=cache)
    s = FakeSystem()
    again = tune.tune(s, steps=32, cache=cache)
    assert again["best"] == first["best"]
    assert s.steps == 0                            # served from the cache: nothing timed
    assert s.set_calls == [first["best"]]


class PhaseSystem(FakeSystem):
    """Per-phase timings and rebuild counters as the library reports them: a step phase of a
    fixed cost per step and rebuilds of a fixed cost whose number per trial varies."""

    def __init__(self, rebuilds_per_trial):
        super().__init__()
        self.plan = list(rebuilds_per_trial)
        self.rebuilds = 0
        self.reorders = 0
        self.timing_on = False
        self.ph = None

    def props(self):
        return [{"rebuilds": self.rebuilds, "reorders": self.reorders}]

    def set_timing(self, on=True):
        self.timing_on = on

    def integrate(self, n):
        super().integrate(n)
        if self.timing_on:
            k = self.plan.pop(0)
            self.rebuilds += k
            self.reorders += 1                  # one reorder of 0.3 ms in each trial
            self.ph = {"step": (0.2 * n, n, n), "bin": (0.1 * k, n, n), "reorder": (0.3, 1, 1),
                       "build": (0.9 * k, n, n), "props": (0.0, 0, 0), "other": (0.0, 0, 0)}

    def timing(self):
        return self.ph


def test_score_does_not_depend_on_the_rebuilds_that_fell_in_a_trial():
    # the same shape timed twice, with 9 and then 14 rebuilds falling into the 100 timed steps:
    # the score is step time + time per rebuild x the rebuild rate over the search, so the
    # second trial scores the same shape no worse than the first
    # (reorders every 100 steps: 0.3 ms x 1/100 per step)
    s = PhaseSystem([9, 14])
    rate = tune._Rate()
    a = tune._time_steps(s, 100, rate)
    b = tune._time_steps(s, 100, rate)
    assert a == pytest.approx(0.2 + 1.0 * 9 / 100 + 0.003)
    assert b == pytest.approx(0.2 + 1.0 * 23 / 200 + 0.003)
    # at every rebuild (-1) the same reorder costs 0.3 ms x the rebuild rate
    s.t["reorder_every"] = -1
    s.plan = [10]
    c = tune._time_steps(s, 100, rate)
    assert c == pytest.approx(0.2 + 1.0 * 33 / 300 + 0.3 * 33 / 300)
    # whole-step timing would have scored the second trial 0.05 ms worse
    assert abs(b - a) < 0.05
