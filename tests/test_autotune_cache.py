"""The autotuner's host logic on the CPU, with fake grids whose timing source is a
table: it times every applicable PCG launch shape (and every z-slab depth of the
momentum and right-hand-side kernels), keeps the fastest, writes the JSON cache and
takes the choice from it on the next call without timing, restores the caller's solver
controls and the state, ignores an unreadable cache and re-tunes when the cached shape
is not one it knows."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1808_04099_gb300 import autotune, bcm  # noqa: E402


class FakeSpec:
    def __init__(self, B, n_cubes):
        self.B = B
        self.n_cubes = n_cubes


class FakeGrid:
    """The grid calls the tuner makes; solve_pressure_iters 'runs' for the table's time
    of the current shape (us per iteration) and records the call."""

    def __init__(self, table, B=16, precision=bcm.PREC_F32_REFINE, corr_us=0.0):
        self.spec = FakeSpec(B, 1024)
        self.corr_us = corr_us  # the x += e launch after every form but the streaming one
        self.precision = precision
        self.device = "cpu"
        self.table = table
        self.shape = (1, 1, 1)
        self.max_cycles = 7
        self.solves = 0
        self.p = torch.arange(10, dtype=torch.float64)
        self.last_iters = 0
        self.profiling = False

    def field(self, fid):
        assert fid == bcm.P
        return self.p

    def set_launch(self, slabs_a=1, slabs_b=1, persistent=1):
        self.shape = (int(persistent), int(slabs_a), int(slabs_b))

    def get_solver(self):
        return {"inner_rtol": 0.0, "max_cycles": self.max_cycles, "check_every": 8,
                "barrier_timeout_s": 2.0, "recycle": 1}

    def set_solver(self, max_cycles=0, **_):
        if max_cycles > 0:
            self.max_cycles = max_cycles

    def profile(self, on):
        self.profiling = bool(on)

    def solve_pressure_iters(self, iters):
        assert self.profiling and self.max_cycles == 1
        self.solves += 1
        self.last_iters = iters
        self.p.add_(1.0)  # the solve changes the pressure; the tuner restores it
        return [{"cg_iters": iters}]

    def profile_read(self, reset=True):
        us = self.table[self.shape]
        ms = 1e-3 * us * self.last_iters
        if self.shape[0]:  # persistent: one launch for all iterations
            prof = {"pcg": (ms, 1), "cg_a": (0.0, 0), "cg_b": (0.0, 0)}
        else:  # two launches per iteration, split evenly
            n = self.last_iters
            prof = {"pcg": (0.0, 0), "cg_a": (0.5 * ms, n), "cg_b": (0.5 * ms, n)}
        if self.corr_us and self.shape[0] != 1:
            prof["add_correction"] = (1e-3 * self.corr_us * self.last_iters, 1)
        return prof, 0


def table(best):
    t = {s: 100.0 + 3.0 * i for i, s in enumerate(autotune.SHAPES)}
    t[best] = 10.0
    return t


def test_tunes_writes_cache_and_reuses_it(tmp_path):
    cache = str(tmp_path / "launch.json")
    g = FakeGrid(table((1, 2, 1)))
    p0 = g.p.clone()
    times = autotune.tune(g, iters=5, cache_path=cache, device_name="fake GB300")
    assert g.shape == (1, 2, 1)
    assert min(times, key=times.get) == "1,2,1"
    assert times["1,2,1"] == pytest.approx(10.0)
    assert g.max_cycles == 7                      # the caller's control is back
    assert torch.equal(g.p, p0)                   # and the pressure
    timed = {s for s in autotune.SHAPES if not (s[0] and s[1] > 1 and g.spec.B != 16)}
    assert g.solves == 2 * len(timed)             # a warm-up pass and a timed pass each
    data = json.load(open(cache))
    (key,) = data.keys()
    assert key.startswith("fake GB300|B16|prec1|cubes1024")
    assert data[key]["best"] == [1, 2, 1]
    # second call: from the cache, no timing
    g2 = FakeGrid(table((0, 1, 2)))
    times2 = autotune.tune(g2, iters=5, cache_path=cache, device_name="fake GB300")
    assert g2.solves == 0 and g2.shape == (1, 2, 1) and times2 == data[key]["times"]
    # another device name: its own entry
    g3 = FakeGrid(table((0, 1, 2)))
    autotune.tune(g3, iters=5, cache_path=cache, device_name="other")
    assert g3.shape == (0, 1, 2) and g3.solves > 0
    assert len(json.load(open(cache))) == 2


def test_the_correction_launch_is_charged_to_the_forms_that_need_it():
    t = table((0, 1, 1))
    t[(0, 1, 1)], t[(1, 1, 1)] = 9.0, 10.0  # streaming: its x += e inside the launch
    g = FakeGrid(t, corr_us=2.0)
    times = autotune.tune(g, iters=5, use_cache=False)
    assert times["0,1,1"] == pytest.approx(11.0) and times["1,1,1"] == pytest.approx(10.0)
    assert g.shape == (1, 1, 1)


def test_fp64_and_small_cubes_skip_the_shapes_they_cannot_run(tmp_path):
    g = FakeGrid(table((5, 1, 1)), B=8, precision=bcm.PREC_F64)
    times = autotune.tune(g, iters=3, use_cache=False)
    assert "5,1,1" not in times                   # the fused form: FP32 on 16^3 only
    assert all(not (int(k.split(",")[0]) and int(k.split(",")[1]) > 1) for k in times)
    assert g.shape == tuple(map(int, min(times, key=times.get).split(",")))


def test_unreadable_or_stale_cache_is_retuned(tmp_path):
    cache = tmp_path / "launch.json"
    cache.write_text("{not json")
    g = FakeGrid(table((3, 1, 1)))
    autotune.tune(g, iters=4, cache_path=str(cache), device_name="d")
    assert g.shape == (3, 1, 1) and g.solves > 0
    data = json.loads(cache.read_text())
    (key,) = data.keys()
    data[key]["best"] = [9, 9, 9]                 # a shape the tuner does not know
    cache.write_text(json.dumps(data))
    g2 = FakeGrid(table((2, 1, 1)))
    autotune.tune(g2, iters=4, cache_path=str(cache), device_name="d")
    assert g2.solves > 0 and g2.shape == (2, 1, 1)
    assert json.loads(cache.read_text())[key]["best"] == [2, 1, 1]
    assert np.isfinite(list(json.loads(cache.read_text())[key]["times"].values())).all()


class FakeStencilGrid:
    """The calls of the stencil-slab tuner; a step 'runs' the momentum and right-hand
    side for the table's times of the current slab depth and changes the state."""

    def __init__(self, table, B=16):
        self.spec = FakeSpec(B, 1024)
        self.precision = bcm.PREC_F32_REFINE
        self.device = "cpu"
        self.table = table
        self.slabs = 0
        self.fields = {f: torch.full((8,), float(f)) for f in autotune.STATE_FIELDS}
        self.steps_taken = 5
        self.last = 0
        self.profiling = False

    def field(self, fid):
        return self.fields[fid]

    def get_stencil_slabs(self):
        return self.slabs

    def set_stencil_slabs(self, s):
        self.slabs = int(s)

    def step(self, n=1, stats=True, **_):
        if n:
            assert self.profiling
            for t in self.fields.values():
                t.add_(1.0)
        self.steps_taken += n
        self.last = n
        return [{"steps": self.steps_taken}] if stats else None

    def set_step(self, s):
        self.steps_taken = s

    def profile(self, on):
        self.profiling = bool(on)

    def profile_read(self, reset=True):
        us_m, us_r = self.table[self.slabs]
        n = self.last
        return {"momentum": (1e-3 * us_m * n, n), "rhs": (1e-3 * us_r * n, n)}, 0


def test_stencil_slabs_tuned_state_restored_and_cached(tmp_path):
    cache = str(tmp_path / "launch.json")
    table = {1: (300.0, 200.0), 2: (250.0, 180.0), 4: (200.0, 150.0)}
    g = FakeStencilGrid(table)
    before = {f: t.clone() for f, t in g.fields.items()}
    times = autotune.tune_stencils(g, steps=3, cache_path=cache, device_name="d")
    assert times == {1: pytest.approx(500.0), 2: pytest.approx(430.0), 4: pytest.approx(350.0)}
    assert g.slabs == 4 and g.steps_taken == 5
    assert all(torch.equal(g.fields[f], before[f]) for f in before)
    g2 = FakeStencilGrid({1: (1.0, 1.0), 2: (9.0, 9.0), 4: (9.0, 9.0)})
    assert autotune.tune_stencils(g2, cache_path=cache, device_name="d") == times
    assert g2.slabs == 4 and g2.steps_taken == 5  # from the cache: no steps
    g3 = FakeStencilGrid(table, B=8)
    assert autotune.tune_stencils(g3, cache_path=cache, device_name="d") == {}
    assert g3.slabs == 0
