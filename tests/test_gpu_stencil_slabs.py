"""The momentum and right-hand-side kernels at every z-slab depth of a 16^3 cube
(bcm_set_stencil_slabs 1, 2, 4 and the default) against the oracle, FP64 and mixed, on
a sphere channel and a two-level grid with a rotating body; the stencil tuner on the
GPU picks one of them and leaves the state as it found it."""
import numpy as np
import pytest

from paper_1808_04099_gb300 import workloads as W
from _util import assert_close, oracle_run, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import autotune, bcm  # noqa: E402

GRIDS = {
    "sphere": lambda: W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0), radius=0.2,
                                       center=(0.6, 0.5, 0.5)),
    "two_level": lambda: W.two_level_channel(2, 1, 1, 16, (1, 0, 0), (2, 1, 1), 1 / 32., 1,
                                             seed=5),
}


def velocity(g):
    return np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])


@pytest.mark.parametrize("name", sorted(GRIDS))
@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
def test_every_slab_depth_matches_oracle(name, prec):
    spec = GRIDS[name]()
    state = W.initial_state(spec, seed=63, noise=1e-3)
    ost, _ = oracle_run(spec, state, 2, 1e-13)
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    runs = []
    for slabs in (0, 1, 2, 4):
        g = bcm.Grid(spec, prec)
        g.load_state(state)
        g.set_stencil_slabs(slabs)
        assert g.get_stencil_slabs() == slabs
        st = g.step(2, rtol=1e-13 if prec == bcm.PREC_F64 else 1e-12)
        assert all(s["converged"] == 1 for s in st)
        if prec == bcm.PREC_F64:
            assert_close(velocity(g), ref, g.numpy(bcm.P), ost["p"], spec, 1e-10)
        else:
            # the velocity within 1e-6; the pressure of this grid is ~1e-3 of the velocity,
            # so the FP32 rounding of the state moves it by ~1e-3 of itself (R13)
            assert rel_l2(velocity(g), ref) <= 1e-6
        runs.append((velocity(g), g.numpy(bcm.P)))
        del g
    for v, p in runs[1:]:  # the same arithmetic in another tiling
        assert np.abs(v - runs[0][0]).max() <= 1e-12 * np.abs(runs[0][0]).max()
        assert np.abs(p - runs[0][1]).max() <= 1e-9 * np.abs(runs[0][1]).max()


def test_stencil_tuner_on_the_gpu(tmp_path):
    spec = W.config_sphere(2)
    g = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g.load_state(W.initial_state(spec))
    g.step(1, rtol=1e-8)
    before = velocity(g)
    step0 = g.step(0)[0]["steps"]
    times = autotune.tune_stencils(g, steps=2, cache_path=str(tmp_path / "c.json"))
    assert set(times) == {1, 2, 4} and all(t > 0 for t in times.values())
    assert g.get_stencil_slabs() == min(times, key=times.get)
    assert np.array_equal(velocity(g), before) and g.step(0)[0]["steps"] == step0
    print("momentum + rhs us per step by slabs:", {k: round(v, 1) for k, v in times.items()})
