"""The batched form: many tanks stepped by one launch per kernel over packed
block tables.  Each tank of a batch must equal, bit for bit, the same tank run
alone through the single-tank path (the per-cell arithmetic and the order of
every reduction are the same), and the FP64 batch must match the oracle
within 1e-11 like the single-tank path."""
import numpy as np
import pytest

import oracle
from paper_1201_0351_gb300 import inputs as I

from parity import assert_f64_parity, macro_errors, velocity_check

pytestmark = pytest.mark.gpu


def _scenes():
    """Uneven small tanks: moving free boxes, a tank without bodies, a
    periodic one, and the two smallest heeled-box tanks of the sweep."""
    out = [I.random_box_scene(40, 30, 22, seed=11, nboxes=2, speed=0.02),
           I.random_box_scene(26, 34, 20, seed=12, nboxes=1, speed=0.03),
           I.random_box_scene(20, 20, 16, seed=13, nboxes=0),
           I.random_box_scene(24, 18, 18, seed=14, nboxes=1, periodic=1, speed=0.02)]
    sweep = sorted(I.batched_sweep_tanks(64), key=lambda s: s.nx)
    return out + sweep[:2]


def _alone(sc, storage, steps):
    from paper_1201_0351_gb300 import lbm_fs

    sim = lbm_fs.Simulation(sc, storage=storage)
    sim.step(steps)
    g = sim.fields(want_f=True)
    b = [sim.body(k) for k in range(len(sc.boxes))]
    st = sim.stats()
    sim.close()
    return g, b, st


def _batched(scenes, storage, steps, use_graphs=True, autotune=False, lanes=0):
    from paper_1201_0351_gb300 import lbm_fs

    bt = lbm_fs.Batch(scenes, storage=storage, use_graphs=use_graphs)
    if lanes:
        cfg = bt.config()
        bt.set_config(cfg["zb"], cfg["bulk_blocks"], cfg["list_cells"], lanes)
    if autotune:
        cfg = bt.autotune()
        assert 1 <= cfg["zb"] <= 8 and cfg["bulk_ms"] > 0.0
    bt.step(steps)
    bt.sync()
    res = []
    for t, sc in zip(bt.tanks, scenes):
        res.append((t.fields(want_f=True), [t.body(k) for k in range(len(sc.boxes))], t.stats()))
    launches = bt.launches()
    bt.close()
    return res, launches


def _same(a, b):
    g1, b1, s1 = a
    g2, b2, s2 = b
    for key in ("flags", "f", "fill", "mass", "rho", "u"):
        assert np.array_equal(g1[key], g2[key]), key
    for x, y in zip(b1, b2):
        for key in ("F", "T", "center", "quat", "vel", "omega"):
            assert np.array_equal(x[key], y[key]), key
    for key in ("liquid_mass", "covered", "uncovered", "lost_excess", "n_interface", "n_general"):
        assert s1[key] == s2[key], (key, s1[key], s2[key])
    # the moving-wall mass source is summed by device atomics in arrival order,
    # so its last bits differ between any two runs (alone or batched)
    assert abs(s1["wall_source"] - s2["wall_source"]) <= 1e-12 * max(1.0, abs(s2["wall_source"]))


@pytest.mark.parametrize("storage,lanes", [("f64", 1), ("f16s", 1), ("f16s", 3)])
def test_batch_equals_tanks_run_alone(storage, lanes):
    """every kernel once per step for the tanks of each lane (concurrent
    chains of launches), every tank bit for bit as alone"""
    scenes = _scenes()
    steps = 40
    res, (launches, nsteps) = _batched(scenes, storage, steps, lanes=lanes)
    assert nsteps == steps and launches == 17 * lanes * steps
    for sc, r in zip(scenes, res):
        _same(r, _alone(sc, storage, steps))


def test_batch_f64_matches_oracle():
    scenes = _scenes()
    steps = 40
    res, _ = _batched(scenes, "f64", steps)
    for sc, (g, gb, gs) in zip(scenes, res):
        ref = oracle.OracleSim(sc)
        ref.step(steps)
        assert ref.error == 0
        o = ref.fields(want_f=True)
        ob = [ref.body(k) for k in range(len(sc.boxes))]
        assert_f64_parity(g, o, gb, ob)


def test_batch_f16s_against_oracle():
    """FP16-shifted storage in the batch (the sweep's storage) against the
    FP64 oracle: density within 2e-3, classes identical, velocity within 2e-3
    of the largest speed plus the rounding floor, torque within 2e-3 of its
    scale."""
    scenes = sorted(I.batched_sweep_tanks(64), key=lambda s: s.nx)[:3]
    steps = 60
    res, _ = _batched(scenes, "f16s", steps)
    for sc, (g, gb, gs) in zip(scenes, res):
        ref = oracle.OracleSim(sc)
        ref.step(steps)
        o = ref.fields(want_f=True)
        e = macro_errors(g, o)
        assert e["flag_diff"] == 0 and e["rho"] <= 2e-3, (sc.name, e)
        e_liq, e_if, bound, umax = velocity_check(g, o, "f16s", 2e-3, steps)
        assert e_liq <= bound and e_if <= bound, (sc.name, e_liq, e_if, bound)
        ob = ref.body(0)
        lever = float(np.linalg.norm(sc.boxes[0].half))  # torque scale: force scale x half diagonal
        assert abs(gb[0]["T"][0] - ob["T"][0]) <= 2e-3 * gb[0]["S"] * lever, (gb[0]["T"], ob["T"])


def test_batch_of_more_than_64_tanks():
    """Tanks beyond the 64 of one launch go to a second group of launches."""
    scenes = [I.random_box_scene(12 + k % 5, 12 + k % 3, 12, seed=100 + k, nboxes=(k % 2), speed=0.02)
              for k in range(70)]
    steps = 12
    res, (launches, _) = _batched(scenes, "f32", steps, lanes=1)
    assert launches == 2 * 17 * steps
    for k in (0, 63, 64, 69):
        _same(res[k], _alone(scenes[k], "f32", steps))


def test_autotune_leaves_state_unchanged():
    scenes = _scenes()
    a, _ = _batched(scenes, "f32", 20, autotune=True)
    b, _ = _batched(scenes, "f32", 20, autotune=False)
    for x, y in zip(a, b):
        _same(x, y)


def test_batch_graph_and_stream_agree():
    """captured graphs and direct launches, both with two concurrent lanes"""
    scenes = _scenes()[:3]
    a, _ = _batched(scenes, "f32", 15, use_graphs=True, lanes=2)
    b, _ = _batched(scenes, "f32", 15, use_graphs=False, lanes=2)
    for x, y in zip(a, b):
        _same(x, y)


def test_box_added_between_batch_steps():
    from paper_1201_0351_gb300 import lbm_fs

    base = I.random_box_scene(30, 26, 20, seed=21, nboxes=0)
    extra = I.random_box_scene(30, 26, 20, seed=22, nboxes=1, speed=0.02).boxes[0]
    bt = lbm_fs.Batch([base, base], storage="f64")
    bt.step(5)
    bt.tanks[1].add_box(extra)
    bt.step(10)
    g = bt.tanks[1].fields(want_f=True)
    gb = bt.tanks[1].body(0)
    bt.close()
    sim = lbm_fs.Simulation(base, storage="f64")
    sim.step(5)
    sim.add_box(extra)
    sim.step(10)
    s = sim.fields(want_f=True)
    sb = sim.body(0)
    sim.close()
    assert np.array_equal(g["f"], s["f"]) and np.array_equal(g["flags"], s["flags"])
    assert np.array_equal(gb["F"], sb["F"])


def test_member_tank_cannot_be_stepped_or_destroyed():
    from paper_1201_0351_gb300 import lbm_fs

    bt = lbm_fs.Batch([I.random_box_scene(16, 16, 12, seed=3, nboxes=0)], storage="f32")
    h = bt.tanks[0].h
    for call in (lambda: lbm_fs.lbm_fs_step(h, 1), lambda: lbm_fs.lbm_fs_destroy(h),
                 lambda: lbm_fs.lbm_fs_kernel_times(h, 1)):
        with pytest.raises(lbm_fs.LbmFsError) as e:
            call()
        assert e.value.code == lbm_fs.LBM_FS_ESTATE
    bt.step(2)
    bt.sync()
    bt.close()
