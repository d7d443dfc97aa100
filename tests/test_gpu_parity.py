"""GPU path (through the C ABI) against the CPU oracle, element by element.

Double precision: cell classes identical, populations / fill / mass within
1e-11 relative, forces within 1e-11 of |F| (or of the link-term sum S when F
cancels) after the stated number of steps.  Reduced precision: errors of the
macroscopic fields against the oracle within the stated tolerances.
"""
import dataclasses

import numpy as np
import pytest

from paper_1201_0351_gb300 import inputs as I

from parity import assert_f64_parity, macro_errors, run_both, velocity_check

pytestmark = pytest.mark.gpu


def test_closed_tank_fixed_box_200_steps():
    """32^3 closed tank, fixed 8x8x6 box at the surface, 200 steps."""
    g, o, gb, ob, gs, _ = run_both(I.closed_tank_32(), 200)
    assert_f64_parity(g, o, gb, ob)


def test_channel_free_box_200_steps():
    """96x32x32 channel, periodic in x, body force, free box of density 0.5."""
    g, o, gb, ob, gs, _ = run_both(I.channel_96x32x32(), 200)
    assert_f64_parity(g, o, gb, ob)


def test_ragged_moving_boxes():
    """odd sizes (ragged x tiles), two moving rotated boxes: conversions
    and cover / uncover every few steps"""
    sc = I.random_box_scene(37, 23, 19, seed=5, nboxes=2, speed=0.02)
    g, o, gb, ob, gs, ref = run_both(sc, 90, chunks=3)
    L = ref.ledger()
    assert L["covered"] > 0 and L["uncovered"] > 0
    assert_f64_parity(g, o, gb, ob)


def test_periodic_moving_box_galilean():
    n = 16
    u0 = np.array([6e-3, -2.5e-3, 1.5e-3])
    fl, fi, rh = I.uniform_state(n, n, n, I.LIQUID)
    box = I.Box(center=(8.2, 7.7, 8.4), half=(3.1, 2.2, 2.6), quat=I.heel_quat(17.0, (0.0, 0.6, 0.8)),
                density_ratio=1.0, vel=tuple(u0), mode=I.MODE_FREE)
    sc = I.Scenario("galilean", n, n, n, 7, 0.8, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 1.0, 1e-2, fl, fi, rh, [box], 0,
                    np.tile(u0, n ** 3))
    g, o, gb, ob, gs, _ = run_both(sc, 200)
    assert_f64_parity(g, o, gb, ob)
    assert np.abs(gb[0]["vel"] - u0).max() < 1e-12


def test_surface_conversions_filled_and_emptied():
    """interface cells that fill and empty in the first step (Sec. 2.2 rules)"""
    n = 12
    flags = np.full((n, n, n), I.GAS, np.uint8)
    fill = np.zeros((n, n, n))
    flags[:5] = I.LIQUID
    fill[:5] = 1.0
    flags[5] = I.INTERFACE
    fill[5] = 0.5
    fill[5, 3, 3] = 1.6
    fill[5, 3, 4] = -0.5
    fill[5, 8, 8] = -0.4
    fill[5, 6, 9] = 1.3
    sc = I.Scenario("conv", n, n, n, 0, 0.7, (0.0, 0.0, -1e-5), (0.0, 0.0, 0.0), 1.0, 1e-2, flags.reshape(-1),
                    fill.reshape(-1), np.ones(n ** 3), [], 0)
    g, o, gb, ob, gs, ref = run_both(sc, 5)
    assert_f64_parity(g, o, gb, ob)


def test_no_bodies_and_all_gas_columns():
    sc = I.closed_tank_32(with_box=False)
    g, o, gb, ob, gs, _ = run_both(sc, 50)
    assert_f64_parity(g, o, gb, ob)


def test_shear_wave_periodic_thin():
    """fully periodic 1 x 4 x 32 grid (neighbours wrap onto the cell itself)"""
    L = 32
    fl, fi, rh = I.uniform_state(1, 4, L, I.LIQUID)
    z = np.arange(L) + 0.5
    vel = np.zeros((L, 4, 1, 3))
    vel[..., 0] = 1e-3 * np.sin(2 * np.pi * z / L)[:, None, None]
    sc = I.Scenario("sw", 1, 4, L, 7, 0.6, (0, 0, 0), (0, 0, 0), 1.0, 1e-2, fl, fi, rh, [], 0, vel.reshape(-1))
    g, o, gb, ob, gs, _ = run_both(sc, 100)
    assert_f64_parity(g, o, gb, ob)


def test_graph_and_stream_launch_agree():
    sc = I.random_box_scene(30, 26, 22, seed=3, nboxes=2, speed=0.02)
    from paper_1201_0351_gb300 import lbm_fs
    out = []
    for graphs in (True, False):
        sim = lbm_fs.Simulation(sc, storage="f64", use_graphs=graphs)
        sim.step(30)
        out.append((sim.fields(want_f=True), sim.body(0)))
        sim.close()
    assert np.array_equal(out[0][0]["flags"], out[1][0]["flags"])
    assert np.array_equal(out[0][0]["f"], out[1][0]["f"])
    assert np.array_equal(out[0][1]["F"], out[1][1]["F"])


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16s", 2e-3)])
def test_reduced_precision_closed_tank(storage, tol):
    """FP32 / FP16-shifted storage against the FP64 oracle after 200 steps of
    the closed tank with the fixed box: density relative error, buoyancy, and
    velocity within tol of the largest oracle speed plus the storage's
    rounding floor (at rest the speeds are ~1e-5, near that floor)."""
    g, o, gb, ob, gs, ref = run_both(I.closed_tank_32(), 200, storage=storage)
    e = macro_errors(g, o)
    e_liq, e_if, bound, umax = velocity_check(g, o, storage, tol, 200)
    print(storage, e, "liquid", e_liq, "interface", e_if, "bound", bound)
    assert e["flag_diff"] == 0, e
    assert e["rho"] <= tol, e
    assert e_liq <= bound and e_if <= bound, (e_liq, e_if, bound)
    fz = ob[0]["F"][2]
    assert abs(gb[0]["F"][2] - fz) <= tol * gb[0]["S"], (gb[0]["F"], ob[0]["F"])


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16s", 2e-3)])
def test_reduced_precision_channel_velocity(storage, tol):
    """Body-force driven channel with the free box, after 200 steps: density
    error, and the velocity error of liquid and interface cells within tol of
    the largest oracle speed plus the storage's rounding floor."""
    g, o, gb, ob, gs, ref = run_both(I.channel_96x32x32(), 200, storage=storage)
    e = macro_errors(g, o)
    e_liq, e_if, bound, umax = velocity_check(g, o, storage, tol, 200)
    print(storage, e, "liquid", e_liq, "interface", e_if, "bound", bound, "tol*umax", tol * umax)
    assert e["flag_diff"] == 0 and e["rho"] <= tol, e
    assert e_liq <= bound and e_if <= bound, (e_liq, e_if, bound)


def test_mass_ledger_identity_f64():
    sc = I.random_box_scene(40, 30, 22, seed=5, nboxes=3, speed=0.02)
    from paper_1201_0351_gb300 import lbm_fs
    sim = lbm_fs.Simulation(sc, storage="f64")
    sim.step(80)
    s = sim.stats()
    sim.close()
    resid = s["liquid_mass"] - s["mass0"] - (s["uncovered"] - s["covered"] - s["lost_excess"] + s["wall_source"])
    assert abs(resid) <= 1e-12 * s["mass0"], s
    assert s["covered"] > 0 and abs(s["wall_source"]) > 1e-3


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_reduced_precision_mass_drift(storage):
    """Total liquid mass drift below 1e-9 per 10^4 steps (closed tank with the
    fixed box: no moving-wall source, so M - M0 - ledger measures rounding
    drift alone)."""
    from paper_1201_0351_gb300 import lbm_fs
    steps = 400
    sim = lbm_fs.Simulation(I.closed_tank_32(), storage=storage)
    sim.step(steps)
    s = sim.stats()
    sim.close()
    resid = s["liquid_mass"] - s["mass0"] - (s["uncovered"] - s["covered"] - s["lost_excess"] + s["wall_source"])
    drift_per_1e4 = abs(resid) / s["mass0"] * (1e4 / steps)
    print(storage, "drift per 1e4 steps", drift_per_1e4)
    assert drift_per_1e4 < 1e-9, s


@pytest.mark.parametrize("storage", ["f32", "f16s"])
@pytest.mark.parametrize("variant,dims", [("pipe", (40, 30, 22)), ("pipe", (37, 23, 19)), ("tma", (40, 30, 22))])
def test_bulk_kernel_variants_match_plain_kernel(storage, variant, dims, monkeypatch):
    """The software-pipelined and the TMA-staged bulk kernels read the same
    populations as the plain one (through shared memory instead of direct
    loads): results are bit-identical, also for an odd cell count."""
    from paper_1201_0351_gb300 import lbm_fs
    sc = I.random_box_scene(*dims, seed=5, nboxes=2, speed=0.02)
    out = []
    for v in (variant, "plain"):
        monkeypatch.setenv("LBMFS_BULK", v)
        sim = lbm_fs.Simulation(sc, storage=storage)
        sim.step(40)
        out.append((sim.fields(want_f=True), sim.body(0)))
        sim.close()
    assert np.array_equal(out[0][0]["flags"], out[1][0]["flags"])
    assert np.array_equal(out[0][0]["f"], out[1][0]["f"])
    assert np.array_equal(out[0][1]["F"], out[1][1]["F"])


def test_box_reaching_a_wall_is_reported():
    """A free box coasting through an all-gas tank (uniform gas pressure, no
    net force) reaches the far wall: the library stops with a contact error
    rather than running on without a contact model."""
    from paper_1201_0351_gb300 import lbm_fs

    n = 40
    flags = np.full(n * n * n, I.GAS, np.uint8)
    sc = I.Scenario("coasting_box", n, n, n, 0, 0.7, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 1.0, 1e-2, flags,
                    np.zeros(n ** 3), np.ones(n ** 3),
                    [I.Box(center=(20.3, 20.2, 20.1), half=(4.0, 3.0, 3.0), vel=(0.1, 0.0, 0.0), mode=I.MODE_FREE,
                           density_ratio=0.5)], 200)
    sim = lbm_fs.Simulation(sc, storage="f32")
    sim.step(100)
    sim.sync()  # still 11 cells from the wall
    sim.step(100)
    with pytest.raises(lbm_fs.LbmFsError) as e:
        sim.sync()
    sim.close()
    assert e.value.code == lbm_fs.LBM_FS_EUNSTABLE and "wall" in str(e.value)


@pytest.mark.parametrize("fill_value", [0.3, 0.95])
def test_neighbour_conversion_rule_parity(fill_value):
    """A lone splash cell (no liquid neighbour) and an enclosed interface cell
    (no gas neighbour) convert as in the oracle."""
    import test_oracle_conversions as T

    g, o, gb, ob, gs, ref = run_both(T._pool_with_cell(I.INTERFACE, fill_value), 20, storage="f64")
    assert_f64_parity(g, o, gb, ob)


def test_rising_droplet_crosses_skipped_tiles():
    """A droplet launched upward through an all-gas column: the bulk kernel
    skips tiles above the previous step's fluid top, so the drop rising by
    many planes checks that the tracked top follows it (F64 parity after 300
    steps, the top plane risen by at least 8 cells, no error status)."""
    n, nz = 16, 40
    drop = I.droplet(n, 4.0, sigma=0.0, seed_offset=(8.0, 8.0, 6.0))
    pad = (nz - n) * n * n
    flags = np.concatenate([drop.flags, np.full(pad, I.GAS, np.uint8)])
    fill = np.concatenate([drop.fill, np.zeros(pad)])
    sc = dataclasses.replace(drop, name="rising_droplet", nz=nz, flags=flags, fill=fill, rho=np.ones(n * n * nz),
                             vel=np.tile([0.0, 0.0, 0.05], n * n * nz))
    g, o, gb, ob, gs, _ = run_both(sc, 300, chunks=3)
    assert gs["status"] == 0
    assert_f64_parity(g, o, gb, ob)
    fluid_z = np.nonzero((g["flags"] == I.LIQUID) | (g["flags"] == I.INTERFACE))[0] // (n * n)
    assert fluid_z.max() >= 10 + 8, fluid_z.max()


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16s", 2e-3)])
def test_reduced_precision_box_across_periodic_seams(storage, tol):
    """A moving, rotated box whose cell range wraps around the periodic seams
    on every axis (the float force kernel maps the wrapped rows to threads):
    after 120 steps its force and torque match the oracle within the storage's
    tolerance of the link-term sum S, the density within the tolerance and the
    velocity within tol of the largest speed plus the rounding floor."""
    n = 16
    u0 = np.array([6e-3, -2.5e-3, 1.5e-3])
    fl, fi, rh = I.uniform_state(n, n, n, I.LIQUID)
    box = I.Box(center=(1.3, 14.6, 0.8), half=(3.1, 2.2, 2.6), quat=I.heel_quat(17.0, (0.0, 0.6, 0.8)),
                density_ratio=1.0, vel=(0.0, 0.0, 0.0), mode=I.MODE_FIXED)
    sc = I.Scenario("periodic_seams", n, n, n, 7, 0.8, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 1.0, 1e-2, fl, fi, rh,
                    [box], 0, np.tile(u0, n ** 3))
    g, o, gb, ob, gs, _ = run_both(sc, 120, storage=storage)
    e = macro_errors(g, o)
    e_liq, e_if, bound, umax = velocity_check(g, o, storage, tol, 120)
    print(storage, e, "liquid", e_liq, "bound", bound, "tol*umax", tol * umax)
    assert e["flag_diff"] == 0, e
    assert e["rho"] <= tol and e_liq <= bound and e_if <= bound, (e, e_liq, e_if, bound)
    for key in ("F", "T"):
        assert np.abs(np.asarray(gb[0][key]) - np.asarray(ob[0][key])).max() <= tol * ob[0]["S"], (key, gb[0], ob[0])
