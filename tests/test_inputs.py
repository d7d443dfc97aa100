"""The seeded synthetic workloads (no GPU): the random generator against its
published test vectors, and each workload's sizes, parameters and structure
against its stated recipe (the tank and box shapes of the paper's tests)."""
import math

import numpy as np

from paper_1201_0351_gb300 import inputs as I


def test_splitmix64_published_vectors():
    """splitmix64 (Vigna's reference generator): the outputs for seed 0 and
    for seed 1234567 that its reference implementation prints."""
    r = I.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    r = I.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_uniform_draws_are_53_bit_in_unit_interval():
    r = I.SplitMix64(I.SEED)
    u = np.array([r.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1.0 / 12.0) < 0.005


def test_hydrostatic_initial_state():
    """Filled cells carry rho = rho_G exp(3 g (eta - z_c)), the fill level is
    clamp(eta - z, 0, 1) per column, and the interface layer separates liquid
    from gas."""
    nx, ny, nz, g, eta = 6, 5, 12, 2e-5, 7.3
    flags, fill, rho = I.hydrostatic_tank(nx, ny, nz, lambda X, Y: eta, g, 1.0, 0)
    z = np.repeat(np.arange(nz), nx * ny)
    assert np.array_equal(fill, np.clip(eta - z, 0.0, 1.0))
    filled = fill > 0
    assert np.allclose(rho[filled], np.exp(3.0 * g * (eta - (z[filled] + 0.5))), rtol=0, atol=1e-15)
    assert np.all(rho[~filled] == 1.0)
    assert set(flags[z < 7]) == {I.LIQUID} and set(flags[z == 7]) == {I.INTERFACE} and set(flags[z > 7]) == {I.GAS}


def test_wave_tank_recipe():
    sc = I.wave_tank()
    assert (sc.nx, sc.ny, sc.nz, sc.nx * sc.ny * sc.nz) == (768, 384, 256, 75497472)
    assert (sc.tau, sc.gravity, sc.steps, sc.periodic) == (0.52, (0.0, 0.0, -1e-5), 2000, 0)
    assert len(sc.boxes) == 16
    c = np.array([b.center for b in sc.boxes])
    for b in sc.boxes:
        assert b.half == (12.0, 6.0, 4.0) and b.mode == I.MODE_FREE and 0.4 <= b.density_ratio < 0.6
        x, y, z = b.center
        assert 24.0 <= x < 744.0 and 12.0 <= y < 372.0
        # floating upright at its draft below the local surface
        eta = 128.0 + 8.0 * math.sin(2.0 * math.pi * x / 192.0)
        assert abs((z - 4.0) - (eta - 8.0 * b.density_ratio)) < 1e-12
    d = np.hypot(c[:, None, 0] - c[None, :, 0], c[:, None, 1] - c[None, :, 1])
    assert d[np.triu_indices(16, 1)].min() >= 40.0
    # the surface: the fill of column x sits where 128 + 8 sin(2 pi x_c / 192) puts it
    fill = sc.fill.reshape(256, 384, 768)
    for x in (0, 100, 333, 767):
        eta = 128.0 + 8.0 * math.sin(2.0 * math.pi * (x + 0.5) / 192.0)
        assert abs(fill[:, 7, x].sum() - eta) < 1e-9


def test_batched_sweep_recipe():
    tanks = I.batched_sweep_tanks(64)
    assert len(tanks) == 64
    assert sum(t.nx * t.ny * t.nz for t in tanks) == 38995946
    for t in tanks:
        e = t.nx
        assert t.nx == t.ny == t.nz and 48 <= e <= 112 and t.tau == 0.55 and t.gravity == (0.0, 0.0, -2e-5)
        (b,) = t.boxes
        assert np.allclose(b.half, (0.2 * e, 0.1 * e, 0.06 * e), rtol=0, atol=1e-12)
        assert 0.3 <= b.density_ratio < 0.7 and b.mode == I.MODE_ROT_AXIS_ONLY | I.MODE_DAMP_TRANSLATION
        heel = math.degrees(2.0 * math.atan2(b.quat[1], b.quat[0]))
        assert 0.0 <= heel < 30.0 and b.quat[2] == 0.0 and b.quat[3] == 0.0
        assert abs(b.center[0] - e / 2) < 1e-12 and abs(b.center[1] - e / 2) < 1e-12
    assert len({t.nx for t in tanks}) > 30  # uneven sizes


def test_floating_cubes_recipe():
    sc = I.floating_cubes()
    assert (sc.nx, sc.ny, sc.nz) == (130, 40, 40) and abs(sc.tau - 1.0 / 1.9) < 1e-15
    assert sc.gravity == (0.0, 0.0, -7.5e-4)
    assert [b.density_ratio for b in sc.boxes] == [0.75, 0.5, 0.25]
    for b in sc.boxes:
        assert b.half == (16.0, 8.0, 8.0) and b.rot_axis == (1.0, 0.0, 0.0)
        assert abs(math.degrees(2.0 * math.atan2(b.quat[1], b.quat[0])) - 2.86) < 1e-12
    fill = sc.fill.reshape(40, 40, 130)
    assert abs(fill[:, 20, 65].sum() - 20.0) < 1e-12  # half full
