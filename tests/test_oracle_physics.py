"""Pins of the oracle against closed forms, invariants and the paper's theory
(no GPU).  Each test names the passage it checks.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from paper_1201_0351_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scenario(nx, ny, nz, periodic, tau, flags, fill, rho, boxes=(), gravity=(0.0, 0.0, 0.0),
              body_accel=(0.0, 0.0, 0.0), vel=None, name="pin"):
    return I.Scenario(name, nx, ny, nz, periodic, tau, tuple(gravity), tuple(body_accel), 1.0, 1e-2,
                      flags, fill, rho, list(boxes), 0, vel)


# --------------------------------------------------------------- Sec. 2.1


def _shear_wave_error(L, tau=0.6, U=1e-3, t_per_L2=1000.0 / 32 ** 2):
    steps = int(round(t_per_L2 * L * L))
    fl, fi, rh = I.uniform_state(4, 4, L, I.LIQUID)
    z = np.arange(L) + 0.5
    prof = np.sin(2 * np.pi * z / L)
    vel = np.zeros((L, 4, 4, 3))
    vel[..., 0] = U * prof[:, None, None]
    s = oracle.OracleSim(_scenario(4, 4, L, 7, tau, fl, fi, rh, vel=vel.reshape(-1)))
    s.step(steps)
    u = s.fields()["u"].reshape(L, 4, 4, 3)[:, 0, 0, 0]
    amp = (u * prof).sum() / (prof * prof).sum()
    nu = (tau - 0.5) / 3.0
    expected = U * math.exp(-nu * (2 * math.pi / L) ** 2 * steps)
    return amp / expected - 1.0


def test_shear_wave_decay_second_order():
    """Eq. lbgk + tau = 3 nu + 1/2: a shear wave decays as exp(-nu k^2 t).  The
    lattice's own error is second order in the resolution: it falls by 4 from
    L = 32 to L = 64 (the same diffusive time), and the Richardson extrapolation
    (4 e64 - e32) / 3 removes it to below 1e-4 (a dropped or wrong term in the
    collision would leave an error that does not extrapolate away)."""
    e32 = _shear_wave_error(32)
    e64 = _shear_wave_error(64)
    assert abs(e32) < 1e-2
    assert 3.5 < e32 / e64 < 4.5
    assert abs((4.0 * e64 - e32) / 3.0) < 1e-4


def test_uniform_flow_is_preserved():
    """Galilean invariance of the periodic all-liquid lattice without forces."""
    n = 8
    fl, fi, rh = I.uniform_state(n, n, n, I.LIQUID)
    vel = np.tile([3e-3, -2e-3, 1e-3], n ** 3)
    s = oracle.OracleSim(_scenario(n, n, n, 7, 0.7, fl, fi, rh, vel=vel))
    s.step(50)
    f = s.fields()
    assert np.abs(f["u"] - vel.reshape(-1, 3)).max() < 1e-14
    assert np.abs(f["rho"] - 1.0).max() < 1e-14


def test_hydrostatic_profile_sign_and_slope():
    """Eq. pressure + Eq. forceterm: at rest the density follows
    rho = rho_G exp(3 g (eta - z)); its slope pins the sign of the force term."""
    sc = I.closed_tank_32(with_box=False)
    s = oracle.OracleSim(sc)
    acc, k = np.zeros(32), 0
    for _ in range(30):
        s.step(10)
        if s.time > 100:
            acc += s.fields()["rho"].reshape(32, 32, 32)[:, 16, 16]
            k += 1
    prof = acc / k
    z = np.arange(32) + 0.5
    slope = np.polyfit(z[:16], np.log(prof[:16]), 1)[0]
    assert slope == pytest.approx(-3e-5, rel=1e-2)
    expected = np.exp(3e-5 * (16.5 - z[:16]))
    assert np.abs(prof[:16] - expected).max() < 0.05 * 3e-5 * 16.5
    assert s.error == 0


def _planar(sc, steps, deadband=None):
    if deadband is not None:
        sc = dataclasses.replace(sc, readings=dict(deadband=deadband))
    s = oracle.OracleSim(sc)
    s.step(steps)
    f = s.fields()
    sh = (sc.nz, sc.ny, sc.nx)
    flags = f["flags"].reshape(sh)
    ifc = flags == I.INTERFACE
    u = f["u"].reshape(sh + (3,))
    bulk = u[flags == I.LIQUID].mean(axis=0)
    return (np.unique(np.nonzero(ifc)[0]), np.ptp(f["fill"].reshape(sh)[ifc]), np.abs(u[ifc] - bulk).max(),
            s.error)


def test_planar_surface_stays_planar():
    """Sec. 3.2.1: a planar free surface remains planar and the spurious
    interface velocities (deviation from the bulk velocity) stay below 1e-5 --
    in a closed tank at rest (tau 0.6, below the paper's lowest tau) and in the
    paper's channel (60 x 40 x 30, surface 19.5, walls moving with u = 1e-4,
    g = 1e-5, tau = 0.62)."""
    zs, spread, dev, err = _planar(I.closed_tank_32(with_box=False), 200)
    assert list(zs) == [16] and err == 0
    assert spread < 1e-3  # height variation of the surface, in cells
    assert dev < 1e-5
    ch = dataclasses.replace(I.free_advection_channel(tau=0.62, u=1e-4), boxes=[])
    zs, spread, dev, err = _planar(ch, 150)
    assert list(zs) == [19] and err == 0
    assert spread < 1e-3 and dev < 1e-5


def test_strict_sign_test_breaks_the_planar_bound():
    """The reading of Eq. reconstruct's c.n <= 0 set: with the bare sign test
    (dead band 0) the noise of the estimated normal decides the tangential
    directions of a flat surface cell by cell, and the spurious interface
    velocities of the same closed tank exceed the paper's 1e-5 several times
    over (measured 7e-5); with the default dead band they stay below it (previous
    test).  The surface stays one layer thick either way."""
    zs, spread, dev, err = _planar(I.closed_tank_32(with_box=False), 200, deadband=0.0)
    assert list(zs) == [16] and err == 0
    assert dev > 2e-5


# ----------------------------------------------------------- Sec. 2.2


def test_closed_tank_mass_conservation():
    """Sec. 2.2: the interface mass exchange is antisymmetric and excess mass is
    redistributed, so the liquid mass of a closed tank is conserved (booked
    covered / uncovered / lost mass included)."""
    sc = I.closed_tank_32()
    s = oracle.OracleSim(sc)
    s.step(200)
    L = s.ledger()
    resid = L["M"] - L["M0"] - (L["uncovered"] - L["covered"] - L["lost"] + L["wall"])
    assert abs(resid) <= 1e-13 * L["M0"]
    assert s.error == 0


def _duct(H=16.5, nz=20, tau=0.8, a=1e-6, steps=8000, deadband=None):
    fl, fi, rh = I.hydrostatic_tank(4, 4, nz, lambda X, Y: H, 0.0, 1.0, 3)
    sc = _scenario(4, 4, nz, 3, tau, fl, fi, rh, body_accel=(a, 0.0, 0.0))
    if deadband is not None:
        sc = dataclasses.replace(sc, readings=dict(deadband=deadband))
    s = oracle.OracleSim(sc)
    s.step(steps)
    f = s.fields()
    u = f["u"].reshape(nz, 4, 4, 3)[:, 0, 0, 0]
    flags = f["flags"].reshape(nz, 4, 4)[:, 0, 0]
    return u, flags, (tau - 0.5) / 3.0


@pytest.mark.parametrize("deadband", [None, 0.0])
def test_gravity_driven_layer_profile(deadband):
    """Sec. 2.2 free-surface condition (Eq. reconstruct): a liquid layer driven
    along x over a no-slip floor has the half-Poiseuille profile
    u = (a / nu)(H z - z^2 / 2).  The stress-free plane of the anti-bounce-back
    lies half-way between the interface cell and the gas cell above it (z = 17
    for the interface layer at z = 16); the curvature u'' = -a / nu is exact.
    Holds with the default dead band and with the bare sign test of the
    paper's c.n <= 0 set (the flat layer's normal has no tangential noise)."""
    a = 1e-6
    u, flags, nu = _duct(a=a, deadband=deadband)
    z = np.arange(20) + 0.5
    liq = flags == I.LIQUID
    ex = a / nu * (17.0 * z - z * z / 2.0)
    assert np.sqrt(((u - ex)[liq] ** 2).mean()) / ex[liq].max() < 5e-3
    d2 = u[:14] - 2 * u[1:15] + u[2:16]
    assert np.abs(d2[1:] / (-a / nu) - 1.0).max() < 3e-3


def test_duct_mutations_are_caught():
    """Reflecting the wrong population at a wall (f_q instead of f_qbar) or
    flipping the surface normal both spoil the layer profile."""
    a = 1e-6
    for m in (6, 7):
        oracle.set_mutation(m)
        u, flags, nu = _duct(a=a, steps=3000)
        oracle.set_mutation(0)
        z = np.arange(20) + 0.5
        liq = flags == I.LIQUID
        ex = a / nu * (17.0 * z - z * z / 2.0)
        u0, _, _ = _duct(a=a, steps=3000)
        assert np.abs(u - u0)[liq].max() > 0.05 * ex[liq].max(), m


def test_mass_mutation_is_caught():
    oracle.set_mutation(2)
    s = oracle.OracleSim(I.closed_tank_32())
    s.step(20)
    L = s.ledger()
    assert abs(L["M"] - L["M0"] - (L["uncovered"] - L["covered"] - L["lost"] + L["wall"])) > 1e-9 * L["M0"]


# ---------------------------------------------------- Sec. 2.3 and 2.4


def _box_scene(n, box, fill_fn, rho_fn, g=0.0):
    """Scene at rest with per-cell classes from fill_fn(z, y, x)."""
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    fill = fill_fn(zz, yy, xx).astype(np.float64)
    flags = np.where(fill >= 1.0, I.LIQUID, np.where(fill > 0.0, I.INTERFACE, I.GAS)).astype(np.uint8)
    flags = np.where(fill < 0.0, I.GAS, flags).astype(np.uint8)
    rho = rho_fn(zz, yy, xx).astype(np.float64)
    return _scenario(n, n, n, 0, 0.7, flags.reshape(-1), fill.reshape(-1), rho.reshape(-1), [box],
                     gravity=(0.0, 0.0, -g))


def test_uniform_pressure_gives_zero_force_and_torque():
    """Eqs. momentumexchange / momentuminterface: under a uniform pressure the
    link terms pair up along every lattice line, so F = T = 0 -- for any mix of
    liquid, interface (any fill level) and gas cells around a rotated box."""
    rng = np.random.default_rng(3)
    box = I.Box(center=(8.3, 7.9, 8.1), half=(3.2, 2.1, 2.6), quat=I.heel_quat(23.0, (0.6, 0.0, 0.8)))
    fills = rng.random((16, 16, 16)) * 1.4 - 0.2

    def fill_fn(z, y, x):
        return np.where(z < 6, 1.0, np.where(z > 10, 0.0, fills[z, y, x]))

    s = oracle.OracleSim(_box_scene(16, box, fill_fn, lambda z, y, x: np.ones(z.shape)))
    s.compute_forces()
    b = s.body(0)
    assert b["S"] > 1.0
    assert np.abs(b["F"]).max() <= 1e-14 * b["S"]
    assert np.abs(b["T"]).max() <= 1e-13 * b["S"]


def test_gas_pressure_term_mutation_is_caught():
    """Dropping the (1 - phi) f_eq(rho_G, 0) part of Eq. momentuminterface
    breaks the uniform-pressure balance on interface links."""
    oracle.set_mutation(4)
    box = I.Box(center=(8.0, 8.0, 8.0), half=(3.0, 3.0, 3.0))
    s = oracle.OracleSim(_box_scene(16, box, lambda z, y, x: np.where(z < 5, 0.5, 0.0),
                                    lambda z, y, x: np.ones(z.shape)))
    s.compute_forces()
    b = s.body(0)
    assert np.abs(b["F"]).max() > 1e-3


def _line_sum_fz(obst, rho_eff, w):
    """Independent brute-force sum along lattice lines: every line in a
    direction d with d_z = +1 that crosses the obstacle enters from a fluid
    cell below and leaves into one above; the pair contributes
    2 w_d (rho_eff(entry) - rho_eff(exit)) to F_z."""
    nz, ny, nx = obst.shape
    total = 0.0
    dirs = [((0, 0, 1), w[5]), ((-1, 0, 1), w[7]), ((1, 0, 1), w[8]), ((0, 1, 1), w[9]), ((0, -1, 1), w[10])]
    for (dx, dy, dz), wd in dirs:
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    if not obst[z, y, x]:
                        continue
                    pz, py, px = z - dz, y - dy, x - dx
                    if obst[pz, py, px]:
                        continue  # not the first obstacle cell of its line
                    qz, qy, qx = z, y, x
                    while obst[qz, qy, qx]:
                        qz, qy, qx = qz + dz, qy + dy, qx + dx
                    total += 2.0 * wd * (rho_eff[pz, py, px] - rho_eff[qz, qy, qx])
    return total


def test_submerged_box_line_sum_linear_pressure():
    """Eq. momentumexchange with the force on the body = -(momentum gained by
    the fluid): in a linear pressure field the exact discrete buoyancy of a fully
    submerged box is rho0 g sum_{pairs d} 6 w_d sum_lines (L + 1)."""
    n, g = 20, 1e-4
    box = I.Box(center=(10.0, 10.0, 9.0), half=(4.0, 3.0, 2.5), mode=I.MODE_FIXED)
    s = oracle.OracleSim(_box_scene(n, box, lambda z, y, x: np.ones(z.shape),
                                    lambda z, y, x: 1.0 + 3.0 * g * (15.0 - (z + 0.5)), g=g))
    s.compute_forces()
    b = s.body(0)
    _, w, _ = oracle.lattice()
    obst = (s.fields()["flags"] == oracle.OBSTACLE).reshape(n, n, n)
    # closed form: each line of L obstacle cells spans L + 1 cells of head
    closed = 0.0
    for (dx, dy, dz), wd in [((0, 0, 1), w[5]), ((-1, 0, 1), w[7]), ((1, 0, 1), w[8]), ((0, 1, 1), w[9]),
                             ((0, -1, 1), w[10])]:
        for z in range(n):
            for y in range(n):
                for x in range(n):
                    if obst[z, y, x] and not obst[z - dz, y - dy, x - dx]:
                        L = 0
                        while obst[z + L * dz, y + L * dy, x + L * dx]:
                            L += 1
                        closed += 6.0 * wd * g * (L + 1)
    assert b["F"][2] == pytest.approx(closed, rel=1e-12)
    assert np.abs(b["F"][:2]).max() <= 1e-14 * b["S"]
    assert np.abs(b["T"]).max() <= 1e-13 * b["S"]


def test_force_sign_mutation_is_caught():
    oracle.set_mutation(1)
    n, g = 20, 1e-4
    box = I.Box(center=(10.0, 10.0, 9.0), half=(4.0, 3.0, 2.5))
    s = oracle.OracleSim(_box_scene(n, box, lambda z, y, x: np.ones(z.shape),
                                    lambda z, y, x: 1.0 + 3.0 * g * (15.0 - (z + 0.5)), g=g))
    s.compute_forces()
    assert s.body(0)["F"][2] < 0.0


def _half_submerged(scale, eta_off=0.0, heel=0.0, b=8.0, h=6.0, l=8.0):
    """Fixed box of b x h cross-section straddling a hydrostatic surface."""
    g = 1e-5
    n = int(32 * scale)
    eta = n / 2 + 0.5 + eta_off
    fl, fi, rh = I.hydrostatic_tank(n, n, n, lambda X, Y: eta, g, 1.0, 0)
    box = I.Box(center=(n / 2, n / 2, n / 2 + 0.5), half=(0.5 * l * scale, 0.5 * b * scale, 0.5 * h * scale),
                quat=I.heel_quat(heel), mode=I.MODE_FIXED)
    sc = I.Scenario("half", n, n, n, 0, 0.6, (0.0, 0.0, -g), (0.0, 0.0, 0.0), 1.0, 1e-2, fl, fi, rh, [box], 0)
    return sc, g, eta


def test_half_submerged_box_line_sum():
    """Eq. momentuminterface at rest: an interface cell presses with
    phi rho + (1 - phi) rho_G, a gas cell with rho_G, so the exact t = 0 force on
    a half-submerged box is the line sum over those effective densities."""
    sc, g, eta = _half_submerged(1)
    s = oracle.OracleSim(sc)
    s.compute_forces()
    f = s.fields()
    n = sc.nx
    obst = (f["flags"] == oracle.OBSTACLE).reshape(n, n, n)
    flags0 = sc.flags.reshape(n, n, n)
    rho_eff = np.where(flags0 == I.LIQUID, sc.rho.reshape(n, n, n),
                       np.where(flags0 == I.INTERFACE, sc.fill.reshape(n, n, n) * sc.rho.reshape(n, n, n)
                                + (1 - sc.fill.reshape(n, n, n)) * 1.0, 1.0))
    _, w, _ = oracle.lattice()
    fz = _line_sum_fz(obst, rho_eff, w)
    assert s.body(0)["F"][2] == pytest.approx(fz, rel=1e-9)


def test_archimedes_converges_with_resolution():
    """Sec. 3.2: buoyancy rho g V of the displaced volume; the staircase /
    half-way bounce-back error is first order in the resolution."""
    errs = []
    for scale in (1, 2):
        sc, g, eta = _half_submerged(scale)
        s = oracle.OracleSim(sc)
        s.compute_forces()
        b = s.body(0)
        n = sc.nx
        vol = (8 * scale) * (8 * scale) * (eta - (n / 2 + 0.5 - 3 * scale))
        errs.append(b["F"][2] / (g * vol) - 1.0)
        assert np.abs(b["F"][:2]).max() <= 1e-12 * b["S"]
    assert 0 < errs[0] < 0.3
    assert 0 < errs[1] < 0.7 * errs[0]


def test_closed_tank_box_force_after_200_steps():
    """The 32^3 closed tank with the fixed 8 x 8 x 6 box half immersed: at rest
    the liquid stays hydrostatic, so after 200 steps the buoyancy equals the
    exact t = 0 line sum of Eq. momentumexchange / momentuminterface within 1 %
    and the lateral force vanishes (below 1e-3 of F_z).  Against Archimedes'
    rho g V_displaced (V = 8 * 8 * 3.5 below the surface plane 16.5) the force
    is high by the half-cell offset of the half-way bounce-back pressure (the
    head is measured at the fluid cell centre half a cell below the box's
    floor, and the diagonal lines add one cell each), a first-order staircase
    error that the resolution test above shows shrinking."""
    sc = I.closed_tank_32()
    s0 = oracle.OracleSim(sc)
    s0.compute_forces()
    f0 = s0.body(0)["F"][2]
    s = oracle.OracleSim(sc)
    s.step(200)
    b = s.body(0)
    assert b["F"][2] == pytest.approx(f0, rel=1e-2)
    assert np.abs(b["F"][:2]).max() < 1e-3 * b["F"][2]
    arch = 1e-5 * 8 * 8 * 3.5
    assert 1.0 < b["F"][2] / arch < 1.25
    assert s.error == 0


def test_buoyancy_linear_in_level():
    """Sec. 3.2: with a fixed box and a varying water level the buoyant force is
    continuous and linear in the level (the fill level of the interface cells
    enters Eq. momentuminterface), not a staircase."""
    levels = np.linspace(-0.9, 0.9, 10)
    fz = []
    for off in levels:
        sc, g, eta = _half_submerged(1, eta_off=off)
        s = oracle.OracleSim(sc)
        s.compute_forces()
        fz.append(s.body(0)["F"][2])
    fz = np.array(fz)
    p = np.polyfit(levels, fz, 1)
    resid = fz - np.polyval(p, levels)
    r2 = 1 - (resid ** 2).sum() / ((fz - fz.mean()) ** 2).sum()
    assert r2 > 0.999
    assert p[0] == pytest.approx(g * 64, rel=0.1)


def _golden_box():
    vals = {}
    for line in open(os.path.join(GOLDEN, "wall_sided_box.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _heel_torque(scale, alpha):
    gv = _golden_box()
    b, h, l = gv["b"] * scale, gv["h"] * scale, gv["l"] * scale
    nx, ny, nz = int(l + 8), int(3 * b), int(3 * h)
    g = 1e-4
    eta = math.floor(nz / 2) + 0.5
    fl, fi, rh = I.hydrostatic_tank(nx, ny, nz, lambda X, Y: eta, g, 1.0, 0)
    box = I.Box(center=(nx / 2, ny / 2, eta), half=(l / 2, b / 2, h / 2), quat=I.heel_quat(alpha),
                density_ratio=0.5, mode=I.MODE_FIXED)
    sc = I.Scenario("heel", nx, ny, nz, 0, 1.0, (0.0, 0.0, -g), (0.0, 0.0, 0.0), 1.0, 1e-2, fl, fi, rh, [box], 0)
    s = oracle.OracleSim(sc)
    s.compute_forces()
    d = h / 2
    bm0 = b * b / (12 * d)
    gm0 = d / 2 + bm0 - h / 2
    a = math.radians(alpha)
    gz = math.sin(a) * (gm0 + 0.5 * bm0 * math.tan(a) ** 2)
    return s.body(0)["T"][0], g * l * b * d * gz, gz


def test_wall_sided_righting_moment():
    """Sec. 3.2.2 (Scribanti): the righting moment of the half-immersed heeled
    box, m_s = rho g V GZ, is reproduced by the momentum-exchange torque and the
    error decreases with resolution (the paper's convergence statement)."""
    gv = _golden_box()
    t1, ms1, gz = _heel_torque(1, 10.0)
    assert gz == pytest.approx(gv["GZ_10deg"], abs=1e-4)
    assert t1 < 0  # restoring: opposes the positive heel about x
    e1 = abs(-t1 / ms1 - 1.0)
    assert e1 < 0.1
    t2, ms2, _ = _heel_torque(2, 10.0)
    e2 = abs(-t2 / ms2 - 1.0)
    assert e2 < 0.75 * e1


def test_galilean_body_follows_uniform_flow():
    """Sec. 3.2.1 first series: in uniform liquid flow without gravity a body of
    the liquid's density moves with the flow ('to the last digit'), while it
    covers and uncovers cells (Eq. noslip moving-wall term, obstacle-to-fluid
    rule with f = f_eq(rho, u_w))."""
    n = 16
    u0 = np.array([6e-3, -2.5e-3, 1.5e-3])
    fl, fi, rh = I.uniform_state(n, n, n, I.LIQUID)
    vel = np.tile(u0, n ** 3)
    box = I.Box(center=(8.2, 7.7, 8.4), half=(3.1, 2.2, 2.6), quat=I.heel_quat(17.0, (0.0, 0.6, 0.8)),
                density_ratio=1.0, vel=tuple(u0), mode=I.MODE_FREE)
    s = oracle.OracleSim(_scenario(n, n, n, 7, 0.8, fl, fi, rh, boxes=[box], vel=vel))
    s.step(400)
    b = s.body(0)
    L = s.ledger()
    assert L["covered"] > 10 and L["uncovered"] > 10
    assert np.abs(b["vel"] - u0).max() < 1e-12
    assert np.abs(b["omega"]).max() < 1e-12
    f = s.fields()
    fluid = f["flags"] == I.LIQUID
    assert np.abs(f["u"][fluid] - u0).max() < 1e-12
    assert s.error == 0


def test_mass_ledger_with_moving_free_boxes():
    """Liquid mass changes only through covered / uncovered cells, excess mass
    that finds no interface neighbour, and the moving-wall term of Eq. noslip
    (which adds 6 w rho c.u_w to a liquid cell at a moving obstacle link)."""
    sc = I.random_box_scene(40, 30, 22, seed=5, nboxes=3, speed=0.02)
    s = oracle.OracleSim(sc)
    s.step(80)
    L = s.ledger()
    assert L["covered"] > 1 and L["uncovered"] > 1 and abs(L["wall"]) > 1e-3
    resid = L["M"] - L["M0"] - (L["uncovered"] - L["covered"] - L["lost"] + L["wall"])
    assert abs(resid) <= 1e-12 * L["M0"]
    assert s.error == 0
