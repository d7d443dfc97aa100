"""Pins of the oracle's rigid-body update (the role Sec. 2.3 gives the pe
engine: the body moves under the momentum-exchange force and torque and under
gravity) against closed forms of rigid-body mechanics (no GPU).

The update is driven here by scripted forces and torques (orc_set_body_force +
orc_bodies_step, no fluid), so each pin isolates one part of it:
  * the virtual-mass scheme reaches Newton's acceleration (F + m g) / m of the
    body's own mass m = rho_s V (V = 8 h0 h1 h2 for half extents h, 4/3 pi r^3
    for a sphere), geometrically with the ratio C m_f / (m + C m_f);
  * the angular update reaches Euler's T / I with the textbook moments of a
    cuboid, m (b^2 + c^2) / 12 for full edges b, c, and of a sphere, 2/5 m r^2;
  * about a single axis a the moment is a^T I a in the body frame;
  * a torque-free symmetric top precesses at (I3 - I1) omega3 / I1 (Euler's
    equations), which fixes the sign of the gyroscopic term;
  * the first-order quaternion update by the world-frame angular velocity
    turns the body by 2 atan(|omega| / 2) per step about omega;
  * translation damping is geometric, the semi-implicit position a geometric sum;
  * the two-step force mean removes a force component that flips every step.
Planted mistakes (an inertia factor of 12 with half extents, the virtual mass
left out of the denominator, a flipped gyroscopic term, the body-frame
quaternion product, the volume without its factor 8) each fail one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1201_0351_gb300 import inputs as I

FAR = (100.0, 100.0, 100.0)  # body centre outside the 4^3 grid: no cell is covered


def _rig(box, gravity=(0.0, 0.0, 0.0), periodic=0, n=4, readings=None):
    fl, fi, rh = I.uniform_state(n, n, n, I.GAS, fill=0.0)
    sc = I.Scenario("c5", n, n, n, periodic, 0.6, tuple(gravity), (0.0, 0.0, 0.0), 1.0, 1e-2, fl, fi, rh, [box], 0,
                    readings=readings)
    return oracle.OracleSim(sc)


def _drive(s, steps, F=(0.0, 0.0, 0.0), T=(0.0, 0.0, 0.0)):
    """Apply F(n), T(n) (callables or constants) for `steps` updates; returns
    the body states after each update."""
    out = []
    for k in range(steps):
        f = F(k) if callable(F) else F
        t = T(k) if callable(T) else T
        s.set_body_force(0, f, t)
        s.bodies_step()
        out.append(s.body(0))
    return out


def _box_volume(h):
    return (2 * h[0]) * (2 * h[1]) * (2 * h[2])


def _box_moments(m, h):
    """Principal moments of a solid cuboid with full edges 2 h (textbook)."""
    a, b, c = 2 * h[0], 2 * h[1], 2 * h[2]
    return np.array([m * (b * b + c * c) / 12.0, m * (a * a + c * c) / 12.0, m * (a * a + b * b) / 12.0])


def _rotmat(q):
    """Rotation matrix of the unit quaternion (w, x, y, z), body -> world."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _qmul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw])


# ------------------------------------------------------------- translation


def _newton_error(h=(3.0, 2.0, 1.5), dens=0.5, shape=0):
    F = np.array([2e-3, -1e-3, 5e-4])
    g = np.array([0.0, 0.0, -1e-5])
    box = I.Box(center=FAR, half=h, density_ratio=dens, mode=I.MODE_FREE, shape=shape)
    s = _rig(box, gravity=g)
    st = _drive(s, 300, F=F)
    V = _box_volume(h) if shape == 0 else 4.0 / 3.0 * math.pi * h[0] ** 3
    m = dens * V
    acc = st[-1]["vel"] - st[-2]["vel"]
    expected = (F + m * g) / m
    return np.abs(acc - expected).max() / np.abs(expected).max()


def test_translation_reaches_newton_acceleration():
    """After the virtual-mass transient a constant force gives the body the
    acceleration (F + m g) / m of its own mass m = rho_s V."""
    assert _newton_error() < 1e-12
    assert _newton_error(dens=1.7) < 1e-12
    assert _newton_error(h=(2.5, 2.5, 2.5), shape=I.SHAPE_SPHERE) < 1e-12


def test_virtual_mass_transient_is_geometric():
    """(m + C m_f) dv_{n+1} = F + m g + C m_f dv_n from rest: dv_n = a (1 - r^n)
    with a = (F + m g) / m and r = C m_f / (m + C m_f); C = 0 is the explicit
    Newton update (dv = a from the first step)."""
    h, dens = (3.0, 2.0, 1.5), 0.5
    F = np.array([0.0, 0.0, 3e-3])
    V = _box_volume(h)
    m = dens * V
    a = F[2] / m
    for C in (1.0, 0.5, 0.0):
        s = _rig(I.Box(center=FAR, half=h, density_ratio=dens, mode=I.MODE_FREE),
                 readings=dict(virtual_mass=C))
        st = _drive(s, 40, F=F)
        r = C * V / (m + C * V)
        v = np.array([b["vel"][2] for b in st])
        dv = np.diff(np.concatenate([[0.0], v]))
        n = np.arange(1, 41)
        assert np.abs(dv - a * (1 - r ** n)).max() <= 1e-13 * a, C


def test_neutral_body_stays_at_rest():
    """A fully submerged body of the liquid's density: buoyancy -rho V g
    cancels its weight exactly, so it never moves."""
    h = (3.0, 2.0, 1.5)
    g = -1e-5
    V = _box_volume(h)
    s = _rig(I.Box(center=FAR, half=h, density_ratio=1.0, mode=I.MODE_FREE), gravity=(0.0, 0.0, g))
    st = _drive(s, 50, F=(0.0, 0.0, -V * g))
    assert all(np.all(b["vel"] == 0.0) for b in st)
    assert np.all(st[-1]["center"] == np.array(FAR))


# ---------------------------------------------------------------- rotation


def _euler_error(axis, h=(3.0, 2.0, 1.5), dens=0.5, shape=0, tau=1e-3):
    T = np.zeros(3)
    T[axis] = tau
    s = _rig(I.Box(center=FAR, half=h, density_ratio=dens, mode=I.MODE_FREE, shape=shape))
    st = _drive(s, 300, T=T)
    if shape == 0:
        Iax = _box_moments(dens * _box_volume(h), h)[axis]
    else:
        Iax = 0.4 * dens * (4.0 / 3.0 * math.pi * h[0] ** 3) * h[0] ** 2
    alpha = st[-1]["omega"] - st[-2]["omega"]
    expected = np.zeros(3)
    expected[axis] = tau / Iax
    return np.abs(alpha - expected).max() / abs(expected[axis])


def test_rotation_reaches_euler_acceleration():
    """A constant torque about a principal axis gives the angular acceleration
    T / I with the cuboid's moments m (b^2 + c^2) / 12 (the gyroscopic term
    vanishes about a principal axis)."""
    for axis in range(3):
        assert _euler_error(axis) < 1e-12, axis
    assert _euler_error(1, h=(2.5, 2.5, 2.5), shape=I.SHAPE_SPHERE) < 1e-12


def test_rotation_about_one_axis_uses_its_moment():
    """Rotation about the world x axis only, with the box turned by 30 deg about
    z: the moment is cos^2 I_x + sin^2 I_y, torque components off the axis do
    nothing and the angular velocity stays along the axis."""
    h, dens = (3.0, 2.0, 1.5), 0.5
    q0 = I.heel_quat(30.0, (0.0, 0.0, 1.0))
    box = I.Box(center=FAR, half=h, quat=q0, density_ratio=dens, mode=I.MODE_ROT_AXIS_ONLY, rot_axis=(1.0, 0.0, 0.0))
    s = _rig(box)
    T = (1e-3, 4e-3, -7e-3)
    st = _drive(s, 300, T=T)
    Im = _box_moments(dens * _box_volume(h), h)
    c, sn = math.cos(math.radians(30.0)), math.sin(math.radians(30.0))
    Ia = c * c * Im[0] + sn * sn * Im[1]
    alpha = st[-1]["omega"][0] - st[-2]["omega"][0]
    assert alpha == pytest.approx(T[0] / Ia, rel=1e-12)
    assert all(b["omega"][1] == 0.0 and b["omega"][2] == 0.0 for b in st)
    # the rotation is about world x: the body's x-row of R^T x stays put
    R = _rotmat(st[-1]["quat"])
    assert np.allclose(R.T @ np.array([1.0, 0.0, 0.0]), [c, -sn, 0.0], atol=1e-12)


def _quat_turn_error(h=(3.0, 2.0, 1.5), q0=(1.0, 0.0, 0.0, 0.0), w=0.02, steps=500):
    box = I.Box(center=FAR, half=h, quat=q0, density_ratio=0.5, omega=(0.0, 0.0, w), mode=I.MODE_FREE)
    s = _rig(box)
    st = _drive(s, steps)
    th = steps * 2.0 * math.atan(0.5 * w)
    rz = np.array([math.cos(0.5 * th), 0.0, 0.0, math.sin(0.5 * th)])
    expected = _qmul(rz, np.array(q0))
    q = st[-1]["quat"]
    q = q if np.dot(q, expected) >= 0 else -q
    return np.abs(q - expected).max(), st


def test_quaternion_turns_by_exact_angle():
    """q <- normalise(q + 1/2 (0, w) q): one step is the rotation by
    2 atan(|w| / 2) about w (applied on the world side), so a torque-free body
    spinning about a principal axis, or a cube about any axis (no gyroscopic
    term), ends at rz(n theta) q0."""
    err, st = _quat_turn_error()
    assert err < 1e-12
    assert all(abs(np.linalg.norm(b["quat"]) - 1.0) < 1e-15 for b in st)
    err, _ = _quat_turn_error(h=(2.0, 2.0, 2.0), q0=I.heel_quat(30.0))
    assert err < 1e-12


def _precession_rate(h=(2.0, 2.0, 5.0), dens=0.5, w_perp=2e-3, w3=1e-2, n0=100, n1=300):
    box = I.Box(center=FAR, half=h, density_ratio=dens, omega=(w_perp, 0.0, w3), mode=I.MODE_FREE)
    s = _rig(box)
    st = _drive(s, n1)
    ang = []
    for b in (st[n0 - 1], st[n1 - 1]):
        wb = _rotmat(b["quat"]).T @ b["omega"]
        ang.append(math.atan2(wb[1], wb[0]))
    d = (ang[1] - ang[0] + math.pi) % (2 * math.pi) - math.pi
    Im = _box_moments(dens * _box_volume(h), h)
    return d / (n1 - n0), (Im[2] - Im[0]) * w3 / Im[0], st


def test_symmetric_top_precesses_at_euler_rate():
    """Euler's equations for a torque-free symmetric top (I1 = I2): the
    body-frame (w1, w2) turns at (I3 - I1) w3 / I1 while w3 and |(w1, w2)| stay
    constant; the sign fixes the gyroscopic term -w x (I w).  The update is
    first order in time: over 300 steps at a turn of 7e-3 rad per step the
    perpendicular part grows by a few per cent (explicit Euler alone: 0.8 %)."""
    rate, expected, st = _precession_rate()
    assert rate == pytest.approx(expected, rel=1e-2)
    wb = [_rotmat(b["quat"]).T @ b["omega"] for b in st]
    assert abs(wb[-1][2] / wb[0][2] - 1.0) < 1e-6
    assert abs(np.linalg.norm(wb[-1][:2]) / np.linalg.norm(wb[0][:2]) - 1.0) < 5e-2


# --------------------------------------------------- damping and position


def test_damped_translation_is_geometric():
    """v *= (1 - lambda) every step; the semi-implicit position o += v_{n+1}
    is then the geometric sum o_0 + v_0 (1 - l)(1 - (1 - l)^n) / l."""
    lam = 0.05
    v0 = np.array([1e-2, -2e-3, 5e-3])
    o0 = np.array(FAR)
    box = I.Box(center=FAR, half=(3.0, 2.0, 1.5), density_ratio=0.5, vel=tuple(v0),
                mode=I.MODE_FREE | I.MODE_DAMP_TRANSLATION, lin_damping=lam)
    s = _rig(box)
    st = _drive(s, 100)
    for n in (1, 10, 100):
        k = (1 - lam) ** n
        assert np.abs(st[n - 1]["vel"] - v0 * k).max() <= 1e-14 * np.abs(v0).max()
        assert np.abs(st[n - 1]["center"] - (o0 + v0 * (1 - lam) * (1 - k) / lam)).max() < 1e-12


def test_position_wraps_on_periodic_axes():
    box = I.Box(center=(3.9, 2.0, 100.0), half=(0.2, 0.2, 0.2), density_ratio=0.5, vel=(0.3, -2.5, 0.0),
                mode=I.MODE_FREE)
    s = _rig(box, periodic=3)
    st = _drive(s, 1)
    assert st[0]["center"] == pytest.approx([0.2, 3.5, 100.0], abs=1e-12)


def test_fixed_body_ignores_force_and_torque():
    box = I.Box(center=FAR, half=(3.0, 2.0, 1.5), quat=I.heel_quat(10.0), density_ratio=0.5, mode=I.MODE_FIXED)
    s = _rig(box, gravity=(0.0, 0.0, -1e-5))
    st = _drive(s, 5, F=(1e-2, 0.0, 0.0), T=(0.0, 1e-2, 0.0))
    assert np.all(st[-1]["vel"] == 0) and np.all(st[-1]["omega"] == 0)
    assert np.all(st[-1]["center"] == np.array(FAR)) and np.allclose(st[-1]["quat"], I.heel_quat(10.0), atol=0)


# ---------------------------------------------------------- force mean


def _period_two(force_mean):
    h, dens = (3.0, 2.0, 1.5), 0.5
    A, B = 1e-3, 2e-4
    m = dens * _box_volume(h)
    s = _rig(I.Box(center=FAR, half=h, density_ratio=dens, mode=I.MODE_FREE),
             readings=dict(force_mean=force_mean))
    st = _drive(s, 200, F=lambda k: (B + A * (-1) ** k, 0.0, 0.0))
    v = np.array([b["vel"][0] for b in st])
    dv = np.diff(v)
    return dv - B / m, A / m


def test_force_mean_removes_the_period_two_component():
    """A force B + A (-1)^n: with the two-step mean the update sees B from the
    second step on, so the acceleration settles on B / m without alternating;
    driven by F_n alone it keeps alternating."""
    e, scale = _period_two(True)
    assert np.all(np.diff(np.abs(e[2:])) <= 1e-14 * scale)  # no growth (beyond rounding)
    nz = e[2:][np.abs(e[2:]) > 1e-14 * scale]
    assert np.all(np.sign(nz) == np.sign(nz[0]))  # no alternation
    assert abs(e[-1]) < 1e-12 * scale
    e0, _ = _period_two(False)
    assert np.abs(e0[-20:]).min() > 0.1 * scale
    assert np.all(np.sign(e0[-20:-1]) != np.sign(e0[-19:]))


def test_force_mean_impulse_of_a_pulse():
    """A single force pulse P on the first step (the mean then uses F_0 alone,
    and (F_1 + F_0) / 2 on the second): the body ends with momentum 3/2 P
    with the mean and P without it."""
    h, dens = (3.0, 2.0, 1.5), 0.5
    m = dens * _box_volume(h)
    P = 4e-3
    for mean, factor in ((True, 1.5), (False, 1.0)):
        s = _rig(I.Box(center=FAR, half=h, density_ratio=dens, mode=I.MODE_FREE), readings=dict(force_mean=mean))
        st = _drive(s, 300, F=lambda k: (P if k == 0 else 0.0, 0.0, 0.0))
        assert m * st[-1]["vel"][0] == pytest.approx(factor * P, rel=1e-12)


# ------------------------------------------------ through a full step


def test_free_fall_through_gas_follows_the_closed_form():
    """A box falling through an all-gas tank: the gas pressure pairs up along
    every lattice line (F = T = 0 up to rounding, Eq. momentuminterface with
    phi = 0), so the full step gives the virtual-mass free fall
    v_n = g (n - r (1 - r^n) / (1 - r)), r = C / (rho_s + C), while the box
    covers and uncovers gas cells."""
    n, g, dens = 20, -1e-4, 2.0
    fl, fi, rh = I.uniform_state(n, n, n, I.GAS, fill=0.0)
    box = I.Box(center=(10.2, 9.7, 12.3), half=(3.0, 2.5, 2.0), quat=I.heel_quat(20.0, (0.6, 0.0, 0.8)),
                density_ratio=dens, mode=I.MODE_FREE)
    sc = I.Scenario("fall", n, n, n, 0, 0.6, (0.0, 0.0, g), (0.0, 0.0, 0.0), 1.0, 1e-2, fl, fi, rh, [box], 0)
    s = oracle.OracleSim(sc)
    s.step(60)
    b = s.body(0)
    r = 1.0 / (dens + 1.0)
    k = 60
    vz = g * (k - r * (1 - r ** k) / (1 - r))
    assert np.abs(b["F"]).max() <= 1e-14 * b["S"]
    assert b["vel"][2] == pytest.approx(vz, rel=1e-10)
    assert abs(b["vel"][0]) < 1e-15 and abs(b["vel"][1]) < 1e-15
    assert b["center"][2] < 12.3 - 0.1
    assert s.error == 0


# ------------------------------------------------------ planted mistakes


@pytest.mark.parametrize("mutation", [10, 11, 12, 13, 14])
def test_planted_body_mistakes_are_caught(mutation):
    """Inertia with m/12 on half extents (10), the virtual mass left out of the
    denominator (11), the gyroscopic term with the wrong sign (12), the
    quaternion product on the body side (13) and the box volume without its
    factor 8 (14) each fail a pin above."""
    oracle.set_mutation(mutation)
    try:
        failed = []
        e = _newton_error()
        failed.append(not (e < 1e-12))
        failed.append(not (_euler_error(0) < 1e-12))
        rate, expected, _ = _precession_rate()
        failed.append(abs(rate / expected - 1.0) > 1e-2)
        err, _ = _quat_turn_error(h=(2.0, 2.0, 2.0), q0=I.heel_quat(30.0))
        failed.append(not (err < 1e-12))
    finally:
        oracle.set_mutation(0)
    assert any(failed), mutation
