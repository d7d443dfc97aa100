"""Sphere bodies and moving domain walls in the oracle (Sec. 2.3 Eq. noslip
with a wall velocity at the channel walls; the free-advection set-up of
Sec. 3.2.1 with a spherical particle).

Pins against the mathematics: the discrete volume of a sphere is the number
of cell centres strictly inside it (brute force) and averages to 4/3 pi r^3
along a path; plane Couette flow between a moving and a resting wall is
linear, which half-way bounce-back with the wall term reproduces exactly in
steady state; and a sphere carried by a uniform flow whose walls move with it
keeps the flow's velocity (the moving-wall term preserves the equilibrium,
the paper's first advection series: "matched ... to the last digit")."""
import numpy as np
import pytest

import oracle
from paper_1201_0351_gb300 import inputs as I


def _liquid_box(nx, ny, nz, periodic, tau=0.8, vel=None, wall_vel=None, boxes=()):
    n = nx * ny * nz
    v = None if vel is None else np.tile(np.asarray(vel, float), n)
    return I.Scenario("liquid_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, periodic, tau, (0.0, 0.0, 0.0),
                      (0.0, 0.0, 0.0), 1.0, 1e-2, np.full(n, I.LIQUID, np.uint8), np.ones(n), np.ones(n),
                      list(boxes), 100, vel=v, wall_vel=wall_vel)


def test_sphere_discrete_volume():
    """Radius 5 moved along x in steps of 0.1: each covered-cell count equals
    the brute-force count of centres with |x_c - o| < 5, and the mean over
    one cell of travel is the ideal 523.6 within 1 %."""
    n, radius = 16, 5.0
    counts = []
    for k in range(10):
        c = (8.0 + 0.1 * k, 8.05, 7.95)
        sc = _liquid_box(n, n, n, 0, boxes=[I.Box(center=c, half=(radius, radius, radius), mode=I.MODE_FIXED,
                                                  shape=I.SHAPE_SPHERE)])
        got = int((oracle.OracleSim(sc).fields()["flags"] == oracle.OBSTACLE).sum())
        zc, yc, xc = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
        brute = int((((xc - c[0]) ** 2 + (yc - c[1]) ** 2 + (zc - c[2]) ** 2) < radius ** 2).sum())
        assert got == brute, (c, got, brute)
        counts.append(got)
    ideal = 4.0 / 3.0 * np.pi * radius ** 3
    assert abs(np.mean(counts) - ideal) <= 0.01 * ideal, (counts, ideal)


def test_couette_flow_between_moving_and_resting_wall():
    U, nz = 1e-3, 16
    wall = [0.0] * 18
    wall[12] = U  # face z- moves along x; z+ at rest
    sc = _liquid_box(4, 4, nz, 3, tau=0.8, wall_vel=tuple(wall))
    ref = oracle.OracleSim(sc)
    ref.step(8000)
    assert ref.error == 0
    u = ref.fields()["u"].reshape(nz, 4, 4, 3)
    zc = np.arange(nz) + 0.5
    exact = U * (1.0 - zc / nz)
    assert np.abs(u[..., 0] - exact[:, None, None]).max() <= 1e-9 * U
    assert np.abs(u[..., 1:]).max() <= 1e-10 * U


def test_sphere_follows_uniform_flow_between_moving_walls():
    U = 1e-3
    wall = []
    for _ in range(6):
        wall += [U, 0.0, 0.0]
    sphere = I.Box(center=(12.2, 8.1, 7.9), half=(4.0, 4.0, 4.0), density_ratio=0.5, vel=(U, 0.0, 0.0),
                   mode=I.MODE_FREE, shape=I.SHAPE_SPHERE)
    sc = _liquid_box(24, 16, 16, 1, tau=0.8, vel=(U, 0.0, 0.0), wall_vel=tuple(wall), boxes=[sphere])
    ref = oracle.OracleSim(sc)
    ref.step(100)
    assert ref.error == 0
    b = ref.body(0)
    assert abs(b["vel"][0] - U) <= 1e-10 * U and np.abs(b["vel"][1:]).max() <= 1e-10 * U, b["vel"]
    f = ref.fields()
    fluid = f["flags"] == I.LIQUID
    assert np.abs(f["u"][fluid, 0] - U).max() <= 1e-10 * U
    assert abs(b["center"][0] - (12.2 + 100 * U)) <= 1e-9


def test_resting_walls_mutation_is_caught():
    """With the walls held at rest (the wall term dropped) the same uniform
    flow is braked at the walls: the check above fails."""
    U = 1e-3
    sc = _liquid_box(24, 16, 16, 1, tau=0.8, vel=(U, 0.0, 0.0), wall_vel=None)
    ref = oracle.OracleSim(sc)
    ref.step(100)
    f = ref.fields()
    assert not np.abs(f["u"][:, 0] - U).max() <= 1e-10 * U
