"""Seeded synthetic scenarios (tanks, channels, boxes) for the free-surface LBM.

This module builds INPUT DATA only: grid sizes, physical parameters, the initial
cell classification and fill/density arrays, and the rigid-box list.  It holds
none of the lattice Boltzmann arithmetic (no equilibrium, streaming, collision,
mass exchange, momentum exchange or conversion rule); both the GPU library and
the CPU checker receive exactly these arrays and each applies the method itself.

Initial state (the paper initialises its basins "with hydrostatic pressure",
Sec. 3.2.1 and Sec. 3.2.2, and defines the cell/fill geometry in Sec. 2.1/2.2):

* cell (x, y, z) is the cube [x, x+1] x [y, y+1] x [z, z+1], centre at +0.5;
* fill level per column: phi = clamp(eta(x, y) - z, 0, 1) for a surface height
  eta (lattice units, measured from the floor plane z = 0);
* density: rho = rho_gas * exp(3 g (eta - z_c)) where phi > 0 (the isothermal
  equation of state p = rho / 3 of Eq. pressure integrated under gravity g along
  -z), rho_gas elsewhere;
* classification: 0 < phi < 1 -> interface; phi = 1 with a phi = 0 neighbour in
  the 18-neighbourhood -> interface (phi = 1); phi = 1 -> liquid; phi = 0 -> gas.

Rigid boxes are NOT mapped here: each side discretises them itself (a cell is an
obstacle iff its centre lies strictly inside the box, Sec. 2.3).

Random numbers: splitmix64 (Steele, Lea, Flood 2014), top 53 bits -> U[0, 1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

# Initial-state cell classes, as passed to the libraries (input encoding).
LIQUID = 1
INTERFACE = 2
GAS = 4

# Box motion modes (input encoding).
SHAPE_BOX, SHAPE_SPHERE = 0, 1
MODE_FIXED = 0
MODE_FREE = 1
MODE_ROT_AXIS_ONLY = 2
MODE_DAMP_TRANSLATION = 0x100

SEED = 1201


class SplitMix64:
    """splitmix64: state += 0x9E3779B97F4A7C15, then the two xor-shift-multiply rounds."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class Box:
    center: tuple
    half: tuple
    quat: tuple = (1.0, 0.0, 0.0, 0.0)  # (w, x, y, z), body -> world rotation
    density_ratio: float = 1.0
    vel: tuple = (0.0, 0.0, 0.0)
    omega: tuple = (0.0, 0.0, 0.0)
    mode: int = MODE_FIXED
    rot_axis: tuple = (1.0, 0.0, 0.0)
    lin_damping: float = 0.0
    shape: int = 0  # SHAPE_BOX, or SHAPE_SPHERE of radius half[0]


@dataclasses.dataclass
class Scenario:
    name: str
    nx: int
    ny: int
    nz: int
    periodic: int  # bit0 = x, bit1 = y, bit2 = z; other faces are no-slip walls
    tau: float
    gravity: tuple
    body_accel: tuple
    rho_gas: float
    eps: float
    flags: np.ndarray  # uint8[N], idx = x + nx*(y + ny*z)
    fill: np.ndarray  # float64[N]
    rho: np.ndarray  # float64[N]
    boxes: List[Box]
    steps: int
    vel: Optional[np.ndarray] = None  # float64[3N] (xyz per cell) or None = at rest
    sigma: float = 0.0  # surface tension (Laplace pressure 2 sigma kappa at the interface); 0 = none
    wall_vel: Optional[tuple] = None  # 18 floats: velocity of the faces x-, x+, y-, y+, z-, z+; None = at rest
    # options where the paper is silent, as keyword values (deadband, virtual_mass,
    # force_mean, neighbour_rule); None = each side's defaults (1e-2, 1, True, True)
    readings: Optional[dict] = None

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    def with_boxes(self, boxes: List[Box]) -> "Scenario":
        return dataclasses.replace(self, boxes=list(boxes))


def _neighbour_offsets():
    """The 18 non-rest offsets of the 3x3x3 neighbourhood without its corners."""
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                s = abs(dx) + abs(dy) + abs(dz)
                if s in (1, 2):
                    out.append((dx, dy, dz))
    return out


def classify(fill3: np.ndarray, periodic: int) -> np.ndarray:
    """Initial classes from a (nz, ny, nx) fill array (rule stated in the module doc)."""
    flags = np.where(fill3 >= 1.0, LIQUID, np.where(fill3 > 0.0, INTERFACE, GAS)).astype(np.uint8)
    empty = fill3 <= 0.0
    near_empty = np.zeros_like(empty)
    nz, ny, nx = fill3.shape
    for dx, dy, dz in _neighbour_offsets():
        shifted = np.zeros_like(empty)
        # shifted[z, y, x] = empty[z + dz, y + dy, x + dx] (periodic wrap or outside = False)
        src = empty
        for axis, d, bit, n in ((2, dx, 1, nx), (1, dy, 2, ny), (0, dz, 4, nz)):
            if d == 0:
                continue
            src = np.roll(src, -d, axis=axis)
            if not (periodic & bit):
                sl = [slice(None)] * 3
                sl[axis] = slice(n - 1, n) if d > 0 else slice(0, 1)
                src = src.copy()
                src[tuple(sl)] = False
        shifted |= src
        near_empty |= shifted
    flags[(flags == LIQUID) & near_empty] = INTERFACE
    return flags


def hydrostatic_tank(nx, ny, nz, eta: Callable[[np.ndarray, np.ndarray], np.ndarray],
                     g: float, rho_gas: float, periodic: int):
    """flags, fill, rho (flat, idx order) for a tank filled up to eta(x_c, y_c)."""
    xc = np.arange(nx, dtype=np.float64) + 0.5
    yc = np.arange(ny, dtype=np.float64) + 0.5
    XC, YC = np.meshgrid(xc, yc, indexing="xy")  # (ny, nx)
    eta2 = np.asarray(eta(XC, YC), dtype=np.float64) * np.ones((ny, nx))
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    fill3 = np.clip(eta2[None, :, :] - z, 0.0, 1.0)
    zc = z + 0.5
    rho3 = np.where(fill3 > 0.0, rho_gas * np.exp(3.0 * g * (eta2[None, :, :] - zc)), rho_gas)
    flags3 = classify(fill3, periodic)
    return (flags3.reshape(-1).copy(), fill3.reshape(-1).copy(), rho3.reshape(-1).astype(np.float64).copy())


def uniform_state(nx, ny, nz, cls: int, fill: float = 1.0, rho: float = 1.0):
    n = nx * ny * nz
    return (np.full(n, cls, np.uint8), np.full(n, fill, np.float64), np.full(n, rho, np.float64))


def heel_quat(alpha_deg: float, axis=(1.0, 0.0, 0.0)) -> tuple:
    a = math.radians(alpha_deg)
    s = math.sin(0.5 * a)
    return (math.cos(0.5 * a), s * axis[0], s * axis[1], s * axis[2])


# ----------------------------------------------------------------------------
# Workloads of the paper's kind (closed tank, stratified channel, heeled box,
# batched heel sweep, large wave tank).
# ----------------------------------------------------------------------------

def closed_tank_32(with_box: bool = True, g: float = 1e-5, eta: float = 16.5) -> Scenario:
    """32^3 closed tank, tau 0.6, g along -z, surface at 16.5, one fixed 8x8x6 box
    centred at (16, 16, 16) (spans x, y in [12, 20], z in [13, 19])."""
    n = 32
    flags, fill, rho = hydrostatic_tank(n, n, n, lambda X, Y: eta, g, 1.0, 0)
    boxes = [Box(center=(16.0, 16.0, 16.0), half=(4.0, 4.0, 3.0), mode=MODE_FIXED, density_ratio=0.5)] if with_box else []
    return Scenario("closed_tank_32", n, n, n, 0, 0.6, (0.0, 0.0, -g), (0.0, 0.0, 0.0), 1.0, 1e-2,
                    flags, fill, rho, boxes, 200)


def channel_96x32x32(free_box: bool = True, tau: float = 0.6) -> Scenario:
    """96x32x32 channel, periodic x, walls in y and z, liquid below 16.5, body
    force 1e-6 along +x, one free 8x8x6 box of density ratio 0.5 (draft 3)."""
    nx, ny, nz = 96, 32, 32
    g = 1e-5
    flags, fill, rho = hydrostatic_tank(nx, ny, nz, lambda X, Y: 16.5, g, 1.0, 1)
    boxes = [Box(center=(48.0, 16.0, 16.5), half=(4.0, 4.0, 3.0), density_ratio=0.5, mode=MODE_FREE)] if free_box else []
    return Scenario("channel_96x32x32", nx, ny, nz, 1, tau, (0.0, 0.0, -g), (1e-6, 0.0, 0.0), 1.0, 1e-2,
                    flags, fill, rho, boxes, 5000)


def heeled_box_128(fixed: bool = False, heel_deg: float = 10.0, n: int = 128) -> Scenario:
    """n^3 half-full tank, tau 0.55, g 2e-5; 48x24x16 box (long axis x), density
    0.5, centre on the water line, heeled about x; rotation about x only with
    damped translation (or held fixed)."""
    g = 2e-5
    eta = n / 2 + 0.5
    flags, fill, rho = hydrostatic_tank(n, n, n, lambda X, Y: eta, g, 1.0, 0)
    s = n / 128.0
    mode = MODE_FIXED if fixed else (MODE_ROT_AXIS_ONLY | MODE_DAMP_TRANSLATION)
    box = Box(center=(n / 2, n / 2, eta), half=(24.0 * s, 12.0 * s, 8.0 * s), quat=heel_quat(heel_deg),
              density_ratio=0.5, mode=mode, rot_axis=(1.0, 0.0, 0.0), lin_damping=0.05)
    return Scenario("heeled_box_%d" % n, n, n, n, 0, 0.55, (0.0, 0.0, -g), (0.0, 0.0, 0.0), 1.0, 1e-2,
                    flags, fill, rho, [box], 20000)


def immersed_offset(b: float, h: float, alpha: float, frac: float) -> float:
    """Height of the box centre above the water line such that a b x h rectangle
    heeled by alpha (radians) has the immersed area fraction frac (bisection on the
    clipped polygon's area; geometry used to place boxes, not LBM arithmetic)."""
    corners = [(-0.5 * b, -0.5 * h), (0.5 * b, -0.5 * h), (0.5 * b, 0.5 * h), (-0.5 * b, 0.5 * h)]
    ca, sa = math.cos(alpha), math.sin(alpha)
    rot = [(ca * x - sa * y, sa * x + ca * y) for x, y in corners]

    def area_below(level):  # area of the rotated rectangle with y < level
        pts = []
        for i in range(4):
            p, q = rot[i], rot[(i + 1) % 4]
            pin, qin = p[1] < level, q[1] < level
            if pin:
                pts.append(p)
            if pin != qin:
                t = (level - p[1]) / (q[1] - p[1])
                pts.append((p[0] + t * (q[0] - p[0]), level))
        a = 0.0
        for i in range(len(pts)):
            x0, y0 = pts[i]
            x1, y1 = pts[(i + 1) % len(pts)]
            a += x0 * y1 - x1 * y0
        return abs(a) * 0.5

    lo, hi = -h - b, h + b
    target = frac * b * h
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if area_below(mid) < target:
            lo = mid
        else:
            hi = mid
    level = 0.5 * (lo + hi)  # water line in the box-centred frame
    return -level  # centre height above the water line


def batched_sweep_tanks(count: int = 64, seed: int = SEED) -> List[Scenario]:
    """Tanks of edge E = 48 + floor(65 U), box 0.4E x 0.2E x 0.12E, heel U(0, 30) deg
    about x, density U(0.3, 0.7), surface E/2 + 0.5, centre placed at the draft of
    the exact clipped-rectangle solve; rotation about x only, damped translation."""
    rng = SplitMix64(seed)
    out = []
    g = 2e-5
    for k in range(count):
        e = 48 + int(math.floor(65.0 * rng.uniform()))
        heel = 30.0 * rng.uniform()
        dens = 0.3 + 0.4 * rng.uniform()
        eta = e / 2 + 0.5
        flags, fill, rho = hydrostatic_tank(e, e, e, lambda X, Y, eta=eta: eta, g, 1.0, 0)
        b, h = 0.2 * e, 0.12 * e
        zc = eta + immersed_offset(b, h, math.radians(heel), dens)
        box = Box(center=(e / 2, e / 2, zc), half=(0.2 * e, 0.1 * e, 0.06 * e), quat=heel_quat(heel),
                  density_ratio=dens, mode=MODE_ROT_AXIS_ONLY | MODE_DAMP_TRANSLATION,
                  rot_axis=(1.0, 0.0, 0.0), lin_damping=0.05)
        out.append(Scenario("sweep_tank_%02d_E%d" % (k, e), e, e, e, 0, 0.55, (0.0, 0.0, -g), (0.0, 0.0, 0.0),
                            1.0, 1e-2, flags, fill, rho, [box], 5000))
    return out


def wave_tank(nx: int = 768, ny: int = 384, nz: int = 256, nboxes: int = 16, seed: int = SEED) -> Scenario:
    """Wave tank: tau 0.52, g 1e-5, surface 128 + 8 sin(2 pi x / 192) (scaled with
    nz / 256 for reduced sizes), free 24x12x8 boxes (long axis x) of density
    U(0.4, 0.6), centres by rejection sampling with minimum spacing 40, floating at
    their draft below the local surface."""
    g = 1e-5
    sz = nz / 256.0
    depth, amp, wl = 128.0 * sz, 8.0 * sz, 192.0 * nx / 768.0

    def eta(X, Y):
        return depth + amp * np.sin(2.0 * np.pi * X / wl)

    flags, fill, rho = hydrostatic_tank(nx, ny, nz, eta, g, 1.0, 0)
    rng = SplitMix64(seed)
    boxes: List[Box] = []
    hx, hy, hz = 12.0, 6.0, 4.0
    x_lo, x_hi = 24.0, nx - 24.0
    y_lo, y_hi = 12.0, ny - 12.0
    tries = 0
    while len(boxes) < nboxes and tries < 100000:
        tries += 1
        x = x_lo + (x_hi - x_lo) * rng.uniform()
        y = y_lo + (y_hi - y_lo) * rng.uniform()
        dens = 0.4 + 0.2 * rng.uniform()
        if any((b.center[0] - x) ** 2 + (b.center[1] - y) ** 2 < 40.0 ** 2 for b in boxes):
            continue
        zc = depth + amp * math.sin(2.0 * math.pi * x / wl) - dens * 2 * hz + hz
        boxes.append(Box(center=(x, y, zc), half=(hx, hy, hz), density_ratio=dens, mode=MODE_FREE))
    return Scenario("wave_tank_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, 0, 0.52, (0.0, 0.0, -g), (0.0, 0.0, 0.0),
                    1.0, 1e-2, flags, fill, rho, boxes, 2000)


def crop(sc: Scenario, nx: int, ny: int, nz: Optional[int] = None, name: Optional[str] = None,
         x0: int = 0, y0: int = 0) -> Scenario:
    """The nx x ny (x nz) window of a scenario starting at column (x0, y0), with
    the boxes whose extent lies inside it, shifted to the window (a bounded
    sample of a large workload; walls on the cut faces)."""
    nz = sc.nz if nz is None else nz
    sh = (sc.nz, sc.ny, sc.nx)
    f3 = sc.flags.reshape(sh)[:nz, y0:y0 + ny, x0:x0 + nx]
    p3 = sc.fill.reshape(sh)[:nz, y0:y0 + ny, x0:x0 + nx]
    r3 = sc.rho.reshape(sh)[:nz, y0:y0 + ny, x0:x0 + nx]
    boxes = []
    for b in sc.boxes:
        r = math.sqrt(sum(h * h for h in b.half))
        cx_, cy_ = b.center[0] - x0, b.center[1] - y0
        if r + 1 < cx_ < nx - r - 1 and r + 1 < cy_ < ny - r - 1:
            boxes.append(dataclasses.replace(b, center=(cx_, cy_, b.center[2])))
    return dataclasses.replace(sc, name=name or sc.name + "_crop%dx%dx%d" % (nx, ny, nz), nx=nx, ny=ny, nz=nz,
                               periodic=sc.periodic & 0, flags=np.ascontiguousarray(f3).reshape(-1).copy(),
                               fill=np.ascontiguousarray(p3).reshape(-1).copy(),
                               rho=np.ascontiguousarray(r3).reshape(-1).copy(), boxes=boxes)


def random_box_scene(nx, ny, nz, seed: int, nboxes: int = 1, periodic: int = 0, g: float = 1e-5,
                     tau: float = 0.6, eta_frac: float = 0.5, speed: float = 0.02) -> Scenario:
    """Small seeded scene for parity sweeps: a tank with a tilted surface and
    moving free boxes with random orientation and velocity (exercises conversions
    and obstacle cover / uncover every few steps)."""
    rng = SplitMix64(seed)
    e0 = eta_frac * nz + 0.3
    sx = 0.6 * (rng.uniform() - 0.5)
    sy = 0.6 * (rng.uniform() - 0.5)

    def eta(X, Y):
        return e0 + sx * (X - nx / 2) * 0.1 + sy * (Y - ny / 2) * 0.1

    flags, fill, rho = hydrostatic_tank(nx, ny, nz, eta, g, 1.0, periodic)
    boxes = []
    for _ in range(nboxes):
        # bodies must not touch each other or the walls (contacts are not modelled)
        for _try in range(1000):
            half = (1.5 + 2.0 * rng.uniform(), 1.5 + 2.0 * rng.uniform(), 1.2 + 1.5 * rng.uniform())
            c = (nx * (0.2 + 0.6 * rng.uniform()), ny * (0.2 + 0.6 * rng.uniform()), e0 + 2.0 * (rng.uniform() - 0.5))
            r = math.sqrt(sum(h * h for h in half))
            ok = all(r + 2.0 < c[k] < n - r - 2.0 for k, n in enumerate((nx, ny, nz)))
            ok = ok and all(math.dist(c, b.center) > r + math.sqrt(sum(h * h for h in b.half)) + 2.0 for b in boxes)
            if ok:
                break
        else:
            raise ValueError("no room for %d boxes in %dx%dx%d" % (nboxes, nx, ny, nz))
        ax = (rng.uniform() - 0.5, rng.uniform() - 0.5, rng.uniform() - 0.5)
        nrm = math.sqrt(sum(a * a for a in ax)) or 1.0
        ang = 40.0 * rng.uniform()
        q = heel_quat(ang, tuple(a / nrm for a in ax))
        vel = tuple(speed * (rng.uniform() - 0.5) for _ in range(3))
        om = tuple(0.01 * (rng.uniform() - 0.5) for _ in range(3))
        dens = 0.4 + 0.4 * rng.uniform()
        boxes.append(Box(center=c, half=half, quat=q, density_ratio=dens, vel=vel, omega=om, mode=MODE_FREE))
    return Scenario("random_%dx%dx%d_s%d" % (nx, ny, nz, seed), nx, ny, nz, periodic, tau, (0.0, 0.0, -g),
                    (0.0, 0.0, 0.0), 1.0, 1e-2, flags, fill, rho, boxes, 100)


def droplet(n: int = 30, radius: float = 7.0, sigma: float = 4e-3, tau: float = 0.8, bubble: bool = False,
            seed_offset: Optional[Sequence[float]] = None) -> Scenario:
    """A liquid sphere of the given radius in gas (or, with bubble=True, a gas
    sphere in liquid) at the centre of an n^3 closed box, no gravity, density
    1 everywhere: the interface layer takes the cells whose centres lie within
    half a cell of the sphere, with fill level clamp(R + 1/2 - r) (liquid side
    inward); surface tension sigma."""
    c = np.array([n / 2.0, n / 2.0, n / 2.0]) if seed_offset is None else np.array(seed_offset, float)
    z, y, x = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    depth = (radius + 0.5 - r) if not bubble else (r - radius + 0.5)  # > 1: liquid, < 0: gas
    fill = np.clip(depth, 0.0, 1.0)
    flags = np.where(depth >= 1.0, LIQUID, np.where(depth <= 0.0, GAS, INTERFACE)).astype(np.uint8)
    # the interface layer must separate liquid from gas along every D3Q19
    # link: a liquid cell with a gas cell among its 18 neighbours becomes
    # interface (cells beyond the closed box's walls do not count)
    fl3 = flags.reshape(n, n, n)
    pad = np.pad(fl3, 1, constant_values=0)
    near_gas = np.zeros_like(fl3, dtype=bool)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if abs(dx) + abs(dy) + abs(dz) in (1, 2):
                    near_gas |= pad[1 + dz:n + 1 + dz, 1 + dy:n + 1 + dy, 1 + dx:n + 1 + dx] == GAS
    fl3 = np.where((fl3 == LIQUID) & near_gas, INTERFACE, fl3)
    flags = fl3.reshape(-1)
    fill = np.where(flags == LIQUID, 1.0, np.where(flags == GAS, 0.0, np.clip(fill.reshape(-1), 0.01, 0.99)))
    rho = np.ones(n ** 3)
    name = "%s_%d_R%g" % ("bubble" if bubble else "droplet", n, radius)
    return Scenario(name, n, n, n, 0, tau, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 1.0, 1e-2, flags,
                    fill.astype(np.float64), rho, [], 400, sigma=sigma)


def floating_cubes(steps: int = 40000, free_rotation: bool = False, scale: int = 1,
                   damping: float = 0.0) -> Scenario:
    """The floating-cube equilibrium of Sec. 3.2.2: a 130x40x40 basin filled to
    half height, tau 1/1.9, g 7.5e-4, three 32x16x16 boxes (the 2D cube of side
    s = 16 extended to 2s along its rolling axis x) of densities 0.75, 0.5 and
    0.25, placed at the draft of their 2.86 deg initial heel.  Rotation about
    x only, or free in all three axes (free_rotation); damping > 0 damps the
    translation by that fraction per step.  scale > 1 refines the lattice
    (every length times scale, g / scale so that the hydrostatic density
    variation 3 g depth stays the same).  Stable heels: atan(1/2) = 26.565 deg
    for 0.25 and 0.75, 45 deg for 0.5."""
    nx, ny, nz = 130 * scale, 40 * scale, 40 * scale
    g, eta, s = 7.5e-4 / scale, 20.0 * scale, 16.0 * scale
    flags, fill, rho = hydrostatic_tank(nx, ny, nz, lambda X, Y: eta, g, 1.0, 0)
    mode = MODE_FREE if free_rotation else MODE_ROT_AXIS_ONLY
    if damping > 0.0:
        mode |= MODE_DAMP_TRANSLATION
    boxes = []
    for k, dens in enumerate((0.75, 0.5, 0.25)):
        heel = 2.86
        zc = eta + immersed_offset(s, s, math.radians(heel), dens)
        boxes.append(Box(center=(nx * (2 * k + 1) / 6.0, ny / 2.0, zc), half=(s, s / 2, s / 2), quat=heel_quat(heel),
                         density_ratio=dens, mode=mode, rot_axis=(1.0, 0.0, 0.0), lin_damping=damping))
    return Scenario("floating_cubes_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, 0, 1.0 / 1.9, (0.0, 0.0, -g),
                    (0.0, 0.0, 0.0), 1.0, 1e-2, flags, fill, rho, boxes, steps)


def free_advection_channel(tau: float = 0.8, u: float = 1e-4, g: float = 1e-5, steps: int = 20000,
                           nx: int = 60, ny: int = 40, nz: int = 30, radius: float = 6.0,
                           depth: float = 19.5) -> Scenario:
    """The free-advection test of Sec. 3.2.1: a 60x40x30 channel, periodic in
    x, filled to `depth` (19.5), whose bottom and long side walls move with
    (u, 0, 0) (the top, in the gas, rests); the liquid starts uniform at u; a
    sphere of diameter 12 and density 0.5 floats half immersed at the centre,
    starting at rest, and should end up moving with the liquid."""
    flags, fill, rho = hydrostatic_tank(nx, ny, nz, lambda X, Y: depth, g, 1.0, 1)
    vel = np.zeros((nx * ny * nz, 3))
    vel[(flags == LIQUID) | (flags == INTERFACE), 0] = u
    wall = [0.0] * 18
    for face in (2, 3, 4):  # y-, y+, z-
        wall[3 * face] = u
    sphere = Box(center=(nx / 2.0, ny / 2.0, depth), half=(radius, radius, radius), density_ratio=0.5,
                 mode=MODE_FREE, shape=SHAPE_SPHERE)
    return Scenario("free_advection_%dx%dx%d_tau%g_u%g" % (nx, ny, nz, tau, u), nx, ny, nz, 1, tau, (0.0, 0.0, -g),
                    (0.0, 0.0, 0.0), 1.0, 1e-2, flags, fill, rho, [sphere], steps, vel=vel.reshape(-1),
                    wall_vel=tuple(wall))
