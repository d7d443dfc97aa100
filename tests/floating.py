"""Floating stability of a long box of square cross-section (Sec. 3.2.2),
from the exact immersed polygon: the heel at which a square of density ratio
s floats in stable equilibrium, and that heel for a weakly compressible
lattice liquid whose density rises with depth.

The immersed part of the heeled square is the polygon below the waterline
whose area is s times the square's; the waterline is found by bisection.  The
buoyancy acts at that polygon's centroid B, the weight at the square's centre
G; the moment vanishes where B lies straight below G.  A square's stable heels
are atan(1/2) = 26.565 deg for s = 1/4 and 3/4 and 45 deg for
0.2817 < s < 0.7183 (the paper's Sec. 3.2.2), and change quickly with s just
inside those intervals."""
import math


def _clip_below(pts, level):
    out = []
    for k in range(len(pts)):
        p, q = pts[k], pts[(k + 1) % len(pts)]
        pin, qin = p[1] < level, q[1] < level
        if pin:
            out.append(p)
        if pin != qin:
            t = (level - p[1]) / (q[1] - p[1])
            out.append((p[0] + t * (q[0] - p[0]), level))
    return out


def _area_centroid(pts):
    a = cx = cy = 0.0
    for k in range(len(pts)):
        x0, y0 = pts[k]
        x1, y1 = pts[(k + 1) % len(pts)]
        c = x0 * y1 - x1 * y0
        a += c
        cx += (x0 + x1) * c
        cy += (y0 + y1) * c
    a *= 0.5
    return a, cx / (6.0 * a), cy / (6.0 * a)


def immersed(s, theta):
    """(horizontal offset of B from G, depth of B below the waterline) for a
    unit square of density ratio s heeled by theta (radians)."""
    c, sn = math.cos(theta), math.sin(theta)
    pts = [(c * x - sn * y, sn * x + c * y) for x, y in ((-.5, -.5), (.5, -.5), (.5, .5), (-.5, .5))]
    lo, hi = -1.0, 1.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        poly = _clip_below(pts, mid)
        if len(poly) < 3 or _area_centroid(poly)[0] < s:
            lo = mid
        else:
            hi = mid
    level = 0.5 * (lo + hi)
    _, bx, by = _area_centroid(_clip_below(pts, level))
    return bx, level - by


def stable_heel(s, step=0.05):
    """The stable heel (deg, in (0, 45]) of a square of density ratio s: the
    first angle where the offset of B changes sign from the upright side."""
    prev = immersed(s, math.radians(step))[0]
    a = step
    while a < 45.0 - step:
        a2 = a + step
        cur = immersed(s, math.radians(a2))[0]
        if prev == 0.0 or (prev > 0) != (cur > 0):
            return a + step * prev / (prev - cur) if prev != cur else a
        prev, a = cur, a2
    return 45.0


def stable_heel_compressible(s, side, g):
    """The stable heel for a liquid of density exp(3 g depth) below its surface
    (the lattice's equation of state p = rho / 3 under gravity g): the body
    floats on the mean density around its immersed part, taken at the depth
    of its centre of buoyancy, i.e. with the density ratio s / exp(3 g d_B)."""
    th = stable_heel(s)
    _, depth = immersed(s, math.radians(th))
    return stable_heel(s / math.exp(3.0 * g * depth * side))
