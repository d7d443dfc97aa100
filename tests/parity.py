"""Helpers of the GPU-vs-oracle parity tests: run both sides on one scenario
and compare element by element."""
import numpy as np

import oracle
from paper_1201_0351_gb300 import lbm_fs

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def run_both(sc, steps, storage="f64", use_graphs=True, chunks=1):
    sim = lbm_fs.Simulation(sc, storage=storage, use_graphs=use_graphs)
    ref = oracle.OracleSim(sc)
    per = steps // chunks
    for _ in range(chunks):
        sim.step(per)
        ref.step(per)
    g = sim.fields(want_f=True)
    o = ref.fields(want_f=True)
    gb = [sim.body(b) for b in range(len(sc.boxes))]
    ob = [ref.body(b) for b in range(len(sc.boxes))]
    gs = sim.stats()
    sim.close()
    assert ref.error == 0, "oracle reported error bits %d" % ref.error
    return g, o, gb, ob, gs, ref


def assert_f64_parity(g, o, gb, ob, rel=1e-11):
    """Flags identical; f, fill and mass within rel (f relative to w_q);
    forces within rel of |F| (or of S when |F| < 1e-3 S)."""
    diff = np.nonzero(g["flags"] != o["flags"])[0]
    assert diff.size == 0, "cell classes differ at %d cells, first %s" % (diff.size, diff[:10])
    df = np.abs(g["f"] - o["f"]) / W[:, None]
    assert df.max() <= rel, "max |df|/w = %.3g" % df.max()
    # fill level, mass and density are O(1) per cell (a fraction, and
    # densities near 1): relative to max(|x|, 1)
    for key in ("fill", "mass", "rho"):
        d = np.abs(g[key] - o[key]) / np.maximum(np.abs(o[key]), 1.0)
        assert d.max() <= rel, "%s: max rel diff %.3g" % (key, d.max())
    for a, b in zip(gb, ob):
        for key in ("F", "T"):
            scale = np.maximum(np.abs(b[key]), 1e-3 * b["S"])
            assert np.all(np.abs(a[key] - b[key]) <= rel * np.maximum(scale, 1e-300) + 1e-300), \
                "%s: gpu %s oracle %s" % (key, a[key], b[key])
        for key in ("center", "quat", "vel", "omega"):
            assert np.abs(a[key] - b[key]).max() <= rel * max(1.0, np.abs(b[key]).max()), \
                "%s: gpu %s oracle %s" % (key, a[key], b[key])


def macro_errors(g, o):
    """Errors of a reduced-precision run against the oracle, over cells whose
    class agrees: max relative density error, max velocity error relative to
    the largest oracle speed, number of differing classes."""
    same = (g["flags"] == o["flags"]) & ((o["flags"] == 1) | (o["flags"] == 2))
    drho = np.abs(g["rho"][same] - o["rho"][same]) / o["rho"][same]
    umax = np.linalg.norm(o["u"][same], axis=1).max()
    du = np.linalg.norm(g["u"][same] - o["u"][same], axis=1).max()
    return dict(rho=float(drho.max()), u=float(du / umax) if umax > 0 else float(du), u_abs=float(du),
                u_max=float(umax), flag_diff=int((g["flags"] != o["flags"]).sum()))


# unit roundoff of one stored population deviation f_q - w_q: FP32, and the
# 11-bit significand of the scaled half of the FP16-shifted storage
UNIT_ROUNDOFF = {"f32": 2.0 ** -24, "f16s": 2.0 ** -11}
# roundings of a population's size per step: the relaxation, the equilibrium
# and force terms of the float collision, and the store
ROUNDINGS_PER_STEP = 4


def rounding_floor(o, storage, steps):
    """Velocity that a float storage's rounding can leave after `steps` steps.
    Each step rounds every stored deviation d_q = f_q - w_q (and the collision
    terms of its size, ROUNDINGS_PER_STEP of them) to the storage's unit
    roundoff u, which moves a cell's momentum sum_q c_qk d_q by up to
    4 u V, V = the largest sum_q |c_qk| |d_q| over the oracle's fluid cells and
    the three axes.  The roundings of successive steps are independent, so
    they add like a random walk: 4 u V sqrt(steps)."""
    import oracle

    c, w, _ = oracle.lattice()
    fluid = (o["flags"] == 1) | (o["flags"] == 2)
    d = np.abs(o["f"][:, fluid] - w[:, None])
    V = max(float((np.abs(c[:, k])[:, None] * d).sum(axis=0).max()) for k in range(3))
    return ROUNDINGS_PER_STEP * UNIT_ROUNDOFF[storage] * V * float(np.sqrt(steps))


def velocity_check(g, o, storage, tol, steps):
    """Largest velocity errors over liquid and over interface cells whose class
    agrees, and the bound both must meet: tol times the largest oracle speed
    plus the rounding floor."""
    same = g["flags"] == o["flags"]
    fluid = same & ((o["flags"] == 1) | (o["flags"] == 2))
    umax = float(np.linalg.norm(o["u"][fluid], axis=1).max())
    du = np.linalg.norm(g["u"] - o["u"], axis=1)
    e_liq = float(du[same & (o["flags"] == 1)].max()) if (same & (o["flags"] == 1)).any() else 0.0
    e_if = float(du[same & (o["flags"] == 2)].max()) if (same & (o["flags"] == 2)).any() else 0.0
    bound = tol * umax + rounding_floor(o, storage, steps)
    return e_liq, e_if, bound, umax
