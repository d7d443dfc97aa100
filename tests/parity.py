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
