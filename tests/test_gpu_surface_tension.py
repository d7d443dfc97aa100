"""Surface tension on the GPU (Sec. 2.2 Laplace pressure in the interface
boundary condition) against the oracle: FP64 bit parity on a droplet and a
bubble, reduced-precision storages within their tolerances, and the batched
form on a droplet next to another tank."""
import numpy as np
import pytest

import oracle
from paper_1201_0351_gb300 import inputs as I

from parity import assert_f64_parity, macro_errors, run_both

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bubble,n,radius,steps", [(False, 24, 5.0, 120), (True, 22, 6.0, 80)])
def test_f64_parity_with_surface_tension(bubble, n, radius, steps):
    sc = I.droplet(n, radius, sigma=4e-3, bubble=bubble)
    g, o, gb, ob, gs, ref = run_both(sc, steps, storage="f64")
    assert_f64_parity(g, o, gb, ob)


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16s", 2e-3)])
def test_reduced_precision_droplet(storage, tol):
    """Density within the storage's tolerance of the oracle after the droplet
    has reached its Laplace overpressure, classes identical."""
    sc = I.droplet(24, 5.0, sigma=4e-3)
    g, o, gb, ob, gs, ref = run_both(sc, 300, storage=storage)
    e = macro_errors(g, o)
    assert e["flag_diff"] == 0 and e["rho"] <= tol, e
    inside = (o["flags"] == I.LIQUID)
    jump_g = g["rho"][inside].mean() - 1.0
    jump_o = o["rho"][inside].mean() - 1.0
    assert jump_o > 0.0 and abs(jump_g - jump_o) <= tol * 10 + 0.02 * jump_o, (jump_g, jump_o)


def test_batch_with_surface_tension_equals_alone():
    from paper_1201_0351_gb300 import lbm_fs

    scenes = [I.droplet(20, 4.5, sigma=4e-3), I.closed_tank_32()]
    bt = lbm_fs.Batch(scenes, storage="f64")
    bt.step(30)
    got = [t.fields(want_f=True) for t in bt.tanks]
    bt.close()
    for sc, g in zip(scenes, got):
        sim = lbm_fs.Simulation(sc, storage="f64")
        sim.step(30)
        s = sim.fields(want_f=True)
        sim.close()
        assert np.array_equal(g["f"], s["f"]) and np.array_equal(g["flags"], s["flags"])
