"""The liquid cells next to an obstacle take the general gather (per-direction
source classes, bounce-back, the moving-body term of Eq. noslip).  The bulk
kernel lists them and a kernel of their own steps them, so that their
dependent loads hold none of the bulk kernel's warps; the list's length of the
last step is lbm_fs_stats' n_general.  Its results are covered by every FP64
parity test with a body (they match the oracle bit for bit); here the list
itself: it holds exactly the liquid cells with an obstacle among their 18
neighbours, in every storage, and a tank without a body or a moving wall lists
none."""
import numpy as np
import pytest

from paper_1201_0351_gb300 import inputs as I
from paper_1201_0351_gb300 import lbm_fs

pytestmark = pytest.mark.gpu

OBSTACLE = 8  # cell class of a body's cells in the read-back flags

D3Q19_MOVING = [(cx, cy, cz) for cx in (-1, 0, 1) for cy in (-1, 0, 1) for cz in (-1, 0, 1)
                if 0 < abs(cx) + abs(cy) + abs(cz) <= 2]


def _next_to_obstacle(flags):
    """liquid cells with an obstacle among their 18 neighbours (closed grid:
    nothing beyond the faces)"""
    nz, ny, nx = flags.shape
    pad = np.zeros((nz + 2, ny + 2, nx + 2), np.uint8)
    pad[1:-1, 1:-1, 1:-1] = flags
    near = np.zeros(flags.shape, bool)
    for cx, cy, cz in D3Q19_MOVING:
        near |= pad[1 + cz:nz + 1 + cz, 1 + cy:ny + 1 + cy, 1 + cx:nx + 1 + cx] == OBSTACLE
    return int(((flags == I.LIQUID) & near).sum())


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_general_list_holds_the_cells_next_to_an_obstacle(storage):
    sc = I.closed_tank_32()
    sim = lbm_fs.Simulation(sc, storage=storage)
    expected = []
    for _ in range(3):
        # the bulk kernel of the next step sees the classes read here
        expected.append(_next_to_obstacle(sim.flags().reshape(sc.nz, sc.ny, sc.nx)))
        sim.step(1)
        assert sim.stats()["n_general"] == expected[-1], (expected, sim.stats()["n_general"])
    sim.close()
    assert expected[0] > 100  # the fixed 8x8x6 box below the surface


def test_general_list_empty_without_bodies():
    sim = lbm_fs.Simulation(I.closed_tank_32(with_box=False), storage="f32")
    sim.step(2)
    st = sim.stats()
    sim.close()
    assert st["n_general"] == 0 and st["status"] == 0
