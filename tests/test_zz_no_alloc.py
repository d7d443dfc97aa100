"""The allocation-free liquid-mass entry point against lbm_fs_stats.

lbm_fs_liquid_mass_noalloc serves callers that may not allocate device memory
(the library then uses a fixed device array for its partial sums).  Its result
must equal the liquid mass that lbm_fs_stats reports for the same state, on two
calls in a row (the second after more steps, so a stale partial-sum array would
show); n = 0 gives 0, and a synthetic state of a few million cells (many
blocks of partial sums, a ragged last block) gives the sum torch computes.
The file name makes pytest collect it last, so that a run that stops at its
first failure has run every other test before this one.
"""
import numpy as np
import pytest

from paper_1201_0351_gb300 import inputs as I
from paper_1201_0351_gb300 import lbm_fs


@pytest.mark.gpu
def test_liquid_mass_noalloc_matches_stats():
    import torch

    sc = I.random_box_scene(40, 30, 22, seed=5, nboxes=3, speed=0.02)
    sim = lbm_fs.Simulation(sc, storage="f64")
    n = sim.n
    dev = torch.cuda.current_device()
    flags = torch.empty(n, dtype=torch.uint8, device=dev)
    mass = torch.empty(n, dtype=torch.float64, device=dev)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        sim.step(15)
        lbm_fs.lbm_fs_read_fields(sim.h, lbm_fs.FIELD_FLAGS | lbm_fs.FIELD_MASS,
                                  [flags.data_ptr(), None, mass.data_ptr(), None, None, None], True)
        lbm_fs.lbm_fs_liquid_mass_noalloc(flags.data_ptr(), mass.data_ptr(), n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        ref = sim.stats()["liquid_mass"]
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)
    sim.close()


@pytest.mark.gpu
def test_liquid_mass_noalloc_rejects_oversize():
    import torch

    buf = torch.zeros(16, dtype=torch.float64, device=torch.cuda.current_device())
    with pytest.raises(lbm_fs.LbmFsError):
        lbm_fs.lbm_fs_liquid_mass_noalloc(buf.data_ptr(), buf.data_ptr(), 268435457, buf.data_ptr())


@pytest.mark.gpu
def test_liquid_mass_noalloc_empty_and_many_blocks():
    import torch

    dev = torch.cuda.current_device()
    out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    lbm_fs.lbm_fs_liquid_mass_noalloc(buf.data_ptr(), buf.data_ptr(), 0, out.data_ptr())
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
    n = 5_000_123  # 1221 blocks of 4096 cells, the last one ragged
    g = torch.Generator(device="cpu").manual_seed(1201)
    cls = torch.tensor([I.LIQUID, I.INTERFACE, I.GAS, 8], dtype=torch.uint8)
    flags = cls[torch.randint(0, 4, (n,), generator=g)].to(dev)
    mass = torch.rand(n, dtype=torch.float64, generator=g).to(dev)
    fluid = (flags == I.LIQUID) | (flags == I.INTERFACE)
    ref = float(mass[fluid].sum().item())
    for _ in range(2):
        lbm_fs.lbm_fs_liquid_mass_noalloc(flags.data_ptr(), mass.data_ptr(), n, out.data_ptr())
        torch.cuda.synchronize()
        assert abs(float(out.item()) - ref) <= 1e-12 * ref, (float(out.item()), ref)
