"""The allocation-free liquid-mass entry point against lbm_fs_stats.

lbm_fs_liquid_mass_noalloc serves callers that may not allocate device memory
(the library then uses a fixed device array for its partial sums).  Its result
must equal the liquid mass that lbm_fs_stats reports for the same state, on two
calls in a row (the second after more steps, so a stale partial-sum array would
show).  This file is collected last on purpose.
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
