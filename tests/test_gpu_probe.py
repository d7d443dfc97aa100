"""The FP64 rate probe that the double-storage roofline is quoted against.

lbm_fs_fp64_rate times independent chains of one double-precision operation
on every SM.  Its rate must be positive, the same within a few per cent for
add, multiply and fused multiply-add (one pipe executes all three), and must
not depend on the chain length once the chains are long; bad arguments give
LBM_FS_EINVAL without a launch.
"""
import pytest

from paper_1201_0351_gb300 import lbm_fs


@pytest.mark.gpu
def test_fp64_rate_consistent():
    rates = [lbm_fs.lbm_fs_fp64_rate(op, 1 << 14) for op in (0, 1, 2)]
    assert all(r > 1e10 for r in rates), rates
    assert max(rates) <= 1.05 * min(rates), rates
    longer = lbm_fs.lbm_fs_fp64_rate(1, 1 << 15)
    assert abs(longer - rates[1]) <= 0.05 * rates[1], (longer, rates[1])


@pytest.mark.gpu
@pytest.mark.parametrize("op,iters", [(-1, 16), (3, 16), (0, 0), (1, -5)])
def test_fp64_rate_rejects_bad_arguments(op, iters):
    with pytest.raises(lbm_fs.LbmFsError) as e:
        lbm_fs.lbm_fs_fp64_rate(op, iters)
    assert e.value.code == lbm_fs.LBM_FS_EINVAL
