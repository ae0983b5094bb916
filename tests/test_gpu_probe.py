"""di_probe_l2: the measured ceilings of the push's and the exact residual's
memory operations (scattered reductions, fetch-and-adds, gathers) that the
bench reports the push against."""
import pytest

from paper_1202_6168_gb300 import binding as di

pytestmark = pytest.mark.gpu


def test_every_mode_measures_a_positive_rate():
    rates = {m: di.probe_l2(m, 1 << 20, 1 << 24)[0] for m in di.PROBE_MODES}
    assert all(r > 0 for r in rates.values()), rates
    # a coalesced warp reduction carries eight FP32 adds per L2 sector, so it
    # retires several times more adds per second than scattered ones
    assert rates["red_f32_coalesced"] > 2 * rates["red_f32"]


def test_bad_arguments_are_rejected():
    lib = di.lib()
    rate = di.ctypes.c_double()
    for mode, slots, ops in ((5, 1 << 20, 1 << 20), (-1, 1 << 20, 1 << 20), (0, 1000, 1 << 20),
                             (0, 3 << 20, 1 << 20), (0, 1 << 20, 0)):
        assert lib.di_probe_l2(mode, slots, ops, di.ctypes.byref(rate), None, None) == di.DI_EINVAL
    assert lib.di_probe_l2(0, 1 << 20, 1 << 20, None, None, None) == di.DI_EINVAL
