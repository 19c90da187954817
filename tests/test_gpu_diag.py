"""The measurement diagnostics on the GPU: the integer-throughput peaks that are
the roofline's denominator, and the dependent-L2-load time that is the unit of a
round's latency chain.  Bounds are loose physical limits, not tuned values."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_16721_gb300 import mh as m
    return m


def test_integer_peaks_are_physical(mh):
    import torch
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    lop3, ms = mh.mh_int_peak(0)
    popc, _ = mh.mh_int_peak(1)
    assert ms > 0
    # at most 128 results per clock per SM at a clock below 3 GHz; at least a few per clock
    assert 1e11 < lop3 < sms * 128 * 3e9
    assert 1e10 < popc <= lop3 * 1.05


def test_l2_dependent_load_time(mh):
    ns = mh.mh_l2_latency()
    assert 50.0 < ns < 5000.0
    assert mh.load().mh_l2_latency(None) == mh.MH_EINVAL
