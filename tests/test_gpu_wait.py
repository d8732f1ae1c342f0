"""The bounded device-side wait of the transform kernel: single-CTA jobs stage their cells with
bulk (TMA) copies and wait for them on an mbarrier with a time limit. A wait that runs out is
reported through a device status word (zx_wait_status) instead of hanging the kernel. The
probe waits on a barrier that nothing completes, so the error path runs without a fault."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0810_3203_gb300 as m
    m.load()
    return m


def round_trip_ok(tg, N, l, n, stride):
    x = workloads.residues(11, n, N, stride=stride, cells=1 << l)
    d = torch.from_numpy(x.view(np.int64)).cuda()
    tg.tft_ex(d, l, n, n, N, 0, stride)
    tg.itft_ex(d, l, n, n, 0, N, 0, stride, scale=1)
    back = d.cpu().numpy().view(np.uint64).reshape(-1, stride)[:n, :N // 64 + 1]
    return np.array_equal(back, x.reshape(-1, stride)[:n, :N // 64 + 1])


def test_wait_that_runs_out_is_reported_then_cleared(tg):
    assert tg.wait_status() == tg.ZX_OK
    tg.wait_probe(2000)
    assert tg.wait_status() == tg.ZX_ETIMEOUT
    # read and cleared: the next read is clean, and the context still runs transforms
    assert tg.wait_status() == tg.ZX_OK
    # even stride: 16-byte aligned cells, so the jobs take the bulk loads
    assert round_trip_ok(tg, 32768, 12, 3000, 514)
    assert tg.wait_status() == tg.ZX_OK


@pytest.mark.parametrize("N,stride_extra", [(4096, 1), (8192, 1), (16384, 1), (32768, 1), (32768, 0)])
def test_bulk_and_plain_loads_round_trip(tg, N, stride_extra):
    """K = 4 .. 32 words per lane with 16-byte aligned cells (bulk loads), and an odd stride
    (plain loads), on a ragged length; no wait gives up."""
    stride = N // 64 + 1 + stride_extra
    assert round_trip_ok(tg, N, 13, 5001, stride)
    assert tg.wait_status() == tg.ZX_OK


def test_probe_rejects_bad_limits(tg):
    for bad in (0, -1, 1000001):
        with pytest.raises(tg.TftError):
            tg.wait_probe(bad)
