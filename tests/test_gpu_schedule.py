"""GPU parity of the persistent form (one launch per transform, jobs claimed in dependency order;
zx_transform_schedule): the same TFT / ITFT outputs as the oracle, bit for bit, with the form
pinned on for the rings used. Covers the benchmark's l = 16 transform on its 16-byte aligned
layout (bulk loads) and smaller rings with random weights and ragged lengths."""
import random

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RINGS = (4096, 8192, 32768)


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0810_3203_gb300 as m
    m.load()
    before = {N: m.config_get(N) for N in RINGS}
    for N in RINGS:
        m.config_set(N, dict(before[N], fused=1))
    yield m
    for N in RINGS:
        m.config_set(N, before[N])


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def from_dev(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def bad_cells(a, b, count, stride, W):
    A = a[:count * stride].reshape(count, stride)[:, :W]
    B = b[:count * stride].reshape(count, stride)[:, :W]
    return np.nonzero(~np.all(A == B, axis=1))[0]


def test_benchmark_tft_on_the_bulk_layout(tg, orc):
    N, l, n = 32768, 16, 40000
    W = N // 64 + 1
    st = W + 1  # 514 limbs: 16-byte aligned cells
    assert tg.transform_schedule(0, l, n, n, N)
    x = workloads.structured_residues(11, n, N, stride=st, cells=1 << l)
    d = to_dev(x)
    tg.tft_ex(d, l, n, n, N, 0, st)
    got = from_dev(d)
    ref = x.copy()
    orc.tft(ref, l, n, n, 0, N, stride=st)
    bad = bad_cells(got, ref, n, st, W)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5]}"
    assert tg.wait_status() == tg.ZX_OK


def test_benchmark_itft_on_the_bulk_layout(tg, orc):
    N, l, n, f, e = 32768, 16, 52000, 1, 12345
    W = N // 64 + 1
    st = W + 1
    x = workloads.residues(13, n + f, N, stride=st, cells=1 << l)
    d = to_dev(x)
    tg.itft_ex(d, l, n + f, n, f, N, e, st, scale=0)
    got = from_dev(d)
    ref = x.copy()
    orc.itft(ref, l, n + f, n, f, e, N, stride=st)
    bad = bad_cells(got, ref, n + f, st, W)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5]}"
    assert tg.wait_status() == tg.ZX_OK


@pytest.mark.parametrize("N,l", [(4096, 10), (4096, 11), (4096, 12), (8192, 13)])
def test_smaller_rings(tg, orc, N, l):
    rng = random.Random(N + l)
    W = N // 64 + 1
    L = 1 << l
    for _ in range(3):
        z = rng.randint(L // 2, L)
        n = rng.randint(L // 3, L)
        e = rng.randrange(2 * N)
        assert tg.transform_schedule(0, l, z, n, N)
        x = workloads.residues(rng.randrange(1 << 30), z, N, cells=L)
        d = to_dev(x)
        tg.tft_ex(d, l, z, n, N, e)
        got = from_dev(d)
        ref = x.copy()
        orc.tft(ref, l, z, n, e, N)
        assert bad_cells(got, ref, n, W, W).size == 0, ("tft", N, l, z, n, e)
        nn = rng.randint(1, z - 1)
        f = 1
        x = workloads.residues(rng.randrange(1 << 30), z, N, cells=L)
        d = to_dev(x)
        tg.itft_ex(d, l, z, nn, f, N, e, scale=1)
        got = from_dev(d)
        ref = x.copy()
        orc.itft(ref, l, z, nn, f, e, N)
        # the outputs below nn carry the division by L (scale=1), the f = 1 output does not
        p = (1 << N) + 1
        want = orc.cells_to_ints(ref, N, nn + f)
        want = [v * pow(2, -l, p) % p for v in want[:nn]] + want[nn:]
        assert orc.cells_to_ints(got, N, nn + f) == want, ("itft", N, l, z, nn, f, e)
    assert tg.wait_status() == tg.ZX_OK
