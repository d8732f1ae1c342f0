"""GPU parity of the two ways the per-pass kernel moves cells (zx_tune_info.tma): one tensor (TMA)
copy per cell, for rings of 8 or more words per lane on 16-byte aligned buffers with an even
stride >= W + 1, and row copies with 16-byte stores otherwise. Both must give the oracle's TFT
(Algorithm 1) and exact ITFT (Algorithm 2) bit for bit; the tensor stores must leave the limbs
past a cell's top limb untouched; a buffer that is not 16-byte aligned must take the row path.
"""
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


def limbs(N):
    return N // 64 + 1


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def from_dev(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def bad_cells(a, b, count, stride, W):
    A = a[:count * stride].reshape(count, stride)[:, :W]
    B = b[:count * stride].reshape(count, stride)[:, :W]
    return np.nonzero(~np.all(A == B, axis=1))[0]


class pinned_tma:
    """Pin the tma setting of ring N for the block, then restore the configuration."""

    def __init__(self, tg, N, tma):
        self.tg, self.N, self.tma = tg, N, tma

    def __enter__(self):
        self.before = self.tg.config_get(self.N)
        self.tg.config_set(self.N, dict(self.before, tma=self.tma))

    def __exit__(self, *exc):
        self.tg.config_set(self.N, self.before)


@pytest.mark.parametrize("N,l,n", [(8192, 12, 3001), (16384, 12, 2500), (32768, 13, 7777)])
@pytest.mark.parametrize("tma", [1, 0])
def test_tft_and_exact_itft_match_the_oracle(tg, orc, N, l, n, tma):
    W = limbs(N)
    st = W + 1  # even for these rings: the tensor path qualifies when tma = 1
    x = workloads.structured_residues(11 + l + tma, n, N, stride=st, cells=1 << l)
    with pinned_tma(tg, N, tma):
        d = to_dev(x)
        tg.tft_ex(d, l, n, n, N, 5, st)
        got = from_dev(d)
        ref = x.copy()
        orc.tft(ref, l, n, n, 5, N, stride=st)
        bad = bad_cells(got, ref, n, st, W)
        assert bad.size == 0, f"TFT: {bad.size} cells differ, first {bad[:5]}"
        nn, f = n - 7, 1
        d = to_dev(x)
        tg.itft_ex(d, l, n, nn, f, N, 3, st, scale=0)
        got = from_dev(d)
        ref = x.copy()
        orc.itft(ref, l, n, nn, f, 3, N, stride=st)
        bad = bad_cells(got, ref, nn + f, st, W)
        assert bad.size == 0, f"ITFT: {bad.size} cells differ, first {bad[:5]}"


def test_scaled_round_trip_on_the_tensor_path(tg):
    """TFT then ITFT with the division by L (the final pass scales its cells on the way out)."""
    N, l, n = 16384, 13, 6000
    W = limbs(N)
    st = W + 1
    x = workloads.residues(23, n, N, stride=st, cells=1 << l)
    with pinned_tma(tg, N, 1):
        d = to_dev(x)
        tg.tft_ex(d, l, n, n, N, 0, st)
        tg.itft_ex(d, l, n, n, 0, N, 0, st, scale=1)
        back = from_dev(d)
    assert bad_cells(back, x, n, st, W).size == 0


def test_limbs_past_the_top_limb_are_never_written(tg, orc):
    """Cells of 516 limbs (three past W = 513): the tensor stores write the N-bit part and the top
    limb only, so a sentinel in the other limbs of every cell survives a TFT and an ITFT."""
    N, l, n = 32768, 13, 5000
    W = limbs(N)
    st = W + 3
    L = 1 << l
    x = workloads.residues(31, n, N, stride=st, cells=L)
    sentinel = np.uint64(0xA5A5A5A5DEADBEEF)
    x.reshape(L, st)[:, W:] = sentinel
    with pinned_tma(tg, N, 1):
        d = to_dev(x)
        tg.tft_ex(d, l, n, n, N, 0, st)
        got = from_dev(d)
        assert np.all(got.reshape(L, st)[:, W:] == sentinel)
        ref = x.copy()
        orc.tft(ref, l, n, n, 0, N, stride=st)
        assert bad_cells(got, ref, n, st, W).size == 0
        tg.itft_ex(d, l, n, n, 0, N, 0, st, scale=1)
        back = from_dev(d)
        assert np.all(back.reshape(L, st)[:, W:] == sentinel)
        assert bad_cells(back, x, n, st, W).size == 0


def test_a_buffer_that_is_not_16_byte_aligned_takes_the_row_path(tg, orc):
    """The same transform on a buffer that starts 8 bytes into an allocation (tensor copies need
    16-byte aligned cells, so the launches fall back to row copies) against the oracle."""
    N, l, n = 8192, 12, 3001
    W = limbs(N)
    st = W + 1
    x = workloads.residues(41, n, N, stride=st, cells=1 << l)
    with pinned_tma(tg, N, 1):
        base = torch.zeros(x.size + 1, dtype=torch.int64, device="cuda")
        d = base[1:]
        assert d.data_ptr() % 16 == 8
        d.copy_(torch.from_numpy(x.view(np.int64)))
        tg.tft_ex(d, l, n, n, N, 0, st)
        got = from_dev(d)
    ref = x.copy()
    orc.tft(ref, l, n, n, 0, N, stride=st)
    assert bad_cells(got, ref, n, st, W).size == 0


def test_the_setting_round_trips_through_the_configuration(tg):
    N = 32768
    before = tg.config_get(N)
    assert before["tma"] == 1
    try:
        tg.config_set(N, dict(before, tma=0))
        assert tg.config_get(N)["tma"] == 0
        with pytest.raises(tg.TftError):
            tg.config_set(N, dict(before, tma=2))
    finally:
        tg.config_set(N, before)
    assert tg.config_get(N) == before


def test_batched_products_on_large_rings_take_either_path(tg, orc):
    """zx_mul_batch merges the transforms of many products into shared launches (job_kernel with
    segment tables); these shapes (coefficients of about 3800 and 7800 bits) land on the rings
    N = 8192 and 16384, whose 8 and 16 words per lane fill all 32 lanes, where the merged launches
    use tensor copies. The batch must give the same words with tma on and off, the same as zx_mul
    alone, and the oracle's schoolbook product for its smallest product."""
    shapes = [(609, 1088, 3801, False), (959, 796, 3889, True), (1366, 814, 3829, True), (1338, 1130, 3995, False),
              (652, 1242, 7799, False), (1471, 1340, 7986, False), (59, 138, 7935, True), (293, 1307, 7706, False),
              (310, 1120, 7757, True), (1483, 1213, 4067, False)]
    rings = [tg.zx_plan(lf, b, lg, b, s)["N"] for lf, lg, b, s in shapes]
    assert set(rings) == {8192, 16384}, rings
    results = {}
    for tma in (1, 0):
        with pinned_tma(tg, 8192, tma), pinned_tma(tg, 16384, tma):
            items, host = [], []
            for k, (lf, lg, bits, signed) in enumerate(shapes):
                m = (bits + (1 if signed else 0) + 63) // 64
                f = workloads.coefficients(500 + 2 * k, lf, bits, m, signed)
                g = workloads.coefficients(501 + 2 * k, lg, bits, m, signed)
                mh = tg.zx_plan(lf, bits, lg, bits, signed)["limbs_h"]
                F = torch.from_numpy(f.view(np.int64)).cuda()
                G = torch.from_numpy(g.view(np.int64)).cuda()
                H = torch.full(((lf + lg - 1) * mh,), -1, dtype=torch.int64, device="cuda")
                items.append((F, lf, m, G, lg, m, H, mh, signed, bits, bits))
                host.append((f, g, m, mh))
            tg.zx_mul_batch(items)
            torch.cuda.synchronize()
            results[tma] = [it[6].cpu().numpy().view(np.uint64).copy() for it in items]
            if tma == 1:
                for (F, lf, m, G, lg, _, H, mh, signed, bits, _), got in zip(items, results[1]):
                    alone = torch.full_like(H, -1)
                    tg.zx_mul(F, lf, m, G, lg, m, alone, mh, signed, bits, bits)
                    torch.cuda.synchronize()
                    assert np.array_equal(alone.cpu().numpy().view(np.uint64), got), (lf, lg, bits, signed)
                smallest = sorted(range(len(shapes)), key=lambda k: shapes[k][0] * shapes[k][1])[:1]
                for k in smallest:
                    lf, lg, bits, signed = shapes[k]
                    f, g, m, mh = host[k]
                    assert np.array_equal(results[1][k], orc.zx_schoolbook(f, lf, m, g, lg, m, mh, signed))
    for a, b in zip(results[1], results[0]):
        assert np.array_equal(a, b)
