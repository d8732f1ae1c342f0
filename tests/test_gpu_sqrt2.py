"""GPU parity of the transforms with omega = sqrt2 = 2^(3N/4) - 2^(N/4) over Z/(2^N+1) (L | 4N;
the sqrt2 trick, not in the paper) and of the products that use them, word for word against
the oracle (pinned in test_oracle_sqrt2.py) and against schoolbook products."""
import random

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


def run(fn, x, *args, **kw):
    d = torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
    fn(d, *args, **kw)
    torch.cuda.synchronize()
    return d.cpu().numpy().view(np.uint64)


def same(a, b, count, W):
    return np.array_equal(a[:count * W].reshape(count, W), b[:count * W].reshape(count, W))


@pytest.mark.parametrize("N,l", [(64, 8), (64, 5), (128, 9), (1024, 12), (4096, 14), (16384, 16)])
def test_sqrt2_transforms_match_oracle(tg, orc, N, l):
    L, W = 1 << l, N // 64 + 1
    rng = random.Random(N + l)
    trials = 1 if l >= 16 else 3
    for t in range(trials):
        z = [rng.randint(L // 2, L), rng.randint(1, L), L][t]
        n = [rng.randint(L // 2, L), rng.randint(1, L), L][t]
        e = [rng.randrange(4 * N), 1, 0][t]
        gen = workloads.structured_residues if t == 1 else workloads.residues
        x = gen(900 + t + l, z, N, cells=L)
        ref = x.copy()
        orc.sqrt2_tft(ref, l, z, n, e, N)
        assert same(run(tg.tft_sqrt2, x, l, z, n, N, e), ref, n, W), ("TFT", z, n, e)
        nn = min(n, z)
        f = 1 if nn < z else 0
        ref = x.copy()
        orc.sqrt2_itft(ref, l, z, nn, f, e, N)
        assert same(run(tg.itft_sqrt2, x, l, z, nn, f, N, e), ref, nn + f, W), ("ITFT", z, nn, f, e)


def test_sqrt2_round_trip_scaled(tg):
    N, l, n = 16384, 16, 40000
    W = N // 64 + 1
    x = workloads.residues(31, n, N, cells=1 << l)
    d = torch.from_numpy(x.view(np.int64)).cuda()
    tg.tft_sqrt2(d, l, n, n, N, 3)
    tg.itft_sqrt2(d, l, n, n, 0, N, 3, scale=1)
    torch.cuda.synchronize()
    assert same(d.cpu().numpy().view(np.uint64), x, n, W)


@pytest.mark.parametrize("lf,lg,bits,signed", [(3000, 3000, 64, False), (2500, 1800, 300, True), (700, 900, 20, False)])
def test_products_over_sqrt2_rings_match_schoolbook(tg, orc, lf, lg, bits, signed):
    p = tg.zx_plan(lf, bits, lg, bits, signed)
    assert p["sqrt2"] == 1, p  # the ring is half the size omega = 2 would need
    mf = (bits + (1 if signed else 0) + 63) // 64
    f = workloads.coefficients(lf + 7, lf, bits, mf, signed)
    g = workloads.coefficients(lg + 9, lg, bits, mf, signed)
    mh = p["limbs_h"]
    F = torch.from_numpy(f.view(np.int64)).cuda()
    G = torch.from_numpy(g.view(np.int64)).cuda()
    H = torch.full(((lf + lg - 1) * mh,), -1, dtype=torch.int64, device="cuda")
    tg.zx_mul(F, lf, mf, G, lg, mf, H, mh, signed, bits, bits)
    torch.cuda.synchronize()
    assert np.array_equal(H.cpu().numpy().view(np.uint64), orc.zx_schoolbook(f, lf, mf, g, lg, mf, mh, signed))


def test_large_sqrt2_product_eval_mod(tg, orc):
    """20000 x 20000 coefficients of 1024 bits: L = 2^16 over Z/(2^16384+1), checked at random
    points modulo a 61-bit prime."""
    lf = lg = 20000
    bits, m = 1024, 16
    p = tg.zx_plan(lf, bits, lg, bits)
    assert (p["N"], p["sqrt2"]) == (16384, 1)
    f = workloads.coefficients(41, lf, bits, m)
    g = workloads.coefficients(42, lg, bits, m)
    mh = p["limbs_h"]
    F = torch.from_numpy(f.view(np.int64)).cuda()
    G = torch.from_numpy(g.view(np.int64)).cuda()
    H = torch.zeros((lf + lg - 1) * mh, dtype=torch.int64, device="cuda")
    tg.zx_mul(F, lf, m, G, lg, m, H, mh, False, bits, bits)
    h = H.cpu().numpy().view(np.uint64)
    P = (1 << 61) - 1
    rng = random.Random(5)
    for _ in range(3):
        t = rng.randrange(P)
        lhs = orc.poly_eval_mod(f, lf, m, False, t, P) * orc.poly_eval_mod(g, lg, m, False, t, P) % P
        assert lhs == orc.poly_eval_mod(h, lf + lg - 1, mh, False, t, P)


def test_largest_transform_the_library_takes(tg, orc):
    """The largest transform: omega = sqrt2 over Z/(2^32768+1) at L = 4N = 2^17 (537 MB of
    cells), z = n = 100000 with the stride padded to 16 bytes. Every TFT output against the
    oracle's Algorithm 1, every ITFT output (with f = 1) against the oracle's Algorithm 2, and
    the scaled round trip restoring the input."""
    N, l, n = 32768, 17, 100000
    W = N // 64 + 1
    st = W + (W & 1)
    x = workloads.residues(41, n, N, stride=st, cells=1 << l)
    cols = lambda a, k: a.reshape(-1, st)[:k, :W]
    ref = x.copy()
    orc.sqrt2_tft(ref, l, n, n, 5, N, stride=st)
    got = run(tg.tft_sqrt2, x, l, n, n, N, 5, st)
    assert np.array_equal(cols(got, n), cols(ref, n)), "TFT"
    ref = x.copy()
    orc.sqrt2_itft(ref, l, n, n - 1, 1, 5, N, stride=st)
    got = run(tg.itft_sqrt2, x, l, n, n - 1, 1, N, 5, st)
    assert np.array_equal(cols(got, n), cols(ref, n)), "ITFT"
    d = torch.from_numpy(x.view(np.int64)).cuda()
    tg.tft_sqrt2(d, l, n, n, N, 0, st)
    tg.itft_sqrt2(d, l, n, n, 0, N, 0, st, scale=1)
    torch.cuda.synchronize()
    assert np.array_equal(cols(d.cpu().numpy().view(np.uint64), n), cols(x, n)), "round trip"
