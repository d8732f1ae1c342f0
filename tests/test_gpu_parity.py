"""GPU parity: the CUDA path through the C ABI against the oracle, bit for bit.

All arithmetic is exact, so the tolerance is zero: every defined output cell must equal the
oracle's (Sec. 2 definitions: TFT outputs a-hat_0..a-hat_{n-1}; ITFT outputs L a_0..L a_{n-1}
and a-hat_n when f = 1). Cells outside the defined outputs are scratch and are not compared.
"""
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


def limbs(N):
    return N // 64 + 1


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def from_dev(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def cells_eq(a, b, count, stride, W):
    A = a[:count * stride].reshape(count, stride)[:, :W]
    B = b[:count * stride].reshape(count, stride)[:, :W]
    bad = np.nonzero(~np.all(A == B, axis=1))[0]
    return bad


def special_inputs(x, N, stride, idx):
    """Put the residues 0, 1, 2^N and 2^N - 1 into cells idx (edge values of the ring)."""
    W = limbs(N)
    vals = [0, 1, 1 << N, (1 << N) - 1]
    for k, i in enumerate(idx):
        v = vals[k % 4]
        x[i * stride:i * stride + W] = [(v >> (64 * t)) & 0xFFFFFFFFFFFFFFFF for t in range(W)]


def gpu_tft(tg, x, l, z, n, e, N, stride):
    d = to_dev(x)
    tg.tft_ex(d, l, z, n, N, e, stride)
    return from_dev(d)


def gpu_itft(tg, x, l, z, n, f, e, N, stride, scale=0):
    d = to_dev(x)
    tg.itft_ex(d, l, z, n, f, N, e, stride, scale)
    return from_dev(d)


CASES = [  # (N, l) covering K = 1 .. 32 and one- and multi-pass plans
    (64, 3), (128, 5), (192, 6), (256, 7), (1024, 8), (1024, 11), (2048, 6), (3072, 9),
    (4096, 9), (4096, 10), (8192, 7), (16384, 6), (32768, 5), (32768, 7),
]


@pytest.mark.parametrize("N,l", CASES)
def test_tft_parity(tg, orc, N, l):
    L = 1 << l
    rng = random.Random(N * 31 + l)
    for t in range(3):
        z = [L, rng.randint(1, L), 1][t]
        n = [L, rng.randint(1, L), rng.randint(1, L)][t]
        e = [0, rng.randrange(2 * N), rng.randrange(2 * N)][t]
        stride = limbs(N) + [0, 1, 3][t]
        x = workloads.residues(1000 + t, z, N, stride=stride, cells=L)
        special_inputs(x, N, stride, [0, z // 2, z - 1])
        ref = x.copy()
        orc.tft(ref, l, z, n, e, N, stride=stride)
        got = gpu_tft(tg, x, l, z, n, e, N, stride)
        bad = cells_eq(got, ref, n, stride, limbs(N))
        assert bad.size == 0, f"N={N} l={l} z={z} n={n} e={e}: {bad.size} cells differ, first {bad[:5]}"


@pytest.mark.parametrize("N,l", CASES)
def test_itft_parity(tg, orc, N, l):
    L = 1 << l
    rng = random.Random(N * 17 + l)
    for t in range(4):
        f = t % 2
        n = [L - f, rng.randint(1 - f, L - f), rng.randint(0, 3), rng.randint(1 - f, L - f)][t]
        n = max(n, 1 - f)
        z = [max(n, 1), rng.randint(max(n, 1), L), L, max(n, 1)][t]
        e = [0, rng.randrange(2 * N), rng.randrange(2 * N), 0][t]
        stride = limbs(N) + (t % 2)
        x = workloads.residues(2000 + t, z, N, stride=stride, cells=L)
        special_inputs(x, N, stride, [0, z - 1])
        ref = x.copy()
        orc.itft(ref, l, z, n, f, e, N, stride=stride)
        got = gpu_itft(tg, x, l, z, n, f, e, N, stride)
        bad = cells_eq(got, ref, n + f, stride, limbs(N))
        assert bad.size == 0, f"N={N} l={l} z={z} n={n} f={f} e={e}: {bad.size} cells differ, first {bad[:5]}"


@pytest.mark.parametrize("N,l", [(128, 5), (1024, 8), (4096, 10), (8192, 7), (32768, 7), (32768, 12)])
def test_structured_inputs(tg, orc, N, l):
    """Inputs with long runs of equal bits (0, 2^N, 2^N - 1, runs of ones, small packed-like
    values): carries and borrows cross many words and lanes, and some results are the zero cell."""
    L = 1 << l
    W = limbs(N)
    rng = random.Random(N + l)
    for t in range(3):
        z = [L, rng.randint(1, L), max(1, L // 2 + 1)][t]
        n = [L, rng.randint(1, z), rng.randint(1, L)][t]
        e = [0, rng.randrange(2 * N), 1][t]
        x = workloads.structured_residues(7000 + 10 * t + l, z, N, cells=L)
        ref = x.copy()
        orc.tft(ref, l, z, n, e, N)
        got = gpu_tft(tg, x, l, z, n, e, N, W)
        bad = cells_eq(got, ref, n, W, W)
        assert bad.size == 0, f"TFT N={N} l={l} z={z} n={n} e={e}: {bad.size} cells differ, first {bad[:5]}"
        nn = min(n, z)
        ref = x.copy()
        orc.itft(ref, l, z, nn, 0, e, N)
        got = gpu_itft(tg, x, l, z, nn, 0, e, N, W)
        bad = cells_eq(got, ref, nn, W, W)
        assert bad.size == 0, f"ITFT N={N} l={l} z={z} n={nn} e={e}: {bad.size} cells differ, first {bad[:5]}"


def test_exhaustive_small(tg, orc):
    """Every (z, n) and (z, n, f) for L = 16 over Z/(2^64+1)."""
    N, l = 64, 4
    L, W = 1 << l, limbs(N)
    for z in range(1, L + 1):
        x = workloads.residues(z, z, N, cells=L)
        for n in range(1, L + 1):
            ref = x.copy()
            orc.tft(ref, l, z, n, 5, N)
            assert cells_eq(gpu_tft(tg, x, l, z, n, 5, N, W), ref, n, W, W).size == 0, (z, n)
        for n in range(0, z + 1):
            for f in (0, 1):
                if not 1 <= n + f <= L:
                    continue
                ref = x.copy()
                orc.itft(ref, l, z, n, f, 9, N)
                got = gpu_itft(tg, x, l, z, n, f, 9, N, W)
                assert cells_eq(got, ref, n + f, W, W).size == 0, (z, n, f)


def test_roundtrip_small_workload(tg, orc):
    """TFT then ITFT over Z/(2^1024+1), L = 256, n = z = 200: brute force and recovery."""
    w = workloads.ROUNDTRIP_SMALL
    N, l, n = w["N"], w["l"], w["n"]
    W = limbs(N)
    x = workloads.residues(w["seed"], n, N, cells=1 << l)
    brute = orc.dft_brute(x, l, n, n, 0, N)
    d = to_dev(x)
    tg.tft(d, l, n, N)
    hat = from_dev(d)
    assert cells_eq(hat, brute, n, W, W).size == 0
    tg.itft(d, l, n, N)
    back = from_dev(d)
    assert cells_eq(back, x, n, W, W).size == 0


def test_itft_scale(tg, orc):
    N, l, n = 4096, 9, 300
    W = limbs(N)
    x = workloads.residues(5, n, N, cells=1 << l)
    d = to_dev(x)
    tg.tft(d, l, n, N)
    hat = from_dev(d)
    tg.itft_ex(d, l, n, n, 0, N, 0, W, 0)
    unscaled = from_dev(d)
    ref = hat.copy()
    orc.itft(ref, l, n, n, 0, 0, N)
    assert cells_eq(unscaled, ref, n, W, W).size == 0


@pytest.mark.parametrize("n", workloads.TRANSFORM_LARGE["ns"])
def test_large_transform_roundtrip(tg, n):
    """Z/(2^32768+1), l = 16: TFT then ITFT restores every input cell."""
    w = workloads.TRANSFORM_LARGE
    N, l = w["N"], w["l"]
    W = limbs(N)
    x = workloads.residues(w["seed"], n, N, cells=1 << l)
    d = to_dev(x)
    tg.tft(d, l, n, N)
    tg.itft(d, l, n, N)
    back = from_dev(d)
    assert cells_eq(back, x, n, W, W).size == 0


def test_large_transform_tft_vs_oracle(tg, orc):
    """Z/(2^32768+1), l = 16, n = 40000: every TFT output against the oracle's Algorithm 1."""
    w = workloads.TRANSFORM_LARGE
    N, l, n = w["N"], w["l"], 40000
    W = limbs(N)
    x = workloads.residues(w["seed"], n, N, cells=1 << l)
    d = to_dev(x)
    tg.tft(d, l, n, N)
    got = from_dev(d)
    ref = x.copy()
    orc.tft(ref, l, n, n, 0, N)
    bad = cells_eq(got, ref, n, W, W)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5]}"


def test_invalid_arguments(tg):
    x = torch.zeros(16 * 2, dtype=torch.int64, device="cuda")
    with pytest.raises(tg.TftError) as ei:
        tg.tft_ex(x, 8, 1, 1, 64, 0, 2)  # L = 256 does not divide 2N = 128
    assert ei.value.code == tg.ZX_EINVAL
    with pytest.raises(tg.TftError) as ei:
        tg.tft_ex(x, 2, 5, 1, 64, 0, 2)  # z > L
    assert ei.value.code == tg.ZX_EINVAL
    with pytest.raises(tg.TftError) as ei:
        tg.itft_ex(x, 2, 1, 2, 0, 64, 0, 2)  # n > z
    assert ei.value.code == tg.ZX_EINVAL
    with pytest.raises(tg.TftError) as ei:
        tg.tft_ex(x, 2, 1, 1, 1088, 0, 18)  # N > 1024 not a multiple of 1024
    assert ei.value.code == tg.ZX_EUNSUPPORTED


@pytest.mark.parametrize("n,f,e", [(40000, 0, 0), (52000, 1, 12345)])
def test_large_itft_vs_oracle(tg, orc, n, f, e):
    """Z/(2^32768+1), l = 16, 16-byte aligned cells as the benchmark lays them out: every output of
    the exact ITFT (Algorithm 2 with its partial rows, z = n + f) against the oracle's, with the
    weight zeta = 2^e and without the final division by L."""
    w = workloads.TRANSFORM_LARGE
    N, l = w["N"], w["l"]
    W = limbs(N)
    st = W + (W & 1)
    z = n + f
    x = workloads.residues(w["seed"] + 7, z, N, stride=st, cells=1 << l)
    d = to_dev(x)
    tg.itft_ex(d, l, z, n, f, N, e, st, scale=0)
    got = from_dev(d)
    ref = x.copy()
    orc.itft(ref, l, z, n, f, e, N, stride=st)
    bad = cells_eq(got, ref, n + f, st, W)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5]}"


@pytest.mark.parametrize("n", [32769, 65536])
def test_large_tft_on_the_bulk_layout(tg, orc, n):
    """Z/(2^32768+1), l = 16, on the benchmark's 16-byte aligned 514-limb cells (bulk loads):
    every TFT output against the oracle's Algorithm 1, at the sweep's two ends (one cell past
    L/2, whose top column pass has n2 = 1, and the full length)."""
    w = workloads.TRANSFORM_LARGE
    N, l = w["N"], w["l"]
    W = limbs(N)
    st = W + 1
    x = workloads.residues(w["seed"] + n, n, N, stride=st, cells=1 << l)
    d = to_dev(x)
    tg.tft_ex(d, l, n, n, N, 0, st)
    got = from_dev(d)
    ref = x.copy()
    orc.tft(ref, l, n, n, 0, N, stride=st)
    bad = cells_eq(got, ref, n, st, W)
    assert bad.size == 0, f"{bad.size} cells differ, first {bad[:5]}"


@pytest.mark.parametrize("N,l,n", [(4096, 12, 3001), (32768, 13, 7777)])
def test_structured_residues_on_the_bulk_layout(tg, orc, N, l, n):
    """Residues with long runs of equal bits (carries and borrows that cross many lanes) on the
    bulk-load path (even strides, N >= 4096): TFT and exact ITFT against the oracle."""
    W = limbs(N)
    st = W + 1
    x = workloads.structured_residues(5 + l, n, N, stride=st, cells=1 << l)
    d = to_dev(x)
    tg.tft_ex(d, l, n, n, N, 0, st)
    got = from_dev(d)
    ref = x.copy()
    orc.tft(ref, l, n, n, 0, N, stride=st)
    assert cells_eq(got, ref, n, st, W).size == 0
    nn, f = n - 5, 1
    d = to_dev(x)
    tg.itft_ex(d, l, n, nn, f, N, 3, st, scale=0)
    got = from_dev(d)
    ref = x.copy()
    orc.itft(ref, l, n, nn, f, 3, N, stride=st)
    assert cells_eq(got, ref, nn + f, st, W).size == 0
