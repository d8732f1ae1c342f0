"""GPU parity of the transforms over the Schoenhage-Nussbaumer coefficient ring (Sec. 5.2):
R = S[y]/(y^(M/2)+1), S = Z/mZ, omega = y. Word for word against the oracle (pinned in
test_oracle_sn.py), from single-job transforms to multi-pass plans."""
import random

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P61 = (1 << 61) - 1


@pytest.fixture(scope="module")
def tg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0810_3203_gb300 as m
    m.load()
    return m


def rand_cells(rng, count, L, M, m):
    H = M // 2
    x = np.zeros(L * H, dtype=np.uint64)
    for i in range(count):
        r = rng.random()
        if r < 0.05:
            continue  # zero element
        if r < 0.1:
            x[i * H:(i + 1) * H] = np.uint64(m - 1)
        else:
            x[i * H:(i + 1) * H] = np.array([rng.randrange(m) for _ in range(H)], dtype=np.uint64)
    return x


def gpu(fn, x, *args, **kw):
    d = torch.from_numpy(x.view(np.int64)).cuda()
    fn(d, *args, **kw)
    torch.cuda.synchronize()
    return d.cpu().numpy().view(np.uint64)


CASES = [(2, 3, 1), (8, 5, 3), (64, 65537, 6), (256, P61, 8), (512, (1 << 62) + 3, 9), (2048, (1 << 40) + 15, 11)]


@pytest.mark.parametrize("M,m,l", CASES)
def test_sn_transforms_match_oracle(tg, orc, M, m, l):
    rng = random.Random(M + l)
    L, H = 1 << l, M // 2
    for t in range(3):
        z = [L, rng.randint(1, L), max(1, L // 3)][t]
        n = [L, rng.randint(1, L), rng.randint(1, L)][t]
        e = [0, rng.randrange(M), M - 1][t]
        x = rand_cells(rng, z, L, M, m)
        ref = x.copy()
        orc.sn_tft(ref, l, z, n, e, M, m)
        got = gpu(tg.sn_tft, x, l, z, n, M, m, e)
        assert np.array_equal(got[:n * H], ref[:n * H]), ("TFT", M, m, l, z, n, e)
        nn = min(n, z)
        f = 1 if nn < z and nn + 1 <= L else 0
        ref = x.copy()
        orc.sn_itft(ref, l, z, nn, f, e, M, m)
        got = gpu(tg.sn_itft, x, l, z, nn, f, M, m, e)
        assert np.array_equal(got[:(nn + f) * H], ref[:(nn + f) * H]), ("ITFT", M, m, l, z, nn, f, e)


@pytest.mark.parametrize("M,m,l", [(64, 65537, 6), (2048, P61, 11)])
def test_sn_round_trip(tg, M, m, l):
    rng = random.Random(l)
    L, H = 1 << l, M // 2
    n = max(1, L - L // 3)
    x = rand_cells(rng, n, L, M, m)
    d = torch.from_numpy(x.view(np.int64)).cuda()
    tg.sn_tft(d, l, n, n, M, m, 5)
    tg.sn_itft(d, l, n, n, 0, M, m, 5, scale=1)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy().view(np.uint64)[:n * H], x[:n * H])


def test_sn_exhaustive_small(tg, orc):
    M, m, l = 16, 65537, 4
    L, H = 1 << l, M // 2
    rng = random.Random(3)
    for z in range(1, L + 1):
        x = rand_cells(rng, z, L, M, m)
        for n in range(1, L + 1):
            ref = x.copy()
            orc.sn_tft(ref, l, z, n, 3, M, m)
            assert np.array_equal(gpu(tg.sn_tft, x, l, z, n, M, m, 3)[:n * H], ref[:n * H]), (z, n)
        for n in range(0, z + 1):
            for f in (0, 1):
                if not 1 <= n + f <= L:
                    continue
                ref = x.copy()
                orc.sn_itft(ref, l, z, n, f, 7, M, m)
                got = gpu(tg.sn_itft, x, l, z, n, f, M, m, 7)
                assert np.array_equal(got[:(n + f) * H], ref[:(n + f) * H]), (z, n, f)


def test_sn_invalid_arguments(tg):
    x = torch.zeros(64, dtype=torch.int64, device="cuda")
    for args, code in (((x, 3, 1, 1, 4, 5), tg.ZX_EINVAL),        # L = 8 does not divide M = 4
                       ((x, 1, 1, 1, 6, 5), tg.ZX_EINVAL),        # M not a power of two
                       ((x, 1, 1, 1, 8, 6), tg.ZX_EINVAL),        # even modulus
                       ((x, 2, 1, 1, 4096, 5), tg.ZX_EUNSUPPORTED)):
        with pytest.raises(tg.TftError) as ei:
            tg.sn_tft(*args)
        assert ei.value.code == code
