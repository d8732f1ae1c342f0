"""GPU parity under every launch configuration, and the autotuner (zx_tune).

Any split and any job size give the same outputs (Sec. 2 decomposition), so the transforms
must match the oracle word for word whatever configuration a ring runs with; the tuner must
leave its buffer restored and the fastest configuration in place.
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


def cells(a, count, W):
    return a[:count * W].reshape(count, W)


def configs(N):
    out = []
    for ls_max in (4, 5, 6, 8):
        for ls_c in (3, 4, 5):
            for mw in (8, 16):
                for sp in (0, 1):
                    out.append({"ls_max": ls_max, "ls_c": ls_c, "max_warps": mw, "split": sp})
    return out


@pytest.mark.parametrize("N,l", [(1024, 11), (4096, 11), (32768, 9)])
def test_parity_under_every_configuration(tg, orc, N, l):
    L, W = 1 << l, N // 64 + 1
    rng = random.Random(N + l)
    tried = 0
    try:
        for cfg in configs(N):
            try:
                tg.config_set(N, cfg)
            except tg.TftError:
                continue  # does not fit this ring
            tried += 1
            z, n = rng.randint(L // 2, L), rng.randint(1, L)
            e = rng.randrange(2 * N)
            x = workloads.residues(100 + tried, z, N, cells=L)
            ref = x.copy()
            orc.tft(ref, l, z, n, e, N)
            d = torch.from_numpy(x.view(np.int64)).cuda()
            tg.tft_ex(d, l, z, n, N, e)
            got = d.cpu().numpy().view(np.uint64)
            assert np.array_equal(cells(got, n, W), cells(ref, n, W)), (cfg, z, n, e)
            nn = min(n, z)
            ref = x.copy()
            orc.itft(ref, l, z, nn, 1 if nn < z else 0, e, N)
            d = torch.from_numpy(x.view(np.int64)).cuda()
            f = 1 if nn < z else 0
            tg.itft_ex(d, l, z, nn, f, N, e)
            got = d.cpu().numpy().view(np.uint64)
            assert np.array_equal(cells(got, nn + f, W), cells(ref, nn + f, W)), (cfg, z, nn, f, e)
    finally:
        tg.config_set(N)
    assert tried >= 8


def test_tune_restores_buffer_and_keeps_fastest(tg, orc):
    N, l, n = 4096, 12, 3000
    W = N // 64 + 1
    x = workloads.residues(77, n, N, cells=1 << l)
    d = torch.from_numpy(x.view(np.int64)).cuda()
    try:
        info = tg.tune(d, l, n, N, reps=1)
        torch.cuda.synchronize()
        back = d.cpu().numpy().view(np.uint64)
        assert np.array_equal(cells(back, n, W), cells(x, n, W))
        assert info["candidates"] >= 4 and info["best_ms"] > 0
        assert tg.config_get(N) == {k: info[k] for k in ("ls_max", "ls_c", "max_warps", "split", "fused", "max_cluster_log2", "tma")}
        # the tuned configuration computes the same transform as the oracle
        ref = x.copy()
        orc.tft(ref, l, n, n, 0, N)
        tg.tft(d, l, n, N)
        got = d.cpu().numpy().view(np.uint64)
        assert np.array_equal(cells(got, n, W), cells(ref, n, W))
    finally:
        tg.config_set(N)


def test_tune_sqrt2_ring(tg):
    """L = 4N: the tuner times the omega = sqrt2 transforms products use on that ring."""
    N, l, n = 1024, 12, 3000
    W = N // 64 + 1
    x = workloads.residues(78, n, N, cells=1 << l)
    d = torch.from_numpy(x.view(np.int64)).cuda()
    try:
        info = tg.tune(d, l, n, N, reps=1)
        torch.cuda.synchronize()
        assert info["best_ms"] > 0
        assert np.array_equal(cells(d.cpu().numpy().view(np.uint64), n, W), cells(x, n, W))
    finally:
        tg.config_set(N)


def test_fewest_pass_configuration_at_the_benchmark_size(tg, orc):
    """split 2 with clusters of at most 4 CTAs (three passes for the l = 16 TFT: 64-cell column
    jobs on 4-CTA clusters, then 32-cell rows) on the benchmark's 514-limb layout: every TFT
    output at n = 40000 and every exact ITFT output at n = 45000, f = 1, against the oracle."""
    N, l = 32768, 16
    W = N // 64 + 1
    st = W + 1
    before = tg.config_get(N)
    tg.config_set(N, dict(before, ls_c=4, split=2, max_cluster_log2=2))
    try:
        n = 40000
        x = workloads.residues(61, n, N, stride=st, cells=1 << l)
        d = torch.from_numpy(x.view(np.int64)).cuda()
        tg.tft_ex(d, l, n, n, N, 0, st)
        got = d.cpu().numpy().view(np.uint64)
        ref = x.copy()
        orc.tft(ref, l, n, n, 0, N, stride=st)
        A = got[:n * st].reshape(n, st)[:, :W]
        B = ref[:n * st].reshape(n, st)[:, :W]
        assert np.array_equal(A, B)
        n, f = 45000, 1
        x = workloads.residues(62, n + f, N, stride=st, cells=1 << l)
        d = torch.from_numpy(x.view(np.int64)).cuda()
        tg.itft_ex(d, l, n + f, n, f, N, 77, st, scale=0)
        got = d.cpu().numpy().view(np.uint64)
        ref = x.copy()
        orc.itft(ref, l, n + f, n, f, 77, N, stride=st)
        A = got[:(n + f) * st].reshape(n + f, st)[:, :W]
        B = ref[:(n + f) * st].reshape(n + f, st)[:, :W]
        assert np.array_equal(A, B)
    finally:
        tg.config_set(N, before)
    assert tg.wait_status() == tg.ZX_OK


@pytest.mark.parametrize("N,l,n", [(32768, 16, 40000), (4096, 12, 3001)])
def test_streaming_launch_form(tg, orc, N, l, n):
    """fused = 3: every per-pass launch of single-CTA jobs runs as a persistent loop that
    prefetches a CTA's next job into L2: TFT and exact ITFT outputs against the oracle."""
    W = N // 64 + 1
    st = W + 1
    before = tg.config_get(N)
    tg.config_set(N, dict(before, fused=3))
    try:
        x = workloads.residues(63 + l, n, N, stride=st, cells=1 << l)
        d = torch.from_numpy(x.view(np.int64)).cuda()
        tg.tft_ex(d, l, n, n, N, 0, st)
        got = d.cpu().numpy().view(np.uint64)
        ref = x.copy()
        orc.tft(ref, l, n, n, 0, N, stride=st)
        assert np.array_equal(got[:n * st].reshape(n, st)[:, :W], ref[:n * st].reshape(n, st)[:, :W])
        nn, f = n - 3, 1
        d = torch.from_numpy(x.view(np.int64)).cuda()
        tg.itft_ex(d, l, n, nn, f, N, 5, st, scale=0)
        got = d.cpu().numpy().view(np.uint64)
        ref = x.copy()
        orc.itft(ref, l, n, nn, f, 5, N, stride=st)
        k = nn + f
        assert np.array_equal(got[:k * st].reshape(k, st)[:, :W], ref[:k * st].reshape(k, st)[:, :W])
    finally:
        tg.config_set(N, before)
    assert tg.wait_status() == tg.ZX_OK
