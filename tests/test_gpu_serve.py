"""GPU tests of the serving loop (zx_server_*): continuous batching of Z[x] products.

Requests arrive from the host while earlier ones run; every result must be the same word for
word as the product computed alone by zx_mul (itself pinned against the oracle's schoolbook
product in test_gpu_zx.py), and a sample is compared with the oracle directly.
"""
import random
import time

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


def operands(tg, k, lf, lg, bits, signed, seed):
    m = (bits + (1 if signed else 0) + 63) // 64
    f = workloads.coefficients(seed + 2 * k, lf, bits, m, signed)
    g = workloads.coefficients(seed + 2 * k + 1, lg, bits, m, signed)
    mh = tg.zx_plan(lf, bits, lg, bits, signed)["limbs_h"]
    F = torch.from_numpy(f.view(np.int64)).cuda()
    G = torch.from_numpy(g.view(np.int64)).cuda()
    H = torch.full(((lf + lg - 1) * mh,), -1, dtype=torch.int64, device="cuda")
    return (f, g, m, mh), (F, lf, m, G, lg, m, H, mh, signed, bits, bits)


def test_results_same_alone_and_in_the_mix(tg, orc):
    rng = random.Random(21)
    shapes = [(rng.randint(1, 3000), rng.randint(1, 3000), rng.randint(1, 3000), rng.random() < 0.3)
              for _ in range(48)]
    shapes[5] = (1, 1, 1, False)
    shapes[9] = (20000, 13000, 64, False)  # l = 16: the largest ring buffers of the mix
    data = [operands(tg, k, *s, 500) for k, s in enumerate(shapes)]
    torch.cuda.synchronize()
    with tg.Server(slots=3) as srv:
        ids = {}
        for k, (_, it) in enumerate(data):
            ids[srv.submit(*it)] = k
            if k >= 16:  # a burst first, then requests that arrive while batches run
                time.sleep(rng.random() * 0.002)
        srv.drain(120.0)
        done = []
        while len(done) < len(data):
            got = srv.poll()
            assert got or len(done) == len(data)
            done += got
        stats = srv.stats()
    assert sorted(ids[r] for r, _, _ in done) == list(range(len(data)))
    assert all(st == tg.ZX_OK and lat > 0 for _, st, lat in done)
    assert stats["completed"] == len(data) and stats["max_wave_products"] > 1
    for (host, (F, lf, m, G, lg, _, H, mh, signed, bits, _)) in data:
        alone = torch.full_like(H, -1)
        tg.zx_mul(F, lf, m, G, lg, m, alone, mh, signed, bits, bits)
        torch.cuda.synchronize()
        assert torch.equal(alone, H), (lf, lg, bits, signed)
    for k in (0, 5, 17, 30):
        f, g, m, mh = data[k][0]
        lf, lg, bits, signed = shapes[k]
        h = data[k][1][6].cpu().numpy().view(np.uint64)
        assert np.array_equal(h, orc.zx_schoolbook(f, lf, m, g, lg, m, mh, signed)), shapes[k]


def test_arena_admission_and_refusal(tg):
    """A product larger than the arena is refused at submission; products that fit the arena
    only one or two at a time still all complete (admission waits for memory to free up)."""
    big = operands(tg, 0, 6000, 6000, 500, False, 900)[1]
    small = [operands(tg, k, 700, 900, 300, False, 950)[1] for k in range(12)]
    need = tg.zx_plan(700, 300, 900, 300)["scratch_bytes"]
    with tg.Server(arena_bytes=2 * need + 65536, slots=2) as srv:
        with pytest.raises(tg.TftError) as ei:
            srv.submit(*big)
        assert ei.value.code == tg.ZX_ENOMEM
        for it in small:
            srv.submit(*it)
        srv.drain(60.0)
        done = srv.poll()
        stats = srv.stats()
    assert len(done) == len(small) and all(st == tg.ZX_OK for _, st, _ in done)
    assert stats["arena_peak_bytes"] <= stats["arena_bytes"] and stats["waves"] >= len(small) // 2
    for (F, lf, m, G, lg, _, H, mh, s, b, _) in small:
        alone = torch.full_like(H, -1)
        tg.zx_mul(F, lf, m, G, lg, m, alone, mh, s, b, b)
        torch.cuda.synchronize()
        assert torch.equal(alone, H)
