"""GPU parity of batched Z[x] products (zx_mul_batch) against the oracle.

The batch shares launches between products of one ring and overlaps rings on forked streams,
so these tests mix lengths, coefficient sizes, signedness and rings in one call. Small
products are compared word for word with the oracle's schoolbook product; the 512-product
mixed workload (lengths uniform in [200, 20000], coefficient bits uniform in [64, 1024]) is
checked for every product by evaluation at random points modulo a 61-bit prime (a property
that holds at any size) and, for its smallest products, word for word against schoolbook.
"""
import random

import numpy as np
import pytest

import workloads

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


def make_batch(tg, shapes, seed):
    """shapes: (len_f, len_g, bits, signed). Returns host operands and device tensors."""
    host, items = [], []
    for k, (lf, lg, bits, signed) in enumerate(shapes):
        m = (bits + (1 if signed else 0) + 63) // 64
        f = workloads.coefficients(seed + 2 * k, lf, bits, m, signed)
        g = workloads.coefficients(seed + 2 * k + 1, lg, bits, m, signed)
        mh = tg.zx_plan(lf, bits, lg, bits, signed)["limbs_h"]
        F = torch.from_numpy(f.view(np.int64)).cuda()
        G = torch.from_numpy(g.view(np.int64)).cuda()
        H = torch.full(((lf + lg - 1) * mh,), -1, dtype=torch.int64, device="cuda")
        host.append((f, g, m, mh))
        items.append((F, lf, m, G, lg, m, H, mh, signed, bits, bits))
    return host, items


def test_mixed_batch_matches_schoolbook(tg, orc):
    rng = random.Random(11)
    shapes = [(1, 1, 1, False), (1, 7, 64, True), (3, 2, 63, False), (200, 1, 1024, True)]
    for _ in range(28):
        shapes.append((rng.randint(1, 400), rng.randint(1, 400), rng.randint(1, 2500), rng.random() < 0.4))
    host, items = make_batch(tg, shapes, 100)
    rings = {tg.zx_plan(lf, b, lg, b, s)["N"] for lf, lg, b, s in shapes}
    assert len(rings) >= 6, rings
    tg.zx_mul_batch(items)
    torch.cuda.synchronize()
    for (lf, lg, bits, signed), (f, g, m, mh), it in zip(shapes, host, items):
        h = it[6].cpu().numpy().view(np.uint64)
        ref = orc.zx_schoolbook(f, lf, m, g, lg, m, mh, signed)
        assert np.array_equal(h, ref), (lf, lg, bits, signed)


def test_batch_equals_one_at_a_time(tg):
    """Each product's words are the same alone (zx_mul) and inside a batch."""
    rng = random.Random(12)
    shapes = [(rng.randint(500, 3000), rng.randint(500, 3000), rng.randint(64, 1500), rng.random() < 0.5)
              for _ in range(12)]
    _, items = make_batch(tg, shapes, 200)
    tg.zx_mul_batch(items)
    torch.cuda.synchronize()
    for (F, lf, m, G, lg, _, H, mh, signed, bits, _) in items:
        alone = torch.full_like(H, -1)
        tg.zx_mul(F, lf, m, G, lg, m, alone, mh, signed, bits, bits)
        torch.cuda.synchronize()
        assert torch.equal(alone, H), (lf, lg, bits, signed)


def test_mixed_workload_512_products(tg, orc):
    shapes = [(lf, lg, bits, False) for lf, lg, bits in workloads.batch_shapes()]
    host, items = make_batch(tg, shapes, workloads.BATCH_MIXED["seed"] * 1000)
    tg.zx_mul_batch(items)
    torch.cuda.synchronize()
    rng = random.Random(13)
    for (lf, lg, bits, _), (f, g, m, mh), it in zip(shapes, host, items):
        h = it[6].cpu().numpy().view(np.uint64)
        t = rng.randrange(P61)
        lhs = orc.poly_eval_mod(f, lf, m, False, t, P61) * orc.poly_eval_mod(g, lg, m, False, t, P61) % P61
        assert lhs == orc.poly_eval_mod(h, lf + lg - 1, mh, False, t, P61), (lf, lg, bits)
    smallest = sorted(range(len(shapes)), key=lambda k: shapes[k][0] * shapes[k][1])[:3]
    for k in smallest:
        lf, lg, bits, _ = shapes[k]
        f, g, m, mh = host[k]
        h = items[k][6].cpu().numpy().view(np.uint64)
        assert np.array_equal(h, orc.zx_schoolbook(f, lf, m, g, lg, m, mh, False)), (lf, lg, bits)


def test_batch_edge_cases(tg):
    tg.zx_mul_batch([])  # empty batch: nothing to do
    _, items = make_batch(tg, [(5, 5, 100, False), (4, 3, 70, True)], 300)
    # host operand: rejected, nothing launched
    F, lf, m, G, lg, _, H, mh, s, b, _ = items[1]
    bad = items[:1] + [(F.cpu().numpy().view(np.uint64), lf, m, G, lg, m, H, mh, s, b, b)]
    with pytest.raises(tg.TftError) as ei:
        tg.zx_mul_batch(bad)
    assert ei.value.code == tg.ZX_EINVAL
    # output too small in the second product
    small = items[:1] + [(F, lf, m, G, lg, m, H, 1, s, b, b)]
    with pytest.raises(tg.TftError) as ei:
        tg.zx_mul_batch(small)
    assert ei.value.code == tg.ZX_EBUFSIZE
    assert "product 1" in str(ei.value)
