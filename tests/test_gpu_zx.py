"""GPU parity of Z[x] products (Sec. 5.1 with the TFT route of Sec. 2) against the oracle.

Exact integer results: the GPU product must equal the oracle's schoolbook product word for
word. For the 3000 x 2500 product of 2000-bit coefficients the oracle's TFT-based product
(itself pinned against schoolbook products in test_oracle_zx.py) is the reference, plus
spot checks modulo a 61-bit prime.
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


def product(tg, f, lf, mf, g, lg, mg, signed, bits, on_device):
    p = tg.zx_plan(lf, bits, lg, bits, signed)
    mh = p["limbs_h"] + 1
    lh = lf + lg - 1
    if on_device:
        F = torch.from_numpy(f.view(np.int64)).cuda()
        G = torch.from_numpy(g.view(np.int64)).cuda()
        H = torch.zeros(lh * mh, dtype=torch.int64, device="cuda")
        tg.zx_mul(F, lf, mf, G, lg, mg, H, mh, signed, bits, bits)
        torch.cuda.synchronize()
        h = H.cpu().numpy().view(np.uint64)
    else:
        h = np.zeros(lh * mh, np.uint64)
        tg.zx_mul(f, lf, mf, g, lg, mg, h, mh, signed, bits, bits)
    return h, mh


@pytest.mark.parametrize("lf,lg,bits,signed,dev", [
    (1, 1, 1, False, True), (1, 1, 64, True, False), (2, 1, 63, False, True),
    (17, 33, 100, False, True), (100, 100, 64, True, True), (257, 255, 300, True, False),
    (1000, 3, 1024, False, True), (513, 511, 1000, True, True), (60, 70, 5000, False, True),
])
def test_zx_mul_matches_schoolbook(tg, orc, lf, lg, bits, signed, dev):
    mf = (bits + (1 if signed else 0) + 63) // 64
    f = workloads.coefficients(lf + 101 * lg, lf, bits, mf, signed)
    g = workloads.coefficients(lf + 103 * lg + 1, lg, bits, mf, signed)
    h, mh = product(tg, f, lf, mf, g, lg, mf, signed, bits, dev)
    ref = orc.zx_schoolbook(f, lf, mf, g, lg, mf, mh, signed)
    assert np.array_equal(h, ref)


def test_extreme_coefficients(tg, orc):
    # every coefficient at the bound: the largest product coefficients, and all -2^b + 1 values
    for signed in (False, True):
        bits, lf, lg = 191, 70, 90
        mf = 3 if not signed else 4
        f = np.zeros(lf * mf, np.uint64)
        g = np.zeros(lg * mf, np.uint64)
        val = (1 << bits) - 1
        for i in range(lf):
            v = -val if signed else val
            v &= (1 << (64 * mf)) - 1
            f[i * mf:(i + 1) * mf] = [(v >> (64 * k)) & 0xFFFFFFFFFFFFFFFF for k in range(mf)]
        for i in range(lg):
            v = val & ((1 << (64 * mf)) - 1)
            g[i * mf:(i + 1) * mf] = [(v >> (64 * k)) & 0xFFFFFFFFFFFFFFFF for k in range(mf)]
        h, mh = product(tg, f, lf, mf, g, lg, mf, signed, bits, True)
        ref = orc.zx_schoolbook(f, lf, mf, g, lg, mf, mh, signed)
        assert np.array_equal(h, ref)


def test_medium_product_workload(tg, orc):
    """f of length 3000 times g of length 2500, 2000-bit unsigned coefficients."""
    w = workloads.PRODUCT_MEDIUM
    lf, lg, bits = w["len_f"], w["len_g"], w["bits"]
    mf = (bits + 63) // 64
    f = workloads.coefficients(w["seed"], lf, bits, mf)
    g = workloads.coefficients(w["seed"] + 1, lg, bits, mf)
    p = tg.zx_plan(lf, bits, lg, bits)
    assert (p["l"], p["N"], p["n"]) == (13, 4096, 5499)
    h, mh = product(tg, f, lf, mf, g, lg, mf, False, bits, True)
    ref, l, N = orc.zx_mul(f, lf, mf, g, lg, mf, mh, False, bits, bits)
    assert (l, N) == (13, 4096)
    assert np.array_equal(h, ref)
    P = (1 << 61) - 1
    rng = random.Random(7)
    for _ in range(3):
        t = rng.randrange(P)
        lhs = orc.poly_eval_mod(f, lf, mf, False, t, P) * orc.poly_eval_mod(g, lg, mf, False, t, P) % P
        assert lhs == orc.poly_eval_mod(h, lf + lg - 1, mh, False, t, P)


def test_buffer_too_small_reports_needed_limbs(tg):
    lf, lg, bits = 10, 10, 500
    f = workloads.coefficients(1, lf, bits, 8)
    g = workloads.coefficients(2, lg, bits, 8)
    h = np.zeros((lf + lg - 1) * 2, np.uint64)
    with pytest.raises(tg.TftError) as ei:
        tg.zx_mul(f, lf, 8, g, lg, 8, h, 2, False, bits, bits)
    assert ei.value.code == tg.ZX_EBUFSIZE


def test_concurrent_calls_from_two_threads(tg):
    """Two host threads call zx_mul at the same time, each on its own stream: every call forks
    its g transform onto its thread's helper stream and joins it back with events, so the
    results are the same as those of the calls made one after another."""
    import threading

    shapes = [(700, 900, 300), (2500, 1800, 500), (64, 3000, 128), (4000, 4000, 700), (1, 1, 64), (300, 5, 1000)]
    jobs = []
    for k, (lf, lg, bits) in enumerate(shapes * 2):
        m = (bits + 63) // 64
        F = torch.from_numpy(workloads.coefficients(500 + 2 * k, lf, bits, m).view(np.int64)).cuda()
        G = torch.from_numpy(workloads.coefficients(501 + 2 * k, lg, bits, m).view(np.int64)).cuda()
        mh = tg.zx_plan(lf, bits, lg, bits)["limbs_h"]
        jobs.append((F, lf, m, G, lg, mh, bits))
    ref = []
    for F, lf, m, G, lg, mh, bits in jobs:
        H = torch.zeros((lf + lg - 1) * mh, dtype=torch.int64, device="cuda")
        tg.zx_mul(F, lf, m, G, lg, m, H, mh, False, bits, bits)
        ref.append(H)
    torch.cuda.synchronize()
    outs = [torch.full_like(r, -1) for r in ref]
    errors = []

    def worker(part):
        try:
            s = torch.cuda.Stream()
            for _ in range(3):
                for i in part:
                    F, lf, m, G, lg, mh, bits = jobs[i]
                    tg.zx_mul(F, lf, m, G, lg, m, outs[i], mh, False, bits, bits, stream=s)
            s.synchronize()
        except Exception as exc:  # reported below, on the main thread
            errors.append(exc)

    threads = [threading.Thread(target=worker, args=(list(range(t, len(jobs), 2)),)) for t in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(120)
    assert not errors, errors
    torch.cuda.synchronize()
    for i, (r, o) in enumerate(zip(ref, outs)):
        assert torch.equal(r, o), i
