"""zx_mul_noalloc through the C ABI: the product for callers that cannot allocate device memory
(for example code whose GPU memory is entirely reserved by another allocator) must equal
zx_mul's result exactly, on two calls in a row that share the library's fixed scratch array.

This file is named so that pytest collects it last; it also passes when run alone in a fresh
process, where its first call performs the per-device set-up of the scratch array.
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


def operands(seed, lf, lg, bits, signed):
    mf = (bits + (1 if signed else 0) + 63) // 64
    f = workloads.coefficients(seed, lf, bits, mf, signed)
    g = workloads.coefficients(seed + 1, lg, bits, mf, signed)
    return mf, torch.from_numpy(f.view(np.int64)).cuda(), torch.from_numpy(g.view(np.int64)).cuda()


def both_products(tg, seed, lf, lg, bits, signed):
    mf, F, G = operands(seed, lf, lg, bits, signed)
    mh = tg.zx_plan(lf, bits, lg, bits, signed)["limbs_h"]
    lh = lf + lg - 1
    ref = torch.zeros(lh * mh, dtype=torch.int64, device="cuda")
    tg.zx_mul(F, lf, mf, G, lg, mf, ref, mh, signed, bits, bits)
    out = torch.full((lh * mh,), -1, dtype=torch.int64, device="cuda")
    tg.zx_mul_noalloc(F, lf, mf, G, lg, mf, out, mh, signed, bits, bits)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy()


def test_noalloc_matches_zx_mul_on_two_calls_in_a_row(tg):
    # first call: a 3000 x 2500 product of 2000-bit coefficients (the medium workload)
    w = workloads.PRODUCT_MEDIUM
    ref1, out1 = both_products(tg, w["seed"], w["len_f"], w["len_g"], w["bits"], False)
    assert np.array_equal(ref1, out1)
    # second call reuses the same scratch with a different ring and signed coefficients
    ref2, out2 = both_products(tg, 77, 700, 900, 333, True)
    assert np.array_equal(ref2, out2)


def test_noalloc_rejects_oversized_and_host_operands(tg):
    lf = lg = 20000
    bits = 64
    p = tg.zx_plan(lf, bits, lg, bits)
    assert 2 * (1 << p["l"]) * p["stride_limbs"] * 8 > 16 * 2 ** 20
    mf, F, G = operands(5, lf, lg, bits, False)
    H = torch.zeros((lf + lg - 1) * p["limbs_h"], dtype=torch.int64, device="cuda")
    with pytest.raises(tg.TftError) as ei:
        tg.zx_mul_noalloc(F, lf, mf, G, lg, mf, H, p["limbs_h"], False, bits, bits)
    assert ei.value.code == tg.ZX_EUNSUPPORTED and "16 MiB" in str(ei.value)
    f = workloads.coefficients(1, 4, 64, 1)
    with pytest.raises(tg.TftError) as ei:
        tg.zx_mul_noalloc(f, 4, 1, f, 4, 1, np.zeros(7, np.uint64), 2)
    assert ei.value.code == tg.ZX_EINVAL


def test_noalloc_on_the_sqrt2_ring(tg):
    # 1500 x 1500 coefficients of 500 bits: zx_plan picks omega = sqrt2 (a ring of N = 1024
    # instead of 2048), whose plans and kernels this entry point shares with zx_mul
    assert tg.zx_plan(1500, 500, 1500, 500)["sqrt2"] == 1
    ref, out = both_products(tg, 91, 1500, 1500, 500, False)
    assert np.array_equal(ref, out)


def test_noalloc_allocates_nothing_on_a_side_stream(tg):
    """A shape seen for the first time (its plans are written into the fixed array) on a stream
    other than the default one: no device memory is taken from the driver or from PyTorch's
    allocator, and the result equals zx_mul's. The same ring and transform length ran just
    before, so no kernel of the call is loaded for the first time during it."""
    lf, lg, bits = 2400, 1700, 700
    ref0, out0 = both_products(tg, 31, lf, lg, bits, False)  # warm: kernels of this ring
    assert np.array_equal(ref0, out0)
    mf, F, G = operands(32, lg, lf, bits, False)  # swapped lengths: same n, new plans
    mh = tg.zx_plan(lg, bits, lf, bits)["limbs_h"]
    lh = lf + lg - 1
    ref = torch.zeros(lh * mh, dtype=torch.int64, device="cuda")
    tg.zx_mul(F, lg, mf, G, lf, mf, ref, mh, False, bits, bits)
    out = torch.full((lh * mh,), -1, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    with torch.cuda.stream(side):
        tg.zx_mul_noalloc(F, lg, mf, G, lf, mf, out, mh, False, bits, bits, stream=side)
    side.synchronize()
    free1, torch1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert (free1, torch1) == (free0, torch0)
    assert torch.equal(out, ref)


def test_noalloc_captured_call_replays(tg):
    """A call of a shape planned before runs inside a captured CUDA graph and replays to the same
    result; a shape planned for the first time is refused while the stream is capturing."""
    lf, lg, bits = 1200, 1100, 450
    mf, F, G = operands(41, lf, lg, bits, False)
    mh = tg.zx_plan(lf, bits, lg, bits)["limbs_h"]
    lh = lf + lg - 1
    ref = torch.zeros(lh * mh, dtype=torch.int64, device="cuda")
    tg.zx_mul(F, lf, mf, G, lg, mf, ref, mh, False, bits, bits)
    out = torch.zeros(lh * mh, dtype=torch.int64, device="cuda")
    tg.zx_mul_noalloc(F, lf, mf, G, lg, mf, out, mh, False, bits, bits)  # plans this shape
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    out.fill_(-1)
    torch.cuda.synchronize()
    refused = None
    with torch.cuda.graph(graph, stream=side):
        tg.zx_mul_noalloc(F, lf, mf, G, lg, mf, out, mh, False, bits, bits, stream=side)
        try:  # a shape not planned yet
            tg.zx_mul_noalloc(F, lf - 1, mf, G, lg, mf, out, mh, False, bits, bits, stream=side)
        except tg.TftError as e:
            refused = e
    assert refused is not None and refused.code == tg.ZX_EINVAL
    for _ in range(2):
        out.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
