"""The C ABI library builds, loads without a GPU, and exports every entry point the header
declares; host-only planning calls answer without touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "tftgpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_0810_3203_gb300 as tg
    tg.build.build()
    return tg.load(build_if_missing=False)


def test_exports_every_declared_function(lib):
    import paper_0810_3203_gb300 as tg
    declared = header_functions()
    assert set(declared) == set(tg.EXPORTS), declared
    so = C.CDLL(tg.library_path())
    for name in declared:
        assert hasattr(so, name), name


def test_status_strings(lib):
    assert lib.zx_strerror(0) == b"ok"
    assert lib.zx_strerror(6) == b"unsupported size"
    assert b"sm_103a" in lib.zx_version()


def test_plan_medium_product():
    import paper_0810_3203_gb300 as tg
    p = tg.zx_plan(3000, 2000, 2500, 2000)
    assert (p["l"], p["N"], p["n"], p["K"]) == (13, 4096, 5499, 4)
    assert p["limbs_h"] * 64 >= 2000 + 2000 + 12
    assert p["tft_passes"] == 2 and p["itft_passes"] >= 2


def test_sqrt2_halves_the_large_rings():
    """With omega = sqrt2 (L | 4N) a product of length L needs a ring of L/4 bits: the mixed
    batch's largest products run over Z/(2^16384+1) instead of Z/(2^32768+1)."""
    import paper_0810_3203_gb300 as tg
    p = tg.zx_plan(20000, 1024, 20000, 1024)
    assert (p["l"], p["N"], p["sqrt2"]) == (16, 16384, 1)
    p = tg.zx_plan(12000, 700, 9000, 700)
    assert (p["l"], p["N"], p["sqrt2"]) == (15, 8192, 1)
    p = tg.zx_plan(3000, 2000, 2500, 2000)  # 4012 bits needed: the ring is the same either way
    assert (p["N"], p["sqrt2"]) == (4096, 0)


def test_zero_padded_product_length():
    """Sec. 6: the product's length is padded with known zeros to whole rows of the top-level
    split, so the ITFT is the TFT's steps reversed: as many passes as the TFT, no last row."""
    import paper_0810_3203_gb300 as tg
    p = tg.zx_plan(3000, 2000, 2500, 2000)
    assert p["n_fft"] == 5504  # 43 rows of 2^7 cells (split 2^6 x 2^7), n = 5499
    assert p["itft_passes"] == p["tft_passes"] == 2
    for lf, lg, bits in ((20000, 20000, 1024), (16385, 1, 64), (12000, 9000, 700), (150, 150, 3000)):
        p = tg.zx_plan(lf, bits, lg, bits)
        n, nf, L = p["n"], p["n_fft"], 1 << p["l"]
        assert n <= nf <= L and (nf - n) * 32 <= max(n, 32 * (1 << (p["l"] - p["l"] // 2)))
        shape = tg.transform_plan(1, p["l"], nf, nf, p["N"])
        exact = tg.transform_plan(1, p["l"], n, n, p["N"])
        assert p["itft_passes"] == shape["passes"] <= exact["passes"]
        if nf > n and exact["passes"] > 1:  # over global memory: no last row at the top level
            assert shape["passes"] < exact["passes"]
    # n = 39999 at L = 2^16: padded to whole rows at every level, the ITFT is the TFT reversed
    p = tg.zx_plan(20000, 1024, 20000, 1024)
    assert p["itft_passes"] == p["tft_passes"], p


def test_plan_sizes_follow_the_ring_rule():
    import paper_0810_3203_gb300 as tg
    for lf, lg, bits in ((1, 1, 1), (100, 100, 64), (20000, 20000, 1024), (5, 70000, 10)):
        if lf + lg - 1 > 65536:
            with pytest.raises(tg.TftError) as ei:
                tg.zx_plan(lf, bits, lg, bits)
            assert ei.value.code == tg.ZX_EUNSUPPORTED
            continue
        p = tg.zx_plan(lf, bits, lg, bits)
        L = 1 << p["l"]
        # omega = 2 needs L | 2N; omega = sqrt2 (chosen when it allows a smaller ring) L | 4N
        assert L >= lf + lg - 1 and ((4 if p["sqrt2"] else 2) * p["N"]) % L == 0
        if p["sqrt2"]:
            assert (2 * p["N"]) % L != 0  # only chosen where omega = 2 would need a bigger ring
        assert p["N"] >= 2 * bits + (min(lf, lg) - 1).bit_length()
        assert p["N"] <= 1024 or p["N"] % 1024 == 0


def test_rejects_bad_arguments_without_a_device(lib):
    # argument checks come before any CUDA call
    assert lib.tft_ex(None, 3, 1, 1, 64, 0, 2, None) == 1
    assert lib.tft_ex(C.c_void_p(8), 8, 1, 1, 64, 0, 2, None) == 1
    assert lib.itft_ex(C.c_void_p(8), 2, 1, 3, 0, 64, 0, 2, 0, None) == 1
    assert lib.tft_ex(C.c_void_p(8), 2, 1, 1, 1088, 0, 18, None) == 6
    assert b"1024" in lib.zx_last_error()


def test_launch_configuration_get_set_without_a_device():
    import paper_0810_3203_gb300 as tg
    N = 32768
    default = tg.config_get(N)
    assert default["max_warps"] in (8, 16) and default["split"] in (0, 1)
    shape = tg.transform_plan(0, 16, 40000, 40000, N)
    try:
        # cluster jobs of 16 CTAs with 16 cells each: 256-cell jobs, the paper's two passes
        tg.config_set(N, {"ls_max": 4, "ls_c": 4, "max_warps": 8, "split": 1})
        assert tg.config_get(N)["ls_c"] == 4
        two = tg.transform_plan(0, 16, 40000, 40000, N)
        assert two["passes"] == 2 and two["cluster_l"] == 4 and two["passes"] < shape["passes"]
        with pytest.raises(tg.TftError) as ei:
            tg.config_set(N, {"ls_max": 9, "ls_c": 3, "max_warps": 8, "split": 0})  # 512 cells of 4 KB
        assert ei.value.code == tg.ZX_EINVAL
    finally:
        tg.config_set(N)
    assert tg.config_get(N) == default
    assert tg.transform_plan(0, 16, 40000, 40000, N) == shape


def test_recursive_pointwise_plans_follow_the_ring_rules(lib):
    """The inner ring of the recursive pointwise products: 2^k pieces of M = N / 2^k bits (whole
    32-bit words), N' >= 2M + k + 1 so that every c_t (|c_t| < 2^k 2^{2M}) is determined by its
    residue, 2^k | N' (theta = 2^{N'/2^k} has theta^{2^k} = -1), N' a supported ring."""
    import paper_0810_3203_gb300 as tg
    for N in (2048, 3072, 4096, 8192, 12288, 16384, 20480, 32768):
        p = tg.pointwise_plan(N, 2)
        k, Ni = p["k"], p["N_inner"]
        M = N >> k
        assert p["method"] == 2 and k >= 2 and M % 32 == 0 and M << k == N, (N, p)
        assert Ni >= 2 * M + k + 1 and Ni % (1 << k) == 0, (N, p)
        assert (Ni <= 1024 and Ni % 64 == 0) or (Ni % 1024 == 0 and Ni <= 32768), (N, p)
        assert p["stride_inner"] >= Ni // 64 + 1 and p["stride_inner"] % 2 == 0
        assert 0 < p["cost_recursive"] and p["cost_schoolbook"] == (N // 32) ** 2
        assert tg.pointwise_plan(N, 1)["method"] == 1 and tg.pointwise_plan(N, 1)["k"] == 0
        assert tg.pointwise_plan(N)["method"] in (1, 2)
    # the schoolbook kernel is the faster one on every supported ring (measured), so auto keeps it
    for N in (1024, 4096, 32768):
        assert tg.pointwise_plan(N)["method"] == 1
    with pytest.raises(tg.TftError) as ei:
        tg.pointwise_plan(64, 2)  # four pieces of 16 bits: not whole 32-bit words
    assert ei.value.code == tg.ZX_EUNSUPPORTED
    with pytest.raises(tg.TftError) as ei:
        tg.pointwise_plan(4096, 5)
    assert ei.value.code == tg.ZX_EINVAL
    assert lib.zx_pointwise(None, None, 1, 4096, 65, 1, None) == tg.ZX_EINVAL


def test_whole_transforms_above_64_cells_take_two_passes(lib):
    """A whole transform of more than 64 cells is never a single job (that job would run all l
    levels on one CTA while the other SMs idle): it takes the Bailey split, whose jobs spread
    over the SMs; up to 64 cells it stays one job."""
    import paper_0810_3203_gb300 as tg
    for N in (128, 1024, 4096):
        for l in range(1, 12):
            if (2 * N) % (1 << l):
                continue
            L = 1 << l
            shape = tg.transform_plan(0, l, L, L, N)
            if l <= 6:
                assert shape["passes"] == 1 and shape["jobs"] == 1, (N, l, shape)
            else:
                assert shape["passes"] >= 2 and shape["jobs"] > 1, (N, l, shape)


def test_transform_jobs_reports_sizes_and_rejects_bad_arguments(lib):
    import numpy as np
    import paper_0810_3203_gb300 as tg
    i64, u32 = C.c_int64, C.c_uint32
    nj, ni = i64(0), i64(0)
    # sizes first (no buffers): ZX_EBUFSIZE with both lengths written
    rc = lib.zx_transform_jobs(0, 10, 700, 900, 0, 1024, 0, 0, 0, None, 0, C.byref(nj), None, 0, C.byref(ni))
    assert rc == tg.ZX_EBUFSIZE and nj.value > 4 and ni.value > 1
    J, I = np.zeros(nj.value, np.int64), np.zeros(ni.value, np.uint32)
    ok = lib.zx_transform_jobs(0, 10, 700, 900, 0, 1024, 0, 0, 0, J.ctypes.data_as(C.POINTER(i64)), J.size,
                               C.byref(nj), I.ctypes.data_as(C.POINTER(u32)), I.size, C.byref(ni))
    assert ok == tg.ZX_OK
    # header: passes, launches, jobs (the launches' counts add up), images
    plan = tg.transform_jobs(0, 10, 700, 900, 1024)
    assert int(J[0]) == plan["passes"] and int(J[1]) == len(plan["launches"])
    assert int(J[2]) == sum(len(L["jobs"]) for L in plan["launches"]) and int(J[3]) == len(plan["images"])
    # one word short on either buffer
    rc = lib.zx_transform_jobs(0, 10, 700, 900, 0, 1024, 0, 0, 0, J.ctypes.data_as(C.POINTER(i64)), J.size - 1,
                               C.byref(nj), I.ctypes.data_as(C.POINTER(u32)), I.size, C.byref(ni))
    assert rc == tg.ZX_EBUFSIZE
    bad = [(2, 10, 700, 900, 0, 1024, 0),   # kind
           (0, 12, 700, 900, 0, 1024, 0),   # L does not divide 2N
           (0, 10, 700, 1025, 0, 1024, 0),  # n > L
           (1, 10, 700, 701, 0, 1024, 0),   # ITFT with z < n
           (0, 10, 700, 900, 0, 1000, 0),   # N not a multiple of 64
           (0, 10, 700, 900, 0, 1024, 1)]   # mode 1 (S[y] rings have their own planner)
    for kind, l, z, n, f, N, mode in bad:
        rc = lib.zx_transform_jobs(kind, l, z, n, f, N, 0, 0, mode, None, 0, C.byref(nj), None, 0, C.byref(ni))
        assert rc in (tg.ZX_EINVAL, tg.ZX_EUNSUPPORTED), (kind, l, z, n, f, N, mode, rc)
