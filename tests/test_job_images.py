"""CPU check of the on-chip schedules (job images) that the GPU kernel executes.

A job image lists, per cluster CTA and stage, the base-case butterflies of Algorithm 1 / 2
(Secs. 3-4) on shared-memory slots, plus the layout exchanges between CTAs. This test runs
an image with Python integers (cell = value x with a pending rotation t, i.e. x 2^t), then
compares the cells it stores with the oracle's TFT / ITFT. It checks the schedule and the
slot bookkeeping, not the GPU's limb arithmetic (that is the GPU parity tests' job).
"""
import random

import pytest

from jobsim import Fermat, SnRing, run_image


@pytest.fixture(scope="module")
def tg():
    import paper_0810_3203_gb300 as m
    m.build.build()
    m.load(build_if_missing=False)
    return m


def oracle_tft(orc, vals, l, z, n, e, N):
    x = orc.cells_from_ints(vals, N, count=1 << l)
    orc.tft(x, l, z, n, e, N)
    return orc.cells_to_ints(x, N, n)


def oracle_itft(orc, vals, l, z, n, f, e, N):
    x = orc.cells_from_ints(vals, N, count=1 << l)
    orc.itft(x, l, z, n, f, e, N)
    return orc.cells_to_ints(x, N, n + f)


@pytest.mark.parametrize("ls,lc", [(2, 1), (3, 0), (4, 2), (5, 1), (5, 2), (6, 2), (6, 3), (7, 2), (8, 3), (8, 4)])
def test_tft_images(tg, orc, ls, lc):
    N = 256 if ls <= 8 else 1024
    L, p = 1 << ls, (1 << N) + 1
    rng = random.Random(ls * 10 + lc)
    for _ in range(6):
        z, n, e = rng.randint(1, L), rng.randint(1, L), rng.randrange(2 * N)
        vals = [rng.randrange(p) for _ in range(z)]
        img = tg.job_program(0, ls, lc, z, n, N)
        got = run_image(img, ls, N, e, vals, z, n)
        assert [got[m] for m in range(n)] == oracle_tft(orc, vals, ls, z, n, e, N), (ls, lc, z, n, e)


@pytest.mark.parametrize("ls,lc", [(2, 1), (3, 0), (4, 2), (5, 1), (5, 2), (6, 2), (6, 3), (7, 2), (8, 3), (8, 4)])
def test_itft_images(tg, orc, ls, lc):
    N = 256
    L, p = 1 << ls, (1 << N) + 1
    rng = random.Random(ls * 100 + lc)
    for t in range(8):
        f = t % 2
        n = rng.randint(1 - f, L - f)
        z = rng.randint(max(n, 1), L)
        e = rng.randrange(2 * N)
        vals = [rng.randrange(p) for _ in range(z)]
        img = tg.job_program(1, ls, lc, z, n, N, f)
        esc = (2 * N - ls) % (2 * N)
        got = run_image(img, ls, N, e, vals, z, n + f, nscale=n, escale=esc)
        ref = oracle_itft(orc, vals, ls, z, n, f, e, N)
        scaled = [v * pow(2, esc, p) % p for v in ref[:n]] + ref[n:]
        assert [got[m] for m in range(n + f)] == scaled, (ls, lc, z, n, f, e)


def test_cluster_job_every_itft_case(tg, orc):
    """An 8-CTA job of 64 cells: every (z, n, f) of the ITFT and every (z, n) of the TFT."""
    ls, lc, N = 6, 3, 64
    L, p = 1 << ls, (1 << N) + 1
    rng = random.Random(64)
    for z in range(1, L + 1, 3):
        vals = [rng.randrange(p) for _ in range(z)]
        for n in range(0, z + 1, 2):
            for f in (0, 1):
                if not 1 <= n + f <= L:
                    continue
                img = tg.job_program(1, ls, lc, z, n, N, f)
                got = run_image(img, ls, N, 5, vals, z, n + f)
                assert [got[m] for m in range(n + f)] == oracle_itft(orc, vals, ls, z, n, f, 5, N), (z, n, f)
            if n >= 1:
                img = tg.job_program(0, ls, lc, z, n, N)
                got = run_image(img, ls, N, 7, vals, z, n)
                assert [got[m] for m in range(n)] == oracle_tft(orc, vals, ls, z, n, 7, N), (z, n)


@pytest.mark.parametrize("ls,lc", [(3, 0), (4, 2), (6, 3), (8, 4)])
def test_sqrt2_images(tg, orc, ls, lc):
    """Schedules with exponents of sqrt2 (mod 4N) at L = 4N: the odd powers appear."""
    N = (1 << ls) // 4 if (1 << ls) >= 256 else 64
    L = 1 << ls
    R = Fermat(N, mode=2)
    rng = random.Random(ls * 13 + lc)
    for t in range(6):
        z, n, e = rng.randint(1, L), rng.randint(1, L), rng.randrange(4 * N)
        vals = [rng.randrange(R.p) for _ in range(z)]
        img = tg.job_program(0, ls, lc, z, n, N, mode=2)
        got = run_image(img, ls, N, e, vals, z, n, ring=R)
        x = orc.cells_from_ints(vals, N, count=L)
        orc.sqrt2_tft(x, ls, z, n, e, N)
        assert [got[m] for m in range(n)] == orc.cells_to_ints(x, N, n), (z, n, e)
        f = t % 2
        nn = rng.randint(1 - f, z - f if z - f >= 1 - f else 1 - f)
        nn = max(1 - f, min(nn, L - f, z))
        img = tg.job_program(1, ls, lc, z, nn, N, f, mode=2)
        esc = (4 * N - 2 * ls) % (4 * N)
        got = run_image(img, ls, N, e, vals, z, nn + f, nscale=nn, escale=esc, ring=R)
        x = orc.cells_from_ints(vals, N, count=L)
        orc.sqrt2_itft(x, ls, z, nn, f, e, N)
        ref = orc.cells_to_ints(x, N, nn + f)
        scaled = [R.pow(v, esc) for v in ref[:nn]] + ref[nn:]
        assert [got[m] for m in range(nn + f)] == scaled, (z, nn, f, e)


@pytest.mark.parametrize("ls", [2, 3, 4, 5])
def test_sn_images(tg, orc, ls):
    """Schedules over S[y]/(y^H+1): rotations are negacyclic shifts, and the ITFT base case's
    doublings and halvings are scalar flags."""
    M, m = 32, 65537
    H, L = M // 2, 1 << ls
    R = SnRing(H, m)
    rng = random.Random(ls)
    for t in range(6):
        z = rng.randint(1, L)
        e = rng.randrange(M)
        vals = [tuple(rng.randrange(m) for _ in range(H)) for _ in range(z)]
        f = t % 2
        n = max(1 - f, min(rng.randint(0, z), L - f))
        img = tg.job_program(1, ls, 0, z, n, H, f, mode=1)
        got = run_image(img, ls, H, e, vals, z, n + f, ring=R)
        x = orc.sn_cells([list(v) for v in vals], M, count=L)
        orc.sn_itft(x, ls, z, n, f, e, M, m)
        assert [list(got[i]) for i in range(n + f)] == orc.sn_vals(x, M, n + f), (z, n, f, e)
        nt = rng.randint(1, L)
        img = tg.job_program(0, ls, 0, z, nt, H, mode=1)
        got = run_image(img, ls, H, e, vals, z, nt, ring=R)
        x = orc.sn_cells([list(v) for v in vals], M, count=L)
        orc.sn_tft(x, ls, z, nt, e, M, m)
        assert [list(got[i]) for i in range(nt)] == orc.sn_vals(x, M, nt), (z, nt, e)
