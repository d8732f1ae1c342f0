"""CPU check of the on-chip schedules (job images) that the GPU kernel executes.

A job image lists, per cluster CTA and stage, the base-case butterflies of Algorithm 1 / 2
(Secs. 3-4) on shared-memory slots, plus the layout exchanges between CTAs. This test runs
an image with Python integers (cell = value x with a pending rotation t, i.e. x 2^t), then
compares the cells it stores with the oracle's TFT / ITFT. It checks the schedule and the
slot bookkeeping, not the GPU's limb arithmetic (that is the GPU parity tests' job).
"""
import random

import numpy as np
import pytest

OP_BF, OP_CROSS, OP_TAG = 1, 2, 3
OPF_S, OPF_D, OPF_S_TO_J, OPF_D_TO_I, OPF_COPY = 1, 2, 4, 8, 16
STAGE_PROG, STAGE_XCHG, STAGE_SWAP = 0, 1, 2


@pytest.fixture(scope="module")
def tg():
    import paper_0810_3203_gb300 as m
    m.build.build()
    m.load(build_if_missing=False)
    return m


def job_cell(layout, rank, slot, C, L2, b):
    if C == 1:
        return slot
    if layout == 0:
        return rank * L2 + slot
    return (slot // b) * L2 + rank * b + slot % b


def ops_of(img, off):
    nlev = int(img[off])
    nops = int(img[off + 1])
    starts = [int(v) for v in img[off + 2:off + 3 + nlev]]
    base = off + ((3 + nlev + 1) & ~1)
    ops = []
    for k in range(nops):
        w = [int(v) for v in img[base + 10 * k:base + 10 * k + 10]]
        ops.append(dict(i=w[0] & 0xFFFF, j=w[0] >> 16, kind=w[1] & 0xFF, flags=(w[1] >> 8) & 0xFF,
                        ra=(w[2], w[3]), rb=(w[4], w[5]), p0=(w[6], w[7]), p1=(w[8], w[9])))
    return starts, ops


def run_image(img, ls, N, e, inputs, nload, nstore, nscale=0, escale=0):
    """Execute a job image on Python integers; returns the stored cell values {cell: value}."""
    p, twoN = (1 << N) + 1, 2 * N
    nst, C, load_l, store_l = (int(v) for v in img[:4])
    lc = C.bit_length() - 1
    nslots = 1 << (ls - lc)
    L2, b = nslots, nslots // C
    rot = lambda a: (a[0] * e + a[1]) % twoN
    state = [[(0, 0)] * nslots for _ in range(C)]
    for c in range(C):
        for s in range(nslots):
            m = job_cell(load_l, c, s, C, L2, b)
            state[c][s] = (inputs[m] if m < nload else 0, 0)
    for st in range(nst):
        ent = 4 + st * (2 + C)
        typ, arg = int(img[ent]), int(img[ent + 1])
        if typ == STAGE_PROG:
            for c in range(C):
                off = int(img[ent + 2 + c])
                if not off:
                    continue
                starts, ops = ops_of(img, off)
                sc = state[c]
                for v in range(len(starts) - 1):
                    touched = set()
                    for o in ops[starts[v]:starts[v + 1]]:
                        for cell in {o["i"], o["j"]}:
                            assert cell not in touched, "ops of one level share a cell"
                            touched.add(cell)
                        xi, ti = sc[o["i"]]
                        xj, tj = sc[o["j"]]
                        if o["kind"] == OP_TAG:
                            if o["flags"] & OPF_COPY:
                                sc[o["j"]] = (xi, (ti + rot(o["rb"])) % twoN)
                            sc[o["i"]] = (xi, (ti + rot(o["ra"])) % twoN)
                            continue
                        A = xi * pow(2, ti + rot(o["ra"]), p) % p
                        B = xj * pow(2, tj + rot(o["rb"]), p) % p
                        if o["kind"] == OP_BF:
                            if o["flags"] & OPF_S:
                                dst = o["j"] if o["flags"] & OPF_S_TO_J else o["i"]
                                sc[dst] = ((A + B) % p, rot(o["p0"]))
                            if o["flags"] & OPF_D:
                                dst = o["i"] if o["flags"] & OPF_D_TO_I else o["j"]
                                sc[dst] = ((A - B) % p, rot(o["p1"]))
                        else:
                            D = (A - B) % p
                            sc[o["j"]] = (D, rot(o["p1"]))
                            sc[o["i"]] = ((A + D) % p, 0)
        else:
            only = arg if typ == STAGE_SWAP else -1
            new = [list(row) for row in state]
            for x in range(C):
                for y in range(C):
                    if y == x or not (only < 0 or x == only or y == only):
                        continue
                    for i in range(b):
                        new[x][y * b + i] = state[y][x * b + i]
            state = new
    out = {}
    for c in range(C):
        for s in range(nslots):
            m = job_cell(store_l, c, s, C, L2, b)
            if m < nstore:
                x, t = state[c][s]
                t += escale if m < nscale else 0
                out[m] = x * pow(2, t, p) % p
    return out


def oracle_tft(orc, vals, l, z, n, e, N):
    x = orc.cells_from_ints(vals, N, count=1 << l)
    orc.tft(x, l, z, n, e, N)
    return orc.cells_to_ints(x, N, n)


def oracle_itft(orc, vals, l, z, n, f, e, N):
    x = orc.cells_from_ints(vals, N, count=1 << l)
    orc.itft(x, l, z, n, f, e, N)
    return orc.cells_to_ints(x, N, n + f)


@pytest.mark.parametrize("ls,lc", [(2, 1), (3, 0), (4, 2), (5, 2), (6, 3), (7, 2), (8, 3), (8, 4)])
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


@pytest.mark.parametrize("ls,lc", [(2, 1), (3, 0), (4, 2), (5, 2), (6, 3), (7, 2), (8, 3), (8, 4)])
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
