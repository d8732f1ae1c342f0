"""Pins for the oracle's Algorithm 1 (TFT) and Algorithm 2 (ITFT).

Routes checked against each other and against the mathematics:
  * Algorithm 1/2 (Secs. 3-4) against the brute-force DFT (Eq. dft), which is itself pinned
    in test_oracle_dft.py;
  * the ITFT against its definition (Sec. 2): mixed input built from brute-force a-hat and L a;
  * independence of the split (Sec. 2: any 1 < L1 < L; L1 = 2 is van der Hoeven's form);
  * the base-case bounds of Theorems 1 and 2;
  * every proof case (a)-(d) of Theorem 2;
  * the intermediate cell states drawn in Figs. 3-10 (fixtures in tests/golden/).
"""
import os
import random

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_res(rng, N, k):
    p = (1 << N) + 1
    # mostly uniform, with the special residues 0 and 2^N mixed in
    out = []
    for _ in range(k):
        r = rng.random()
        out.append(0 if r < 0.03 else (1 << N) if r < 0.06 else rng.randrange(p))
    return out


def brute(orc, vals, l, z, n, e, N):
    x = orc.cells_from_ints(vals, N, count=1 << l)
    return orc.cells_to_ints(orc.dft_brute(x, l, z, n, e, N), N, n)


def run_tft(orc, vals, l, z, n, e, N, **kw):
    x = orc.cells_from_ints(vals, N, count=1 << l)
    cnt = orc.tft(x, l, z, n, e, N, **kw)
    return orc.cells_to_ints(x, N, n), cnt


def itft_case(orc, rng, l, z, n, f, e, N):
    """Random a (z non-zero entries): mixed ITFT input and expected output (Sec. 2)."""
    L, p = 1 << l, (1 << N) + 1
    a = rand_res(rng, N, z)
    hat = brute(orc, a, l, z, min(L, n + 1), e, N)
    inp = hat[:n] + [(L * v) % p for v in a[n:z]]
    exp = [(L * v) % p for v in a[:n]] + ([hat[n]] if f else [])
    return inp, exp


def run_itft(orc, inp, l, z, n, f, e, N, **kw):
    x = orc.cells_from_ints(inp, N, count=1 << l)
    cnt = orc.itft(x, l, z, n, f, e, N, **kw)
    return orc.cells_to_ints(x, N, n + f), cnt


def tft_bound(n, l):
    L = 1 << l
    return min((n - 1) * l / 2 + L - 1, L * l / 2)


def itft_bound(n, f, l):
    L = 1 << l
    return min((n + f - 1) * l / 2 + L - 1, L * l / 2)


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_tft_matches_definition_random(orc, policy):
    rng = random.Random(11 + policy)
    for l in range(1, 8):
        L = 1 << l
        for N in (64, 128, 192):
            if (2 * N) % L:
                continue
            for t in range(6):
                z, n, e = rng.randint(1, L), rng.randint(1, L), rng.randrange(2 * N)
                a = rand_res(rng, N, z)
                got, cnt = run_tft(orc, a, l, z, n, e, N, policy=policy, seed=t)
                assert got == brute(orc, a, l, z, n, e, N), (l, N, z, n, e)
                assert cnt <= tft_bound(n, l)


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_itft_matches_definition_random(orc, policy):
    rng = random.Random(21 + policy)
    for l in range(1, 8):
        L = 1 << l
        for N in (64, 128):
            if (2 * N) % L:
                continue
            for t in range(6):
                f = rng.randint(0, 1)
                n = rng.randint(1 - f, L - f)
                z = rng.randint(max(n, 1), L)
                e = rng.randrange(2 * N)
                inp, exp = itft_case(orc, rng, l, z, n, f, e, N)
                got, cnt = run_itft(orc, inp, l, z, n, f, e, N, policy=policy, seed=t)
                assert got == exp, (l, N, z, n, f, e)
                assert cnt <= itft_bound(n, f, l)


@pytest.mark.parametrize("l", [1, 2, 3, 4, 5])
def test_exhaustive_small(orc, l):
    """Every (z, n) for the TFT and every (z, n, f) for the ITFT, balanced and D&C splits."""
    L, N = 1 << l, 64
    rng = random.Random(l)
    for z in range(1, L + 1):
        a = rand_res(rng, N, z)
        e = rng.randrange(2 * N)
        ref = brute(orc, a, l, z, L, e, N)
        for n in range(1, L + 1):
            for pol in (0, 1):
                got, cnt = run_tft(orc, a, l, z, n, e, N, policy=pol)
                assert got == ref[:n]
                assert cnt <= tft_bound(n, l)
        for n in range(0, z + 1):
            for f in (0, 1):
                if not (1 <= n + f <= L):
                    continue
                inp, exp = itft_case(orc, rng, l, z, n, f, e, N)
                for pol in (0, 1):
                    got, cnt = run_itft(orc, inp, l, z, n, f, e, N, policy=pol)
                    assert got == exp, (z, n, f, pol)
                    assert cnt <= itft_bound(n, f, l)


@pytest.mark.slow
def test_sampled_l6_l7(orc):
    rng = random.Random(99)
    for l, N in ((6, 64), (7, 128)):
        L = 1 << l
        for _ in range(25):
            z, n, e = rng.randint(1, L), rng.randint(1, L), rng.randrange(2 * N)
            a = rand_res(rng, N, z)
            ref = brute(orc, a, l, z, n, e, N)
            for pol in (0, 1, 2):
                assert run_tft(orc, a, l, z, n, e, N, policy=pol, seed=_)[0] == ref
            f = rng.randint(0, 1)
            nn = rng.randint(1 - f, min(z, L - f))
            inp, exp = itft_case(orc, rng, l, z, nn, f, e, N)
            for pol in (0, 1, 2):
                assert run_itft(orc, inp, l, z, nn, f, e, N, policy=pol, seed=_)[0] == exp


def test_roundtrip_and_plain_dft(orc):
    # z = n = L, f = 0, zeta = 1: the plain DFT and its inverse (Sec. 2)
    N, l = 256, 7
    L, p = 1 << l, (1 << N) + 1
    rng = random.Random(5)
    a = rand_res(rng, N, L)
    hat, _ = run_tft(orc, a, l, L, L, 0, N)
    assert hat == brute(orc, a, l, L, L, 0, N)
    back, _ = run_itft(orc, hat, l, L, L, 0, 0, N)
    assert back == [(L * v) % p for v in a]
    # truncated round trip ITFT(TFT(a)) = L a (Sec. 2, R[X] product with z = n)
    for n in (1, 37, 64, 65, 100):
        hat, _ = run_tft(orc, a[:n], l, n, n, 0, N)
        back, _ = run_itft(orc, hat, l, n, n, 0, 0, N)
        assert back == [(L * v) % p for v in a[:n]]


def test_split_independence_l8(orc):
    N, l = 128, 8
    L = 1 << l
    rng = random.Random(8)
    for z, n in ((200, 200), (17, 255), (256, 1), (129, 130)):
        a = rand_res(rng, N, z)
        e = rng.randrange(2 * N)
        outs = [run_tft(orc, a, l, z, n, e, N, policy=pol, seed=s)[0]
                for pol, s in ((0, 0), (1, 0), (2, 1), (2, 2), (3, 0))]
        assert all(o == outs[0] for o in outs)
        f = 1 if n < L else 0
        zz = max(z, n)
        inp, exp = itft_case(orc, rng, l, zz, n, f, e, N)
        for pol, s in ((0, 0), (1, 0), (2, 3)):
            assert run_itft(orc, inp, l, zz, n, f, e, N, policy=pol, seed=s)[0] == exp


def test_theorem_bounds_counting(orc):
    # count-only recursion (no arithmetic) at the large transform's sizes, l = 16
    l = 16
    L = 1 << l
    for n in (32769, 40000, 45000, 52000, 65536, 1, 2, 12345):
        c = orc.tft(None, l, n, n, 0, 32768)
        assert c <= tft_bound(n, l)
        c2 = orc.itft(None, l, n, n, 0, 0, 32768)
        assert c2 <= itft_bound(n, 0, l)
    # a full transform runs every butterfly: L l / 2 base cases
    assert orc.tft(None, l, L, L, 0, 32768) == L * l // 2
    assert orc.itft(None, l, L, L, 0, 0, 32768) == L * l // 2
    for l in range(1, 11):
        L = 1 << l
        for n in range(1, L + 1, max(1, L // 37)):
            for pol in (0, 1, 2):
                assert orc.tft(None, l, L, n, 0, 1 << 12, policy=pol, seed=n) <= tft_bound(n, l)
                for f in (0, 1):
                    if n + f <= L:
                        assert orc.itft(None, l, L, n, f, 0, 1 << 12, policy=pol,
                                        seed=n) <= itft_bound(n, f, l)


def proof_case(L2, z, n):
    z1, n2, z2 = z // L2, n % L2, z % L2
    if z1 == 0:
        return "a"
    if n2 == 0:
        return "b"
    return "c" if n2 <= z2 else "d"


def test_itft_proof_cases_all_hit(orc):
    # Theorem 2's proof cases (a) z1 = 0, (b) n2 = 0, (c) n2 <= z2, (d) n2 > z2, at l = 6
    N, l, l1 = 64, 6, 3
    L, L2 = 1 << l, 1 << (l - l1)
    rng = random.Random(6)
    seen = set()
    for z in range(1, L + 1):
        for n in range(0, z + 1):
            for f in (0, 1):
                if not (1 <= n + f <= L) or rng.random() > 0.15:
                    continue
                e = rng.randrange(2 * N)
                inp, exp = itft_case(orc, rng, l, z, n, f, e, N)
                got, _ = run_itft(orc, inp, l, z, n, f, e, N, policy=3, top_l1=l1)
                assert got == exp
                seen.add(proof_case(L2, z, n))
    assert seen == {"a", "b", "c", "d"}


# ---------------------------------------------------------------- Figs. 3-10
def load_grids(name):
    blocks, cur = [], None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.rstrip("\n")
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = {"name": line.strip("[]"), "grid": []}
            blocks.append(cur)
        elif "=" in line:
            k, v = (s.strip() for s in line.split("=", 1))
            cur[k] = v if k in ("source", "kind") else int(v)
        else:
            cur["grid"].append(line.strip())
    return blocks


def column_b(orc, a, l, l1, e, N):
    """b_k of Eq. (b-cols): brute-force weighted DFT of each column of a (length L1)."""
    L, L1, L2 = 1 << l, 1 << l1, 1 << (l - l1)
    w = 2 * N // L
    b = [0] * L
    for k2 in range(L2):
        col = [a[k2 + L2 * m] if k2 + L2 * m < len(a) else 0 for m in range(L1)]
        out = brute(orc, col, l1, L1, L1, (e + k2 * w) % (2 * N), N)
        for k1 in range(L1):
            b[k2 + L2 * k1] = out[k1]
    return b


@pytest.mark.parametrize("blk", load_grids("fig3_5_tft_cell_states.txt"), ids=lambda b: b["name"])
def test_tft_figure_states(orc, blk):
    N, l, l1 = 64, 6, 3
    L, p = 1 << l, (1 << N) + 1
    z, n = blk["z"], blk["n"]
    rows = blk["grid"]
    assert len(rows) == 8 and all(len(r) == 8 for r in rows)
    labels = "".join(rows)
    # the input diagram's `a` cells are exactly the first z cells
    if blk["phase"] == 0:
        assert [c == "a" for c in labels] == [i < z for i in range(L)]
    rng = random.Random(blk["name"])
    for e in (0, rng.randrange(2 * N)):
        a = rand_res(rng, N, z)
        x = orc.cells_from_ints(a, N, count=L)
        orc.tft_phases(x, l, l1, z, n, e, N, blk["phase"])
        cells = orc.cells_to_ints(x, N, L)
        hat = brute(orc, a, l, z, L, e, N)
        b = column_b(orc, a, l, l1, e, N)
        for i, c in enumerate(labels):
            if c == "a":
                assert cells[i] == a[i]
            elif c == "b":
                assert cells[i] == b[i], (i, blk["name"])
            elif c == "A":
                assert cells[i] == hat[i], (i, blk["name"])
            elif c in ".?":
                if c == "." and i >= z and blk["phase"] == 0:
                    assert cells[i] == 0
            else:
                raise AssertionError(c)
        assert p > 0


@pytest.mark.parametrize("blk", load_grids("fig6_10_itft_cell_states.txt"), ids=lambda b: b["name"])
def test_itft_figure_states(orc, blk):
    N, l, l1 = 64, 6, 3
    L, L2, p = 1 << l, 1 << (l - l1), (1 << N) + 1
    z, n = blk["z"], blk["n"]
    labels = "".join(blk["grid"])
    assert len(labels) == L
    rng = random.Random(blk["name"])
    for f in (0, 1):
        for e in (0, rng.randrange(2 * N)):
            a = rand_res(rng, N, z)
            hat = brute(orc, a, l, z, L, e, N)
            b = column_b(orc, a, l, l1, e, N)
            inp = hat[:n] + [(L * v) % p for v in a[n:z]]
            x = orc.cells_from_ints(inp, N, count=L)
            orc.itft_phases(x, l, l1, z, n, f, e, N, blk["phase"])
            cells = orc.cells_to_ints(x, N, L)
            for i, c in enumerate(labels):
                if c == "a":
                    assert cells[i] == (L * a[i]) % p, (i, blk["name"], f)
                elif c == "b" or (c == "B" and f == 1):
                    assert cells[i] == (L2 * b[i]) % p, (i, blk["name"], f)
                elif c == "A" or (c == "F" and f == 1):
                    assert cells[i] == hat[i], (i, blk["name"], f)
                else:
                    assert c in ".?BF"


def test_section6_partition_example():
    vals = {}
    for line in open(os.path.join(GOLDEN, "sec6_partition_example.txt")):
        line = line.split("#")[0].strip()
        if "=" in line:
            k, v = (s.strip() for s in line.split("="))
            vals[k] = float(v) if "." in v else int(v)
    n, l, l1, l2 = vals["n"], vals["l"], vals["l1"], vals["l2"]
    # the paper's split rule: L1 = 2^floor(l/2), L2 = 2^ceil(l/2)
    assert (l1, l2) == (l // 2, (l + 1) // 2)
    L2 = 1 << l2
    assert (n // L2, n % L2) == (vals["n1"], vals["n2"])
    assert -(-n // L2) * L2 == vals["padded_n"]
    assert (vals["padded_n"] - n) / n <= vals["max_penalty"]
    assert (1 << (l - 1)) < n <= (1 << l)


def test_section5_ring_size(orc):
    # 8000-bit coefficients at length 16384 give ~16000-bit Fourier coefficients (Sec. 5.1)
    l, N = orc.zx_plan(16384, 8000, 16384, 8000, False)
    assert l == 15 and abs(N - 16000) / 16000 < 0.05
