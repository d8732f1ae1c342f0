"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only draws random words (splitmix64,
Steele-Lea-Flood 2014) and shapes them like the paper's workloads. Both the CPU oracle
and the GPU library receive the arrays it returns.

Workload shapes (Harvey, arXiv 0810.3203, Sec. 5.1 uses random non-negative coefficients):
  * ROUNDTRIP_SMALL   TFT then ITFT over Z/(2^1024+1), l = 8, n = z = 200
  * PRODUCT_MEDIUM    f of length 3000 times g of length 2500, 2000-bit unsigned coefficients
  * TRANSFORM_LARGE   TFT + ITFT over Z/(2^32768+1), l = 16, n in {32769, 40000, 45000, 52000, 65536}
  * BATCH_MIXED       512 products, lengths U[200, 20000], bits U[64, 1024]
  * SERVE_POISSON     Poisson arrivals, lengths log-uniform [2^8, 2^15], bits log-uniform [64, 4096]
  * SMOOTHNESS_SWEEP  equal lengths 512 .. 16384 in 5% steps, 8000-bit coefficients (Sec. 5.1)
"""
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

ROUNDTRIP_SMALL = dict(N=1024, l=8, n=200, z=200, seed=0)
PRODUCT_MEDIUM = dict(len_f=3000, len_g=2500, bits=2000, seed=1)
TRANSFORM_LARGE = dict(N=32768, l=16, ns=(32769, 40000, 45000, 52000, 65536), seed=3)
BATCH_MIXED = dict(count=512, len_lo=200, len_hi=20000, bits_lo=64, bits_hi=1024, seed=4)
SERVE_POISSON = dict(rate=2000.0, len_lo=2 ** 8, len_hi=2 ** 15, bits_lo=64, bits_hi=4096, seed=5)
SMOOTHNESS_SWEEP = dict(len_lo=512, len_hi=16384, step=1.05, bits=8000, seed=6)
# Sec. 5.2 shape: a polynomial of about 5 * 10^5 coefficients modulo a 41-bit odd modulus, cut
# into pieces of M/4 coefficients, each piece an element of S[y]/(y^(M/2)+1) with its upper
# half zero; transform length 2^11 = M, n = 2000 nonzero elements
SN_TRANSFORM = dict(M=2048, m=(1 << 40) + 15, l=11, n=2000, seed=7)


def splitmix64(seed, count, offset=0):
    """Words offset .. offset+count-1 of the splitmix64 stream started at `seed`."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def limbs_for(N):
    return N // 64 + 1


def residues(seed, count, N, stride=None, cells=None, offset=0):
    """`count` uniform residues in [0, 2^N) as cells of `stride` limbs (default N/64+1).

    The array holds `cells` cells (default `count`); cells past `count`, the top limb and
    any padding limbs are zero.
    """
    W = limbs_for(N)
    stride = stride or W
    cells = cells if cells is not None else count
    assert stride >= W and cells >= count
    x = np.zeros((cells, stride), dtype=np.uint64)
    if count:
        x[:count, :W - 1] = splitmix64(seed, count * (W - 1), offset).reshape(count, W - 1)
    return x.reshape(-1)


def structured_residues(seed, count, N, stride=None, cells=None):
    """`count` residues in [0, 2^N] drawn from shapes with long runs of equal bits, which make
    carries and borrows travel far: 0, 1, 2^N, 2^N - 1, powers of two, 2^N - 2^k, runs of ones
    (2^a - 1) 2^b, small values (below 2^64 or 2^1024, like packed coefficients) and uniform
    values. Same cell layout as residues()."""
    W = limbs_for(N)
    stride = stride or W
    cells = cells if cells is not None else count
    x = np.zeros((cells, stride), dtype=np.uint64)
    words = splitmix64(seed, 4 * count).tolist()
    for i in range(count):
        kind, a, b, c = (int(v) for v in words[4 * i:4 * i + 4])
        kind %= 10
        if kind == 0:
            v = 0
        elif kind == 1:
            v = 1
        elif kind == 2:
            v = 1 << N
        elif kind == 3:
            v = (1 << N) - 1
        elif kind == 4:
            v = 1 << (a % N)
        elif kind == 5:
            v = (1 << N) - (1 << (a % N))
        elif kind == 6:
            lo, hi = sorted((a % N, b % N))
            v = ((1 << (hi - lo + 1)) - 1) << lo
            v = min(v, (1 << N) - 1)
        elif kind == 7:
            v = c
        elif kind == 8:
            v = int.from_bytes(np.asarray(splitmix64(c, 16), dtype=np.uint64).tobytes(), "little") % (1 << min(N, 1024))
        else:
            v = int.from_bytes(np.asarray(splitmix64(c, W - 1), dtype=np.uint64).tobytes(), "little")
        for t in range(W):
            x[i, t] = np.uint64((v >> (64 * t)) & 0xFFFFFFFFFFFFFFFF)
    return x.reshape(-1)


def sn_elements(seed, count, M, m, cells=None, nonzero=None):
    """`count` elements of S[y]/(y^(M/2)+1), S = Z/mZ: the first `nonzero` coefficients
    (default M/4, a piece of the input polynomial) uniform in [0, m), the rest zero; cells of
    M/2 uint64, `cells` cells in all (the ones past `count` zero)."""
    H = M // 2
    nonzero = M // 4 if nonzero is None else nonzero
    cells = cells if cells is not None else count
    x = np.zeros((cells, H), dtype=np.uint64)
    if count and nonzero:
        w = splitmix64(seed, count * nonzero).reshape(count, nonzero)
        x[:count, :nonzero] = w % np.uint64(m)
    return x.reshape(-1)


def coefficients(seed, length, bits, limbs, signed=False, offset=0):
    """`length` coefficients uniform in [0, 2^bits) (signed: |c| < 2^bits, random sign),
    stored in `limbs` little-endian uint64 limbs, two's complement when signed."""
    assert limbs * 64 >= bits + (1 if signed else 0)
    words = splitmix64(seed, length * limbs, offset).reshape(length, limbs)
    full, rem = divmod(bits, 64)
    words[:, full + (1 if rem else 0):] = 0
    if rem:
        words[:, full] &= np.uint64((1 << rem) - 1)
    if signed:
        sign = splitmix64(seed ^ 0x5151, length, offset) & np.uint64(1)
        neg = sign.astype(bool)
        # two's complement negation of the selected rows
        inv = ~words[neg]
        carry = np.ones(inv.shape[0], dtype=np.uint64)
        for k in range(limbs):
            s = inv[:, k] + carry
            carry = ((s < carry) & (carry > 0)).astype(np.uint64)
            inv[:, k] = s
        words[neg] = inv
    return words.reshape(-1)


def _uniform_ints(seed, count, lo, hi, offset=0):
    w = splitmix64(seed, count, offset)
    return [lo + int(v) % (hi - lo + 1) for v in w.tolist()]


def _log_uniform_ints(seed, count, lo, hi, offset=0):
    w = splitmix64(seed, count, offset)
    out = []
    for v in w.tolist():
        u = (int(v) >> 11) / float(1 << 53)
        out.append(int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))))
    return out


def batch_shapes(count=BATCH_MIXED["count"], seed=BATCH_MIXED["seed"], len_lo=BATCH_MIXED["len_lo"],
                 len_hi=BATCH_MIXED["len_hi"], bits_lo=BATCH_MIXED["bits_lo"],
                 bits_hi=BATCH_MIXED["bits_hi"]):
    """(len_f, len_g, bits) per product of the mixed batch."""
    lf = _uniform_ints(seed, count, len_lo, len_hi, 0)
    lg = _uniform_ints(seed, count, len_lo, len_hi, count)
    bits = _uniform_ints(seed, count, bits_lo, bits_hi, 2 * count)
    return list(zip(lf, lg, bits))


def serve_requests(count, seed=SERVE_POISSON["seed"], rate=SERVE_POISSON["rate"],
                   len_lo=SERVE_POISSON["len_lo"], len_hi=SERVE_POISSON["len_hi"],
                   bits_lo=SERVE_POISSON["bits_lo"], bits_hi=SERVE_POISSON["bits_hi"]):
    """(arrival_time_s, len_f, len_g, bits) for a Poisson stream of requests."""
    w = splitmix64(seed, count, 0)
    t, arrivals = 0.0, []
    for v in w.tolist():
        u = ((int(v) >> 11) + 0.5) / float(1 << 53)
        t += -math.log(u) / rate
        arrivals.append(t)
    lf = _log_uniform_ints(seed, count, len_lo, len_hi, count)
    lg = _log_uniform_ints(seed, count, len_lo, len_hi, 2 * count)
    bits = _log_uniform_ints(seed, count, bits_lo, bits_hi, 3 * count)
    return list(zip(arrivals, lf, lg, bits))


def smoothness_lengths(lo=SMOOTHNESS_SWEEP["len_lo"], hi=SMOOTHNESS_SWEEP["len_hi"],
                       step=SMOOTHNESS_SWEEP["step"]):
    out, v = [], float(lo)
    while v <= hi:
        out.append(int(v))
        v *= step
    return out
