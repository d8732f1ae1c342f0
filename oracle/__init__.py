"""ctypes front end of the C oracle (test infrastructure only).

The oracle is the slow, plain CPU ground truth for the TFT/ITFT over Z/(2^N+1) and for
Z[x] products (Harvey, arXiv 0810.3203: Eq. dft, Algorithms 1 and 2, Sec. 5.1). Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.

Cells are numpy uint64 arrays: cell i occupies limbs [i*stride, i*stride + W) with
W = N/64 + 1 little-endian limbs holding a canonical residue in [0, 2^N].
"""
import ctypes as C

import numpy as np

from . import build as _build

SPLIT_BALANCED, SPLIT_DC, SPLIT_RANDOM, SPLIT_TOP = 0, 1, 2, 3

_lib = None
_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)


class _Poly(C.Structure):
    _fields_ = [("len", C.c_int64), ("limbs", C.c_int64), ("is_signed", C.c_int),
                ("bits", C.c_int64), ("data", _u64p)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        i64, i32, u64 = C.c_int64, C.c_int, C.c_uint64
        for name in ("orc_ring_add", "orc_ring_sub", "orc_ring_mul"):
            getattr(L, name).argtypes = [_u64p, _u64p, _u64p, i64]
        L.orc_ring_mul2exp.argtypes = [_u64p, _u64p, i64, i64]
        L.orc_ring_div2.argtypes = [_u64p, _u64p, i64]
        L.orc_ring_reduce.argtypes = [_u64p, _u64p, i64, i64]
        L.orc_dft_brute.argtypes = [_u64p, _u64p, i64, i32, i64, i64, i64, i64]
        L.orc_tft.argtypes = [_u64p, i64, i32, i64, i64, i64, i64, i32, i32, u64, _i64p]
        L.orc_itft.argtypes = [_u64p, i64, i32, i64, i64, i32, i64, i64, i32, i32, u64, _i64p]
        L.orc_tft_phases.argtypes = [_u64p, i64, i32, i32, i64, i64, i64, i64, i32]
        L.orc_itft_phases.argtypes = [_u64p, i64, i32, i32, i64, i64, i32, i64, i64, i32]
        for name in ("orc_sn_add", "orc_sn_sub", "orc_sn_mul"):
            getattr(L, name).argtypes = [_u64p, _u64p, _u64p, i64, u64]
        L.orc_sn_ypow.argtypes = [_u64p, _u64p, i64, i64, u64]
        L.orc_sn_half.argtypes = [_u64p, _u64p, i64, u64]
        L.orc_sn_dft_brute.argtypes = [_u64p, _u64p, i64, i32, i64, i64, i64, i64, u64]
        L.orc_sn_tft.argtypes = [_u64p, i64, i32, i64, i64, i64, i64, u64, i32, i32, u64, _i64p]
        L.orc_sn_itft.argtypes = [_u64p, i64, i32, i64, i64, i32, i64, i64, u64, i32, i32, u64, _i64p]
        L.orc_sqrt2_dft_brute.argtypes = [_u64p, _u64p, i64, i32, i64, i64, i64, i64]
        L.orc_sqrt2_tft.argtypes = [_u64p, i64, i32, i64, i64, i64, i64, i32, i32, u64, _i64p]
        L.orc_sqrt2_itft.argtypes = [_u64p, i64, i32, i64, i64, i32, i64, i64, i32, i32, u64, _i64p]
        L.orc_zx_mul.argtypes = [C.POINTER(_Poly)] * 3 + [C.POINTER(i32), _i64p]
        L.orc_zx_plan.argtypes = [i64, i64, i64, i64, i32, C.POINTER(i32), _i64p]
        L.orc_zx_schoolbook.argtypes = [C.POINTER(_Poly)] * 3
        L.orc_poly_eval_mod.argtypes = [C.POINTER(_Poly), u64, u64]
        L.orc_poly_eval_mod.restype = u64
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.uint64 and a.flags.c_contiguous
    return a.ctypes.data_as(_u64p)


def limbs(N):
    return N // 64 + 1


# ---------------------------------------------------------------- conversions
def int_to_limbs(v, n):
    """Non-negative Python int -> n little-endian uint64 limbs."""
    assert v >= 0 and v < (1 << (64 * n))
    return np.array([(v >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(n)], dtype=np.uint64)


def limbs_to_int(a):
    v = 0
    for i, x in enumerate(np.asarray(a, dtype=np.uint64).tolist()):
        v |= int(x) << (64 * i)
    return v


def cells_from_ints(vals, N, count=None, stride=None):
    W = limbs(N)
    stride = stride or W
    count = count if count is not None else len(vals)
    x = np.zeros(count * stride, dtype=np.uint64)
    for i, v in enumerate(vals):
        x[i * stride:i * stride + W] = int_to_limbs(v, W)
    return x


def cells_to_ints(x, N, count, stride=None):
    W = limbs(N)
    stride = stride or W
    return [limbs_to_int(x[i * stride:i * stride + W]) for i in range(count)]


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what}: precondition violated")


# ---------------------------------------------------------------- ring (Python ints in/out)
def _ring2(name, a, b, N):
    W = limbs(N)
    r = np.zeros(W, np.uint64)
    A, B = int_to_limbs(a, W), int_to_limbs(b, W)
    _check(getattr(lib(), name)(_p(r), _p(A), _p(B), N), name)
    return limbs_to_int(r)


def ring_add(a, b, N):
    return _ring2("orc_ring_add", a, b, N)


def ring_sub(a, b, N):
    return _ring2("orc_ring_sub", a, b, N)


def ring_mul(a, b, N):
    return _ring2("orc_ring_mul", a, b, N)


def ring_mul2exp(a, k, N):
    W = limbs(N)
    r = np.zeros(W, np.uint64)
    _check(lib().orc_ring_mul2exp(_p(r), _p(int_to_limbs(a, W)), k, N), "mul2exp")
    return limbs_to_int(r)


def ring_div2(a, N):
    W = limbs(N)
    r = np.zeros(W, np.uint64)
    _check(lib().orc_ring_div2(_p(r), _p(int_to_limbs(a, W)), N), "div2")
    return limbs_to_int(r)


def ring_reduce(x, N):
    n = max(1, (x.bit_length() + 63) // 64)
    r = np.zeros(limbs(N), np.uint64)
    _check(lib().orc_ring_reduce(_p(r), _p(int_to_limbs(x, n)), n, N), "reduce")
    return limbs_to_int(r)


# ---------------------------------------------------------------- transforms (arrays)
def dft_brute(x, l, z, n, e, N, stride=None):
    """Eq. (dft) by definition; returns a new array holding cells 0..n-1."""
    stride = stride or limbs(N)
    out = np.zeros((1 << l) * stride, np.uint64)
    _check(lib().orc_dft_brute(_p(out), _p(x), stride, l, z, n, e, N), "dft_brute")
    return out


def tft(x, l, z, n, e, N, stride=None, policy=SPLIT_BALANCED, top_l1=0, seed=0):
    """Algorithm 1 in place on x (None: count only). Returns the base-case count."""
    stride = stride or limbs(N)
    cnt = C.c_int64(0)
    ptr = _p(x) if x is not None else None
    _check(lib().orc_tft(ptr, stride, l, z, n, e, N, policy, top_l1, seed, C.byref(cnt)), "tft")
    return cnt.value


def itft(x, l, z, n, f, e, N, stride=None, policy=SPLIT_BALANCED, top_l1=0, seed=0):
    """Algorithm 2 in place on x (None: count only). Returns the base-case count."""
    stride = stride or limbs(N)
    cnt = C.c_int64(0)
    ptr = _p(x) if x is not None else None
    _check(lib().orc_itft(ptr, stride, l, z, n, f, e, N, policy, top_l1, seed, C.byref(cnt)), "itft")
    return cnt.value


def tft_phases(x, l, l1, z, n, e, N, stop_after, stride=None):
    stride = stride or limbs(N)
    _check(lib().orc_tft_phases(_p(x), stride, l, l1, z, n, e, N, stop_after), "tft_phases")


def itft_phases(x, l, l1, z, n, f, e, N, stop_after, stride=None):
    stride = stride or limbs(N)
    _check(lib().orc_itft_phases(_p(x), stride, l, l1, z, n, f, e, N, stop_after), "itft_phases")


# ---------------------------------------------------------------- Z[x]
def _poly(arr, length, nlimbs, signed, bits=0):
    assert arr.dtype == np.uint64 and arr.size >= length * nlimbs
    return _Poly(length, nlimbs, 1 if signed else 0, bits, _p(arr))


def zx_plan(len_f, bits_f, len_g, bits_g, signed):
    l, N = C.c_int(0), C.c_int64(0)
    _check(lib().orc_zx_plan(len_f, bits_f, len_g, bits_g, 1 if signed else 0,
                             C.byref(l), C.byref(N)), "zx_plan")
    return l.value, N.value


def zx_mul(f, len_f, limbs_f, g, len_g, limbs_g, limbs_h, signed=False, bits_f=0, bits_g=0):
    """Oracle Schoenhage-Strassen product; returns (h array, l, N)."""
    len_h = len_f + len_g - 1
    h = np.zeros(len_h * limbs_h, np.uint64)
    P = _poly(h, len_h, limbs_h, signed)
    F, G = _poly(f, len_f, limbs_f, signed, bits_f), _poly(g, len_g, limbs_g, signed, bits_g)
    l, N = C.c_int(0), C.c_int64(0)
    _check(lib().orc_zx_mul(C.byref(P), C.byref(F), C.byref(G), C.byref(l), C.byref(N)), "zx_mul")
    return h, l.value, N.value


def zx_schoolbook(f, len_f, limbs_f, g, len_g, limbs_g, limbs_h, signed=False):
    len_h = len_f + len_g - 1
    h = np.zeros(len_h * limbs_h, np.uint64)
    P = _poly(h, len_h, limbs_h, signed)
    F, G = _poly(f, len_f, limbs_f, signed), _poly(g, len_g, limbs_g, signed)
    _check(lib().orc_zx_schoolbook(C.byref(P), C.byref(F), C.byref(G)), "zx_schoolbook")
    return h


def poly_eval_mod(f, length, nlimbs, signed, t, P):
    F = _poly(f, length, nlimbs, signed)
    return int(lib().orc_poly_eval_mod(C.byref(F), t, P))


# ---------------------------------------------------------------- S[y]/(y^{M/2}+1), S = Z/mZ
def sn_cells(vals, M, count=None, stride=None):
    """Elements given as lists of M/2 ints mod m -> uint64 cells (zero-filled to `count`)."""
    H = M // 2
    stride = stride or H
    count = count if count is not None else len(vals)
    x = np.zeros(count * stride, dtype=np.uint64)
    for i, v in enumerate(vals):
        x[i * stride:i * stride + H] = np.asarray(v, dtype=np.uint64)
    return x


def sn_vals(x, M, count, stride=None):
    H = M // 2
    stride = stride or H
    return [[int(w) for w in x[i * stride:i * stride + H]] for i in range(count)]


def _sn2(name, a, b, M, m):
    r = np.zeros(M // 2, dtype=np.uint64)
    _check(getattr(lib(), name)(_p(r), _p(np.asarray(a, dtype=np.uint64)), _p(np.asarray(b, dtype=np.uint64)), M, m), name)
    return [int(w) for w in r]


def sn_add(a, b, M, m):
    return _sn2("orc_sn_add", a, b, M, m)


def sn_sub(a, b, M, m):
    return _sn2("orc_sn_sub", a, b, M, m)


def sn_mul(a, b, M, m):
    return _sn2("orc_sn_mul", a, b, M, m)


def sn_ypow(a, k, M, m):
    r = np.zeros(M // 2, dtype=np.uint64)
    _check(lib().orc_sn_ypow(_p(r), _p(np.asarray(a, dtype=np.uint64)), k, M, m), "orc_sn_ypow")
    return [int(w) for w in r]


def sn_half(a, M, m):
    r = np.zeros(M // 2, dtype=np.uint64)
    _check(lib().orc_sn_half(_p(r), _p(np.asarray(a, dtype=np.uint64)), M, m), "orc_sn_half")
    return [int(w) for w in r]


def sn_dft_brute(x, l, z, n, e, M, m, stride=None):
    stride = stride or M // 2
    out = np.zeros_like(x)
    _check(lib().orc_sn_dft_brute(_p(out), _p(x), stride, l, z, n, e, M, m), "orc_sn_dft_brute")
    return out


def sn_tft(x, l, z, n, e, M, m, stride=None, policy=SPLIT_BALANCED, top_l1=0, seed=0):
    """In place: Algorithm 1 over S[y]/(y^{M/2}+1). Returns the base-case count."""
    cnt = C.c_int64(0)
    _check(lib().orc_sn_tft(_p(x), stride or M // 2, l, z, n, e, M, m, policy, top_l1, seed, C.byref(cnt)),
           "orc_sn_tft")
    return cnt.value


def sn_itft(x, l, z, n, f, e, M, m, stride=None, policy=SPLIT_BALANCED, top_l1=0, seed=0):
    """In place: Algorithm 2 over S[y]/(y^{M/2}+1): L a_0 .. L a_{n-1} (then a-hat_n if f)."""
    cnt = C.c_int64(0)
    _check(lib().orc_sn_itft(_p(x), stride or M // 2, l, z, n, f, e, M, m, policy, top_l1, seed, C.byref(cnt)),
           "orc_sn_itft")
    return cnt.value


# ---------------------------------------------------------------- omega = sqrt2 over Z/(2^N+1)
def sqrt2_dft_brute(x, l, z, n, e, N, stride=None):
    stride = stride or limbs(N)
    out = np.zeros_like(x)
    _check(lib().orc_sqrt2_dft_brute(_p(out), _p(x), stride, l, z, n, e, N), "orc_sqrt2_dft_brute")
    return out


def sqrt2_tft(x, l, z, n, e, N, stride=None, policy=SPLIT_BALANCED, top_l1=0, seed=0):
    cnt = C.c_int64(0)
    _check(lib().orc_sqrt2_tft(_p(x), stride or limbs(N), l, z, n, e, N, policy, top_l1, seed, C.byref(cnt)),
           "orc_sqrt2_tft")
    return cnt.value


def sqrt2_itft(x, l, z, n, f, e, N, stride=None, policy=SPLIT_BALANCED, top_l1=0, seed=0):
    cnt = C.c_int64(0)
    _check(lib().orc_sqrt2_itft(_p(x), stride or limbs(N), l, z, n, f, e, N, policy, top_l1, seed, C.byref(cnt)),
           "orc_sqrt2_itft")
    return cnt.value
