"""Python binding of libtftgpu: truncated Fourier transforms over Z/(2^N+1) and
Schoenhage-Strassen products in Z[x] on a GB300 GPU.

Method: D. Harvey, "A cache-friendly truncated FFT" (arXiv 0810.3203), Algorithms 1 and 2.

Every function here only marshals arguments for the C ABI declared in include/tftgpu.h:
device tensors become raw pointers, streams become cudaStream_t handles. All arithmetic runs
in the CUDA kernels of the library. If the library is missing or fails to load, every call
raises; there is no CPU fallback.

Tensors: ring buffers are torch int64 tensors on a CUDA device (the bit patterns are the
uint64 limbs), shape (cells * stride_limbs,) or (cells, stride_limbs), contiguous.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

ZX_OK, ZX_EINVAL, ZX_ENOMEM, ZX_ECUDA, ZX_ETIMEOUT, ZX_EBUFSIZE, ZX_EUNSUPPORTED = range(7)
ZX_HOST, ZX_DEVICE = 0, 1

# every entry point the header declares (checked by tests/test_abi.py)
EXPORTS = ("tft", "tft_ex", "itft", "itft_ex", "zx_plan", "zx_mul", "zx_mul_batch",
           "zx_transform_plan", "zx_mul_noalloc", "zx_job_program", "zx_strerror", "zx_last_error",
           "zx_version", "zx_server_create", "zx_server_submit", "zx_server_poll", "zx_server_drain",
           "zx_server_stats", "zx_server_destroy", "zx_tune", "zx_config_get", "zx_config_set", "sn_tft", "sn_itft", "tft_sqrt2", "itft_sqrt2",
           "zx_pointwise", "zx_pointwise_plan", "zx_wait_status", "zx_wait_probe", "zx_transform_jobs",
           "zx_transform_schedule")

_lib = None


class TftError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        detail = _lib.zx_last_error().decode() if _lib is not None else ""
        name = _lib.zx_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {name} ({detail})")


class ZxPoly(C.Structure):
    _fields_ = [("len", C.c_int64), ("limbs", C.c_int64), ("is_signed", C.c_int32),
                ("where", C.c_int32), ("bits", C.c_int64), ("data", C.c_void_p)]


class ZxPlanInfo(C.Structure):
    _fields_ = [("l", C.c_int32), ("K", C.c_int32), ("N", C.c_int64), ("n", C.c_int64),
                ("stride_limbs", C.c_int64), ("limbs_h", C.c_int64), ("scratch_bytes", C.c_int64),
                ("tft_passes", C.c_int32), ("itft_passes", C.c_int32), ("n_fft", C.c_int64),
                ("sqrt2", C.c_int32), ("pad", C.c_int32)]


class ZxTuneInfo(C.Structure):
    _fields_ = [("ls_max", C.c_int32), ("ls_c", C.c_int32), ("max_warps", C.c_int32), ("split", C.c_int32),
                ("candidates", C.c_int32), ("best_ms", C.c_float), ("default_ms", C.c_float), ("fused", C.c_int32),
                ("max_cluster_log2", C.c_int32), ("tma", C.c_int32)]


class ZxServerInfo(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("pending", C.c_int64),
                ("waves", C.c_int64), ("max_wave_products", C.c_int64), ("slots", C.c_int32),
                ("max_waves_in_flight", C.c_int32), ("arena_bytes", C.c_int64),
                ("arena_peak_bytes", C.c_int64), ("time_scale", C.c_double)]


class ZxPointwiseInfo(C.Structure):
    _fields_ = [("method", C.c_int32), ("k", C.c_int32), ("N_inner", C.c_int64), ("stride_inner", C.c_int64),
                ("cost_recursive", C.c_double), ("cost_schoolbook", C.c_double)]


class ZxTransformInfo(C.Structure):
    _fields_ = [("passes", C.c_int32), ("launches", C.c_int32), ("jobs", C.c_int64),
                ("onchip_l", C.c_int32), ("K", C.c_int32), ("cluster_l", C.c_int32), ("pad", C.c_int32)]


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libtftgpu.so (building it first when asked). Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libtftgpu.so is not built ({path})")
        _build.build()
    L = C.CDLL(path)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    L.tft.argtypes = [vp, i32, i64, i64, vp]
    L.tft_ex.argtypes = [vp, i32, i64, i64, i64, i64, i64, vp]
    L.itft.argtypes = [vp, i32, i64, i64, vp]
    L.itft_ex.argtypes = [vp, i32, i64, i64, i32, i64, i64, i64, i32, vp]
    L.zx_plan.argtypes = [i64, i64, i64, i64, i32, C.POINTER(ZxPlanInfo)]
    L.zx_mul.argtypes = [C.POINTER(ZxPoly), C.POINTER(ZxPoly), C.POINTER(ZxPoly), vp]
    L.zx_mul_batch.argtypes = [C.POINTER(ZxPoly), C.POINTER(ZxPoly), C.POINTER(ZxPoly), i32, vp]
    L.zx_transform_plan.argtypes = [i32, i32, i64, i64, i32, i64, C.POINTER(ZxTransformInfo)]
    L.zx_mul_noalloc.argtypes = [C.POINTER(ZxPoly), C.POINTER(ZxPoly), C.POINTER(ZxPoly), vp]
    L.zx_job_program.argtypes = [i32, i32, i32, i64, i64, i32, i64, i32, C.POINTER(C.c_uint32), i64,
                                 C.POINTER(C.c_int64)]
    L.zx_server_create.argtypes = [i64, i32, C.POINTER(vp)]
    L.zx_server_submit.argtypes = [vp, C.POINTER(ZxPoly), C.POINTER(ZxPoly), C.POINTER(ZxPoly),
                                   C.POINTER(C.c_int64)]
    L.zx_server_poll.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double), i32,
                                 C.POINTER(C.c_int)]
    L.zx_server_drain.argtypes = [vp, C.c_double]
    L.zx_server_stats.argtypes = [vp, C.POINTER(ZxServerInfo)]
    L.zx_server_destroy.argtypes = [vp]
    L.zx_tune.argtypes = [vp, i32, i64, i64, i64, i32, vp, C.POINTER(ZxTuneInfo)]
    L.zx_config_get.argtypes = [i64, C.POINTER(ZxTuneInfo)]
    L.zx_config_set.argtypes = [i64, C.POINTER(ZxTuneInfo)]
    L.zx_transform_schedule.argtypes = [i32, i32, i64, i64, i32, i64, i64, i32, i32, i32, C.POINTER(C.c_int64), i64,
                                        C.POINTER(C.c_int64)]
    L.tft_sqrt2.argtypes = [vp, i32, i64, i64, i64, i64, i64, vp]
    L.itft_sqrt2.argtypes = [vp, i32, i64, i64, i32, i64, i64, i64, i32, vp]
    L.sn_tft.argtypes = [vp, i32, i64, i64, i64, C.c_uint64, i64, i64, vp]
    L.sn_itft.argtypes = [vp, i32, i64, i64, i32, i64, C.c_uint64, i64, i64, i32, vp]
    L.zx_pointwise.argtypes = [vp, vp, i64, i64, i64, i32, vp]
    L.zx_pointwise_plan.argtypes = [i64, i32, C.POINTER(ZxPointwiseInfo)]
    L.zx_transform_jobs.argtypes = [i32, i32, i64, i64, i32, i64, i64, i32, i32, C.POINTER(C.c_int64), i64,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_uint32), i64, C.POINTER(C.c_int64)]
    L.zx_wait_status.argtypes = [vp]
    L.zx_wait_probe.argtypes = [i64, vp]
    L.zx_strerror.argtypes = [i32]
    L.zx_strerror.restype = C.c_char_p
    L.zx_last_error.argtypes = []
    L.zx_last_error.restype = C.c_char_p
    L.zx_version.restype = C.c_char_p
    for name in ("tft", "tft_ex", "itft", "itft_ex", "zx_plan", "zx_mul", "zx_mul_batch",
                 "zx_transform_plan", "zx_mul_noalloc", "zx_job_program", "zx_server_create",
                 "zx_server_submit", "zx_server_poll", "zx_server_drain", "zx_server_stats",
                 "zx_server_destroy", "zx_tune", "zx_config_get", "zx_config_set", "sn_tft", "sn_itft", "tft_sqrt2", "itft_sqrt2",
                 "zx_pointwise", "zx_pointwise_plan"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc, where):
    if rc != ZX_OK:
        raise TftError(rc, where)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dev_ptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)) or not t.is_contiguous():
        raise TypeError("expected a contiguous 64-bit integer tensor")
    return C.c_void_p(t.data_ptr())


def limbs(N):
    return N // 64 + 1


def tft(x, l, n, N, stream=None):
    """In-place TFT with z = n, zeta = 1, stride N/64 + 1 (Algorithm 1)."""
    _check(load().tft(_dev_ptr(x), l, n, N, _stream(stream)), "tft")


def tft_ex(x, l, z, n, N, e=0, stride_limbs=None, stream=None):
    """In-place TFT(2^l, 2^e, z, n) on cells of stride_limbs limbs (Algorithm 1)."""
    s = stride_limbs or limbs(N)
    _check(load().tft_ex(_dev_ptr(x), l, z, n, N, e, s, _stream(stream)), "tft_ex")


def itft(x, l, n, N, stream=None):
    """In-place inverse of tft: returns a_i (scaled by 1/L) (Algorithm 2)."""
    _check(load().itft(_dev_ptr(x), l, n, N, _stream(stream)), "itft")


def itft_ex(x, l, z, n, f, N, e=0, stride_limbs=None, scale=0, stream=None):
    """In-place ITFT(2^l, 2^e, z, n, f) (Algorithm 2); scale=1 divides the L a_i by L."""
    s = stride_limbs or limbs(N)
    _check(load().itft_ex(_dev_ptr(x), l, z, n, f, N, e, s, scale, _stream(stream)), "itft_ex")


def zx_plan(len_f, bits_f, len_g, bits_g, is_signed=False):
    info = ZxPlanInfo()
    _check(load().zx_plan(len_f, bits_f, len_g, bits_g, 1 if is_signed else 0, C.byref(info)), "zx_plan")
    return {k: getattr(info, k) for k, _ in ZxPlanInfo._fields_}


def transform_plan(kind, l, z, n, N, f=0):
    """Launch plan of a TFT (kind 0) or ITFT (kind 1): passes, launches, jobs, onchip_l, K."""
    info = ZxTransformInfo()
    _check(load().zx_transform_plan(kind, l, z, n, f, N, C.byref(info)), "zx_transform_plan")
    return {k: getattr(info, k) for k, _ in ZxTransformInfo._fields_}


def pointwise_plan(N, method=0):
    """Pointwise method for ring N (zx_pointwise_plan): method 1 schoolbook, 2 recursive, with
    the inner ring of the recursion and both cost estimates."""
    info = ZxPointwiseInfo()
    _check(load().zx_pointwise_plan(N, method, C.byref(info)), "zx_pointwise_plan")
    return {k: getattr(info, k) for k, _ in ZxPointwiseInfo._fields_}


def pointwise(a, b, n, N, stride_limbs, method=0, stream=None):
    """a_i <- a_i b_i mod 2^N + 1 for i < n (zx_pointwise) on device tensors of canonical cells."""
    _check(load().zx_pointwise(_dev_ptr(a), _dev_ptr(b), n, N, stride_limbs, method, _stream(stream)), "zx_pointwise")


def job_program(kind, ls, lc, z, n, N, f=0, mode=0):
    """Job image of one on-chip sub-transform (see zx_job_program in include/tftgpu.h), as a
    numpy uint32 array. mode: 0 omega = 2, 1 omega = y over S[y]/(y^N+1), 2 omega = sqrt2."""
    size = C.c_int64(0)
    load().zx_job_program(kind, ls, lc, z, n, f, N, mode, None, 0, C.byref(size))
    buf = np.zeros(max(1, size.value), np.uint32)
    _check(load().zx_job_program(kind, ls, lc, z, n, f, N, mode, buf.ctypes.data_as(C.POINTER(C.c_uint32)),
                                 buf.size, C.byref(size)), "zx_job_program")
    return buf[:size.value]


def _poly(data, length, nlimbs, signed, bits):
    import torch
    if isinstance(data, torch.Tensor):
        ptr, where = _dev_ptr(data).value, ZX_DEVICE
    else:
        assert isinstance(data, np.ndarray) and data.dtype == np.uint64 and data.flags.c_contiguous
        ptr, where = data.ctypes.data, ZX_HOST
    return ZxPoly(length, nlimbs, 1 if signed else 0, where, bits, ptr)


def zx_mul(f, len_f, limbs_f, g, len_g, limbs_g, h, limbs_h, signed=False, bits_f=0, bits_g=0,
           stream=None):
    """h = f * g in Z[x]. f, g, h are CUDA int64 tensors or numpy uint64 arrays (host)."""
    F = _poly(f, len_f, limbs_f, signed, bits_f)
    G = _poly(g, len_g, limbs_g, signed, bits_g)
    H = _poly(h, len_f + len_g - 1, limbs_h, signed, 0)
    _check(load().zx_mul(C.byref(F), C.byref(G), C.byref(H), _stream(stream)), "zx_mul")


def zx_mul_noalloc(f, len_f, limbs_f, g, len_g, limbs_g, h, limbs_h, signed=False, bits_f=0,
                   bits_g=0, stream=None):
    """zx_mul for callers that cannot allocate: every operand a CUDA tensor; the library's
    fixed 20 MiB device array holds the ring buffers (see include/tftgpu.h)."""
    F = _poly(f, len_f, limbs_f, signed, bits_f)
    G = _poly(g, len_g, limbs_g, signed, bits_g)
    H = _poly(h, len_f + len_g - 1, limbs_h, signed, 0)
    _check(load().zx_mul_noalloc(C.byref(F), C.byref(G), C.byref(H), _stream(stream)), "zx_mul_noalloc")


def zx_mul_batch(items, stream=None):
    """items: list of (f, len_f, limbs_f, g, len_g, limbs_g, h, limbs_h, signed, bits_f, bits_g)
    with device tensors."""
    n = len(items)
    Fs, Gs, Hs = (ZxPoly * n)(), (ZxPoly * n)(), (ZxPoly * n)()
    for i, (f, lf, mf, g, lg, mg, h, mh, sg, bf, bg) in enumerate(items):
        Fs[i] = _poly(f, lf, mf, sg, bf)
        Gs[i] = _poly(g, lg, mg, sg, bg)
        Hs[i] = _poly(h, lf + lg - 1, mh, sg, 0)
    _check(load().zx_mul_batch(Fs, Gs, Hs, n, _stream(stream)), "zx_mul_batch")


def tune(x, l, n, N, stride_limbs=None, reps=2, stream=None):
    """Time the launch configurations of ring N on TFT + ITFT round trips of length n over the
    device buffer x (restored afterwards) and keep the fastest for later plans (zx_tune)."""
    info = ZxTuneInfo()
    s = stride_limbs or limbs(N)
    _check(load().zx_tune(_dev_ptr(x), l, n, N, s, reps, _stream(stream), C.byref(info)), "zx_tune")
    return {k: getattr(info, k) for k, _ in ZxTuneInfo._fields_}


def tft_sqrt2(x, l, z, n, N, e=0, stride_limbs=None, stream=None):
    """In-place TFT with omega = sqrt2 (L | 4N); e is the exponent of zeta in units of sqrt2."""
    s = stride_limbs or limbs(N)
    _check(load().tft_sqrt2(_dev_ptr(x), l, z, n, N, e, s, _stream(stream)), "tft_sqrt2")


def itft_sqrt2(x, l, z, n, f, N, e=0, stride_limbs=None, scale=0, stream=None):
    """In-place ITFT with omega = sqrt2 (L | 4N); scale=1 divides the L a_i by L."""
    s = stride_limbs or limbs(N)
    _check(load().itft_sqrt2(_dev_ptr(x), l, z, n, f, N, e, s, scale, _stream(stream)), "itft_sqrt2")


def sn_tft(x, l, z, n, M, m, e=0, stride=None, stream=None):
    """In-place TFT over S[y]/(y^(M/2)+1), S = Z/mZ (Algorithm 1 with omega = y, zeta = y^e)."""
    _check(load().sn_tft(_dev_ptr(x), l, z, n, M, m, e, stride or M // 2, _stream(stream)), "sn_tft")


def sn_itft(x, l, z, n, f, M, m, e=0, stride=None, scale=0, stream=None):
    """In-place ITFT over S[y]/(y^(M/2)+1) (Algorithm 2); scale=1 multiplies by L^-1 mod m."""
    _check(load().sn_itft(_dev_ptr(x), l, z, n, f, M, m, e, stride or M // 2, scale, _stream(stream)), "sn_itft")


def config_get(N):
    """Launch configuration used for ring N: ls_max, ls_c, max_warps, split, fused, max_cluster_log2,
    tma."""
    info = ZxTuneInfo()
    _check(load().zx_config_get(N, C.byref(info)), "zx_config_get")
    return {k: getattr(info, k) for k in ("ls_max", "ls_c", "max_warps", "split", "fused", "max_cluster_log2", "tma")}


def config_set(N, cfg=None):
    """Pin the launch configuration of ring N (a dict like config_get's; fused, max_cluster_log2
    and tma keep their current values when left out), or restore the default."""
    if cfg is None:
        _check(load().zx_config_set(N, None), "zx_config_set")
        return
    cur = config_get(N)  # fields the dict leaves out keep their current values
    info = ZxTuneInfo(cfg["ls_max"], cfg["ls_c"], cfg["max_warps"], cfg["split"], 0, 0.0, 0.0,
                      cfg.get("fused", cur["fused"]), cfg.get("max_cluster_log2", cur["max_cluster_log2"]),
                      cfg.get("tma", cur["tma"]))
    _check(load().zx_config_set(N, C.byref(info)), "zx_config_set")


class Server:
    """Continuous-batching request loop on the current device (zx_server_* in the C ABI).

    submit() queues one product of device tensors and returns its id at once; poll() returns
    finished requests as (id, status, latency_seconds); drain() waits until nothing is queued
    or running. The tensors of a request must stay alive until poll() has returned it."""

    def __init__(self, arena_bytes=0, slots=3):
        self._h = C.c_void_p()
        _check(load().zx_server_create(arena_bytes, slots, C.byref(self._h)), "zx_server_create")
        self._keep = {}

    def submit(self, f, len_f, limbs_f, g, len_g, limbs_g, h, limbs_h, signed=False, bits_f=0, bits_g=0):
        F = _poly(f, len_f, limbs_f, signed, bits_f)
        G = _poly(g, len_g, limbs_g, signed, bits_g)
        H = _poly(h, len_f + len_g - 1, limbs_h, signed, 0)
        rid = C.c_int64()
        _check(load().zx_server_submit(self._h, C.byref(F), C.byref(G), C.byref(H), C.byref(rid)),
               "zx_server_submit")
        self._keep[rid.value] = (f, g, h)
        return rid.value

    def poll(self, max_items=1024):
        ids = (C.c_int64 * max_items)()
        st = (C.c_int32 * max_items)()
        lat = (C.c_double * max_items)()
        n = C.c_int()
        _check(load().zx_server_poll(self._h, ids, st, lat, max_items, C.byref(n)), "zx_server_poll")
        out = [(ids[k], st[k], lat[k]) for k in range(n.value)]
        for rid, _, _ in out:
            self._keep.pop(rid, None)
        return out

    def drain(self, timeout_s=-1.0):
        _check(load().zx_server_drain(self._h, timeout_s), "zx_server_drain")

    def stats(self):
        info = ZxServerInfo()
        _check(load().zx_server_stats(self._h, C.byref(info)), "zx_server_stats")
        return {k: getattr(info, k) for k, _ in ZxServerInfo._fields_}

    def close(self):
        if self._h:
            load().zx_server_destroy(self._h)
            self._h = C.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def transform_jobs(kind, l, z, n, N, f=0, e=0, scale=0, mode=0):
    """The launches of one transform's plan (see zx_transform_jobs in include/tftgpu.h): a dict
    with 'passes' and 'launches', each launch a dict of ls, lc, warps, program_words and its
    'jobs' (dicts of the 9 descriptor fields), and 'images' (numpy uint32 job images)."""
    nj, ni = C.c_int64(0), C.c_int64(0)
    load().zx_transform_jobs(kind, l, z, n, f, N, e, scale, mode, None, 0, C.byref(nj), None, 0, C.byref(ni))
    J = np.zeros(max(1, nj.value), np.int64)
    I = np.zeros(max(1, ni.value), np.uint32)
    _check(load().zx_transform_jobs(kind, l, z, n, f, N, e, scale, mode, J.ctypes.data_as(C.POINTER(C.c_int64)),
                                    J.size, C.byref(nj), I.ctypes.data_as(C.POINTER(C.c_uint32)), I.size,
                                    C.byref(ni)), "zx_transform_jobs")
    passes, nlaunch, _, nimg = (int(v) for v in J[:4])
    fields = ("cell0", "mstride", "e", "nload", "nstore", "nscale", "escale", "pad", "image")
    launches, k = [], 4
    for _ in range(nlaunch):
        ls, lc, warps, pw, count = (int(v) for v in J[k:k + 5])
        k += 5
        jobs = [dict(zip(fields, (int(v) for v in J[k + 9 * t:k + 9 * t + 9]))) for t in range(count)]
        k += 9 * count
        launches.append(dict(ls=ls, lc=lc, warps=warps, program_words=pw, jobs=jobs))
    off = [int(v) for v in I[:nimg + 1]]
    images = [I[nimg + 1 + off[t]:nimg + 1 + off[t + 1]].copy() for t in range(nimg)]
    return dict(passes=passes, launches=launches, images=images)


def transform_schedule(kind, l, z, n, N, f=0, e=0, scale=0, mode=0, slots=0):
    """The persistent form of a transform's plan (zx_transform_schedule in include/tftgpu.h): a
    list of (job, deps) in claim order, job indexing transform_jobs' jobs launch by launch and
    deps the claim positions it waits for; empty when the plan runs as one launch per pass."""
    w = C.c_int64(0)
    load().zx_transform_schedule(kind, l, z, n, f, N, e, scale, mode, slots, None, 0, C.byref(w))
    W = np.zeros(max(1, w.value), np.int64)
    _check(load().zx_transform_schedule(kind, l, z, n, f, N, e, scale, mode, slots,
                                        W.ctypes.data_as(C.POINTER(C.c_int64)), W.size, C.byref(w)),
           "zx_transform_schedule")
    out, k = [], 1
    for _ in range(int(W[0])):
        job, nd = int(W[k]), int(W[k + 1])
        out.append((job, [int(v) for v in W[k + 2:k + 2 + nd]]))
        k += 2 + nd
    return out


def wait_status(stream=None):
    """Synchronise the stream, then read and clear the device's bounded-wait status: the
    status code, ZX_OK or ZX_ETIMEOUT (a transform kernel's bulk-load wait gave up)."""
    return load().zx_wait_status(_stream(stream))


def wait_probe(limit_us, stream=None):
    """Enqueue one warp that waits limit_us microseconds on a barrier nothing completes and
    reports it as a transform's wait that gave up (the error path, taken without a fault)."""
    _check(load().zx_wait_probe(limit_us, _stream(stream)), "zx_wait_probe")


def version():
    return load().zx_version().decode()
