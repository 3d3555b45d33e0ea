"""Thin ctypes binding of ``liblc.so`` (C ABI in ``include/lc.h``).

Argument marshalling only: every step of the connected-components path runs in
the library's CUDA kernels.  Functions carry the C names (``lc_create``,
``lc_run``, ...); :class:`LocalContraction` and :func:`connected_components`
wrap them for torch tensors.  PyTorch supplies device memory and streams.

There is no fallback: if the library has not been built, or CUDA is not
available, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

(LC_OK, LC_ERR_INVALID, LC_ERR_OOM, LC_ERR_CUDA, LC_ERR_NO_CONVERGENCE, LC_ERR_TIMEOUT,
 LC_ERR_INTERNAL, LC_ERR_CANCELLED) = range(8)
LC_VARIANT_FOREST, LC_VARIANT_TWO_HOP, LC_VARIANT_TREE = 0, 1, 2

# every symbol include/lc.h declares (checked by the CPU test suite)
LC_DEDUP_HASH, LC_DEDUP_SORT = 0, 1
EXPORTED = ("lc_create", "lc_configure", "lc_set_merge_to_large", "lc_set_dedup", "lc_set_param", "lc_run", "lc_run_host",
            "lc_last_stats", "lc_last_dedup", "lc_dedup_fallbacks", "lc_profile", "lc_kernel_stats", "lc_destroy", "lc_status_str",
            "lc_rank_probe", "lc_run_static", "lc_batch_create", "lc_batch_run",
            "lc_server_create", "lc_server_submit", "lc_server_wait", "lc_server_result",
            "lc_server_cancel", "lc_server_stats", "lc_server_destroy", "lc_fail_alloc")
LC_STATIC_MAX_N, LC_STATIC_MAX_M = 131072, 524288

_lib = None


class LCError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (status %d)" % (what, lc_status_str(code), code))
        self.code = code


def load(path: str | None = None):
    """Load liblc.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LC_SO
    if not os.path.exists(path):
        raise RuntimeError("liblc.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    u32, u64, i32, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
    pu32, pu64 = ctypes.POINTER(u32), ctypes.POINTER(u64)
    lib.lc_create.argtypes = [u32, p, p, u64, u64, p, ctypes.POINTER(p)]
    lib.lc_configure.argtypes = [p, i32, u64]
    lib.lc_set_merge_to_large.argtypes = [p, p, u32]
    lib.lc_set_merge_to_large.restype = i32
    lib.lc_set_dedup.argtypes = [p, i32]
    lib.lc_set_param.argtypes = [p, ctypes.c_char_p, u64]
    lib.lc_run.argtypes = [p, p, pu32, pu64, pu64, u32]
    lib.lc_run_host.argtypes = [p, p, p, p, pu32, pu64, pu64, u32]
    lib.lc_last_stats.argtypes = [p, pu32, pu64, pu64, u32]
    lib.lc_last_dedup.argtypes = [p, pu32, pu64, pu32, u32]
    lib.lc_last_dedup.restype = i32
    lib.lc_dedup_fallbacks.argtypes = [p, pu64]
    lib.lc_profile.argtypes = [p, i32]
    lib.lc_kernel_stats.argtypes = [p, u32, ctypes.POINTER(ctypes.c_char_p), pu64,
                                    ctypes.POINTER(ctypes.c_double)]
    lib.lc_destroy.argtypes = [p]
    lib.lc_status_str.argtypes = [i32]
    lib.lc_status_str.restype = ctypes.c_char_p
    lib.lc_rank_probe.argtypes = [u64, u32, u32, u32, p, p]
    lib.lc_run_static.argtypes = [u32, p, p, u64, u64, p, p, pu32, pu64, pu64, u32]
    lib.lc_batch_create.argtypes = [u32, p, p, p, p, p, p, ctypes.POINTER(p)]
    lib.lc_batch_run.argtypes = [p, p, p, p, p, u32]
    lib.lc_server_create.argtypes = [u64, u32, ctypes.POINTER(p)]
    lib.lc_server_submit.argtypes = [p, u32, p, p, u64, u64, p, pu64]
    lib.lc_server_wait.argtypes = [p, u64, ctypes.c_double, pu32, ctypes.POINTER(ctypes.c_double)]
    lib.lc_server_result.argtypes = [p, u64, ctypes.c_double, pu32, ctypes.POINTER(ctypes.c_double),
                                     pu64, pu64, u32]
    lib.lc_server_cancel.argtypes = [p, u64]
    lib.lc_fail_alloc.argtypes = [u64]
    lib.lc_server_stats.argtypes = [p, pu64, pu64, pu64]
    lib.lc_server_destroy.argtypes = [p]
    for name in EXPORTED:
        if name != "lc_status_str":
            getattr(lib, name).restype = i32
    _lib = lib
    return lib


def lc_status_str(code: int) -> str:
    return load().lc_status_str(code).decode()


def _check(code: int, what: str) -> None:
    if code != LC_OK:
        raise LCError(code, what)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev_ptr(t, n: int, what: str) -> int:
    if t is None:
        return 0
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if t.element_size() != 4 or not t.is_contiguous() or t.numel() < n:
        raise ValueError("%s must be a contiguous 32-bit tensor with >= %d elements" % (what, n))
    return t.data_ptr()


# ------------------------------------------------------------ C names

def lc_create(n: int, d_src: int, d_dst: int, m: int, seed: int, stream: int) -> int:
    out = ctypes.c_void_p()
    _check(load().lc_create(n, d_src, d_dst, m, seed, stream, ctypes.byref(out)), "lc_create")
    return out.value


def lc_configure(ctx: int, variant: int, finish_edges: int = 0) -> None:
    _check(load().lc_configure(ctx, variant, finish_edges), "lc_configure")


def lc_set_merge_to_large(ctx: int, alpha) -> None:
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.uint32).reshape(-1))
    _check(load().lc_set_merge_to_large(ctx, a.ctypes.data if a.size else None, a.size),
           "lc_set_merge_to_large")


def lc_set_dedup(ctx: int, mode: int) -> None:
    _check(load().lc_set_dedup(ctx, mode), "lc_set_dedup")


def lc_set_param(ctx: int, name: str, value: int) -> None:
    _check(load().lc_set_param(ctx, name.encode(), value), "lc_set_param")


def lc_run(ctx: int, d_labels: int, cap: int = 1024):
    R = ctypes.c_uint32(0)
    n_i = (ctypes.c_uint64 * cap)()
    m_i = (ctypes.c_uint64 * cap)()
    _check(load().lc_run(ctx, d_labels, ctypes.byref(R), n_i, m_i, cap), "lc_run")
    r = R.value
    return r, list(n_i[:r]), list(m_i[:r])


def lc_run_host(ctx: int, h_src: np.ndarray, h_dst: np.ndarray, h_labels: np.ndarray,
                cap: int = 1024):
    R = ctypes.c_uint32(0)
    n_i = (ctypes.c_uint64 * cap)()
    m_i = (ctypes.c_uint64 * cap)()
    _check(load().lc_run_host(ctx, h_src.ctypes.data, h_dst.ctypes.data, h_labels.ctypes.data,
                              ctypes.byref(R), n_i, m_i, cap), "lc_run_host")
    r = R.value
    return r, list(n_i[:r]), list(m_i[:r])


def lc_last_dedup(ctx: int, cap: int = 1024) -> tuple[list[int], list[int]]:
    """(kept_i, passes_i) of each phase's deduplication in the last run."""
    R = ctypes.c_uint32(0)
    kept = (ctypes.c_uint64 * cap)()
    passes = (ctypes.c_uint32 * cap)()
    _check(load().lc_last_dedup(ctx, ctypes.byref(R), kept, passes, cap), "lc_last_dedup")
    r = min(R.value, cap)
    return [int(kept[i]) for i in range(r)], [int(passes[i]) for i in range(r)]


def lc_last_stats(ctx: int, cap: int = 1024) -> tuple[list[int], list[int]]:
    """(m'_i, emitted_i) of the last run."""
    R = ctypes.c_uint32(0)
    mp = (ctypes.c_uint64 * cap)()
    em = (ctypes.c_uint64 * cap)()
    _check(load().lc_last_stats(ctx, ctypes.byref(R), mp, em, cap), "lc_last_stats")
    r = min(R.value, cap)
    return list(mp[:r]), list(em[:r])


def lc_dedup_fallbacks(ctx: int) -> int:
    c = ctypes.c_uint64()
    _check(load().lc_dedup_fallbacks(ctx, ctypes.byref(c)), "lc_dedup_fallbacks")
    return int(c.value)


def lc_profile(ctx: int, on: bool) -> None:
    _check(load().lc_profile(ctx, 1 if on else 0), "lc_profile")


def lc_kernel_stats(ctx: int) -> dict:
    """{kernel name: (launches, device ms)} since the last lc_profile call."""
    out = {}
    k = 0
    lib = load()
    while True:
        name = ctypes.c_char_p()
        launches = ctypes.c_uint64()
        ms = ctypes.c_double()
        if lib.lc_kernel_stats(ctx, k, ctypes.byref(name), ctypes.byref(launches),
                               ctypes.byref(ms)) != LC_OK:
            return out
        out[name.value.decode()] = (int(launches.value), float(ms.value))
        k += 1


def lc_destroy(ctx: int) -> None:
    if ctx:
        _check(load().lc_destroy(ctx), "lc_destroy")


def lc_run_static(n: int, d_src: int, d_dst: int, m: int, seed: int, stream: int,
                  d_labels: int, cap: int = 1024):
    """Allocation-free run for n <= LC_STATIC_MAX_N, m <= LC_STATIC_MAX_M (all
    scratch in the library's static device array; see include/lc.h)."""
    R = ctypes.c_uint32(0)
    n_i = (ctypes.c_uint64 * cap)()
    m_i = (ctypes.c_uint64 * cap)()
    _check(load().lc_run_static(n, d_src, d_dst, m, seed, stream, d_labels, ctypes.byref(R), n_i,
                                m_i, cap), "lc_run_static")
    r = R.value
    return r, list(n_i[:r]), list(m_i[:r])


def lc_batch_create(k: int, h_n: np.ndarray, h_eoff: np.ndarray, d_src: int, d_dst: int,
                    h_seeds: np.ndarray, stream: int) -> int:
    h_n = np.ascontiguousarray(h_n, dtype=np.uint32)
    h_eoff = np.ascontiguousarray(h_eoff, dtype=np.uint64)
    h_seeds = np.ascontiguousarray(h_seeds, dtype=np.uint64)
    out = ctypes.c_void_p()
    _check(load().lc_batch_create(k, h_n.ctypes.data, h_eoff.ctypes.data, d_src, d_dst,
                                  h_seeds.ctypes.data, stream, ctypes.byref(out)),
           "lc_batch_create")
    return out.value


def lc_batch_run(ctx: int, k: int, d_labels: int, cap: int = 256):
    """Returns (rounds[k], n_i[k, cap], m_i[k, cap]) as numpy arrays."""
    rounds = np.zeros(k, dtype=np.uint32)
    n_i = np.zeros((k, cap), dtype=np.uint64)
    m_i = np.zeros((k, cap), dtype=np.uint64)
    _check(load().lc_batch_run(ctx, d_labels, rounds.ctypes.data, n_i.ctypes.data,
                               m_i.ctypes.data, cap), "lc_batch_run")
    return rounds, n_i, m_i


def lc_rank_probe(seed: int, i: int, v0: int, count: int, d_out: int, stream: int) -> None:
    _check(load().lc_rank_probe(seed, i, v0, count, d_out, stream), "lc_rank_probe")


# ------------------------------------------------------------ wrappers

@dataclass
class Result:
    rounds: int
    n_i: list
    m_i: list


def _apply_tuned(ctx: int, n: int, m: int, kind: str = "single") -> dict:
    """Speed parameters measured by the autotuner (tune.py) for the size class
    of this kind nearest to (n, m), set on the context; {} when the table has
    none."""
    from . import tune
    applied = {}
    for name, value in tune.params_for(n, m, kind).items():
        try:
            lc_set_param(ctx, name, int(value))
            applied[name] = int(value)
        except LCError:
            pass  # a value this context cannot take (it changes speed only)
    return applied


class LocalContraction:
    """One graph resident on the device.

    ``src``/``dst`` are CUDA int32/uint32 tensors of length m (kept alive by this
    object; never written).  With ``src is None`` the context owns its input
    buffers and :meth:`run_host` takes host arrays.
    """

    def __init__(self, n: int, src=None, dst=None, m: int | None = None, seed: int = 0,
                 stream=None, variant: int = LC_VARIANT_FOREST, finish_edges: int = 0,
                 dedup: int = LC_DEDUP_HASH, merge_alpha=(), tuned: bool = True):
        if src is None:
            if m is None:
                raise ValueError("m is required when the context owns its inputs")
            self.m = int(m)
        else:
            self.m = int(src.numel())
            if dst is None or dst.numel() != self.m:
                raise ValueError("src and dst must have the same length")
        self.n = int(n)
        self._src, self._dst = src, dst  # keep the caller's buffers alive
        self.stream = stream
        self.ctx = lc_create(self.n, _dev_ptr(src, self.m, "src"), _dev_ptr(dst, self.m, "dst"),
                             self.m, seed, _stream_handle(stream))
        if variant != LC_VARIANT_FOREST or finish_edges:
            lc_configure(self.ctx, variant, finish_edges)
        if dedup != LC_DEDUP_HASH:
            lc_set_dedup(self.ctx, dedup)
        if len(merge_alpha):
            lc_set_merge_to_large(self.ctx, merge_alpha)
        self.params = _apply_tuned(self.ctx, self.n, self.m) if tuned else {}

    def run(self, labels=None, cap: int = 1024):
        import torch
        if labels is None:
            dev = self._src.device if self._src is not None else torch.device("cuda")
            labels = torch.empty(self.n, dtype=torch.int32, device=dev)
        r, n_i, m_i = lc_run(self.ctx, _dev_ptr(labels, self.n, "labels"), cap)
        return labels, Result(r, n_i, m_i)

    def run_host(self, h_src: np.ndarray, h_dst: np.ndarray, h_labels: np.ndarray | None = None,
                 cap: int = 1024):
        for a in (h_src, h_dst):
            if a.dtype != np.uint32 or not a.flags.c_contiguous or a.size != self.m:
                raise ValueError("host edges must be contiguous uint32 arrays of length m")
        if h_labels is None:
            h_labels = np.empty(self.n, dtype=np.uint32)
        r, n_i, m_i = lc_run_host(self.ctx, h_src, h_dst, h_labels, cap)
        return h_labels, Result(r, n_i, m_i)

    def mprime(self) -> list[int]:
        return lc_last_stats(self.ctx)[0]

    def emitted(self) -> list[int]:
        return lc_last_stats(self.ctx)[1]

    def set_param(self, name: str, value: int) -> None:
        lc_set_param(self.ctx, name, value)

    def profile(self, on: bool) -> None:
        lc_profile(self.ctx, on)

    def kernel_stats(self) -> dict:
        return lc_kernel_stats(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            lc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchLocalContraction:
    """k independent graphs run together; results equal k separate runs.

    n: uint32[k] vertex counts; eoff: uint64[k+1] edge offsets into the CUDA
    32-bit tensors src/dst (local ids); seeds: uint64[k] rank seeds.
    """

    def __init__(self, n, eoff, src, dst, seeds, stream=None, variant: int = LC_VARIANT_FOREST,
                 tuned: bool = True):
        self.n = np.ascontiguousarray(n, dtype=np.uint32)
        self.k = int(self.n.shape[0])
        self.eoff = np.ascontiguousarray(eoff, dtype=np.uint64)
        self.voff = np.zeros(self.k + 1, dtype=np.int64)
        np.cumsum(self.n, out=self.voff[1:])
        m = int(self.eoff[-1])
        self._src, self._dst = src, dst
        self.ctx = lc_batch_create(self.k, self.n, self.eoff, _dev_ptr(src, m, "src") if m else 0,
                                   _dev_ptr(dst, m, "dst") if m else 0, seeds,
                                   _stream_handle(stream))
        if variant != LC_VARIANT_FOREST:
            lc_configure(self.ctx, variant, 0)
        self.params = _apply_tuned(self.ctx, int(self.voff[-1]), m, "batch") if tuned else {}

    def run(self, labels=None, cap: int = 256):
        import torch
        total = int(self.voff[-1])
        if labels is None:
            dev = self._src.device if self._src is not None else torch.device("cuda")
            labels = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        rounds, n_i, m_i = lc_batch_run(self.ctx, self.k, _dev_ptr(labels, total, "labels"), cap)
        return labels, rounds, n_i, m_i

    def set_param(self, name: str, value: int) -> None:
        lc_set_param(self.ctx, name, value)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            lc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (see lc_server_* in include/lc.h).

    submit() takes host uint32 arrays (kept alive until wait() returns; pinned
    memory lets the copies overlap) and returns a job id; wait(id) returns
    (labels, rounds, latency_s)."""

    def __init__(self, budget_bytes: int = 0, slots: int = 32):
        out = ctypes.c_void_p()
        _check(load().lc_server_create(budget_bytes, slots, ctypes.byref(out)), "lc_server_create")
        self.srv = out.value
        self._held = {}

    def submit(self, n: int, h_src: np.ndarray, h_dst: np.ndarray, seed: int = 0,
               h_labels: np.ndarray | None = None) -> int:
        m = int(h_src.size)
        for a in (h_src, h_dst):
            if a.dtype != np.uint32 or not a.flags.c_contiguous or a.size != m:
                raise ValueError("host edges must be contiguous uint32 arrays of equal length")
        if h_labels is None:
            h_labels = np.empty(max(n, 1), dtype=np.uint32)
        job = ctypes.c_uint64()
        _check(load().lc_server_submit(self.srv, n, h_src.ctypes.data if m else 0,
                                       h_dst.ctypes.data if m else 0, m, seed,
                                       h_labels.ctypes.data, ctypes.byref(job)), "lc_server_submit")
        self._held[job.value] = (h_src, h_dst, h_labels, n)
        return job.value

    def wait(self, job: int, timeout_s: float = 0.0):
        R = ctypes.c_uint32()
        lat = ctypes.c_double()
        st = load().lc_server_wait(self.srv, job, timeout_s, ctypes.byref(R), ctypes.byref(lat))
        if st == LC_ERR_TIMEOUT:
            raise LCError(st, "lc_server_wait")  # still pending: may be waited on again
        h_src, h_dst, h_labels, n = self._held.pop(job)
        _check(st, "lc_server_wait")
        return h_labels[:n], int(R.value), float(lat.value)

    def result(self, job: int, timeout_s: float = 0.0, cap: int = 1024):
        """wait() plus the job's per-phase sizes: (labels, Result, latency_s)."""
        R = ctypes.c_uint32()
        lat = ctypes.c_double()
        n_i = (ctypes.c_uint64 * cap)()
        m_i = (ctypes.c_uint64 * cap)()
        st = load().lc_server_result(self.srv, job, timeout_s, ctypes.byref(R), ctypes.byref(lat),
                                     n_i, m_i, cap)
        if st == LC_ERR_TIMEOUT:
            raise LCError(st, "lc_server_result")
        h_src, h_dst, h_labels, n = self._held.pop(job)
        _check(st, "lc_server_result")
        r = int(R.value)
        return h_labels[:n], Result(r, list(n_i[:r]), list(m_i[:r])), float(lat.value)

    def cancel(self, job: int) -> bool:
        """True if the job will end cancelled; False if it is unknown or too far along."""
        return load().lc_server_cancel(self.srv, job) == LC_OK

    def stats(self) -> dict:
        c, p, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().lc_server_stats(self.srv, ctypes.byref(c), ctypes.byref(p), ctypes.byref(b)),
               "lc_server_stats")
        return {"completed": c.value, "peak_active": p.value, "bytes_in_use": b.value}

    def close(self) -> None:
        if getattr(self, "srv", None):
            load().lc_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fail_alloc(k: int) -> None:
    """Test hook: the k-th library allocation from now fails (0: off)."""
    _check(load().lc_fail_alloc(k), "lc_fail_alloc")


def connected_components(n: int, src, dst, seed: int = 0, stream=None):
    """Labels (smallest vertex id per component) of the graph (src[j], dst[j]),
    plus the phase count and per-phase sizes.  src/dst: CUDA 32-bit tensors."""
    ctx = LocalContraction(n, src, dst, seed=seed, stream=stream)
    try:
        return ctx.run()
    finally:
        ctx.close()


def rank_probe(seed: int, i: int, v0: int, count: int, stream=None):
    import torch
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    lc_rank_probe(seed, i, v0, count, out.data_ptr() if count else 0, _stream_handle(stream))
    return out
