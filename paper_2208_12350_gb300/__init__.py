"""Python binding of libswgb (batched Smith-Waterman/Gotoh on GB300).

Argument marshalling only: every step of an alignment runs in the CUDA
library behind the C ABI declared in include/swgb.h.  PyTorch supplies
device memory and streams.  There is no CPU fallback: if libswgb.so is
missing or cannot load, load() raises.

Functions keep the C names (sw_plan_create, sw_plan_execute, sw_align_batch,
...) and take torch tensors, numpy arrays or raw integer addresses.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswgb.so")

SW_OK, SW_EINVAL, SW_ERANGE, SW_ENOMEM, SW_ECUDA, SW_ETIMEOUT, SW_EBUDGET = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "SW_OK", -1: "SW_EINVAL", -2: "SW_ERANGE", -3: "SW_ENOMEM", -4: "SW_ECUDA",
                -5: "SW_ETIMEOUT", -6: "SW_EBUDGET"}
SW_MODE_AUTO, SW_MODE_PLAIN, SW_MODE_BATCHED = 0, 1, 2
SW_PLAN_GRAPH = 1
SW_PLAN_ENDS_ONLY = 2
SW_PLAN_PACKED_2BIT = 4
SW_PLAN_NO_S16X2 = 8
SW_PLAN_PAIR_SCRATCH = 16
SW_PLAN_GUARDS = 32
SW_PLAN_ROWS32 = 64
SW_ARITH_S32, SW_ARITH_S16X2 = 0, 1
SW_MAX_LEN = 65535

# Every function the library exports, with its ctypes signature.
_P = ctypes.c_void_p
_I32, _I64, _U32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
_PP = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "sw_last_error": ([], ctypes.c_char_p),
    "sw_ctx_create": ([_I32, _PP], ctypes.c_int),
    "sw_ctx_destroy": ([_P], ctypes.c_int),
    "sw_ctx_sm_count": ([_P, ctypes.POINTER(_I32)], ctypes.c_int),
    "sw_ctx_status": ([_P, ctypes.POINTER(_I32)], ctypes.c_int),
    "sw_default_ctx": ([_I32, _PP], ctypes.c_int),
    "sw_ctx_set_guards": ([_P, _I32], ctypes.c_int),
    "sw_ctx_host_in_place": ([_P, ctypes.POINTER(_I32)], ctypes.c_int),
    "sw_ctx_set_host_in_place": ([_P, _I32], ctypes.c_int),
    "sw_ctx_set_tuning": ([_P, _I32, ctypes.c_double], ctypes.c_int),
    "sw_ctx_set_form": ([_P, _I32, _I32, _I32], ctypes.c_int),
    "sw_ctx_get_tuning": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32)],
                          ctypes.c_int),
    "sw_plan_rows": ([_P, ctypes.POINTER(_I32)], ctypes.c_int),
    "sw_plan_create": ([_P, _P, _P, _I32, _P, _I32, _I32, _I32, _I32, _U32, _PP], ctypes.c_int),
    "sw_plan_execute": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "sw_plan_execute_host": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "sw_plan_info": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                      ctypes.POINTER(_I64)], ctypes.c_int),
    "sw_plan_arith": ([_P, ctypes.POINTER(_I32)], ctypes.c_int),
    "sw_plan_preview": ([_P, _P, _I32, _P, _I32, _I32, _I32, _I32, _U32, _I32, _I32,
                         ctypes.c_double, ctypes.POINTER(_I32), _P, _P], ctypes.c_int),
    "sw_plan_destroy": ([_P], ctypes.c_int),
    "sw_plan_poison_guard": ([_P, _I32], ctypes.c_int),
    "sw_align_batch": ([_P, _P, _P, _P, _I32, _P, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P],
                       ctypes.c_int),
    "sw_align_batch_ex": ([_P, _P, _P, _P, _P, _I32, _P, _I32, _I32, _I32, _I32, _P, _P, _P, _P,
                           _P, _P], ctypes.c_int),
    "sw_check_residues": ([_P, _I64, _I32, _P, _P], ctypes.c_int),
    "sw_static_status": ([ctypes.POINTER(_I32), _P], ctypes.c_int),
    "sw_align_batch_static": ([_P, _P, _P, _P, _I32, _P, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P],
                              ctypes.c_int),
    "sw_autotune": ([_P, _P, _P, _I32, _P, _I32, _I32, _I32, _P, _P, _P, ctypes.c_char_p, _P,
                     ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double),
                     ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "sw_autotune_ex": ([_P, _P, _P, _I32, _P, _I32, _I32, _I32, _P, _P, _P, _U32, ctypes.c_char_p,
                        _P, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "sw_server_create": ([_P, _I64, _I32, _I64, _PP], ctypes.c_int),
    "sw_server_submit": ([_P, _P, _P, _P, _P, _I32, _P, _I32, _I32, _I32, _I32,
                          ctypes.POINTER(_I64)], ctypes.c_int),
    "sw_server_add_pool": ([_P, _P, _P, _P, _P, _I32, _P, _I32, _I32, _I32,
                            ctypes.POINTER(_I32)], ctypes.c_int),
    "sw_server_submit_pool": ([_P, _I32, _I64, _I32, _I32, ctypes.POINTER(_I64)], ctypes.c_int),
    "sw_server_poll": ([_P, _I64, ctypes.POINTER(_I32)], ctypes.c_int),
    "sw_server_wait": ([_P, _I64, _I32, _P, ctypes.POINTER(_I64)], ctypes.c_int),
    "sw_server_stats": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                         ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
    "sw_server_launches": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                            ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "sw_server_destroy": ([_P], ctypes.c_int),
    "sw_pack_2bit": ([_P, _I64, _P], ctypes.c_int),
    "sw_unpack_2bit": ([_P, _I64, _P, _P], ctypes.c_int),
    "sw_cigar_capacity": ([_P, _I32, _P], ctypes.c_int),
    "sw_traceback": ([_P, _P, _P, _P, _P, _I32, _P, _I32, _I32, _I32, _P, _P, _P, _P, _P],
                     ctypes.c_int),
    "sw_cigar_capacity_device": ([_P, _I32, _P, _P], ctypes.c_int),
    "sw_traceback_device": ([_P, _P, _P, _P, _P, _I32, _P, _I32, _I32, _I32, _P, _P, _P, _P, _P],
                            ctypes.c_int),
    "sw_microbench_int": ([_I32, _I32, _I64, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
}

_lib = None


class SwError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def load():
    """Load libswgb.so (built by build.py / __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libswgb.so not built at {LIB_PATH}; run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _check(rc: int, fn: str) -> None:
    if rc != SW_OK:
        raise SwError(fn, rc, load().sw_last_error().decode(errors="replace"))


def _addr(x) -> int | None:
    """Address of a torch tensor / numpy array / int (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _host_i64(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a), dtype=np.int64)
    return a


def _host_i8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int8)


# ----------------------------------------------------------------- context

def sw_ctx_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().sw_ctx_create(device, ctypes.byref(h)), "sw_ctx_create")
    return h.value


def sw_ctx_destroy(ctx: int) -> None:
    _check(load().sw_ctx_destroy(ctx), "sw_ctx_destroy")


def sw_ctx_sm_count(ctx: int) -> int:
    v = _I32()
    _check(load().sw_ctx_sm_count(ctx, ctypes.byref(v)), "sw_ctx_sm_count")
    return v.value


def sw_ctx_status(ctx: int) -> int:
    v = _I32()
    _check(load().sw_ctx_status(ctx, ctypes.byref(v)), "sw_ctx_status")
    return v.value


def sw_default_ctx(device: int = 0) -> int:
    """The library-owned context sw_align_batch uses on `device` (never destroy it)."""
    h = ctypes.c_void_p()
    _check(load().sw_default_ctx(device, ctypes.byref(h)), "sw_default_ctx")
    return h.value


STATUS_REVERSE_MISMATCH = 1
STATUS_BAD_OFFSETS = 2
STATUS_GUARD = 4


def sw_ctx_set_guards(ctx: int, on: bool = True) -> None:
    """Guard regions around the one-shot calls' workspace parts (test aid)."""
    _check(load().sw_ctx_set_guards(ctx, 1 if on else 0), "sw_ctx_set_guards")


def sw_ctx_set_tuning(ctx: int, narrow_log2g: int = -1, cap_fraction: float = 0.5) -> None:
    _check(load().sw_ctx_set_tuning(ctx, narrow_log2g, cap_fraction), "sw_ctx_set_tuning")


def sw_ctx_set_form(ctx: int, arith: int = -1, rows: int = 16, blocks_per_sm: int = 0) -> None:
    """Batched kernel form: arith -1 auto / 0 int32 / 1 packed; rows 16 or 32;
    resident blocks per SM (0: as many as fit)."""
    _check(load().sw_ctx_set_form(ctx, arith, rows, blocks_per_sm), "sw_ctx_set_form")


def sw_ctx_get_tuning(ctx: int) -> dict:
    lg, fr, ar, rw, bl = _I32(), ctypes.c_double(), _I32(), _I32(), _I32()
    _check(load().sw_ctx_get_tuning(ctx, ctypes.byref(lg), ctypes.byref(fr), ctypes.byref(ar),
                                    ctypes.byref(rw), ctypes.byref(bl)), "sw_ctx_get_tuning")
    return {"narrow_log2g": lg.value, "cap_fraction": fr.value, "arith": ar.value,
            "rows": rw.value, "blocks_per_sm": bl.value}


# -------------------------------------------------------------------- plan

def sw_plan_create(ctx: int, q_offsets, r_offsets, score_matrix, gap_open: int, gap_extend: int,
                   mode: int = SW_MODE_AUTO, flags: int = 0) -> int:
    """q_offsets / r_offsets / score_matrix are host arrays (numpy-convertible)."""
    qo, ro = _host_i64(q_offsets), _host_i64(r_offsets)
    mat = _host_i8(score_matrix)
    if mat.ndim != 2 or mat.shape[0] != mat.shape[1]:
        raise ValueError("score_matrix must be square")
    n = len(qo) - 1
    if len(ro) != n + 1:
        raise ValueError("q_offsets and r_offsets differ in length")
    h = ctypes.c_void_p()
    _check(load().sw_plan_create(ctx, qo.ctypes.data, ro.ctypes.data, n, mat.ctypes.data,
                                 mat.shape[0], gap_open, gap_extend, mode, flags,
                                 ctypes.byref(h)), "sw_plan_create")
    return h.value


def sw_plan_execute(plan: int, q_seqs, r_seqs, out, stream=None) -> None:
    """out: a (5, n_pairs) int32 CUDA tensor (score, qend, rend, qstart, rstart) or 5 tensors."""
    outs = [out[k] for k in range(5)]
    _check(load().sw_plan_execute(plan, _addr(q_seqs), _addr(r_seqs), *[_addr(o) for o in outs],
                                  _stream(stream)), "sw_plan_execute")


def sw_ctx_host_in_place(ctx: int) -> bool:
    """Whether sw_plan_execute_host reads page-locked inputs in place."""
    v = _I32()
    _check(load().sw_ctx_host_in_place(ctx, ctypes.byref(v)), "sw_ctx_host_in_place")
    return bool(v.value)


def sw_ctx_set_host_in_place(ctx: int, enable: bool) -> None:
    """Read page-locked host inputs in place (True, the default where the
    device supports it) or copy them to the device first (False)."""
    _check(load().sw_ctx_set_host_in_place(ctx, 1 if enable else 0), "sw_ctx_set_host_in_place")


def sw_plan_execute_host(plan: int, q_seqs, r_seqs, out_host, stream=None) -> None:
    """Host numpy/pinned-torch buffers in and out; out_host is (5, n_pairs) int32."""
    _check(load().sw_plan_execute_host(plan, _addr(q_seqs), _addr(r_seqs), _addr(out_host),
                                       _stream(stream)), "sw_plan_execute_host")


def sw_plan_info(plan: int) -> dict:
    t, p, l = _I32(), _I32(), _I32()
    sb = _I64()
    _check(load().sw_plan_info(plan, ctypes.byref(t), ctypes.byref(p), ctypes.byref(l),
                               ctypes.byref(sb)), "sw_plan_info")
    ar, rw = _I32(), _I32()
    _check(load().sw_plan_arith(plan, ctypes.byref(ar)), "sw_plan_arith")
    _check(load().sw_plan_rows(plan, ctypes.byref(rw)), "sw_plan_rows")
    return {"group_pairs": t.value, "plain_pairs": p.value, "launches": l.value,
            "scratch_bytes": sb.value, "arith": "s16x2" if ar.value == SW_ARITH_S16X2 else "s32",
            "rows": rw.value}


PLAN_KINDS = {0: "int32", 1: "int32-int8-profile", 2: "s16x2", 3: "s16x2-byte-profile",
              4: "s16x2-32-rows"}


def sw_plan_preview(q_offsets, r_offsets, score_matrix, gap_open: int, gap_extend: int,
                    mode: int = SW_MODE_AUTO, flags: int = 0, sm_count: int = 152,
                    narrow_log2g: int = -1, cap_fraction: float = 0.5):
    """Host-only preview of a plan: (kind name, per-pair lane-group log2 width
    (-1 = plain kernel), per-pair queue position).  No GPU needed."""
    q_offsets = _host_i64(q_offsets)
    r_offsets = _host_i64(r_offsets)
    n = len(q_offsets) - 1
    mat = np.ascontiguousarray(score_matrix, dtype=np.int8)
    kind = _I32()
    lg = np.empty(max(n, 1), np.int32)
    rank = np.empty(max(n, 1), np.int32)
    _check(load().sw_plan_preview(_addr(q_offsets), _addr(r_offsets), n, _addr(mat), mat.shape[0],
                                  gap_open, gap_extend, mode, flags, sm_count, narrow_log2g,
                                  cap_fraction, ctypes.byref(kind), _addr(lg), _addr(rank)),
           "sw_plan_preview")
    return PLAN_KINDS[kind.value], lg[:n], rank[:n]


def sw_plan_poison_guard(plan: int, region: int) -> None:
    """Test aid: break one word of guard region `region` of a SW_PLAN_GUARDS plan."""
    _check(load().sw_plan_poison_guard(plan, region), "sw_plan_poison_guard")


def sw_plan_destroy(plan: int) -> None:
    _check(load().sw_plan_destroy(plan), "sw_plan_destroy")


def sw_autotune(ctx: int, q_offsets, r_offsets, score_matrix, gap_open: int, gap_extend: int,
                q_seqs, r_seqs, out, cache_path: str | None = None, stream=None,
                flags: int = 0) -> dict:
    """Measure the candidate tunings on a resident batch (planned with the
    ENDS_ONLY / NO_S16X2 bits of `flags`); sets the best on ctx."""
    qo, ro = _host_i64(q_offsets), _host_i64(r_offsets)
    mat = _host_i8(score_matrix)
    lg, frac, ms = _I32(), ctypes.c_double(), ctypes.c_double()
    _check(load().sw_autotune_ex(ctx, qo.ctypes.data, ro.ctypes.data, len(qo) - 1,
                                 mat.ctypes.data, mat.shape[0], gap_open, gap_extend,
                                 _addr(q_seqs), _addr(r_seqs), _addr(out), flags,
                                 cache_path.encode() if cache_path else None, _stream(stream),
                                 ctypes.byref(lg), ctypes.byref(frac), ctypes.byref(ms)),
           "sw_autotune_ex")
    t = sw_ctx_get_tuning(ctx)
    return {"narrow_log2g": lg.value, "cap_fraction": frac.value, "ms": ms.value,
            "arith": {-1: "auto", 0: "s32", 1: "s16x2"}[t["arith"]], "rows": t["rows"],
            "blocks_per_sm": t["blocks_per_sm"]}


# ---------------------------------------------------------------- one-shot

def sw_align_batch(q_seqs, q_offsets, r_seqs, r_offsets, score_matrix, gap_open: int,
                   gap_extend: int, out, stream=None) -> None:
    """Sequences, offsets and out on the device; score_matrix on the host."""
    mat = _host_i8(score_matrix)
    n = int(q_offsets.shape[0]) - 1
    outs = [out[k] for k in range(5)]
    _check(load().sw_align_batch(_addr(q_seqs), _addr(q_offsets), _addr(r_seqs), _addr(r_offsets),
                                 n, mat.ctypes.data, mat.shape[0], gap_open, gap_extend,
                                 *[_addr(o) for o in outs], _stream(stream)), "sw_align_batch")


def sw_align_batch_ex(ctx: int, q_seqs, q_offsets, r_seqs, r_offsets, score_matrix, gap_open: int,
                      gap_extend: int, mode: int, out, stream=None) -> None:
    mat = _host_i8(score_matrix)
    n = int(q_offsets.shape[0]) - 1
    outs = [out[k] for k in range(5)]
    _check(load().sw_align_batch_ex(ctx, _addr(q_seqs), _addr(q_offsets), _addr(r_seqs),
                                    _addr(r_offsets), n, mat.ctypes.data, mat.shape[0], gap_open,
                                    gap_extend, mode, *[_addr(o) for o in outs], _stream(stream)),
           "sw_align_batch_ex")


SW_STATIC_MAX_PAIRS = 65536
SW_STATIC_MAX_BOUNDARY_WORDS = 8 << 20


def sw_align_batch_static(q_seqs, q_offsets, r_seqs, r_offsets, score_matrix, gap_open: int,
                          gap_extend: int, out, stream=None) -> None:
    """Allocation-free alignment: sequences and out on the device, offsets and
    score_matrix on the host.  The library allocates no device memory for the
    call (see include/swgb.h for the fixed limits and the ordering rule)."""
    qo, ro = _host_i64(q_offsets), _host_i64(r_offsets)
    mat = _host_i8(score_matrix)
    outs = [out[k] for k in range(5)]
    _check(load().sw_align_batch_static(_addr(q_seqs), qo.ctypes.data, _addr(r_seqs),
                                        ro.ctypes.data, len(qo) - 1, mat.ctypes.data,
                                        mat.shape[0], gap_open, gap_extend,
                                        *[_addr(o) for o in outs], _stream(stream)),
           "sw_align_batch_static")


def sw_static_status(stream=None) -> int:
    """Status word of sw_align_batch_static's kernels on `stream` (read and cleared)."""
    v = _I32()
    _check(load().sw_static_status(ctypes.byref(v), _stream(stream)), "sw_static_status")
    return v.value


def sw_check_residues(seqs, n: int, alphabet_size: int, bad_count, stream=None) -> None:
    _check(load().sw_check_residues(_addr(seqs), n, alphabet_size, _addr(bad_count),
                                    _stream(stream)), "sw_check_residues")


MICROBENCH_OPS = {"iadd": 0, "imax": 1, "viaddmax_s32": 2, "vimax3_s32_relu": 3,
                  "viaddmax_s16x2": 4, "vimax_s32_relu": 5, "vimax3_s16x2": 6,
                  "viaddmax_s16x2_relu": 7}


def sw_microbench_int(op: str, device: int = 0, iters: int = 4096) -> tuple[float, float]:
    """(instructions per second over the device, seconds) for one instruction kind."""
    rate, secs = ctypes.c_double(), ctypes.c_double()
    _check(load().sw_microbench_int(MICROBENCH_OPS[op], device, iters, ctypes.byref(rate),
                                    ctypes.byref(secs)), "sw_microbench_int")
    return rate.value, secs.value


# ----------------------------------------------------------------- serving

def sw_server_create(ctx: int, budget_bytes: int, streams: int = 8,
                     staging_bytes: int = 1 << 30) -> int:
    h = ctypes.c_void_p()
    _check(load().sw_server_create(ctx, budget_bytes, streams, staging_bytes, ctypes.byref(h)),
           "sw_server_create")
    return h.value


def sw_server_submit(server: int, q_seqs, q_offsets, r_seqs, r_offsets, score_matrix,
                     gap_open: int, gap_extend: int, timeout_ms: int = 60000) -> int:
    """Host arrays in; returns the request id."""
    q = np.ascontiguousarray(q_seqs, dtype=np.uint8)
    r = np.ascontiguousarray(r_seqs, dtype=np.uint8)
    qo, ro = _host_i64(q_offsets), _host_i64(r_offsets)
    mat = _host_i8(score_matrix)
    rid = _I64()
    _check(load().sw_server_submit(server, q.ctypes.data if q.size else None, qo.ctypes.data,
                                   r.ctypes.data if r.size else None, ro.ctypes.data, len(qo) - 1,
                                   mat.ctypes.data, mat.shape[0], gap_open, gap_extend,
                                   timeout_ms, ctypes.byref(rid)), "sw_server_submit")
    return rid.value


def sw_server_add_pool(server: int, q_seqs, q_offsets, r_seqs, r_offsets, score_matrix,
                       gap_open: int, gap_extend: int) -> int:
    """Upload a batch (host arrays) as a resident pool; returns its id."""
    q = np.ascontiguousarray(q_seqs, dtype=np.uint8)
    r = np.ascontiguousarray(r_seqs, dtype=np.uint8)
    qo, ro = _host_i64(q_offsets), _host_i64(r_offsets)
    mat = _host_i8(score_matrix)
    pid = _I32()
    _check(load().sw_server_add_pool(server, q.ctypes.data if q.size else None, qo.ctypes.data,
                                     r.ctypes.data if r.size else None, ro.ctypes.data,
                                     len(qo) - 1, mat.ctypes.data, mat.shape[0], gap_open,
                                     gap_extend, ctypes.byref(pid)), "sw_server_add_pool")
    return pid.value


def sw_server_submit_pool(server: int, pool_id: int, first_pair: int, n_pairs: int,
                          timeout_ms: int = 60000) -> int:
    """Queue pairs [first_pair, first_pair + n_pairs) of a resident pool; returns the request id."""
    rid = _I64()
    _check(load().sw_server_submit_pool(server, pool_id, first_pair, n_pairs, timeout_ms,
                                        ctypes.byref(rid)), "sw_server_submit_pool")
    return rid.value


def sw_server_poll(server: int, request_id: int) -> bool:
    d = _I32()
    _check(load().sw_server_poll(server, request_id, ctypes.byref(d)), "sw_server_poll")
    return bool(d.value)


def sw_server_wait(server: int, request_id: int, n_pairs: int, timeout_ms: int = 60000,
                   return_done_ns: bool = False):
    """(n_pairs, 5) int32 results of a request; with return_done_ns, also the
    CLOCK_MONOTONIC ns (time.monotonic_ns's clock) at which it finished."""
    out = np.empty((5, n_pairs), dtype=np.int32)
    done = _I64()
    _check(load().sw_server_wait(server, request_id, timeout_ms, out.ctypes.data,
                                 ctypes.byref(done)), "sw_server_wait")
    res = out.T.copy()
    return (res, done.value) if return_done_ns else res


def sw_server_stats(server: int) -> dict:
    v = [_I64() for _ in range(5)]
    _check(load().sw_server_stats(server, *[ctypes.byref(x) for x in v]), "sw_server_stats")
    return dict(zip(["completed", "in_flight", "queued", "device_bytes_in_use",
                     "device_bytes_peak"], [x.value for x in v]))


def sw_server_launches(server: int) -> dict:
    """{"launches", "pairs", "plan_ms"} so far."""
    a, b, c = _I64(), _I64(), ctypes.c_double()
    _check(load().sw_server_launches(server, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "sw_server_launches")
    return {"launches": a.value, "pairs": b.value, "plan_ms": c.value}


def sw_server_destroy(server: int) -> None:
    _check(load().sw_server_destroy(server), "sw_server_destroy")


# ------------------------------------------------------------ 2-bit input

def sw_pack_2bit(codes) -> np.ndarray:
    """Host uint8 codes (0..3) -> (n + 3) // 4 packed bytes."""
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.zeros(max(1, (len(c) + 3) // 4), dtype=np.uint8)
    _check(load().sw_pack_2bit(c.ctypes.data if len(c) else None, len(c), out.ctypes.data),
           "sw_pack_2bit")
    return out[:(len(c) + 3) // 4]


def sw_unpack_2bit(packed, n_res: int, codes, stream=None) -> None:
    """Device packed bytes -> device codes (4-byte aligned), on the stream."""
    _check(load().sw_unpack_2bit(_addr(packed), n_res, _addr(codes), _stream(stream)),
           "sw_unpack_2bit")


# --------------------------------------------------------------- traceback

CIGAR_CODES = "MID"


def sw_cigar_capacity(results) -> np.ndarray:
    """Host (5, n_pairs) int32 results -> int64 offsets of room per pair."""
    res = np.ascontiguousarray(results, dtype=np.int32)
    n = res.shape[1]
    off = np.zeros(n + 1, dtype=np.int64)
    _check(load().sw_cigar_capacity(res.ctypes.data, n, off.ctypes.data), "sw_cigar_capacity")
    return off


def sw_traceback(ctx: int, q_seqs, q_offsets, r_seqs, r_offsets, score_matrix, gap_open: int,
                 gap_extend: int, results, cigar_offsets, out_ops, out_n_ops,
                 stream=None) -> None:
    """Sequences and outputs on the device; offsets, matrix, results (5, n)
    and cigar_offsets on the host.  Asynchronous on the stream."""
    qo, ro = _host_i64(q_offsets), _host_i64(r_offsets)
    mat = _host_i8(score_matrix)
    res = np.ascontiguousarray(results, dtype=np.int32)
    co = _host_i64(cigar_offsets)
    _check(load().sw_traceback(ctx, _addr(q_seqs), qo.ctypes.data, _addr(r_seqs), ro.ctypes.data,
                               len(qo) - 1, mat.ctypes.data, mat.shape[0], gap_open, gap_extend,
                               res.ctypes.data, co.ctypes.data, _addr(out_ops), _addr(out_n_ops),
                               _stream(stream)), "sw_traceback")


def _dev_tensor(x, dtype, name: str):
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == dtype and x.is_contiguous()):
        raise TypeError(f"{name}: a contiguous {dtype} CUDA tensor is required")
    return x


def sw_cigar_capacity_device(results, offsets, stream=None) -> None:
    """results (5, n) int32 and offsets (n + 1,) int64, both on the device;
    offsets gets each aligned pair's op room, offsets[n] the total.
    Asynchronous on the stream."""
    import torch
    res = _dev_tensor(results, torch.int32, "results")
    off = _dev_tensor(offsets, torch.int64, "offsets")
    n = int(res.shape[1]) if res.dim() == 2 else 0
    if res.dim() != 2 or res.shape[0] != 5 or off.numel() != n + 1:
        raise ValueError("results must be (5, n) and offsets (n + 1,)")
    _check(load().sw_cigar_capacity_device(_addr(res), n, _addr(off), _stream(stream)),
           "sw_cigar_capacity_device")


def sw_traceback_device(ctx: int, q_seqs, q_offsets, r_seqs, r_offsets, score_matrix,
                        gap_open: int, gap_extend: int, results, cigar_offsets, out_ops,
                        out_n_ops, stream=None) -> None:
    """Everything on the device but the score matrix: offsets (n + 1,) int64,
    results (5, n) int32, cigar_offsets (n + 1,) int64.  Waits for the
    classification kernels, then enqueues the fill and walk on the stream."""
    import torch
    qo = _dev_tensor(q_offsets, torch.int64, "q_offsets")
    ro = _dev_tensor(r_offsets, torch.int64, "r_offsets")
    res = _dev_tensor(results, torch.int32, "results")
    co = _dev_tensor(cigar_offsets, torch.int64, "cigar_offsets")
    n = int(qo.numel()) - 1
    if ro.numel() != n + 1 or co.numel() != n + 1 or tuple(res.shape) != (5, n):
        raise ValueError("offsets must be (n + 1,) and results (5, n)")
    mat = _host_i8(score_matrix)
    _check(load().sw_traceback_device(ctx, _addr(q_seqs), _addr(qo), _addr(r_seqs), _addr(ro), n,
                                      mat.ctypes.data, mat.shape[0], gap_open, gap_extend,
                                      _addr(res), _addr(co), _addr(out_ops), _addr(out_n_ops),
                                      _stream(stream)), "sw_traceback_device")


def cigar_strings(ops, offsets, n_ops) -> list[str]:
    """Per-pair CIGAR text ('12M1D3M') from run-length ops."""
    ops = np.asarray(ops)
    return ["".join(f"{int(o) >> 4}{CIGAR_CODES[int(o) & 15]}"
                    for o in ops[offsets[p]:offsets[p] + n_ops[p]]) for p in range(len(n_ops))]


# ----------------------------------------------------------------- helpers

class Aligner:
    """A planned batch resident on one device: upload once, execute many times."""

    def __init__(self, q_seqs, q_offsets, r_seqs, r_offsets, score_matrix, gap_open, gap_extend,
                 mode=SW_MODE_AUTO, flags=0, device=0, ctx=None):
        import torch
        self.device = torch.device("cuda", device)
        self._own_ctx = ctx is None
        self.ctx = sw_ctx_create(device) if ctx is None else ctx
        q_offsets = _host_i64(q_offsets)
        r_offsets = _host_i64(r_offsets)
        self.n_pairs = len(q_offsets) - 1
        self.q = torch.from_numpy(np.ascontiguousarray(q_seqs, dtype=np.uint8)).to(self.device)
        self.r = torch.from_numpy(np.ascontiguousarray(r_seqs, dtype=np.uint8)).to(self.device)
        if self.q.numel() == 0:
            self.q = torch.zeros(1, dtype=torch.uint8, device=self.device)
        if self.r.numel() == 0:
            self.r = torch.zeros(1, dtype=torch.uint8, device=self.device)
        self.out = torch.full((5, max(self.n_pairs, 1)), -7, dtype=torch.int32, device=self.device)
        self.plan = sw_plan_create(self.ctx, q_offsets, r_offsets, score_matrix, gap_open,
                                   gap_extend, mode, flags)

    def run(self, stream=None):
        sw_plan_execute(self.plan, self.q, self.r, self.out, stream)
        return self.out

    def results(self) -> np.ndarray:
        """(n_pairs, 5) int32 host array after the last run (synchronises)."""
        return self.out[:, :self.n_pairs].T.contiguous().cpu().numpy()

    def info(self) -> dict:
        return sw_plan_info(self.plan)

    def close(self):
        if self.plan:
            sw_plan_destroy(self.plan)
            self.plan = None
        if self._own_ctx and self.ctx:
            sw_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
