"""CPU oracle for batched Smith-Waterman/Gotoh local alignment.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The CUDA
library (``paper_2208_12350_gb300``) never imports it and shares no code with
it; the two meet only in the seeded inputs of the ``workloads`` package.

Three independent implementations, all plain C built with gcc:

* ``align`` / ``align_batch`` (sw_oracle.c): the paper's method as written,
  a forward pass that fills the scoring matrix and picks the maximal cell,
  then a reverse pass over the reversed prefixes for the start
  (Section II-B.1, Fig. 2, Fig. 8).
* ``brute`` (sw_brute.c): enumeration of every local alignment of short
  sequences, scored by the definition.
* ``track`` (sw_track.c): a forward pass that carries start positions.

All return (score, qend, rend, qstart, rstart) with 0-based inclusive
coordinates, and score 0 with all coordinates -1 when nothing aligns.

``cigar`` / ``cigar_batch`` (sw_cigar.c) give the alignment itself: the
traceback (Fig. 2(c)) of the global Gotoh recurrence over the located
substrings, as run-length ops (length << 4 | code, M = 0, I = 1, D = 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["sw_oracle.c", "sw_brute.c", "sw_track.c", "sw_cigar.c"]
LIB = os.path.join(HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into oracle/liboracle.so with gcc."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared", "-pthread",
           *srcs, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i8p = ctypes.POINTER(ctypes.c_int8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.oracle_align.argtypes = [u8p, i64, u8p, i64, i8p, i32, i32, i32, i32p]
        lib.oracle_align.restype = ctypes.c_int
        lib.track_align.argtypes = [u8p, i64, u8p, i64, i8p, i32, i32, i32, i32p]
        lib.track_align.restype = ctypes.c_int
        lib.brute_align.argtypes = [u8p, i64, u8p, i64, i8p, i32, i32, i32, i32p]
        lib.brute_align.restype = ctypes.c_int64
        lib.oracle_align_batch.argtypes = [u8p, i64p, u8p, i64p, i32, i8p, i32, i32, i32,
                                           i32p, i32p, i32]
        lib.oracle_align_batch.restype = ctypes.c_int
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_cigar.argtypes = [u8p, i64, u8p, i64, i8p, i32, i32, i32, i32p, u32p, i32,
                                     i32p, ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_cigar.restype = ctypes.c_int
        lib.oracle_cigar_batch.argtypes = [u8p, i64p, u8p, i64p, i32, i8p, i32, i32, i32, i32p,
                                           i64p, u32p, i32p, i32p, i32]
        lib.oracle_cigar_batch.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _prep(q, r, matrix):
    q = np.ascontiguousarray(np.asarray(q, dtype=np.uint8))
    r = np.ascontiguousarray(np.asarray(r, dtype=np.uint8))
    mat = np.ascontiguousarray(np.asarray(matrix, dtype=np.int8))
    assert mat.ndim == 2 and mat.shape[0] == mat.shape[1]
    return q, r, mat


class OracleError(RuntimeError):
    pass


def align(q, r, matrix, gap_open: int, gap_extend: int) -> tuple[int, int, int, int, int]:
    """Forward + reverse pass oracle for one pair."""
    q, r, mat = _prep(q, r, matrix)
    out = np.zeros(5, dtype=np.int32)
    rc = _load().oracle_align(_ptr(q, ctypes.c_uint8), len(q), _ptr(r, ctypes.c_uint8), len(r),
                              _ptr(mat, ctypes.c_int8), mat.shape[0], gap_open, gap_extend,
                              _ptr(out, ctypes.c_int32))
    if rc != 0:
        raise OracleError(f"oracle_align returned {rc}")
    return tuple(int(v) for v in out)


def track(q, r, matrix, gap_open: int, gap_extend: int) -> tuple[int, int, int, int, int]:
    """Start-tracking forward-only oracle for one pair."""
    q, r, mat = _prep(q, r, matrix)
    out = np.zeros(5, dtype=np.int32)
    rc = _load().track_align(_ptr(q, ctypes.c_uint8), len(q), _ptr(r, ctypes.c_uint8), len(r),
                             _ptr(mat, ctypes.c_int8), mat.shape[0], gap_open, gap_extend,
                             _ptr(out, ctypes.c_int32))
    if rc != 0:
        raise OracleError(f"track_align returned {rc}")
    return tuple(int(v) for v in out)


def brute(q, r, matrix, gap_open: int, gap_extend: int) -> tuple[int, int, int, int, int]:
    """Enumerate every local alignment (at most 12 residues per sequence)."""
    q, r, mat = _prep(q, r, matrix)
    out = np.zeros(5, dtype=np.int32)
    rc = _load().brute_align(_ptr(q, ctypes.c_uint8), len(q), _ptr(r, ctypes.c_uint8), len(r),
                             _ptr(mat, ctypes.c_int8), mat.shape[0], gap_open, gap_extend,
                             _ptr(out, ctypes.c_int32))
    if rc < 0:
        raise OracleError("brute_align: bad arguments")
    return tuple(int(v) for v in out)


def align_batch(q_seqs, q_offsets, r_seqs, r_offsets, matrix, gap_open: int, gap_extend: int,
                threads: int | None = None) -> np.ndarray:
    """Oracle over a CSR batch on host threads; returns an (n_pairs, 5) int32 array."""
    q_seqs = np.ascontiguousarray(q_seqs, dtype=np.uint8)
    r_seqs = np.ascontiguousarray(r_seqs, dtype=np.uint8)
    q_off = np.ascontiguousarray(q_offsets, dtype=np.int64)
    r_off = np.ascontiguousarray(r_offsets, dtype=np.int64)
    mat = np.ascontiguousarray(matrix, dtype=np.int8)
    n = len(q_off) - 1
    out = np.zeros((n, 5), dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    if n == 0:
        return out
    if threads is None:
        threads = os.cpu_count() or 1
    rc = _load().oracle_align_batch(
        _ptr(q_seqs if len(q_seqs) else np.zeros(1, np.uint8), ctypes.c_uint8), _ptr(q_off, ctypes.c_int64),
        _ptr(r_seqs if len(r_seqs) else np.zeros(1, np.uint8), ctypes.c_uint8), _ptr(r_off, ctypes.c_int64),
        n, _ptr(mat, ctypes.c_int8), mat.shape[0], gap_open, gap_extend,
        _ptr(out, ctypes.c_int32), _ptr(status, ctypes.c_int32), int(threads))
    if rc != 0:
        raise OracleError(f"oracle_align_batch returned {rc} (first failing pair "
                          f"{int(np.flatnonzero(status)[0])})")
    return out


def align_workload(batch, threads: int | None = None, idx=None) -> np.ndarray:
    """Oracle over a workloads.Batch (optionally only the pairs in idx)."""
    if idx is not None:
        batch = batch.subset(idx)
    return align_batch(batch.q_seqs, batch.q_offsets, batch.r_seqs, batch.r_offsets,
                       batch.matrix, batch.gap_open, batch.gap_extend, threads)


CIGAR_CODES = "MID"


def cigar_string(ops) -> str:
    """Run-length ops (length << 4 | code) as text, e.g. '1M1I3M'."""
    return "".join(f"{int(o) >> 4}{CIGAR_CODES[int(o) & 15]}" for o in ops)


def cigar(q, r, matrix, gap_open: int, gap_extend: int, result) -> tuple[list[int], int]:
    """(run-length ops, global score of the span) of one pair's alignment,
    given its (score, qend, rend, qstart, rstart)."""
    q, r, mat = _prep(q, r, matrix)
    res = np.ascontiguousarray(result, dtype=np.int32)
    cap = max(1, len(q) + len(r))
    ops = np.zeros(cap, dtype=np.uint32)
    n_ops = ctypes.c_int32()
    g = ctypes.c_int64()
    rc = _load().oracle_cigar(_ptr(q, ctypes.c_uint8), len(q),
                              _ptr(r, ctypes.c_uint8), len(r), _ptr(mat, ctypes.c_int8),
                              mat.shape[0], gap_open, gap_extend, _ptr(res, ctypes.c_int32),
                              _ptr(ops, ctypes.c_uint32), cap, ctypes.byref(n_ops),
                              ctypes.byref(g))
    if rc != 0:
        raise OracleError(f"oracle_cigar returned {rc}")
    return [int(x) for x in ops[:n_ops.value]], int(g.value)


def cigar_capacity(results) -> np.ndarray:
    """CSR offsets of room for each pair's ops: qend-qstart+1 + rend-rstart+1
    for pairs with a positive score, 0 otherwise."""
    res = np.asarray(results)
    room = np.where(res[:, 0] > 0, (res[:, 1] - res[:, 3] + 1) + (res[:, 2] - res[:, 4] + 1), 0)
    off = np.zeros(len(res) + 1, dtype=np.int64)
    np.cumsum(room, out=off[1:])
    return off


def cigar_batch(q_seqs, q_offsets, r_seqs, r_offsets, matrix, gap_open: int, gap_extend: int,
                results, threads: int | None = None) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(ops, offsets, n_ops) for every pair of a batch, given its
    (n_pairs, 5) results; pair p's ops are ops[offsets[p] : offsets[p] + n_ops[p]]."""
    q_seqs = np.ascontiguousarray(q_seqs, dtype=np.uint8)
    r_seqs = np.ascontiguousarray(r_seqs, dtype=np.uint8)
    q_off = np.ascontiguousarray(q_offsets, dtype=np.int64)
    r_off = np.ascontiguousarray(r_offsets, dtype=np.int64)
    mat = np.ascontiguousarray(matrix, dtype=np.int8)
    res = np.ascontiguousarray(results, dtype=np.int32)
    n = len(q_off) - 1
    off = cigar_capacity(res)
    ops = np.zeros(max(1, int(off[-1])), dtype=np.uint32)
    n_ops = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    if n == 0:
        return ops, off, n_ops
    rc = _load().oracle_cigar_batch(
        _ptr(q_seqs if len(q_seqs) else np.zeros(1, np.uint8), ctypes.c_uint8),
        _ptr(q_off, ctypes.c_int64),
        _ptr(r_seqs if len(r_seqs) else np.zeros(1, np.uint8), ctypes.c_uint8),
        _ptr(r_off, ctypes.c_int64), n, _ptr(mat, ctypes.c_int8), mat.shape[0], gap_open,
        gap_extend, _ptr(res, ctypes.c_int32), _ptr(off, ctypes.c_int64),
        _ptr(ops, ctypes.c_uint32), _ptr(n_ops, ctypes.c_int32), _ptr(status, ctypes.c_int32),
        int(threads or os.cpu_count() or 1))
    if rc != 0:
        raise OracleError(f"oracle_cigar_batch returned {rc} (first failing pair "
                          f"{int(np.flatnonzero(status)[0])})")
    return ops, off, n_ops


def cigar_workload(batch, results, threads: int | None = None):
    """cigar_batch over a workloads.Batch."""
    return cigar_batch(batch.q_seqs, batch.q_offsets, batch.r_seqs, batch.r_offsets,
                       batch.matrix, batch.gap_open, batch.gap_extend, results, threads)
