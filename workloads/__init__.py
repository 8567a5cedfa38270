"""Seeded synthetic workloads for batched Smith-Waterman/Gotoh alignment.

This module only draws inputs.  It holds none of the alignment arithmetic, so
both the CPU oracle (test infrastructure) and the CUDA library's tests and
benchmark can take their inputs from here without sharing any of the method.

The paper evaluates on ADEPT's 30,000-pair DNA set and 4.6 million held-out
pairs (Section III-C), which are not distributed with it and whose length
distribution it does not state.  The five workloads below stand in for them:

  0  dna-1k        1,000 DNA pairs, |q| ~ U[100,150], |r| ~ U[200,300]
  1  dna-100k    100,000 DNA pairs, |q| ~ U[100,300], |r| ~ U[200,1024]
  2  protein-20k  20,000 protein pairs, |q| ~ U[64,400], |r| ~ U[64,1024]
  3  dna-skew-200k 200,000 DNA pairs, |q| lognormal(median 150, sigma 0.6)
                   clipped to [50,1000], |r| lognormal(median 400, sigma 0.6)
                   clipped to [100,4096]
  4  serving       Poisson arrivals of requests of floor(log-uniform[1,4096])
                   pairs, half drawn like workload 1, half like workload 2

DNA is coded A,C,G,T = 0..3 with i.i.d. uniform bases, scored +3/-3 with
gap_open -6 and gap_extend -1.  In 30% of the DNA pairs a mutated copy of the
query (5% substitutions to a different base, 1% single-base indels split
evenly between insertion and deletion) overwrites the reference at a uniform
offset.  Protein residues are coded in BLOSUM order ARNDCQEGHILKMFPSTWYV =
0..19, drawn i.i.d. from the background frequencies BLOSUM62 implies; 30% of
the pairs carry a planted homolog of the query with 30% of its positions
substituted by b != a with probability proportional to p_b exp(lambda s(a,b)).
Scoring is BLOSUM62 with gap_open -11 and gap_extend -1.

Random numbers come from a counter-based generator (the splitmix64 finaliser
applied to key + (counter + 1) * golden-gamma), one stream per purpose, each
draw indexed by the pair or by the global residue position.  The first N pairs
of a workload are therefore identical whatever the total pair count, which
lets a bounded sample of a workload stand for the whole.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

BASE_SEED = 20220825
DNA_ALPHABET = "ACGT"
PROTEIN_ALPHABET = "ARNDCQEGHILKMFPSTWYV"

# ---------------------------------------------------------------- scoring data


def load_blosum62() -> tuple[np.ndarray, str]:
    """Return (20x20 int matrix, residue order) read from blosum62.txt."""
    rows = []
    with open(os.path.join(HERE, "blosum62.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) == 20:  # header line of residue letters
                continue
            rows.append([int(x) for x in parts[1:]])
    s = np.array(rows, dtype=np.int64)
    assert s.shape == (20, 20)
    return s, PROTEIN_ALPHABET


def load_background() -> tuple[float, np.ndarray]:
    """Return (lambda, p) written by derive_background.py."""
    lam = None
    p = []
    with open(os.path.join(HERE, "blosum62_background.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, val = line.split()
            if key == "lambda":
                lam = float(val)
            else:
                p.append(float(val))
    assert lam is not None and len(p) == 20
    return lam, np.array(p, dtype=np.float64)


def dna_matrix(match: int = 3, mismatch: int = -3) -> np.ndarray:
    m = np.full((4, 4), mismatch, dtype=np.int8)
    np.fill_diagonal(m, match)
    return m


# ------------------------------------------------------------------ generator

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def _finalise(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _C1
    z ^= z >> np.uint64(27)
    z *= _C2
    z ^= z >> np.uint64(31)
    return z


class Stream:
    """Counter-based stream: draw k of stream (seed, sid) is a pure function."""

    def __init__(self, seed: int, sid: int):
        k = _finalise(np.array([(seed * 0x100000001B3 + sid * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF],
                               dtype=np.uint64))
        self.key = k[0]

    def u64(self, start: int, n: int) -> np.ndarray:
        c = np.arange(start, start + n, dtype=np.uint64) + np.uint64(1)
        with np.errstate(over="ignore"):
            return _finalise(self.key + c * _GAMMA)

    def uniform(self, start: int, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(start, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


S_QLEN, S_RLEN, S_QRES, S_RRES, S_PLANT, S_EVENT, S_OFFSET = 1, 2, 3, 4, 5, 6, 7


def _lengths(st: Stream, n: int, spec: tuple) -> np.ndarray:
    if spec[0] == "uniform":
        lo, hi = spec[1], spec[2]
        u = st.uniform(0, n)
        return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)
    if spec[0] == "lognormal":
        median, sigma, lo, hi = spec[1:]
        u1 = st.uniform(0, n)
        u2 = st.uniform(n, n)
        z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
        return np.clip(np.rint(median * np.exp(sigma * z)), lo, hi).astype(np.int64)
    raise ValueError(spec)


def _dna_residues(st: Stream, n: int) -> np.ndarray:
    words = st.u64(0, (n + 31) // 32)
    shifts = (np.arange(32, dtype=np.uint64) * np.uint64(2))
    bases = ((words[:, None] >> shifts[None, :]) & np.uint64(3)).astype(np.uint8)
    return bases.reshape(-1)[:n]


def _protein_residues(st: Stream, n: int, p: np.ndarray) -> np.ndarray:
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    out = np.empty(n, dtype=np.uint8)
    chunk = 1 << 22
    for s in range(0, n, chunk):
        u = st.uniform(s, min(chunk, n - s))
        out[s:s + len(u)] = np.minimum(np.searchsorted(cdf, u, side="right"), 19)
    return out


def _offsets(lens: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


@dataclass
class Batch:
    """A batch of (query, reference) pairs in packed CSR form."""

    name: str
    q_seqs: np.ndarray       # uint8, concatenated query residues
    q_offsets: np.ndarray    # int64, n_pairs + 1
    r_seqs: np.ndarray       # uint8, concatenated reference residues
    r_offsets: np.ndarray    # int64, n_pairs + 1
    matrix: np.ndarray       # int8, alphabet x alphabet, row = query residue
    gap_open: int
    gap_extend: int
    planted: np.ndarray = field(default=None)  # bool per pair

    @property
    def alphabet(self) -> int:
        return int(self.matrix.shape[0])

    @property
    def n_pairs(self) -> int:
        return len(self.q_offsets) - 1

    @property
    def q_lens(self) -> np.ndarray:
        return np.diff(self.q_offsets)

    @property
    def r_lens(self) -> np.ndarray:
        return np.diff(self.r_offsets)

    @property
    def cells(self) -> int:
        return int(np.sum(self.q_lens * self.r_lens))

    def pair(self, i: int) -> tuple[np.ndarray, np.ndarray]:
        q = self.q_seqs[self.q_offsets[i]:self.q_offsets[i + 1]]
        r = self.r_seqs[self.r_offsets[i]:self.r_offsets[i + 1]]
        return q, r

    def slice(self, lo: int, hi: int) -> "Batch":
        """Pairs lo..hi-1 as their own batch (contiguous, so no repacking)."""
        qo, ro = self.q_offsets[lo:hi + 1], self.r_offsets[lo:hi + 1]
        return Batch(f"{self.name}[{lo}:{hi}]", self.q_seqs[qo[0]:qo[-1]].copy(), qo - qo[0],
                     self.r_seqs[ro[0]:ro[-1]].copy(), ro - ro[0], self.matrix,
                     self.gap_open, self.gap_extend,
                     None if self.planted is None else self.planted[lo:hi].copy())

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        qs = [self.pair(int(i))[0] for i in idx]
        rs = [self.pair(int(i))[1] for i in idx]
        return make_batch(self.name + "-subset", qs, rs, self.matrix,
                          self.gap_open, self.gap_extend,
                          planted=None if self.planted is None else self.planted[idx])


def make_batch(name, queries, refs, matrix, gap_open, gap_extend, planted=None) -> Batch:
    """Pack lists of residue arrays into a Batch."""
    ql = np.array([len(q) for q in queries], dtype=np.int64)
    rl = np.array([len(r) for r in refs], dtype=np.int64)
    qs = np.concatenate([np.asarray(q, dtype=np.uint8) for q in queries]) if len(queries) and ql.sum() else np.zeros(0, np.uint8)
    rs = np.concatenate([np.asarray(r, dtype=np.uint8) for r in refs]) if len(refs) and rl.sum() else np.zeros(0, np.uint8)
    return Batch(name, qs, _offsets(ql), rs, _offsets(rl), np.asarray(matrix, dtype=np.int8),
                 int(gap_open), int(gap_extend),
                 np.zeros(len(ql), bool) if planted is None else np.asarray(planted, bool))


CONFIGS = {
    0: dict(name="dna-1k", kind="dna", n_pairs=1_000,
            qlen=("uniform", 100, 150), rlen=("uniform", 200, 300)),
    1: dict(name="dna-100k", kind="dna", n_pairs=100_000,
            qlen=("uniform", 100, 300), rlen=("uniform", 200, 1024)),
    2: dict(name="protein-20k", kind="protein", n_pairs=20_000,
            qlen=("uniform", 64, 400), rlen=("uniform", 64, 1024)),
    3: dict(name="dna-skew-200k", kind="dna", n_pairs=200_000,
            qlen=("lognormal", 150.0, 0.6, 50, 1000),
            rlen=("lognormal", 400.0, 0.6, 100, 4096)),
}

PLANT_RATE = 0.30
DNA_SUB, DNA_INDEL = 0.05, 0.01
PROTEIN_SUB = 0.30
DNA_GAPS = (-6, -1)
PROTEIN_GAPS = (-11, -1)


def _plant_dna(q_seqs, q_off, r_seqs, r_off, planted, st_ev, st_off):
    idx = np.flatnonzero(planted)
    if len(idx) == 0:
        return
    starts, ends = q_off[idx], q_off[idx + 1]
    lens = ends - starts
    pos = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)])
    w = st_ev.u64(0, int(q_off[-1]))[pos]
    u = (w >> np.uint64(32)).astype(np.float64) * (2.0 ** -32)
    low = (w & np.uint64(0xFFFFFFFF)).astype(np.int64)
    orig = q_seqs[pos].astype(np.int64)
    dele = u < DNA_INDEL / 2
    ins = (u >= DNA_INDEL / 2) & (u < DNA_INDEL)
    sub = (u >= DNA_INDEL) & (u < DNA_INDEL + DNA_SUB)
    base1 = np.where(sub, (orig + 1 + low % 3) % 4, orig).astype(np.uint8)
    base2 = (low & 3).astype(np.uint8)
    counts = np.where(dele, 0, np.where(ins, 2, 1))
    first = np.cumsum(counts) - counts
    out = np.empty(int(counts.sum()), dtype=np.uint8)
    keep = counts >= 1
    out[first[keep]] = base1[keep]
    out[first[ins] + 1] = base2[ins]
    # per-pair output ranges
    pair_pos_start = np.concatenate([[0], np.cumsum(lens)[:-1]])
    out_start = np.concatenate([first, [len(out)]])[pair_pos_start]
    out_end = np.concatenate([out_start[1:], [len(out)]])
    m = r_off[idx + 1] - r_off[idx]
    L = np.minimum(out_end - out_start, m)
    uo = st_off.uniform(0, len(q_off) - 1)[idx]
    o = np.floor(uo * (m - L + 1)).astype(np.int64)
    for k in range(len(idx)):
        if L[k] > 0:
            dst = r_off[idx[k]] + o[k]
            r_seqs[dst:dst + L[k]] = out[out_start[k]:out_start[k] + L[k]]


def substitution_conditionals(s: np.ndarray, p: np.ndarray, lam: float) -> np.ndarray:
    """Row a: cumulative P(b | a, b != a) proportional to p_b exp(lam s(a,b))."""
    w = p[None, :] * np.exp(lam * s.astype(np.float64))
    np.fill_diagonal(w, 0.0)
    w /= w.sum(axis=1, keepdims=True)
    cdf = np.cumsum(w, axis=1)
    cdf[:, -1] = 1.0
    return cdf


def _plant_protein(q_seqs, q_off, r_seqs, r_off, planted, st_ev, st_off, cond_cdf):
    idx = np.flatnonzero(planted)
    if len(idx) == 0:
        return
    starts, ends = q_off[idx], q_off[idx + 1]
    pos = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)])
    w = st_ev.u64(0, int(q_off[-1]))[pos]
    u = (w >> np.uint64(32)).astype(np.float64) * (2.0 ** -32)
    ub = (w & np.uint64(0xFFFFFFFF)).astype(np.float64) * (2.0 ** -32)
    orig = q_seqs[pos].astype(np.int64)
    sub = u < PROTEIN_SUB
    newb = np.empty_like(orig)
    for a in range(20):
        sel = orig == a
        newb[sel] = np.minimum(np.searchsorted(cond_cdf[a], ub[sel], side="right"), 19)
    hom = np.where(sub, newb, orig).astype(np.uint8)
    lens = ends - starts
    hstart = np.concatenate([[0], np.cumsum(lens)[:-1]])
    m = r_off[idx + 1] - r_off[idx]
    L = np.minimum(lens, m)
    uo = st_off.uniform(0, len(q_off) - 1)[idx]
    o = np.floor(uo * (m - L + 1)).astype(np.int64)
    for k in range(len(idx)):
        if L[k] > 0:
            dst = r_off[idx[k]] + o[k]
            r_seqs[dst:dst + L[k]] = hom[hstart[k]:hstart[k] + L[k]]


def generate(kind: str, n_pairs: int, qlen: tuple, rlen: tuple, seed: int,
             name: str = "custom") -> Batch:
    """Draw n_pairs pairs of the given kind ('dna' or 'protein')."""
    qlens = _lengths(Stream(seed, S_QLEN), n_pairs, qlen)
    rlens = _lengths(Stream(seed, S_RLEN), n_pairs, rlen)
    q_off, r_off = _offsets(qlens), _offsets(rlens)
    planted = Stream(seed, S_PLANT).uniform(0, n_pairs) < PLANT_RATE
    if kind == "dna":
        q = _dna_residues(Stream(seed, S_QRES), int(q_off[-1]))
        r = _dna_residues(Stream(seed, S_RRES), int(r_off[-1]))
        _plant_dna(q, q_off, r, r_off, planted, Stream(seed, S_EVENT), Stream(seed, S_OFFSET))
        return Batch(name, q, q_off, r, r_off, dna_matrix(), *DNA_GAPS, planted)
    if kind == "protein":
        s, _ = load_blosum62()
        lam, p = load_background()
        q = _protein_residues(Stream(seed, S_QRES), int(q_off[-1]), p)
        r = _protein_residues(Stream(seed, S_RRES), int(r_off[-1]), p)
        _plant_protein(q, q_off, r, r_off, planted, Stream(seed, S_EVENT), Stream(seed, S_OFFSET),
                       substitution_conditionals(s, p, lam))
        return Batch(name, q, q_off, r, r_off, s.astype(np.int8), *PROTEIN_GAPS, planted)
    raise ValueError(kind)


def gen_config(k: int, n_pairs: int | None = None, seed: int | None = None) -> Batch:
    """Workload k (0..3); n_pairs < full gives the first n_pairs of it."""
    c = CONFIGS[k]
    n = c["n_pairs"] if n_pairs is None else int(n_pairs)
    s = BASE_SEED + k if seed is None else seed
    return generate(c["kind"], n, c["qlen"], c["rlen"], s, c["name"])


# -------------------------------------------------------------- serving (4)


@dataclass
class Request:
    rid: int
    arrival_s: float
    kind: str
    batch: Batch
    first: int = 0  # index of the request's first pair in its kind's pool


def serving_requests(n_requests: int, rate_per_s: float, seed: int = BASE_SEED + 4,
                     max_pairs: int = 4096, pools: dict | None = None) -> list[Request]:
    """Serving workload: Poisson arrivals at rate_per_s, request sizes
    floor(log-uniform[1, max_pairs]) pairs, half DNA and half protein.

    A DNA request takes the next consecutive pairs of the 100k-pair DNA
    workload, a protein request those of the 20k-pair protein workload
    (wrapping to the start when a pool runs out).  pools may pass those two
    batches in ({"dna": ..., "protein": ...}); otherwise the needed prefixes
    are generated.  Arrival times scale exactly with 1 / rate_per_s, so one
    request list serves a whole rate sweep via arrival_s * old / new rate.
    """
    st = Stream(seed, 11)
    u = st.uniform(0, 3 * n_requests).reshape(3, n_requests)
    gaps = -np.log1p(-u[0]) / rate_per_s
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.clip(np.floor(np.exp(u[1] * math.log(max_pairs))), 1, max_pairs).astype(np.int64)
    kinds = np.where(u[2] < 0.5, "dna", "protein")
    pools = dict(pools or {})
    for kind, cfg in (("dna", 1), ("protein", 2)):
        if kind not in pools:
            need = int(sizes[kinds == kind].sum())
            pools[kind] = gen_config(cfg, n_pairs=max(1, min(need, CONFIGS[cfg]["n_pairs"])))
    cursor = {"dna": 0, "protein": 0}
    out = []
    for i in range(n_requests):
        kind = str(kinds[i])
        pool = pools[kind]
        k = int(min(sizes[i], pool.n_pairs))
        if cursor[kind] + k > pool.n_pairs:
            cursor[kind] = 0
        b = pool.slice(cursor[kind], cursor[kind] + k)
        b.name = f"req{i}-{kind}"
        cursor[kind] += k
        out.append(Request(i, float(arrivals[i]), kind, b, cursor[kind] - k))
    return out
