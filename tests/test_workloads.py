"""The seeded input generators: shapes, ranges, determinism, scoring data."""
import numpy as np
import pytest

import oracle
import workloads as wl


def test_blosum62_properties():
    s, order = wl.load_blosum62()
    assert order == "ARNDCQEGHILKMFPSTWYV"
    assert s.shape == (20, 20)
    assert np.array_equal(s, s.T)
    d = np.diag(s)
    off = s + np.diag(np.full(20, -100))
    assert np.all(d > 0) and np.all(d > off.max(axis=1))
    # a few entries every copy of the published matrix has
    idx = {c: i for i, c in enumerate(order)}
    assert s[idx["W"], idx["W"]] == 11 and s[idx["C"], idx["C"]] == 9
    assert s[idx["A"], idx["A"]] == 4 and s[idx["W"], idx["D"]] == -4
    assert s.min() == -4 and s.max() == 11


def test_implied_background():
    s, _ = wl.load_blosum62()
    lam, p = wl.load_background()
    assert 0.25 < lam < 0.40
    assert np.all(p > 0) and abs(p.sum() - 1) < 1e-12
    resid = np.exp(lam * s) @ p
    assert np.allclose(resid, 1.0, atol=1e-9)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_config_shapes(k):
    c = wl.CONFIGS[k]
    b = wl.gen_config(k, n_pairs=3000)
    assert b.n_pairs == 3000
    q, r = b.q_lens, b.r_lens
    lo_q, hi_q = (c["qlen"][1], c["qlen"][2]) if c["qlen"][0] == "uniform" else c["qlen"][3:5]
    lo_r, hi_r = (c["rlen"][1], c["rlen"][2]) if c["rlen"][0] == "uniform" else c["rlen"][3:5]
    assert q.min() >= lo_q and q.max() <= hi_q
    assert r.min() >= lo_r and r.max() <= hi_r
    assert b.q_seqs.max() < b.alphabet and b.r_seqs.max() < b.alphabet
    assert abs(b.planted.mean() - 0.30) < 0.03
    assert b.q_offsets[0] == 0 and b.q_offsets[-1] == len(b.q_seqs)
    assert b.r_offsets[-1] == len(b.r_seqs)


def test_prefix_property_and_determinism():
    a = wl.gen_config(1, n_pairs=500)
    b = wl.gen_config(1, n_pairs=2000)
    assert np.array_equal(a.q_seqs, b.q_seqs[:len(a.q_seqs)])
    assert np.array_equal(a.r_seqs, b.r_seqs[:len(a.r_seqs)])
    c = wl.gen_config(1, n_pairs=500)
    assert np.array_equal(a.r_seqs, c.r_seqs)


def test_planted_pairs_score_high():
    """Planted DNA pairs align far above random ones (the planting works)."""
    b = wl.gen_config(0, n_pairs=300)
    out = oracle.align_workload(b)
    pl = out[b.planted, 0]
    rnd = out[~b.planted, 0]
    assert np.median(pl) > 2 * b.q_lens[b.planted].min()
    assert np.median(rnd) < 60


def test_lognormal_tail():
    b = wl.gen_config(3, n_pairs=50_000)
    frac = np.mean(b.r_lens >= 1600)
    assert 0.005 < frac < 0.02
    assert abs(np.median(b.q_lens) - 150) < 5 and abs(np.median(b.r_lens) - 400) < 10


def test_serving_requests():
    reqs = wl.serving_requests(40, rate_per_s=100.0)
    assert len(reqs) == 40
    sizes = np.array([r.batch.n_pairs for r in reqs])
    assert sizes.min() >= 1 and sizes.max() <= 4096
    arr = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(arr) >= 0)
    kinds = {r.kind for r in reqs}
    assert kinds == {"dna", "protein"}
