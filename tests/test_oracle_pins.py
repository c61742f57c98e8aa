"""Pins of the CPU oracle against what the paper and the mathematics fix.

The oracle is the parity reference for the CUDA library, so it is checked
here against things other than itself: hand-worked examples (tests/golden/),
special cases that reduce to a library routine (numpy sums, integer matrix
products, sorts), brute force over all subsets on tiny inputs, closed forms
and invariants.  Each test names the part of the paper it pins: Alg. 1
(overlap), Alg. 2 (inhibition), the Section 1.1 learning rule.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1608_01966_gb300 import synth
from conftest import GOLDEN

F32 = np.float32


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------- golden ----

def test_golden_two_frame_example():
    """Alg. 1 + Alg. 2 + learning, hand-worked (tests/golden/sp_two_frame_example.json)."""
    g = _load("sp_two_frame_example.json")
    idx = np.array(g["idx"], np.uint32)
    perm = np.array(g["perm"], np.float32)
    boost = np.array(g["boost"], np.float32)
    C, S = idx.shape
    p = oracle.params(C, S, g["n_in"], thr=g["connect_threshold"], inc=g["perm_inc"],
                      dec=g["perm_dec"], min_overlap=g["min_overlap"],
                      k=g["winners_set_size"])
    for x, e in zip(g["frames"], g["expected"]):
        x = np.array(x, np.uint8)
        raw, ov = oracle.overlap(idx, perm, boost, x, g["connect_threshold"], g["min_overlap"])
        np.testing.assert_array_equal(raw, e["raw"])
        np.testing.assert_array_equal(ov, np.array(e["ov"], np.float32))
        act = oracle.inhibit_global(ov, g["winners_set_size"])
        np.testing.assert_array_equal(act, e["active"])
        oracle.learn(idx, perm, x, act, g["perm_inc"], g["perm_dec"])
        np.testing.assert_array_equal(perm, np.array(e["perm_after"], np.float32))
    # the same two frames through the sequence driver
    perm2 = np.array(g["perm"], np.float32)
    act2 = oracle.run(p, idx, perm2, boost, np.array(g["frames"], np.uint8), True)
    np.testing.assert_array_equal(act2, [e["active"] for e in g["expected"]])
    np.testing.assert_array_equal(perm2, np.array(g["expected"][-1]["perm_after"], np.float32))


def test_golden_inhibition_grid():
    """Alg. 2, global and local (clipped window), hand-worked."""
    g = _load("inhibition_grid_example.json")
    ov = np.array(g["ov"], np.float32)
    for case in g["cases"]:
        if case["mode"] == "local":
            act = oracle.inhibit_local(ov, g["grid_w"], g["grid_h"], case["k"], case["radius"])
        else:
            act = oracle.inhibit_global(ov, case["k"])
        np.testing.assert_array_equal(act, case["active"], err_msg=case["work"])


# ------------------------------------------------------------- Alg. 1 pins ---

def _random_sp(seed, C, S, n_in, lo=0.1, hi=0.3):
    idx = synth.pool_uniform(synth.derive_seed(seed, 1, 0), C, S, n_in)
    perm = synth.perm_uniform(synth.derive_seed(seed, 2, 0), (C, S), lo, hi)
    return idx, perm


def test_overlap_threshold_zero_is_pool_popcount():
    """With threshold 0 every potential synapse is connected, so the raw overlap
    is the number of active input bits in the column's pool."""
    idx, perm = _random_sp(1, 200, 24, 500)
    x = synth.frame_bernoulli(5, 500, 0.3)
    raw, _ = oracle.overlap(idx, perm, np.ones(200, F32), x, 0.0, 0)
    np.testing.assert_array_equal(raw, x[idx].sum(axis=1))


def test_overlap_dense_pool_is_integer_matmul():
    """Dense pools (every column sees the whole input): raw = Conn . x, an integer
    matrix-vector product with Conn[c, i] = [perm[c, i] >= thr]."""
    n = 96
    idx = synth.pool_dense(40, n)
    perm = synth.perm_uniform(3, (40, n), 0.0, 0.4)
    X = np.stack([synth.frame_bernoulli(10 + t, n, 0.4) for t in range(8)])
    conn = (perm >= F32(0.2)).astype(np.int64)
    ref = X.astype(np.int64) @ conn.T  # [frames, C]
    for t in range(8):
        raw, _ = oracle.overlap(idx, perm, np.ones(40, F32), X[t], 0.2, 0)
        np.testing.assert_array_equal(raw, ref[t])


def test_overlap_threshold_above_one_no_connection():
    idx, perm = _random_sp(2, 50, 16, 256, 0.0, 1.0)
    x = np.ones(256, np.uint8)
    raw, ov = oracle.overlap(idx, perm, np.ones(50, F32), x, 1.5, 0)
    assert (raw == 0).all() and (ov == 0).all()
    assert oracle.inhibit_global(ov, 10).sum() == 0


def test_overlap_extremes_and_bounds():
    """All-ones input counts every connected synapse; all-zeros counts none;
    0 <= raw <= #connected <= S."""
    idx, perm = _random_sp(4, 128, 32, 300)
    nconn = (perm >= F32(0.2)).sum(axis=1)
    raw1, _ = oracle.overlap(idx, perm, np.ones(128, F32), np.ones(300, np.uint8), 0.2, 0)
    np.testing.assert_array_equal(raw1, nconn)
    raw0, _ = oracle.overlap(idx, perm, np.ones(128, F32), np.zeros(300, np.uint8), 0.2, 0)
    assert (raw0 == 0).all()
    for s in range(5):
        x = synth.frame_bernoulli(s, 300, 0.2)
        raw, _ = oracle.overlap(idx, perm, np.ones(128, F32), x, 0.2, 0)
        assert (raw >= 0).all() and (raw <= nconn).all()


def test_overlap_subadditive_and_monotone():
    """Counting is monotone in the input and additive over disjoint inputs."""
    idx, perm = _random_sp(6, 64, 20, 200)
    b = np.ones(64, F32)
    a = synth.frame_bernoulli(1, 200, 0.3)
    c = synth.frame_bernoulli(2, 200, 0.3)
    ra, _ = oracle.overlap(idx, perm, b, a, 0.2, 0)
    rc, _ = oracle.overlap(idx, perm, b, c, 0.2, 0)
    r_or, _ = oracle.overlap(idx, perm, b, a | c, 0.2, 0)
    r_and, _ = oracle.overlap(idx, perm, b, a & c, 0.2, 0)
    np.testing.assert_array_equal(r_or + r_and, ra + rc)
    assert (r_or >= np.maximum(ra, rc)).all()


def test_min_overlap_and_boost():
    """Alg. 1's tail: below min_overlap -> 0; otherwise the exact fp32 product
    of the count and the boost (one rounding)."""
    idx, perm = _random_sp(7, 300, 32, 256)
    x = synth.frame_bernoulli(3, 256, 0.5)
    boost = synth.perm_uniform(8, (300,), 0.5, 3.0)
    raw, _ = oracle.overlap(idx, perm, np.ones(300, F32), x, 0.2, 0)
    for m in (0, 1, 3, 5):
        raw_m, ov = oracle.overlap(idx, perm, boost, x, 0.2, m)
        np.testing.assert_array_equal(raw_m, raw)
        keep = raw >= m
        assert (ov[~keep] == 0).all()
        np.testing.assert_array_equal(ov[keep], raw[keep].astype(F32) * boost[keep])
        # with unit boost the boosted overlap is the count itself
        _, ov1 = oracle.overlap(idx, perm, np.ones(300, F32), x, 0.2, m)
        np.testing.assert_array_equal(ov1[keep], raw[keep].astype(F32))


def test_overlap_rejects_out_of_range_index():
    idx = np.array([[0, 9]], np.uint32)
    with pytest.raises(ValueError):
        oracle.overlap(idx, np.ones((1, 2), F32), np.ones(1, F32), np.ones(8, np.uint8), 0.2, 0)


# ------------------------------------------------------------- Alg. 2 pins ---

def _unique_top_set(ov, k):
    """Brute force over all subsets: the winner set is the unique subset of
    nonzero columns of size min(k, #nonzero) whose every member beats every
    nonzero non-member under (ov desc, index asc)."""
    C = len(ov)
    nz = [c for c in range(C) if ov[c] > 0]
    size = min(k, len(nz))
    beats = lambda a, b: ov[a] > ov[b] or (ov[a] == ov[b] and a < b)
    found = [set(W) for W in itertools.combinations(nz, size)
             if all(beats(w, l) for w in W for l in nz if l not in W)]
    assert len(found) == 1
    return found[0]


def test_inhibit_global_brute_force_subsets_with_ties():
    rng = np.random.default_rng(1)
    for trial in range(300):
        C = int(rng.integers(1, 9))
        ov = rng.integers(0, 4, C).astype(F32)  # heavy ties, many zeros
        k = int(rng.integers(0, C + 2))
        act = oracle.inhibit_global(ov, k)
        assert set(np.flatnonzero(act)) == _unique_top_set(ov, k)


def test_inhibit_global_equals_lexsort():
    """Global inhibition = the first k entries of a lexicographic sort on
    (-ov, index), restricted to nonzero overlaps (numpy's lexsort)."""
    rng = np.random.default_rng(2)
    for trial in range(50):
        C = int(rng.integers(1, 3000))
        ov = (rng.integers(0, 30, C) * rng.choice([1.0, 1.25, 0.5], C)).astype(F32)
        k = int(rng.integers(1, 200))
        order = np.lexsort((np.arange(C), -ov))
        order = order[ov[order] > 0][:k]
        ref = np.zeros(C, np.uint8)
        ref[order] = 1
        np.testing.assert_array_equal(oracle.inhibit_global(ov, k), ref)


def test_inhibit_local_rank_by_sort_in_window():
    """Local inhibition restated with a sort: c wins iff ov[c] > 0 and its
    position in the sorted (-ov, index) list of its clipped window is < k."""
    rng = np.random.default_rng(3)
    for trial in range(40):
        gw, gh = int(rng.integers(1, 9)), int(rng.integers(1, 9))
        r = int(rng.integers(0, 4))
        k = int(rng.integers(1, 6))
        ov = rng.integers(0, 4, gw * gh).astype(F32)
        act = oracle.inhibit_local(ov, gw, gh, k, r)
        for j in range(gh):
            for i in range(gw):
                c = j * gw + i
                win = [jj * gw + ii for jj in range(max(0, j - r), min(gh, j + r + 1))
                       for ii in range(max(0, i - r), min(gw, i + r + 1))]
                ranked = sorted(win, key=lambda d: (-ov[d], d))
                assert act[c] == int(ov[c] > 0 and ranked.index(c) < k)


def test_inhibit_local_special_cases():
    rng = np.random.default_rng(4)
    gw, gh = 12, 10
    ov = rng.integers(0, 6, gw * gh).astype(F32)
    # a window that covers the whole grid is global inhibition
    for k in (1, 5, 17):
        np.testing.assert_array_equal(oracle.inhibit_local(ov, gw, gh, k, 12),
                                      oracle.inhibit_global(ov, k))
    # k at least the window size: every nonzero column wins
    np.testing.assert_array_equal(oracle.inhibit_local(ov, gw, gh, 9, 1),
                                  (ov > 0).astype(np.uint8))
    np.testing.assert_array_equal(oracle.inhibit_local(ov, gw, gh, 1, 0),
                                  (ov > 0).astype(np.uint8))


def test_inhibit_invariants_global():
    rng = np.random.default_rng(5)
    for trial in range(100):
        C = int(rng.integers(1, 2000))
        ov = rng.integers(0, 12, C).astype(F32)
        k = int(rng.integers(0, 100))
        act = oracle.inhibit_global(ov, k).astype(bool)
        assert act.sum() == min(k, int((ov > 0).sum()))
        assert (ov[act] > 0).all()
        if act.any() and (~act & (ov > 0)).any():
            assert ov[act].min() >= ov[~act].max()


def test_paper_literal_reading_agrees_without_boundary_ties():
    """The word-for-word Alg. 2 (strict '>' against the n-th largest of the
    other columns, floor 1) equals the rank count when the top k+1 values are
    distinct and exceed 1, and drops the whole tie at the boundary otherwise."""
    ov = np.array([9, 3, 7, 5, 2, 8], F32)
    np.testing.assert_array_equal(oracle.inhibit_paper_literal(ov, 3),
                                  oracle.inhibit_global(ov, 3))
    tie = np.array([9, 5, 7, 5, 2, 8], F32)  # third/fourth place tied at 5
    np.testing.assert_array_equal(oracle.inhibit_paper_literal(tie, 4), [1, 0, 1, 0, 0, 1])
    np.testing.assert_array_equal(oracle.inhibit_global(tie, 4), [1, 1, 1, 0, 0, 1])


# ----------------------------------------------------------- learning pins ---

def test_learning_closed_form_per_synapse():
    """Section 1.1 learning: every potential synapse of a winner becomes
    min(1, fl(p + inc)) if its input bit is 1, else max(0, fl(p - dec)); other
    columns are untouched.  numpy float32 arithmetic is IEEE round-to-nearest."""
    idx, perm0 = _random_sp(9, 150, 40, 400, 0.0, 1.0)
    perm0[0, :4] = [1.0, 0.99, 0.0, 0.01]
    x = synth.frame_bernoulli(4, 400, 0.5)
    x[idx[0, :4]] = [1, 1, 0, 0]
    active = (np.arange(150) % 3 == 0).astype(np.uint8)
    inc, dec = F32(0.05), F32(0.02)
    perm = perm0.copy()
    oracle.learn(idx, perm, x, active, float(inc), float(dec))
    bit = x[idx].astype(bool)
    up = np.minimum(F32(1), perm0 + inc)
    down = np.maximum(F32(0), perm0 - dec)
    ref = np.where(bit, up, down)
    rows = active.astype(bool)
    np.testing.assert_array_equal(perm[rows], ref[rows])
    np.testing.assert_array_equal(perm[~rows], perm0[~rows])
    assert perm[0, 0] == 1.0 and perm[0, 1] == 1.0 and perm[0, 2] == 0.0 and perm[0, 3] == 0.0
    assert perm.min() >= 0 and perm.max() <= 1


def test_learning_identities():
    idx, perm0 = _random_sp(10, 80, 16, 128)
    x = synth.frame_bernoulli(1, 128, 0.4)
    act = np.ones(80, np.uint8)
    p = perm0.copy()
    oracle.learn(idx, p, x, act, 0.0, 0.0)
    np.testing.assert_array_equal(p, perm0)  # inc = dec = 0 -> unchanged
    p = perm0.copy()
    oracle.learn(idx, p, np.ones(128, np.uint8), act, 0.05, 0.02)
    assert (p > perm0).all()  # all-ones input: every permanence rises
    p = perm0.copy()
    oracle.learn(idx, p, np.zeros(128, np.uint8), act, 0.05, 0.02)
    assert (p < perm0).all()  # all-zeros input: every permanence falls
    p = perm0.copy()
    oracle.learn(idx, p, x, np.zeros(80, np.uint8), 0.05, 0.02)
    np.testing.assert_array_equal(p, perm0)  # no winner -> nothing moves


# ------------------------------------------------------------ sequences ------

def test_sequence_invariants_small_config():
    """256 columns x 16 synapses over 32x32 Bernoulli(0.1) frames, 100 frames
    inference then 100 frames learning (inc 0.05, dec 0.02)."""
    C, S, n = 256, 16, 1024
    idx, perm = _random_sp(0x5EED0001, C, S, n)
    boost = np.ones(C, F32)
    frames = np.stack([synth.frame_bernoulli(synth.derive_seed(0x5EED0001, 3, t), n, 0.1)
                       for t in range(200)])
    p = oracle.params(C, S, n, 0.2, 0.05, 0.02, 4, 10)
    perm0 = perm.copy()
    act_inf, ov_inf = oracle.run(p, idx, perm, boost, frames[:100], False, want_ov=True)
    np.testing.assert_array_equal(perm, perm0)  # inference never changes state
    act_l = oracle.run(p, idx, perm, boost, frames[100:], True)
    for act, ov in ((act_inf, ov_inf),):
        assert (act.sum(axis=1) <= 10).all()
        assert ((ov == 0) | (ov >= 4)).all()
    assert (act_l.sum(axis=1) <= 10).all()
    assert perm.min() >= 0 and perm.max() <= 1
    # only columns that ever won changed
    changed = (perm != perm0).any(axis=1)
    assert not (changed & ~act_l.any(axis=0).astype(bool)).any()
    # statistical sanity: mean raw overlap ~ S * P(connected) * p = 16 * 0.5 * 0.1
    raw_all = np.stack([oracle.overlap(idx, perm0, boost, frames[t], 0.2, 0)[0]
                        for t in range(100)])
    assert abs(raw_all.mean() - 0.8) < 0.1


def test_sequence_learning_order_matters():
    """Frame t+1 sees the permanences learned on frame t: running frames one at
    a time through overlap / inhibition / learning equals the sequence driver,
    and differs from applying all learning after the last frame."""
    C, S, n = 64, 16, 256
    idx, perm = _random_sp(21, C, S, n, 0.15, 0.25)
    boost = np.ones(C, F32)
    frames = np.stack([synth.frame_bernoulli(100 + t, n, 0.3) for t in range(30)])
    p = oracle.params(C, S, n, 0.2, 0.05, 0.02, 2, 6)
    seq_perm = perm.copy()
    act_seq = oracle.run(p, idx, seq_perm, boost, frames, True)
    step_perm = perm.copy()
    for t in range(30):
        _, ov = oracle.overlap(idx, step_perm, boost, frames[t], 0.2, 2)
        a = oracle.inhibit_global(ov, 6)
        np.testing.assert_array_equal(a, act_seq[t])
        oracle.learn(idx, step_perm, frames[t], a, 0.05, 0.02)
    np.testing.assert_array_equal(step_perm, seq_perm)
    frozen = perm.copy()
    act_frozen = oracle.run(p, idx, frozen, boost, frames, False)
    assert (act_frozen != act_seq).any()


# ---------------------------------------------------------- duty cycles -----

def test_duty_cycle_closed_forms():
    """d <- d + (a - d)/P: period 1 copies the activity; a constant activity of 1
    from d = 0 gives 1 - (1 - 1/P)^n up to n fp32 roundings."""
    d = np.full(6, 0.3, F32)
    a = np.array([1, 0, 1, 0, 0, 1], np.uint8)
    oracle.duty_update(d, a, 1.0)
    np.testing.assert_array_equal(d, a.astype(F32))
    P, n = 50.0, 200
    d = np.zeros(3, F32)
    for _ in range(n):
        oracle.duty_update(d, np.array([1, 0, 1], np.uint8), P)
    ref = 1 - (1 - 1 / P) ** n
    assert abs(float(d[0]) - ref) < n * 2 ** -23
    assert d[1] == 0 and d[0] == d[2]


def test_step_dispatches_the_paper_literal_reading():
    """orc_step with inhibition 2 applies the word-for-word Alg. 2."""
    idx, perm = _random_sp(30, 80, 16, 256, 0.2, 0.2)
    x = synth.frame_bernoulli(31, 256, 0.5)
    p = oracle.params(80, 16, 256, 0.2, 0.05, 0.02, 1, 7, inhibition=2)
    _, ov = oracle.overlap(idx, perm, np.ones(80, F32), x, 0.2, 1)
    act = oracle.run(p, idx, perm.copy(), np.ones(80, F32), x[None, :], False)[0]
    np.testing.assert_array_equal(act, oracle.inhibit_paper_literal(ov, 7))
