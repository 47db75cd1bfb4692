"""Pins for the oracle's bounded edit distance (Methods, "Local Alignment").

The paper's EditDistance(Read, Reference[p], d_limit) returns the distance when it is
at most d_limit and a special value otherwise, in O(n d_limit) time by tracking the
farthest reach per diagonal.  The oracle's reading: the start is anchored at p and
the end is free in the reference (min over prefixes).  These tests pin the oracle's
farthest-reach implementation (ed_lv) and its textbook table (ed_dp) to things other
than themselves:

* a breadth-first search over edit operations (edit distance as a shortest path
  between strings), exhaustive over a binary alphabet;
* hand-worked values;
* the band theorem: ed_lv(L) == (ed_dp if ed_dp <= L else over), exhaustive over
  ACGT for short strings and random long pairs at 0-30% error with limits up to 800;
* Myers' bit-vector method (anchored start, free end), written here independently:
  exhaustive over short ACGT strings and random pairs up to 1.2 kb.
"""
import itertools
import random
from collections import deque

import numpy as np
import pytest

import oracle


def _all_strings(alphabet, maxlen):
    out = []
    for n in range(maxlen + 1):
        out.extend("".join(p) for p in itertools.product(alphabet, repeat=n))
    return out


def _bfs_distances(x, alphabet, radius, maxlen):
    """Shortest number of single-character edits from x to every string within radius."""
    dist = {x: 0}
    q = deque([x])
    while q:
        u = q.popleft()
        d = dist[u]
        if d == radius:
            continue
        nbrs = set()
        for i in range(len(u)):
            nbrs.add(u[:i] + u[i + 1:])
            for a in alphabet:
                if a != u[i]:
                    nbrs.add(u[:i] + a + u[i + 1:])
        if len(u) < maxlen:
            for i in range(len(u) + 1):
                for a in alphabet:
                    nbrs.add(u[:i] + a + u[i:])
        for v in nbrs:
            if v not in dist:
                dist[v] = d + 1
                q.append(v)
    return dist


def test_dp_matches_edit_graph_bfs_binary_alphabet():
    # every X of length <= 5 and every T of length <= 6 over {A, C}
    alphabet = "AC"
    xs = _all_strings(alphabet, 5)
    ts = _all_strings(alphabet, 6)
    pairs_x, pairs_t, expect = [], [], []
    for x in xs:
        # deleting all of x reaches the empty prefix, so the answer is <= |x|
        dist = _bfs_distances(x, alphabet, radius=len(x), maxlen=len(x) + 6)
        for t in ts:
            best = min(dist.get(t[:j], 99) for j in range(len(t) + 1))
            pairs_x.append(x)
            pairs_t.append(t)
            expect.append(best)
    lv, dp = oracle.ed_pairs(pairs_x, pairs_t, [len(x) for x in pairs_x])
    assert np.array_equal(dp, np.array(expect, dtype=np.int32))
    assert np.array_equal(lv, dp)


@pytest.mark.parametrize("x,t,d", [
    ("ACGT", "ACGT", 0),
    ("ACGT", "ACGTTTTT", 0),          # free end in the reference
    ("ACGT", "TACGT", 1),             # start is anchored: one extra reference base costs 1
    ("ACGT", "AGT", 1),               # one deletion from the reference's view
    ("ACGT", "ACCGT", 1),             # one insertion in the reference
    ("AAAA", "CCCC", 4),              # all substitutions (or delete all four)
    ("", "ACGT", 0),
    ("ACGT", "", 4),
    ("GATTACA", "GATACA", 1),         # one T fewer in the reference
    ("TTTT", "TTTGA", 1),             # best prefix TTT: one deletion
])
def test_hand_worked_values(x, t, d):
    assert oracle.ed_dp(x, t) == d
    assert oracle.ed_lv(x, t, d) == d
    if d > 0:
        assert oracle.ed_lv(x, t, d - 1) == -1


def test_lv_equals_dp_exhaustive_acgt():
    xs = _all_strings("ACGT", 4)
    ts = _all_strings("ACGT", 5)
    rng = random.Random(7)
    px, pt, pl = [], [], []
    for x in xs:
        for t in ts:
            px.append(x)
            pt.append(t)
            pl.append(rng.randint(0, 5))
    lv, dp = oracle.ed_pairs(px, pt, pl)
    L = np.array(pl)
    expect = np.where(dp <= L, dp, -1)
    assert np.array_equal(lv, expect)


def _mutate(rng, s, rate, indel_frac=0.2):
    out = []
    i = 0
    while i < len(s):
        if rng.random() < rate:
            if rng.random() < indel_frac:
                if rng.random() < 0.5:
                    out.append(rng.choice("ACGT"))  # insertion
                    continue
                i += 1  # deletion
                continue
            out.append(rng.choice([a for a in "ACGT" if a != s[i]]))
            i += 1
            continue
        out.append(s[i])
        i += 1
    return "".join(out)


@pytest.mark.parametrize("m,rate", [(100, 0.0), (100, 0.02), (100, 0.1), (250, 0.3),
                                    (1000, 0.05), (3000, 0.1)])
def test_lv_equals_dp_random_pairs(m, rate):
    rng = random.Random(m * 1000 + int(rate * 100))
    px, pt, pfull, pl = [], [], [], []
    for _ in range(4 if m >= 1000 else 40):
        ref = "".join(rng.choice("ACGT") for _ in range(m + m // 2 + 10))
        x = _mutate(rng, ref[:m], rate)
        for L in (0, 1, 3, 8, 20, 64, max(1, int(rate * m * 1.5))):
            px.append(x)
            pt.append(ref[: len(x) + L])  # what the aligner hands the distance: |X| + L bases
            pfull.append(ref)
            pl.append(L)
    lv, _ = oracle.ed_pairs(px, pt, pl, with_dp=False)
    # the full table on the whole reference (no text cut) decides the truth
    _, dp_full = oracle.ed_pairs(px, pfull, pl)
    L = np.array(pl)
    expect = np.where(dp_full <= L, dp_full, -1)
    assert np.array_equal(lv, expect)


def test_lv_long_read_limit_800():
    rng = random.Random(11)
    ref = "".join(rng.choice("ACGT") for _ in range(10_000 + 900))
    x = _mutate(rng, ref[:10_000], 0.05)
    d = oracle.ed_dp(x, ref)
    assert 300 < d < 800
    assert oracle.ed_lv(x, ref[: len(x) + 801], 801) == d
    assert oracle.ed_lv(x, ref[: len(x) + d], d) == d
    assert oracle.ed_lv(x, ref[: len(x) + d], d - 1) == -1


def test_band_theorem_text_cut():
    # a distance <= L never needs more than |X| + L reference bases
    rng = random.Random(3)
    for _ in range(200):
        m = rng.randint(1, 60)
        ref = "".join(rng.choice("ACGT") for _ in range(2 * m + 20))
        x = _mutate(rng, ref[:m], 0.15)
        d_full = oracle.ed_dp(x, ref)
        for L in range(0, 8):
            d_cut = oracle.ed_dp(x, ref[: len(x) + L])
            if d_full <= L:
                assert d_cut == d_full
            else:
                assert d_cut > L


def _bitparallel_prefix_distance(x: str, t: str) -> int:
    """min over j of Lev(x, t[0..j)) by the bit-vector method of Myers (1999) in
    Hyyro's formulation: one machine word (here a Python int) per text column holds
    the vertical differences of the column; the top row's horizontal difference is
    +1 per column because the start is anchored (D[0][j] = j).  Written independently
    of the oracle as a second way to the same integer."""
    m = len(x)
    if m == 0:
        return 0
    mask, high = (1 << m) - 1, 1 << (m - 1)
    peq = {c: sum(1 << i for i, xc in enumerate(x) if xc == c) for c in "ACGT"}
    pv, mv, score = mask, 0, m
    best = score
    for c in t:
        eq = peq.get(c, 0)
        xv = eq | mv
        xh = ((((eq & pv) + pv) & mask) ^ pv) | eq
        ph = (mv | ~(xh | pv)) & mask
        mh = pv & xh
        if ph & high:
            score += 1
        elif mh & high:
            score -= 1
        ph = ((ph << 1) | 1) & mask
        mh = (mh << 1) & mask
        pv = (mh | ~(xv | ph)) & mask
        mv = ph & xv
        best = min(best, score)
    return best


def test_table_equals_bit_parallel_exhaustive():
    # every pair over ACGT with |x| <= 3 and |t| <= 5, and |x| = 4 with |t| <= 4
    for lx in range(0, 5):
        for x in ("".join(p) for p in itertools.product("ACGT", repeat=lx)):
            for lt in range(0, 6 if lx <= 3 else 5):
                for t in ("".join(p) for p in itertools.product("ACGT", repeat=lt)):
                    assert oracle.ed_dp(x, t) == _bitparallel_prefix_distance(x, t), (x, t)


@pytest.mark.parametrize("m,rate", [(60, 0.05), (150, 0.1), (400, 0.2), (1200, 0.05)])
def test_table_and_reach_equal_bit_parallel_random(m, rate):
    rng = random.Random(7 * m + int(rate * 100))
    for _ in range(40):
        x = "".join(rng.choice("ACGT") for _ in range(m))
        t = _mutate(rng, x, rate) + "".join(rng.choice("ACGT") for _ in range(30))
        if rng.random() < 0.3:  # an unrelated window
            t = "".join(rng.choice("ACGT") for _ in range(len(t)))
        d = _bitparallel_prefix_distance(x, t)
        assert oracle.ed_dp(x, t) == d
        L = rng.randint(0, m // 3)
        assert oracle.ed_lv(x, t, L) == (d if d <= L else -1)
