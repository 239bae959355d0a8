"""Pins of the set-level model of the paper's method (oracle/paper_method.py).

* Section 4, equations del / undo-del, and Section 5.1: deletions and
  undeletions must be properly nested; undoing them in reverse order
  restores the list exactly.  After unwind every node keeps the neighbours it
  had when it was deleted: the nearest smaller and larger element among the
  positions before it (the unwind links the GPU path computes directly).
* Section 5, Fig. block-if: the model's (L, s) after each operation.
* Section 6.3, equation (inv): before every output s_A + s_B = h and
  S_A u S_B = H_AB (the h smallest elements of the window).
* Section 6.3, Lemma 1 and its case-analysis table: with S_A non-empty, the
  small sets after delete/undelete and after the advance follow one of the
  table's rows.  Reading of the table used here: the first group holds when
  the deleted a_A is small (a_A <= p_A), the second when it is large
  (p_A < a_A); the second group's row "p_B < a_B" holds as printed only when
  also p_A < a_B; for p_B < a_B < p_A the advance goes to B instead
  (S_A'' = S_A', S_B'' = S_B' + a_B), which this test checks as an extra case.
* The output equals the plain definition (oracle.median_filter), including
  the index of the median element, on random inputs with heavy ties and with
  n not a multiple of k.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle.paper_method import DancingLinks, RankBlock, sort_median, stable_order
from signals import paper_generator


def test_properly_nested_delete_undelete_restores_list():
    rng = np.random.default_rng(0)
    alpha = list(rng.integers(0, 50, size=31))
    dl = DancingLinks(alpha)
    before = (list(dl.prev), list(dl.next), dl.walk())
    assert dl.walk() == sorted(range(31), key=lambda t: (alpha[t], t))
    # the example of Section 5.1: delete 15, delete 3, undelete 3, undelete 15
    dl.remove(15)
    dl.remove(3)
    assert 15 not in dl.walk() and 3 not in dl.walk()
    dl.restore(3)
    dl.restore(15)
    assert (list(dl.prev), list(dl.next), dl.walk()) == before
    # an order that is not properly nested can corrupt the list: with three
    # consecutive elements u < v < w removed in that order, restoring u, w, v
    # leaves u and v unreachable
    u, v, w = before[2][10:13]
    for e in (u, v, w):
        dl.remove(e)
    for e in (u, w, v):
        dl.restore(e)
    assert dl.walk() != before[2] and u not in dl.walk()


@pytest.mark.parametrize("seed", range(6))
def test_unwind_leaves_the_links_of_earlier_neighbours(seed):
    """delete(k-1), ..., delete(0), then undelete(0), ..., undelete(k-1): at
    undelete(i) node i is relinked between the nearest smaller and the
    nearest larger of positions 0 .. i-1 (sentinel k where there is none),
    and the list is then positions 0 .. i in sorted order."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 40))
    alpha = list(rng.integers(0, 8 if seed % 2 else 1000, size=k))
    dl = DancingLinks(alpha)
    for i in reversed(range(k)):
        dl.remove(i)
    assert dl.walk() == []
    _, rank = stable_order(alpha)
    for i in range(k):
        lower = [p for p in range(i) if rank[p] < rank[i]]
        upper = [p for p in range(i) if rank[p] > rank[i]]
        assert dl.prev[i] == (max(lower, key=rank.__getitem__) if lower else k)
        assert dl.next[i] == (min(upper, key=rank.__getitem__) if upper else k)
        dl.restore(i)
        assert dl.walk() == sorted(range(i + 1), key=lambda t: (alpha[t], t))


def test_block_interface_semantics():
    """Fig. block-if on a small block: construct, delete (s = max(0, s-1)),
    undelete (s unchanged), advance, peek (first large or +inf), unwind."""
    alpha = [7, 3, 9, 3, 1]                    # sorted positions: 4, 1, 3, 0, 2
    b = RankBlock(alpha, 2)
    assert b.small() == 2 and b.small_set() == {4, 1} and b.peek() == 3 and b.first_large() == 3
    b.delete(0)                                # a large element: s = 1
    assert b.small() == 1 and b.small_set() == {4} and b.first_large() == 1
    b.delete(4)                                # a small element: s = 0
    assert b.small() == 0 and b.peek() == 3 and b.first_large() == 1
    b.undelete(4)                              # back in L, s unchanged: 1 is now first
    assert b.small() == 0 and b.first_large() == 4 and b.peek() == 1
    b.advance()
    b.advance()
    assert b.small_set() == {4, 1} and b.first_large() == 3
    with pytest.raises(AssertionError):
        b.undelete(4)                          # not the latest deletion
    b.undelete(0)
    b.unwind()
    assert b.members() == set() and b.small() == 0 and b.peek() == float("inf")


def _ordkey(trace_step, side, idx):
    alpha = trace_step["alphaA"] if side == "A" else trace_step["alphaB"]
    return (alpha[idx], 0 if side == "A" else 1, idx)


def _check_invariant(step):
    h = step["h"]
    post = step["post"]
    assert step["sA"] + step["sB"] == h
    window = ([_ordkey(step, "A", i) for i in post["LA"]]
              + [_ordkey(step, "B", i) for i in post["LB"]])
    hab = set(sorted(window)[:h])
    small = ({_ordkey(step, "A", i) for i in post["SA"]}
             | {_ordkey(step, "B", i) for i in post["SB"]})
    assert small == hab


@pytest.mark.parametrize("gen", ["r-small", "r-large", "r-asc", "r-desc", "r-block"])
@pytest.mark.parametrize("k", [1, 3, 5, 9, 17])
def test_invariant_and_definition(gen, k):
    for n in (k, k + 1, 2 * k - 1, 2 * k, 5 * k + 2):
        x = paper_generator(gen, n, seed=n * 31 + k).tolist()
        trace = []
        y, arg = sort_median(x, k, trace=trace)
        ref, ref_arg = oracle.median_filter(np.array(x, dtype=np.int32), k)
        assert y == ref.tolist()
        assert arg == ref_arg.tolist()
        for step in trace:
            _check_invariant(step)


def test_ties_between_blocks_prefer_older_block():
    x = [5, 5, 5, 5, 5, 5, 5, 5, 5]
    y, arg = sort_median(x, 3)
    assert y == [5] * 7
    assert arg == [1, 2, 3, 4, 5, 6, 7]


def _classify(step):
    """Return (row, predicted dict) for one step whose S_A was non-empty."""
    A, B = "A", "B"
    pre, i = step["pre"], step["i"]
    key = lambda s, t: _ordkey(step, s, t)
    SA = sorted(key(A, t) for t in pre["SA"])
    SB = sorted(key(B, t) for t in pre["SB"])
    LA = sorted(key(A, t) for t in pre["LA"])
    LB = sorted(key(B, t) for t in pre["LB"])
    NEG, POS = (-np.inf,), (np.inf,)
    aA, aB = key(A, i), key(B, i)
    pA = SA[-1]
    qA = next((e for e in LA if e not in SA), POS)
    pB = SB[-1] if SB else NEG
    qB = next((e for e in LB if e not in SB), POS)
    sA, sB = set(SA), set(SB)
    if aA <= pA:                                   # deleted element is small
        if aB < pB:
            return 1, dict(mA=sA - {aA}, mB=sB - {pB} | {aB}, pA=sA - {aA}, pB=sB - {pB} | {aB} | {pB})
        if aB < min(qA, qB):
            return 2, dict(mA=sA - {aA}, mB=sB, pA=sA - {aA}, pB=sB | {aB})
        if qB < min(qA, aB):
            return 3, dict(mA=sA - {aA}, mB=sB, pA=sA - {aA}, pB=sB | {qB})
        return 4, dict(mA=sA - {aA}, mB=sB, pA=sA - {aA} | {qA}, pB=sB)
    # deleted element is large
    if pB < aB:
        if pA < aB:
            return 5, dict(mA=sA - {pA}, mB=sB, pA=sA, pB=sB)
        return "5'", dict(mA=sA - {pA}, mB=sB, pA=sA - {pA}, pB=sB | {aB})
    if pB < pA:
        return 6, dict(mA=sA - {pA}, mB=sB - {pB} | {aB}, pA=sA - {pA}, pB=sB - {pB} | {aB} | {pB})
    return 7, dict(mA=sA - {pA}, mB=sB - {pB} | {aB}, pA=sA, pB=sB - {pB} | {aB})


def test_case_analysis_table():
    seen = {}
    rng = np.random.default_rng(5)
    for trial in range(400):
        k = int(rng.choice([3, 5, 7, 9]))
        n = k * int(rng.integers(2, 6))
        x = rng.integers(0, 3 * k, size=n).tolist()
        trace = []
        sort_median(x, k, trace=trace)
        for step in trace:
            if not step["pre"]["SA"]:
                # first case of the proof: S_A empty, nothing moves to A
                assert not step["post"]["SA"]
                continue
            row, pred = _classify(step)
            key = lambda s, t: _ordkey(step, s, t)
            mid_A = {key("A", t) for t in step["mid"]["SA"]}
            mid_B = {key("B", t) for t in step["mid"]["SB"]}
            post_A = {key("A", t) for t in step["post"]["SA"]}
            post_B = {key("B", t) for t in step["post"]["SB"]}
            assert mid_A == pred["mA"] and mid_B == pred["mB"], (row, step)
            assert post_A == pred["pA"] and post_B == pred["pB"], (row, step)
            seen[row] = seen.get(row, 0) + 1
    assert set(seen) == {1, 2, 3, 4, 5, "5'", 6, 7}, seen


def test_exhaustive_small_blocks():
    """Every sequence over {0,1,2} of length 6 with k = 3 (two full blocks)."""
    for seq in itertools.product((0, 1, 2), repeat=6):
        y, arg = sort_median(list(seq), 3)
        ref, ref_arg = oracle.median_filter(np.array(seq, dtype=np.int32), 3)
        assert y == ref.tolist() and arg == ref_arg.tolist()
