"""A set-level model of the paper's median-filter method -- TEST INFRASTRUCTURE ONLY.

Only the tests import this module; no product code does, and it never
supplies expected values to the CUDA path (those come from the plain
definition in ``mf_oracle.c``).  It exists to pin the reasoning behind the
method, written from the paper's definitions rather than from its printed
code:

* Section 5 defines a block data structure as a tuple (alpha, pi, L, s): a
  block of input, the permutation that sorts it, a list L holding a subset of
  the block in sorted order, and a counter s; the first s elements of L are
  "small", the rest "large".  The interface (Fig. block-if) fixes what each
  operation does to (L, s):
    construct  L = every element, s = h
    delete     remove alpha[i] from L, then s = max(0, s - 1)
    undelete   put alpha[i] back into L (s unchanged); deletions and
               undeletions must be properly nested (Section 5.1)
    unwind     delete(k-1), ..., delete(0)
    advance    s = s + 1
    small      s
    peek       the first large element, or +inf when every element is small
  ``RankBlock`` keeps exactly that: L as the sorted list of the live
  elements' ranks in the stable order of the block, and s.  Section 5.2's
  remark that pi^-1 may replace the pairs (alpha[i], i) in comparisons is
  what makes ranks a faithful stand-in for the values.
* Section 4 defines the two list updates behind delete and undelete
  (equations del and undo-del, Knuth's dancing links).  ``DancingLinks``
  applies them to prev / next arrays with a sentinel node, and is used to
  pin the two facts the GPU path builds on: properly nested undeletions
  restore the list exactly, and after unwind every node still holds the
  neighbours it had when it was deleted (the unwind links).
* Section 6.2 (Fig. postprocess) combines the blocks; ``sort_median`` runs
  those steps on ``RankBlock`` states and records the sets S_A, S_B, L_A, L_B
  around every step, so the tests can check the invariant of Section 6.3
  (eq. inv) and the rows of the case-analysis table of Lemma 1.

Readings of the paper used here (each also listed in the design notes):
* n not a multiple of k: the last block has r = n - (b-1) k elements and its
  pair prints r outputs (the paper calls the extension "straightforward").
* Ties: blocks are sorted stably, and peek(A) <= peek(B) advances and prints
  A, so on equal values the older block counts as smaller (Section 6.3).
"""
from __future__ import annotations

import bisect
import math


def stable_order(alpha):
    """pi: positions of the block in the order of the pairs (alpha[i], i)
    (Section 5.2), and pi^-1: the rank of every position."""
    pi = sorted(range(len(alpha)), key=lambda i: (alpha[i], i))
    inv = [0] * len(alpha)
    for r, p in enumerate(pi):
        inv[p] = r
    return pi, inv


class RankBlock:
    """(alpha, pi, L, s) of Section 5 with L kept as sorted ranks."""

    def __init__(self, alpha, h: int):
        self.alpha = list(alpha)
        self.h = h
        self.pi, self.rank = stable_order(self.alpha)
        self.live = list(range(len(self.alpha)))   # construct: every element ...
        self.s = min(h, len(self.live))            # ... and the first h are small
        self._removed = []                         # stack of deleted positions

    # -- the interface's queries ---------------------------------------------
    def small(self) -> int:
        return self.s

    def first_large(self):
        """Position of the first large element of L, or None (peek = +inf)."""
        return self.pi[self.live[self.s]] if self.s < len(self.live) else None

    def peek(self):
        p = self.first_large()
        return math.inf if p is None else self.alpha[p]

    def small_set(self):
        return {self.pi[r] for r in self.live[:self.s]}

    def members(self):
        return {self.pi[r] for r in self.live}

    # -- the interface's updates ----------------------------------------------
    def delete(self, i: int) -> None:
        r = self.rank[i]
        at = bisect.bisect_left(self.live, r)
        assert at < len(self.live) and self.live[at] == r, "delete of an element not in L"
        del self.live[at]
        self._removed.append(i)
        self.s = max(0, self.s - 1)

    def undelete(self, i: int) -> None:
        assert self._removed and self._removed[-1] == i, "undeletions must be properly nested"
        self._removed.pop()
        bisect.insort(self.live, self.rank[i])

    def unwind(self) -> None:
        for i in reversed(range(len(self.alpha))):
            self.delete(i)

    def advance(self) -> None:
        assert self.s < len(self.live), "advance past the end of L"
        self.s += 1


class DancingLinks:
    """prev / next arrays over nodes 0 .. k-1 plus a sentinel node k, linked
    in the stable sorted order of the block; equations del and undo-del of
    Section 4 as the only updates."""

    def __init__(self, alpha):
        self.k = len(alpha)
        pi, _ = stable_order(alpha)
        ring = [self.k] + pi
        self.next = [0] * (self.k + 1)
        self.prev = [0] * (self.k + 1)
        for a, b in zip(ring, ring[1:] + ring[:1]):
            self.next[a] = b
            self.prev[b] = a

    def remove(self, i: int) -> None:         # equation del
        self.next[self.prev[i]] = self.next[i]
        self.prev[self.next[i]] = self.prev[i]

    def restore(self, i: int) -> None:        # equation undo-del
        self.next[self.prev[i]] = i
        self.prev[self.next[i]] = i

    def walk(self):
        out, node = [], self.next[self.k]
        while node != self.k:
            out.append(node)
            node = self.next[node]
        return out


def sort_median(x, k: int, trace=None):
    """Median filter of x with odd window k by the steps of Fig. postprocess.

    Returns (y, argmed) as lists (argmed = index into x of the printed
    element).  If ``trace`` is a list, every printed output after the first
    appends the sets S_A, S_B, L_A, L_B before step (dagger), after the
    delete / undelete, and before the print, with s_A and s_B.
    """
    n = len(x)
    if k < 1 or k % 2 == 0 or k > n:
        raise ValueError("need odd 1 <= k <= n")
    h = (k - 1) // 2
    blocks = [list(x[j:j + k]) for j in range(0, n, k)]

    def sets(A, B):
        return dict(SA=A.small_set(), SB=B.small_set(), LA=A.members(), LB=B.members())

    B = RankBlock(blocks[0], h)
    y, arg = [B.peek()], [B.first_large()]               # step (double dagger)
    for j in range(1, len(blocks)):
        A, B = B, RankBlock(blocks[j], h)
        B.unwind()
        for i in range(len(blocks[j])):
            before = sets(A, B) if trace is not None else None
            A.delete(i)                                  # step (dagger)
            B.undelete(i)
            middle = sets(A, B) if trace is not None else None
            if A.small() + B.small() < h:
                (A if A.peek() <= B.peek() else B).advance()
            take_a = A.peek() <= B.peek()                # step (inverted dagger)
            y.append(A.peek() if take_a else B.peek())
            arg.append((j - 1) * k + A.first_large() if take_a else j * k + B.first_large())
            if trace is not None:
                trace.append(dict(j=j, i=i, h=h, alphaA=A.alpha, alphaB=B.alpha,
                                  pre=before, mid=middle, post=sets(A, B),
                                  sA=A.small(), sB=B.small()))
    return y, arg
