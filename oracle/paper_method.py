"""The paper's own median-filter algorithm on the CPU -- TEST INFRASTRUCTURE ONLY.

Restates, for the tests, the two-phase method of "Median Filtering is
Equivalent to Sorting" (Suomela):

* Section 3 / Section 6.1 -- piecewise stable sort: each block X_j of length
  k = 2h + 1 gets the permutation P_j that sorts the pairs (X_j[i], i).
* Section 5 -- the block data structure: a sorted doubly-linked list over the
  block's indices with a sentinel node k, arrays prev/next of length k + 1,
  a counter s of "small" elements and a pointer m to the first large one
  (Section 5.3 invariants: next[k] = p_0, prev[k] = p_{c-1}, m = p_s).
  Operations construct / delete / undelete / unwind / advance / small / peek
  (Figures "Block data structure interface" and "... implementation").
* Section 6.2 -- post-processing: for each adjacent pair of blocks, delete
  the old block's elements in index order while undoing the new block's
  deletions (Knuth's dancing links, Section 4 equations del / undo-del),
  advance one pointer whenever s_A + s_B < h, and print min(peek A, peek B).

Readings of the paper used here (each also listed in the design notes):
* unwind: the implementation figure prints the *undelete* formulas inside
  unwind; the interface figure defines unwind as delete(k-1), ..., delete(0),
  so this file unlinks with the deletion formulas and then sets m = k, s = 0.
* n not a multiple of k: the last block has r = n - (b-1) k elements and its
  pair emits r outputs (the paper calls the extension "straightforward").
* Ties: the stable sort orders equal values by index inside a block, and
  peek(A) <= peek(B) advances A, so equal values of the older block count as
  smaller (Section 6.3).

It is used to pin the invariant of Section 6.3 (s_A + s_B = h and
S_A u S_B = H_AB before every output), the seven cases of the case-analysis
table, and properly nested delete/undelete.  Expected values for the CUDA
path always come from the plain definition in ``mf_oracle.c``.
"""
from __future__ import annotations

import math


class SortedBlock:
    """One block data structure B = (alpha, pi, L, s) of Section 4."""

    def __init__(self, alpha, h: int):
        # construct(alpha, pi): L holds every element in sorted order, s = h.
        self.alpha = list(alpha)
        self.size = len(self.alpha)
        self.h = h
        self.sentinel = self.size                      # node k
        self.pi = sorted(range(self.size), key=lambda i: (self.alpha[i], i))
        self.prev = [0] * (self.size + 1)
        self.next = [0] * (self.size + 1)
        order = [self.sentinel] + self.pi + [self.sentinel]
        for left, right in zip(order[:-1], order[1:]):
            self.next[left] = right
            self.prev[right] = left
        self.s = h
        self.m = self.pi[h] if h < self.size else self.sentinel

    # -- queries ----------------------------------------------------------
    def at_end(self) -> bool:
        return self.m == self.sentinel

    def peek(self):
        """First large element's value, or +inf if every element is small."""
        return math.inf if self.at_end() else self.alpha[self.m]

    def small(self) -> int:
        return self.s

    def is_small(self, i: int) -> bool:
        """alpha[i] is small iff (alpha[i], i) < (alpha[m], m); alpha[k] = +inf."""
        if self.at_end():
            return True
        return (self.alpha[i], i) < (self.alpha[self.m], self.m)

    def members(self):
        """Indices currently in L, in sorted order."""
        out, node = [], self.next[self.sentinel]
        while node != self.sentinel:
            out.append(node)
            node = self.next[node]
        return out

    def small_set(self):
        return self.members()[: self.s]

    # -- updates ----------------------------------------------------------
    def _unlink(self, i: int) -> None:
        # equation del: prev[next[i]] <- prev[i], next[prev[i]] <- next[i]
        before, after = self.prev[i], self.next[i]
        self.next[before] = after
        self.prev[after] = before

    def _relink(self, i: int) -> None:
        # equation undo-del: prev[next[i]] <- i, next[prev[i]] <- i
        self.next[self.prev[i]] = i
        self.prev[self.next[i]] = i

    def delete(self, i: int) -> None:
        """Remove alpha[i] from L; s becomes max(0, s - 1)."""
        was_small = self.is_small(i)
        self._unlink(i)
        if was_small:
            self.s -= 1
            return
        if self.m == i:
            # i's own pointers still name its old successor
            self.m = self.next[i]
        if self.s > 0:
            self.m = self.prev[self.m]
            self.s -= 1

    def undelete(self, i: int) -> None:
        """Put alpha[i] back into L (only as the inverse of the latest delete)."""
        self._relink(i)
        if self.is_small(i):
            self.m = self.prev[self.m]

    def unwind(self) -> None:
        """delete(k-1), ..., delete(0); afterwards L is empty, m = k, s = 0."""
        for i in range(self.size - 1, -1, -1):
            self._unlink(i)
        self.m = self.sentinel
        self.s = 0

    def advance(self) -> None:
        self.m = self.next[self.m]
        self.s += 1


def sort_median(x, k: int, trace=None):
    """Median filter of x with odd window k by sorting + post-processing.

    Returns (y, argmed) as Python lists (argmed = index into x of the median
    element).  If ``trace`` is a list, one dict per printed output after the
    first is appended with the block states, for the invariant tests.
    """
    n = len(x)
    if k < 1 or k % 2 == 0 or k > n:
        raise ValueError("need odd 1 <= k <= n")
    h = (k - 1) // 2
    nblocks = -(-n // k)
    blocks = [x[j * k:(j + 1) * k] for j in range(nblocks)]

    B = SortedBlock(blocks[0], h)
    y = [B.peek()]
    arg = [B.m]
    for j in range(1, nblocks):
        A = B
        B = SortedBlock(blocks[j], h)
        B.unwind()
        for i in range(len(blocks[j])):
            pre = None
            if trace is not None:
                pre = dict(SA=set(A.small_set()), SB=set(B.small_set()),
                           LA=set(A.members()), LB=set(B.members()))
            A.delete(i)
            B.undelete(i)
            mid = None
            if trace is not None:
                mid = dict(SA=set(A.small_set()), SB=set(B.small_set()),
                           LA=set(A.members()), LB=set(B.members()))
            if A.small() + B.small() < h:
                if A.peek() <= B.peek():
                    A.advance()
                else:
                    B.advance()
            if A.peek() <= B.peek():
                y.append(A.peek())
                arg.append((j - 1) * k + A.m)
            else:
                y.append(B.peek())
                arg.append(j * k + B.m)
            if trace is not None:
                trace.append(dict(
                    j=j, i=i, h=h, alphaA=A.alpha, alphaB=B.alpha,
                    pre=pre, mid=mid,
                    post=dict(SA=set(A.small_set()), SB=set(B.small_set()),
                              LA=set(A.members()), LB=set(B.members())),
                    sA=A.small(), sB=B.small()))
    return y, arg
