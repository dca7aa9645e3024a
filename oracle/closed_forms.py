"""Closed forms of benchmark programs on inputs that admit one.

TEST INFRASTRUCTURE ONLY (imported by tests and by the golden-file script
beside this module).  Shares no code with the GPU library.

Same-generation on a forest (Section 5.2's SG program; its recursive rule
pairs the children of two nodes already known to be of one generation):
with edge(parent, child) only and no cross edges, sg(x, y) holds exactly
when x != y lie in the same tree at the same depth.  Reading the rules
bottom up, round 1 derives the sibling pairs (lowest common ancestor one
level up) and round k the pairs whose lowest common ancestor is k levels up,
since a pair at LCA distance k needs the pair of their parents, at distance
k - 1, to be known first.

  * |sg| = sum over (tree, depth) groups of c (c - 1), c the group size;
  * delta_k = sum over ancestors a of S(a, k)^2
              - sum over non-root nodes c of S(c, k - 1)^2,
    where S(v, j) counts the descendants of v exactly j levels below it
    (S(v, 0) = 1): the ordered pairs under a at distance k, minus those whose
    two ends sit under one child of a (their LCA is lower);
  * iterations = the largest k with delta_k > 0.

Both hold for the program with and without the inequality in the recursive
rule, since a pure forest never derives sg(x, x).
"""
from __future__ import annotations

import numpy as np


def forest_structure(n: int, edges) -> tuple:
    """(parent, depth, root) of a forest given as edge(parent, child) rows in
    which every parent precedes its child (a random recursive forest)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    par = np.full(n, -1, dtype=np.int64)
    if len(e):
        if np.any(e[:, 0] >= e[:, 1]):
            raise ValueError("not a recursive forest: a parent must precede its child")
        if len(np.unique(e[:, 1])) != len(e):
            raise ValueError("not a forest: a node has two parents")
        par[e[:, 1]] = e[:, 0]
    depth = np.zeros(n, dtype=np.int64)
    root = np.arange(n, dtype=np.int64)
    # one sweep in node order: parents precede children
    for v in np.nonzero(par >= 0)[0]:
        p = par[v]
        depth[v] = depth[p] + 1
        root[v] = root[p]
    return par, depth, root


def sg_forest(n: int, edges) -> dict:
    """Closed form of same-generation on a pure forest of n nodes.

    Returns a dict with
      group      -- (n,) int64 id of each node's (tree, depth) group;
      group_size -- (groups,) int64 size c of each group;
      size       -- |sg| = sum c (c - 1);
      deltas     -- [delta_1, ..., delta_K] new pairs of each round;
      iterations -- K, the rounds with a non-empty delta.
    """
    par, depth, root = forest_structure(n, edges)
    key = root * (int(depth.max(initial=0)) + 1) + depth
    _, group, group_size = np.unique(key, return_inverse=True, return_counts=True)
    group = group.astype(np.int64)
    group_size = group_size.astype(np.int64)
    size = int(np.sum(group_size * (group_size - 1)))

    nonroot = par >= 0
    deltas = []
    # anc = each node's ancestor j levels up (-1 once past its root)
    anc = np.arange(n, dtype=np.int64)
    s_prev = np.ones(n, dtype=np.int64)  # S(v, 0) = 1
    while True:
        live = anc >= 0
        anc = np.where(live, par[np.where(live, anc, 0)], -1)
        live = anc >= 0
        if not live.any():
            break
        s = np.bincount(anc[live], minlength=n).astype(np.int64)  # S(v, j)
        d = int(np.sum(s * s)) - int(np.sum(s_prev[nonroot] * s_prev[nonroot]))
        deltas.append(d)
        s_prev = s
    while deltas and deltas[-1] == 0:
        deltas.pop()
    return dict(group=group, group_size=group_size, size=size, deltas=deltas,
                iterations=len(deltas))
