"""Named query patterns as plain edge lists (inputs, no method arithmetic).

A pattern is a small connected simple graph on labels 0..k-1. Matching is
vertex-induced: pattern edges must be present and absent pairs must be absent.
Structures for the named shapes of the GraphZero evaluation (the drawings of its
Fig. 8 are not available, so these are the usual definitions):

* chordal cycle of size k = K_k minus one edge (Sec. 1, Sec. 7.1);
* tailed triangle (paw) = triangle plus one pendant edge (Sec. 5.1);
* house = 4-cycle plus a fifth vertex adjacent to two adjacent cycle vertices;
* hourglass (bowtie) = two triangles sharing one vertex;
* the size-3 chordal cycle K3 - e is the wedge (2-path).
"""
from __future__ import annotations

import numpy as np


def _clique(k):
    return [(i, j) for i in range(k) for j in range(i + 1, k)]


def _chordal(k):
    return [e for e in _clique(k) if e != (k - 2, k - 1)]


def _cycle(k):
    return [(i, (i + 1) % k) for i in range(k)]


EDGES = {
    "edge": (2, [(0, 1)]),
    "wedge": (3, [(0, 1), (0, 2)]),
    "triangle": (3, _clique(3)),
    "path4": (4, [(0, 1), (1, 2), (2, 3)]),
    "star3": (4, [(0, 1), (0, 2), (0, 3)]),
    "c4": (4, _cycle(4)),
    "paw": (4, [(0, 1), (1, 2), (0, 2), (2, 3)]),
    "diamond": (4, _chordal(4)),
    "k4": (4, _clique(4)),
    "c5": (5, _cycle(5)),
    "house": (5, _cycle(4) + [(0, 4), (1, 4)]),
    "hourglass": (5, [(0, 1), (0, 2), (1, 2), (0, 3), (0, 4), (3, 4)]),
    "chordal5": (5, _chordal(5)),
    "k5": (5, _clique(5)),
    "k6": (6, _clique(6)),
    "chordal6": (6, _chordal(6)),
    "chordal7": (7, _chordal(7)),
    # a 6-vertex graph with a trivial automorphism group (no restrictions at all)
    "asym6": (6, [(0, 1), (1, 2), (2, 3), (3, 4), (2, 5), (3, 5), (4, 5), (1, 5)]),
}

#: the five size-3..5 patterns of the arbitrary-pattern workload
PATTERN_SET = ["c4", "diamond", "paw", "house", "chordal5"]
#: the twelve patterns of the batched workload
BATCH_PATTERNS = ["wedge", "triangle", "path4", "star3", "c4", "paw", "diamond", "k4", "k5",
                  "k6", "chordal5", "chordal6"]
#: difference-heavy sparse patterns, placed only on graphs of scale <= 14 in the batch
BATCH_SPARSE = {"wedge", "path4", "star3", "c4", "paw"}
#: request mix of the served workload
SERVED_PATTERNS = ["triangle", "c4", "diamond", "k4", "k5", "chordal5"]


def adjacency(name_or_edges, k: int | None = None) -> np.ndarray:
    """k x k uint8 adjacency (symmetric, zero diagonal)."""
    if isinstance(name_or_edges, str):
        k, edges = EDGES[name_or_edges]
    else:
        edges = name_or_edges
        assert k is not None
    a = np.zeros((k, k), dtype=np.uint8)
    for i, j in edges:
        a[i, j] = a[j, i] = 1
    return a


#: largest R-MAT scale a pattern is placed on in the batched workload. The
#: difference-heavy sparse patterns cost about the sum of cubed degrees on hub
#: vertices; chordal cycles and K6 have counts of 10^12 and more on the
#: skewed graphs above these scales, each costing seconds to minutes alone.
BATCH_MAX_SCALE = {"wedge": 14, "path4": 14, "star3": 14, "c4": 14, "paw": 14, "chordal6": 13,
                   "chordal5": 15, "k6": 16, "diamond": 16, "k5": 18, "triangle": 21, "k4": 21}


def batch_queries(scales=None, per_graph: int = 4, seed: int = 4):
    """Query table of the batched workload: (graph index, pattern name) pairs.

    ``per_graph`` queries on each graph (64 in all for the 16 graphs), every
    pattern of BATCH_PATTERNS at least four times, each only on graphs whose
    scale is at most BATCH_MAX_SCALE[pattern]. Seeded; the table is an input,
    not a result.
    """
    if scales is None:
        scales = [10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 12, 14, 16, 18]
    rng = np.random.default_rng(seed)
    slots = [(g, j) for g in range(len(scales)) for j in range(per_graph)]
    table = {}
    # most constrained patterns first, four copies each, into random eligible slots
    for p in sorted(BATCH_PATTERNS, key=lambda x: (BATCH_MAX_SCALE[x], x)):
        for _ in range(4):
            free = [s for s in slots if s not in table and scales[s[0]] <= BATCH_MAX_SCALE[p]]
            table[free[int(rng.integers(len(free)))]] = p
    for s in slots:
        if s not in table:
            pool = [p for p in BATCH_PATTERNS if scales[s[0]] <= BATCH_MAX_SCALE[p]]
            table[s] = pool[int(rng.integers(len(pool)))]
    return [(g, table[(g, j)]) for g, j in slots]
