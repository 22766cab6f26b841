"""Host-only check of the identity the matrix-product path uses to report
the priority-wedge count without enumerating wedges: a middle v of degree d
with k neighbours ranked above it (Def. 4) is the middle of C(d,2) - C(d-k,2)
wedges whose top vertex outranks it (every pair of v's neighbours except
the pairs ranked both below v). Compared with a direct enumeration of the
wedges u - v - w with u the highest of the three, on small seeded graphs."""
import itertools

import numpy as np

from paper_2308_07932_gb300 import synth


def global_rank(g):
    """Def. 4's total order: by degree, ties by gid (u, or |U| + v)."""
    n = g.nU + g.nV
    deg = np.concatenate([np.diff(g.rowptr), np.bincount(g.col, minlength=g.nV)])
    order = np.lexsort((np.arange(n), deg))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    return rank, deg


def by_identity(g):
    rank, deg = global_rank(g)
    u, v, _ = g.edges()
    a, b = u, g.nU + v
    above = np.zeros(g.nU + g.nV, np.int64)
    np.add.at(above, a, (rank[b] > rank[a]).astype(np.int64))
    np.add.at(above, b, (rank[a] > rank[b]).astype(np.int64))
    c2 = lambda x: x * (x - 1) // 2
    return int((c2(deg) - c2(deg - above)).sum())


def by_enumeration(g):
    rank, _ = global_rank(g)
    u, v, _ = g.edges()
    nbr = [[] for _ in range(g.nU + g.nV)]
    for x, y in zip(u, g.nU + v):
        nbr[x].append(y)
        nbr[y].append(x)
    count = 0
    for mid in range(g.nU + g.nV):
        for x, y in itertools.combinations(nbr[mid], 2):
            top = x if rank[x] > rank[y] else y
            if rank[top] > rank[mid]:
                count += 1
    return count


def test_wedge_count_identity_matches_enumeration():
    graphs = [synth.uniform(3, 40, 30, 300, 0.6), synth.vote(4, 12, 200, 0.4, 2, 0.55, 0.8),
              synth.chung_lu(5, 300, 120, 1500, 2.1, 2.1, 100.0, 0.8),
              synth.from_dense(np.ones((5, 7), np.int8)), synth.from_edges(3, 3, [], [], [])]
    for g in graphs:
        assert by_identity(g) == by_enumeration(g), g.name
