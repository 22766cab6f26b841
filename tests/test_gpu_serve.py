"""Serving engine: asynchronous requests (bb_submit / bb_submit_request /
bb_poll) overlapping on worker slots, a managed cache of resident graphs
under an arena budget with LRU eviction, and sign-flip re-queries. Every
result must equal the oracle's count of the graph as that request sees it,
and be the same whether the request runs alone or in a mix."""
import numpy as np
import pytest

import oracle
import paper_2308_07932_gb300 as pkg
from paper_2308_07932_gb300 import synth

pytestmark = pytest.mark.gpu

MB = 1 << 20


def pool(n, seed0=300, m_lo=1e4, m_hi=3e5):
    """Request graphs drawn like the serving workload (the 2M x 500k
    recipe at log-uniform sizes), smaller so the oracle stays quick."""
    rng = np.random.default_rng(seed0)
    sizes = np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), n)).astype(int)
    return [synth.chung_lu_scaled(seed0 + i, int(m)) for i, m in enumerate(sizes)]


def flipped(g, idx):
    s = g.sign.copy()
    s[idx] = -s[idx]
    return synth.SignedBipartite(g.nU, g.nV, g.rowptr, g.col, s, g.name + "/f")


def trace(graphs, n_req, seed, requery=0.2, flip_frac=0.01):
    """Requests: (key, graph index, flips or None); re-queries pick a key
    already requested and flip flip_frac of its edge signs. Returns the
    requests and, per request, the graph state it must count."""
    rng = np.random.default_rng(seed)
    reqs, states, cur, seen = [], [], {}, []
    for k in range(n_req):
        if seen and rng.random() < requery:
            key = seen[rng.integers(len(seen))]
            g = cur[key]
            idx = rng.choice(g.nE, size=max(1, int(g.nE * flip_frac)), replace=False)
            cur[key] = flipped(g, idx)
            reqs.append((key, None, idx))
        else:
            key = 1000 + k
            gi = int(rng.integers(len(graphs)))
            cur[key] = graphs[gi]
            seen.append(key)
            reqs.append((key, gi, None))
        states.append(cur[key])
    return reqs, states


@pytest.fixture(scope="module")
def graphs():
    return pool(12)


@pytest.fixture(scope="module")
def counts(graphs):
    return {}


def oracle_of(cache, g):
    k = (g.name, g.sign.tobytes().__hash__())
    if k not in cache:
        cache[k] = oracle.count(g, threads=4)
    return cache[k]


def run_mix(ctx, graphs, reqs):
    tickets = []
    for key, gi, flips in reqs:
        g = graphs[gi] if gi is not None else None
        tickets.append(ctx.submit_request(key, g, flips))
    return [t.wait() for t in tickets]


def test_caller_graphs_submitted_together(graphs, counts):
    with pkg.Context(0) as ctx:
        ctx.serve(slots=3)
        res = [ctx.upload(g) for g in graphs[:6]]
        # every graph twice, all outstanding at once: same-graph requests serialise
        tickets = [ctx.submit(r) for r in res] + [ctx.submit(r) for r in res]
        out = [t.wait() for t in tickets]
        for i, o in enumerate(out):
            assert (o.balanced, o.total) == oracle_of(counts, graphs[i % 6])
        for r in res:
            r.free()


def test_default_engine_starts_on_first_submit(graphs, counts):
    with pkg.Context(0) as ctx:
        r = ctx.upload(graphs[0])
        o = ctx.submit(r).wait()
        assert (o.balanced, o.total) == oracle_of(counts, graphs[0])
        with pytest.raises(pkg.BBError):  # no managed cache in the default engine
            ctx.submit_request(1, graphs[0])
        r.free()


def test_mix_equals_alone_and_oracle(graphs, counts):
    reqs, states = trace(graphs, 40, seed=7)
    want = [oracle_of(counts, s) for s in states]
    with pkg.Context(0) as ctx:
        ctx.serve(slots=4, arena_bytes=4096 * MB)
        mixed = run_mix(ctx, graphs, reqs)
        st = ctx.serve_stats()
    assert [(o.balanced, o.total) for o in mixed] == want
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["cache_hits"] == sum(1 for r in reqs if r[1] is None)
    # the same requests one at a time, on a fresh engine
    with pkg.Context(0) as ctx:
        ctx.serve(slots=1, arena_bytes=4096 * MB)
        alone = []
        for key, gi, flips in reqs:
            t = ctx.submit_request(key, graphs[gi] if gi is not None else None, flips)
            alone.append(t.wait())
    assert [(o.balanced, o.total) for o in alone] == want


def test_small_arena_evicts_and_reuploads(graphs, counts):
    sizes = sorted(graphs, key=lambda g: g.nE)
    small = sizes[:6]
    with pkg.Context(0) as ctx:
        # room for about two of these graphs with their build workspace
        ctx.serve(slots=2, arena_bytes=int(2.5 * max(pkg.request_bytes(g) for g in small)))
        outs = []
        for rnd in range(2):
            tickets = [ctx.submit_request(10 + i, g) for i, g in enumerate(small)]
            outs += [t.wait() for t in tickets]
        st = ctx.serve_stats()
        assert st["evictions"] > 0
        assert st["arena_used"] <= st["arena_bytes"]
        for i, o in enumerate(outs):
            assert (o.balanced, o.total) == oracle_of(counts, small[i % len(small)])
        # a key that is not resident needs its CSR
        gone = [k for k in range(10, 16)]
        t = [ctx.submit_request(k) for k in gone]
        n_fail = 0
        for x in t:
            try:
                x.wait()
            except pkg.BBError as e:
                assert e.name == "BB_ERR_INVALID_ARG"
                n_fail += 1
        assert n_fail >= 1


def test_budget_and_invalid_requests(graphs, counts):
    with pkg.Context(0) as ctx:
        ctx.serve(slots=2, arena_bytes=8 * MB)
        big = synth.chung_lu_scaled(5, 400_000)
        with pytest.raises(pkg.BBError) as ei:
            ctx.submit_request(1, big).wait()
        assert ei.value.name == "BB_ERR_BUDGET"
        ctx.serve(slots=2, arena_bytes=1024 * MB)
        dup = synth.SignedBipartite(2, 2, np.array([0, 2, 2], np.int64), np.array([1, 1], np.int32),
                                    np.array([1, 1], np.int8), "dup")
        with pytest.raises(pkg.BBError) as ei:
            ctx.submit_request(2, dup).wait()
        assert ei.value.name == "BB_ERR_INVALID_ARG"
        # a bad flip index fails that request only; the graph stays usable
        g = graphs[0]
        o = ctx.submit_request(3, g).wait()
        assert (o.balanced, o.total) == oracle_of(counts, g)
        with pytest.raises(pkg.BBError) as ei:
            ctx.submit_request(3, None, [g.nE]).wait()
        assert ei.value.name == "BB_ERR_INVALID_ARG"
        o = ctx.submit_request(3).wait()
        assert (o.balanced, o.total) == oracle_of(counts, g)
        # the no-cache flag drops the graph after its count
        ctx.submit_request(4, graphs[1], no_cache=True).wait()
        with pytest.raises(pkg.BBError):
            ctx.submit_request(4).wait()


def test_destroy_with_requests_in_flight(graphs, counts):
    ctx = pkg.Context(0)
    ctx.serve(slots=2, arena_bytes=2048 * MB)
    tickets = [ctx.submit_request(50 + i, graphs[i % len(graphs)]) for i in range(24)]
    ctx.close()  # waits for running requests; queued ones end with BB_ERR_BUSY
    ok = busy = 0
    for i, t in enumerate(tickets):
        try:
            o = t.poll()
            assert o is not None
            assert (o.balanced, o.total) == oracle_of(counts, graphs[i % len(graphs)])
            ok += 1
        except pkg.BBError as e:
            assert e.name == "BB_ERR_BUSY"
            busy += 1
    assert ok + busy == len(tickets)


def test_small_flip_requeries_are_incremental(graphs, counts):
    """Re-queries flipping a handful of edges of a resident graph whose
    counts are known take the incremental walk; every result stays exact."""
    big = sorted(graphs, key=lambda g: g.nE)[-3:]
    reqs, states = trace(big, 30, seed=11, requery=0.6, flip_frac=0.0)
    # flip_frac 0 gives one flipped edge per re-query; add a few more
    rng = np.random.default_rng(4)
    reqs = [(k, gi, None if f is None else np.concatenate([f, rng.choice(states[i].nE, 3)]))
            for i, (k, gi, f) in enumerate(reqs)]
    cur, states = {}, []
    for key, gi, f in reqs:
        if gi is not None:
            cur[key] = big[gi]
        else:
            idx, cnt = np.unique(f, return_counts=True)
            cur[key] = flipped(cur[key], idx[cnt % 2 == 1])  # a repeated index flips back
        states.append(cur[key])
    want = [oracle_of(counts, s) for s in states]
    with pkg.Context(0) as ctx:
        ctx.serve(slots=3, arena_bytes=2048 * MB)
        got = run_mix(ctx, big, reqs)
        st = ctx.serve_stats()
    assert [(o.balanced, o.total) for o in got] == want
    assert st["incremental"] > 0 and st["failed"] == 0
