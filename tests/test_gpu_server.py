"""The continuous-batching server: results against the oracle, bit-identical
alone and in a mix, cancellation, timeouts, admission by memory budget."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cpaa_inputs as ci
from oracle import oracle as O
from tests.gpu_util import upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_01743_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def served(pkg):
    graphs = [ci.chung_lu(5000, 40000, seed=31), ci.chung_lu(60000, 600000, seed=32),
              ci.grid_deleted(100, 120, 0.2, seed=3)]
    G = [upload(pkg, g) for g in graphs]
    S = pkg.Server(4 << 30)
    ids = [S.add_graph(x, 8) for x in G]
    yield pkg, graphs, G, S, ids
    S.close()
    for x in G:
        x.close()


def _queries(graphs, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        gi = int(rng.integers(len(graphs)))
        n = graphs[gi].n
        k = int(rng.integers(1, 17))
        seeds = rng.choice(n, size=k, replace=False).astype(np.int32)
        c = float(rng.choice([0.5, 0.85, 0.95]))
        out.append((gi, seeds, None, c, 1e-6))
    return out


def test_alone_equals_in_mix_and_matches_oracle(served):
    pkg, graphs, G, S, ids = served
    gi = 1
    n = graphs[gi].n
    q = (ids[gi], np.array([5, 123, 40000], dtype=np.int32), None, 0.85, 1e-6)
    alone = np.empty(n)
    st, info = S.wait(S.submit(*q), alone, timeout_us=120_000_000)
    assert st == pkg.CPAA_OK
    # the same query submitted in the middle of a stream of others
    mix = _queries(graphs, 80, seed=5)
    tickets, tq = [], None
    for i, (g2, seeds, w, c, tol) in enumerate(mix):
        tickets.append((g2, seeds, c, S.submit(ids[g2], seeds, w, c, tol)))
        if i == 40:
            tq = S.submit(*q)
    in_mix = np.empty(n)
    st2, info2 = S.wait(tq, in_mix, timeout_us=120_000_000)
    assert st2 == pkg.CPAA_OK and info2.rounds == info.rounds
    assert np.array_equal(alone, in_mix)
    rp, cx = graphs[gi].numpy()
    p = np.zeros(n)
    p[q[1]] = 1.0 / 3
    ref = O.cpaa(rp, cx, p, 0.85, info.rounds)
    assert np.abs(alone - ref).sum() / np.abs(ref).sum() <= 1e-6
    # every query of the mix against the oracle (FP32 serving: relative L1 <= 1e-6)
    out = {}
    for g2, seeds, c, t in tickets:
        pi = np.empty(graphs[g2].n)
        st, inf = S.wait(t, pi, timeout_us=120_000_000)
        assert st == pkg.CPAA_OK
        out[t] = (g2, seeds, c, pi, inf.rounds)
    for t in list(out)[::8]:
        g2, seeds, c, pi, M = out[t]
        rp, cx = graphs[g2].numpy()
        p = np.zeros(graphs[g2].n)
        p[seeds] = 1.0 / len(seeds)
        ref = O.cpaa(rp, cx, p, c, M)
        assert np.abs(pi - ref).sum() / np.abs(ref).sum() <= 1e-6
        assert abs(pi.sum() - 1.0) < 1e-9
    s = S.stats()
    assert s["completed"] >= 82 and s["failed"] == 0
    assert s["p99_us"] >= s["p50_us"] > 0


def test_cancel_and_timeout(pkg):
    g = ci.chung_lu(200000, 2000000, seed=41)
    G = upload(pkg, g)
    S = pkg.Server(1 << 30)
    gid = S.add_graph(G, 1)  # one slot: later queries must queue
    tickets = [S.submit(gid, np.array([i * 7 + 1], dtype=np.int32), None, 0.95, 1e-8) for i in range(12)]
    last = tickets[-1]
    st, _ = S.wait(last, None, timeout_us=0)
    assert st == pkg.CPAA_ETIMEOUT
    assert S.cancel(last) == pkg.CPAA_OK
    st, _ = S.wait(last, None, timeout_us=120_000_000)
    assert st == pkg.CPAA_ECANCELLED
    with pytest.raises(pkg.CpaaError) as e:
        S.wait(last, None, timeout_us=0)
    assert e.value.status == pkg.CPAA_ENOTFOUND
    for t in tickets[:-1]:
        st, info = S.wait(t, None, timeout_us=120_000_000)
        assert st == pkg.CPAA_OK
    assert S.stats()["cancelled"] == 1
    S.close()
    G.close()


def test_invalid_submissions(served):
    pkg, graphs, G, S, ids = served
    n = graphs[0].n
    bad = [
        (ids[0], np.array([n], dtype=np.int32), None, 0.85, 1e-6),          # out of range
        (ids[0], np.array([3, 3], dtype=np.int32), None, 0.85, 1e-6),       # duplicate seed
        (ids[0], np.array([3, 4], dtype=np.int32), np.array([0.5, 0.6]), 0.85, 1e-6),
        (ids[0], np.array([3], dtype=np.int32), None, 1.0, 1e-6),
        (ids[0], np.array([3], dtype=np.int32), None, 0.85, 0.0),
        (ids[0], np.arange(65, dtype=np.int32), None, 0.85, 1e-6),          # too many seeds
    ]
    for q in bad:
        with pytest.raises(pkg.CpaaError) as e:
            S.submit(*q)
        assert e.value.status == pkg.CPAA_EINVAL
    with pytest.raises(pkg.CpaaError) as e:
        S.submit(99, np.array([1], dtype=np.int32), None, 0.85, 1e-6)
    assert e.value.status == pkg.CPAA_ENOTFOUND


def test_admission_needs_memory(pkg):
    g = ci.chung_lu(100000, 800000, seed=42)
    G = upload(pkg, g)
    S = pkg.Server(1 << 20)  # 1 MiB: not even one slot
    with pytest.raises(pkg.CpaaError) as e:
        S.add_graph(G, 4)
    assert e.value.status == pkg.CPAA_ENOMEM
    S.close()
    G.close()


def test_posteriori_rule_alone_equals_in_mix(pkg):
    """Serving under the a-posteriori stopping rule: a query stops at the round
    the oracle's own sums give, no later than the rigorous M, within tol of the
    exact solution, and with the same bits alone and in a mix."""
    graphs = [ci.chung_lu(5000, 40000, seed=31), ci.chung_lu(60000, 600000, seed=32)]
    G = [upload(pkg, g) for g in graphs]
    S = pkg.Server(2 << 30, stop_rule=pkg.CPAA_STOP_POSTERIORI)
    ids = [S.add_graph(x, 8) for x in G]
    try:
        n = graphs[1].n
        rp, cx = graphs[1].numpy()
        seeds = np.array([59990], dtype=np.int32)  # a low-degree seed: kappa = 390
        p = np.zeros(n)
        p[seeds] = 1.0
        truth, _ = O.power(rp, cx, p, 0.85, tol=1e-11)
        alone = np.empty(n)
        st, info = S.wait(S.submit(ids[1], seeds, None, 0.85, 1e-6), alone, timeout_us=120_000_000)
        assert st == pkg.CPAA_OK
        k = O.kappa(rp, p)
        M1 = O.rounds_needed(0.85, 1e-6, k)
        _, _, l1 = O.cpaa(rp, cx, p, 0.85, M1, history=True)
        M2 = O.rounds_posteriori(0.85, 1e-6, l1)
        assert M2 is not None and M2 < M1  # 33 against 34 on this graph
        assert info.rounds == M2
        assert info.bound < 1e-6
        ref = O.cpaa(rp, cx, p, 0.85, info.rounds)
        assert np.abs(alone - ref).sum() / np.abs(ref).sum() <= 1e-6
        assert np.abs(alone - truth).sum() <= 2e-6
        mix = _queries(graphs, 60, seed=9)
        tickets, tq = [], None
        for i, (g2, sd, w, c, tol) in enumerate(mix):
            tickets.append(S.submit(ids[g2], sd, w, c, tol))
            if i == 30:
                tq = S.submit(ids[1], seeds, None, 0.85, 1e-6)
        in_mix = np.empty(n)
        st2, info2 = S.wait(tq, in_mix, timeout_us=120_000_000)
        assert st2 == pkg.CPAA_OK and info2.rounds == info.rounds
        assert np.array_equal(alone, in_mix)
        for t in tickets:
            st3, _ = S.wait(t, None, timeout_us=120_000_000)
            assert st3 == pkg.CPAA_OK
    finally:
        S.close()
        for x in G:
            x.close()


@pytest.mark.parametrize("rule", ["RIGOROUS", "POSTERIORI"])
def test_fused_mode_matches_per_graph_mode(pkg, rule):
    """CPAA_SERVER_FUSED (one launch per round over all graphs, one stream)
    gives the same bits as the per-graph mode, alone and in a mix."""
    graphs = [ci.chung_lu(5000, 40000, seed=31), ci.chung_lu(60000, 600000, seed=32),
              ci.grid_deleted(100, 120, 0.2, seed=3)]
    G = [upload(pkg, g) for g in graphs]
    sr = getattr(pkg, "CPAA_STOP_" + rule)
    qs = _queries(graphs, 40, seed=13)
    out = {}
    try:
        for fused in (False, True):
            S = pkg.Server(2 << 30, stop_rule=sr, fused=fused)
            ids = [S.add_graph(x, 8) for x in G]
            tickets = [S.submit(ids[g2], sd, w, c, tol) for g2, sd, w, c, tol in qs]
            res = []
            for (g2, sd, w, c, tol), t in zip(qs, tickets):
                pi = np.empty(graphs[g2].n)
                st, info = S.wait(t, pi, timeout_us=120_000_000)
                assert st == pkg.CPAA_OK
                res.append((pi, info.rounds))
            out[fused] = res
            S.close()
        for (a, ra), (b, rb) in zip(out[False], out[True]):
            assert ra == rb
            assert np.array_equal(a, b)
        # and against the oracle for a few of them
        for i in (0, 17, 39):
            g2, sd, w, c, tol = qs[i]
            rp, cx = graphs[g2].numpy()
            p = np.zeros(graphs[g2].n)
            p[sd] = 1.0 / len(sd)
            ref = O.cpaa(rp, cx, p, c, out[True][i][1])
            assert np.abs(out[True][i][0] - ref).sum() / np.abs(ref).sum() <= 1e-6
    finally:
        for x in G:
            x.close()


@pytest.mark.parametrize("fused", [False, True])
def test_df64_serving(pkg, fused):
    """Serving in double-float: results within the FP64 bound of the oracle and
    the same bits alone and in a mix, in both launch modes."""
    graphs = [ci.chung_lu(5000, 40000, seed=31), ci.grid_deleted(100, 120, 0.2, seed=3)]
    G = [upload(pkg, g) for g in graphs]
    S = pkg.Server(2 << 30, precision=pkg.CPAA_DF64, fused=fused)
    ids = [S.add_graph(x, 4) for x in G]
    try:
        seeds = np.array([11, 4000], dtype=np.int32)
        alone = np.empty(graphs[0].n)
        st, info = S.wait(S.submit(ids[0], seeds, None, 0.85, 1e-9), alone, timeout_us=120_000_000)
        assert st == pkg.CPAA_OK
        rp, cx = graphs[0].numpy()
        p = np.zeros(graphs[0].n)
        p[seeds] = 0.5
        ref = O.cpaa(rp, cx, p, 0.85, info.rounds)
        assert np.abs(alone - ref).sum() <= 1e-12
        mix = _queries(graphs, 20, seed=2)
        tickets = [S.submit(ids[g2], sd, w, c, tol) for g2, sd, w, c, tol in mix[:10]]
        tq = S.submit(ids[0], seeds, None, 0.85, 1e-9)
        tickets += [S.submit(ids[g2], sd, w, c, tol) for g2, sd, w, c, tol in mix[10:]]
        in_mix = np.empty(graphs[0].n)
        st2, info2 = S.wait(tq, in_mix, timeout_us=120_000_000)
        assert st2 == pkg.CPAA_OK and info2.rounds == info.rounds
        assert np.array_equal(alone, in_mix)
        for t in tickets:
            assert S.wait(t, None, timeout_us=120_000_000)[0] == pkg.CPAA_OK
    finally:
        S.close()
        for x in G:
            x.close()


@pytest.mark.parametrize("prec,fused", [("F32", False), ("F64", False), ("BF16", False), ("DF64", False),
                                        ("F32", True)])
def test_tile_width_follows_live_slots(pkg, prec, fused):
    """A graph's tile is as wide as its highest live slot needs: queries run
    alone compute one column per round, and when the width changes while a
    long query runs, its columns move to the new layout bit for bit (every
    result equals the same query run alone)."""
    import time
    g = ci.chung_lu(300000, 3000000, seed=44)
    G = upload(pkg, g)
    S = pkg.Server(4 << 30, precision=getattr(pkg, "CPAA_" + prec), fused=fused)
    gid = S.add_graph(G, 16)
    n = g.n
    long_q = (np.array([5, 299000, 123456], dtype=np.int32), 0.99, 1e-12)  # 238 rounds
    rng = np.random.default_rng(7)
    short = [(rng.choice(n, size=int(rng.integers(1, 9)), replace=False).astype(np.int32),
              float(rng.choice([0.5, 0.85])), 1e-6) for _ in range(9)]
    try:
        alone = []
        for seeds, c, tol in [long_q] + short:
            pi = np.empty(n)
            st, info = S.wait(S.submit(gid, seeds, None, c, tol), pi, timeout_us=120_000_000)
            assert st == pkg.CPAA_OK
            alone.append((pi, info.rounds))
        s0 = S.stats()
        assert s0["relayouts"] == 0 and s0["round_columns"] == s0["rounds"]
        assert s0["rounds"] == sum(r for _, r in alone)
        # the long query, then a wave of six (slots 1-6: width 8), then, once
        # those are done, two more (width 4), all while the long one may run
        def collect(t):
            pi = np.empty(n)
            st, info = S.wait(t, pi, timeout_us=120_000_000)
            assert st == pkg.CPAA_OK
            return pi, info.rounds

        t_long = S.submit(gid, long_q[0], None, long_q[1], long_q[2])
        time.sleep(0.001)
        wave = [S.submit(gid, sd, None, c, tol) for sd, c, tol in short[:6]]
        res = {1 + i: collect(t) for i, t in enumerate(wave)}
        wave = [S.submit(gid, sd, None, c, tol) for sd, c, tol in short[6:8]]
        res.update({7 + i: collect(t) for i, t in enumerate(wave)})
        res[0] = collect(t_long)
        for i, (pi, r) in res.items():
            assert r == alone[i][1]
            assert np.array_equal(pi, alone[i][0]), i
        s1 = S.stats()
        assert s1["relayouts"] >= 2
        assert s1["round_columns"] > s1["rounds"]
        assert s1["failed"] == 0
        # a lone query after the mix runs at width 1 again
        pi = np.empty(n)
        r0, c0 = s1["rounds"], s1["round_columns"]
        sd, c, tol = short[8]
        st, info = S.wait(S.submit(gid, sd, None, c, tol), pi, timeout_us=120_000_000)
        s2 = S.stats()
        assert np.array_equal(pi, alone[9][0])
        assert s2["rounds"] - r0 == info.rounds
        assert s2["round_columns"] - c0 == info.rounds
    finally:
        S.close()
        G.close()
