"""The serving configuration at its full size: 8 resident Chung-Lu graphs of
10k to 8M vertices (mean degree 16), a stream of mixed personalised queries
(uniform graph, 1-16 seeds, c in {0.5, 0.85, 0.95}, tol 1e-6).

Queries on the 4M- and 8M-vertex graphs are compared with the FP64 oracle run
for the rounds the server ran (FP32 serving: relative L1 <= 1e-6; DF64: L1 <=
1e-12), and each equals, bit for bit, the same query served alone, although
its graph's tile changed width while it ran (a burst of queries joined it)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cpaa_inputs as ci
from oracle import oracle as O

pytestmark = pytest.mark.gpu

SIZES = [10_000, 50_000, 200_000, 500_000, 1_000_000, 2_000_000, 4_000_000, 8_000_000]


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_01743_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def mix_graphs(pkg):
    """The serving workload's graphs (as the benchmark builds them), with host
    copies of the 4M and 8M ones for the oracle."""
    G, host = [], {}
    for i, n in enumerate(SIZES):
        g = ci.chung_lu(n, 8 * n, seed=100 + i, device="cuda")
        G.append(pkg.Graph(g.row_ptr, g.col_idx, n=g.n))
        if n >= 4_000_000:
            host[i] = g.numpy()
        del g
    torch.cuda.empty_cache()
    yield G, host
    for x in G:
        x.close()


def _mix(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        gi = int(rng.integers(len(SIZES)))
        k = int(rng.integers(1, 17))
        seeds = rng.choice(SIZES[gi], size=k, replace=False).astype(np.int32)
        out.append((gi, seeds, float(rng.choice([0.5, 0.85, 0.95]))))
    return out


# the two queries compared with the oracle: a 3-seed one on the 8M graph and a
# 9-seed one on the 4M graph, both c = 0.85, tol 1e-6
T8 = (7, np.array([11, 4_321_987, 7_999_990], dtype=np.int32), 0.85)
T4 = (6, np.array([0, 5, 77, 1000, 65_536, 1_234_567, 2_000_001, 3_333_333, 3_999_999], dtype=np.int32), 0.85)


def _p(n, seeds):
    p = np.zeros(n)
    p[seeds] = 1.0 / len(seeds)
    return p


@pytest.fixture(scope="module")
def oracle_refs(mix_graphs):
    """Oracle results of T8 and T4 for the rounds the rigorous rule gives
    (the same M whatever the serving precision: it depends on c, tol and
    kappa only), computed once."""
    _, host = mix_graphs
    refs = {}
    for gi, seeds, c in (T8, T4):
        rp, cx = host[gi]
        p = _p(SIZES[gi], seeds)
        M = O.rounds_needed(c, 1e-6, O.kappa(rp, p))
        refs[gi] = (M, O.cpaa(rp, cx, p, c, M))
    return refs


def _serve(pkg, G, precision, nmix):
    """Alone runs of T8 and T4, then T8, a burst of 12 queries on its graph
    (width 1 -> 16 while T8 runs), and a random mix with T4 in the middle."""
    S = pkg.Server(64 << 30, precision=precision)
    ids = [S.add_graph(x, 16) for x in G]
    try:
        def collect(t, gi):
            pi = np.empty(SIZES[gi])
            st, info = S.wait(t, pi, timeout_us=600_000_000)
            assert st == pkg.CPAA_OK
            return pi, info.rounds

        alone = {}
        for gi, seeds, c in (T8, T4):
            alone[gi] = collect(S.submit(ids[gi], seeds, None, c, 1e-6), gi)
        r0 = S.stats()["relayouts"]
        t8 = S.submit(ids[T8[0]], T8[1], None, T8[2], 1e-6)
        time.sleep(0.002)
        rng = np.random.default_rng(17)
        burst = [(7, rng.choice(SIZES[7], size=4, replace=False).astype(np.int32), 0.5) for _ in range(12)]
        tickets = [(gi, S.submit(ids[gi], sd, None, c, 1e-6)) for gi, sd, c in burst]
        mix = _mix(nmix, seed=23)
        t4 = None
        for i, (gi, sd, c) in enumerate(mix):
            tickets.append((gi, S.submit(ids[gi], sd, None, c, 1e-6)))
            if i == nmix // 2:
                t4 = S.submit(ids[T4[0]], T4[1], None, T4[2], 1e-6)
        in_mix = {T8[0]: collect(t8, T8[0]), T4[0]: collect(t4, T4[0])}
        sums = []
        for gi, t in tickets:
            pi, _ = collect(t, gi)
            sums.append(pi.sum())
        st = S.stats()
        assert st["failed"] == 0
        assert st["relayouts"] > r0
        assert np.abs(np.array(sums) - 1.0).max() < 1e-9
        return alone, in_mix
    finally:
        S.close()


@pytest.mark.parametrize("prec,bound,relative", [("F32", 1e-6, True), ("DF64", 1e-12, False)])
def test_serving_full_size_against_oracle(pkg, mix_graphs, oracle_refs, prec, bound, relative):
    G, _ = mix_graphs
    alone, in_mix = _serve(pkg, G, getattr(pkg, "CPAA_" + prec), 300 if prec == "F32" else 120)
    for gi in (T8[0], T4[0]):
        M, ref = oracle_refs[gi]
        pa, ra = alone[gi]
        pm, rm = in_mix[gi]
        assert ra == rm == M
        assert np.array_equal(pa, pm), gi
        err = np.abs(pa - ref).sum()
        if relative:
            err /= np.abs(ref).sum()
        print("serving %s, graph %d (n=%d): %d rounds, %s L1 %.3e" %
              (prec, gi, SIZES[gi], M, "relative" if relative else "absolute", err))
        assert err <= bound
