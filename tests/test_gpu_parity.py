"""GPU parity: the CUDA path against the FP64 oracle, through the C ABI.

Tolerances: FP64 path L1 <= 1e-12; FP32 path relative L1 <= 1e-6 (both
against the oracle run for the same number of rounds M).  The BF16 path's
error is measured and only bounded loosely (it is a precision study)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cpaa_inputs as ci
from oracle import oracle as O
from tests.gpu_util import boundary_graphs, solve, upload

pytestmark = pytest.mark.gpu

GRAPHS = boundary_graphs()


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_01743_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def uploaded(pkg):
    return [upload(pkg, g) for g in GRAPHS]


def _p_variants(n):
    uni = np.full(n, 1.0 / n)
    seed = np.zeros(n); seed[n // 2] = 1.0
    ramp = np.arange(1, n + 1, dtype=float); ramp /= ramp.sum()
    return {"uniform": uni, "seed": seed, "ramp": ramp}


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=[g.name for g in GRAPHS])
def test_f64_fixed_rounds_matches_oracle(pkg, uploaded, gi):
    g, G = GRAPHS[gi], uploaded[gi]
    rp, cx = g.numpy()
    for pname, p in _p_variants(g.n).items():
        for M in (1, 2, 3, 17):
            for norm in (0, 1):
                pi, info = solve(pkg, G, p, 0.85, fixed_rounds=M, normalize=norm)
                ref = O.cpaa(rp, cx, p, 0.85, M, normalize=norm)
                assert info.rounds == M
                err = np.abs(pi - ref).sum()
                assert err <= 1e-12, (g.name, pname, M, norm, err)


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=[g.name for g in GRAPHS])
@pytest.mark.parametrize("c", [0.5, 0.85, 0.95])
def test_f64_tolerance_solve(pkg, uploaded, gi, c):
    """M equals the oracle's stopping rule, and the result is within tol of pi*."""
    g, G = GRAPHS[gi], uploaded[gi]
    rp, cx = g.numpy()
    p = _p_variants(g.n)["ramp"]
    tol = 1e-9
    pi, info = solve(pkg, G, p, c, tol)
    k_or = O.kappa(rp, p)
    assert abs(info.kappa - k_or) <= 1e-12 * k_or
    assert info.rounds == O.rounds_needed(c, tol, k_or, 0)
    ref = O.cpaa(rp, cx, p, c, info.rounds)
    assert np.abs(pi - ref).sum() <= 1e-12
    if g.n <= 2500:
        truth = O.lapack_pagerank(rp, cx, p, c)
    else:  # the power method's L1 change stalls near 1e-14 from rounding
        truth, _ = O.power(rp, cx, p, c, tol=1e-11)
    assert np.abs(pi - truth).sum() <= tol


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=[g.name for g in GRAPHS])
def test_f32_matches_oracle(pkg, uploaded, gi):
    g, G = GRAPHS[gi], uploaded[gi]
    rp, cx = g.numpy()
    for pname, p in _p_variants(g.n).items():
        pi, info = solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_F32)
        ref = O.cpaa(rp, cx, p, 0.85, info.rounds)
        rel = np.abs(pi - ref).sum() / np.abs(ref).sum()
        assert rel <= 1e-6, (g.name, pname, rel)


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=[g.name for g in GRAPHS])
def test_df64_matches_oracle(pkg, uploaded, gi):
    """Double-float iterates (pairs of FP32, about 48 significant bits): the
    FP64 bound, L1 <= 1e-12 against the oracle for the same M, at a fixed M and
    from the stopping rule, for three vectors."""
    g, G = GRAPHS[gi], uploaded[gi]
    rp, cx = g.numpy()
    for pname, p in _p_variants(g.n).items():
        pi, info = solve(pkg, G, p, 0.85, 1e-9, precision=pkg.CPAA_DF64)
        ref = O.cpaa(rp, cx, p, 0.85, info.rounds)
        assert np.abs(pi - ref).sum() <= 1e-12, (g.name, pname)
        pi, _ = solve(pkg, G, p, 0.95, fixed_rounds=60, precision=pkg.CPAA_DF64)
        ref = O.cpaa(rp, cx, p, 0.95, 60)
        assert np.abs(pi - ref).sum() <= 1e-12, (g.name, pname, "M=60")


@pytest.mark.parametrize("gi", [0, 3, 12, 13, 14], ids=lambda i: GRAPHS[i].name)
def test_bf16_error_is_bounded(pkg, uploaded, gi):
    g, G = GRAPHS[gi], uploaded[gi]
    rp, cx = g.numpy()
    p = np.full(g.n, 1.0 / g.n)
    pi, info = solve(pkg, G, p, 0.85, 1e-6, precision=pkg.CPAA_BF16)
    ref = O.cpaa(rp, cx, p, 0.85, info.rounds)
    rel = np.abs(pi - ref).sum() / np.abs(ref).sum()
    assert rel <= 5e-2, rel
    assert abs(pi.sum() - 1.0) < 1e-12


def test_mass_invariant_history(pkg, uploaded):
    g, G = GRAPHS[13], uploaded[13]
    rp, cx = g.numpy()
    p = _p_variants(g.n)["seed"]
    M = 30
    hist = np.zeros(2 * (M + 1))
    solve(pkg, G, p, 0.85, fixed_rounds=M, history=hist)
    _, mass, l1 = O.cpaa(rp, cx, p, 0.85, M, history=True)
    assert np.abs(hist[0::2] - 1.0).max() < 1e-12
    assert np.abs(hist[0::2] - mass).max() < 1e-12
    assert np.abs(hist[1::2] - l1).max() < 1e-10 * l1.max()


def test_host_and_device_io_agree_and_repeat_bitwise(pkg, uploaded):
    g, G = GRAPHS[13], uploaded[13]
    p = _p_variants(g.n)["ramp"]
    for prec in (pkg.CPAA_F64, pkg.CPAA_F32, pkg.CPAA_BF16):
        a, _ = solve(pkg, G, p, 0.85, 1e-7, precision=prec)
        b, _ = solve(pkg, G, p, 0.85, 1e-7, precision=prec)
        host_pi = np.empty(g.n)
        G.solve(np.ascontiguousarray(p), 0.85, 1e-7, host_pi, precision=prec)
        assert np.array_equal(a, b)
        assert np.array_equal(a, host_pi)


def test_reversibility_on_gpu(pkg, uploaded):
    """pi_s(t)/d_t = pi_t(s)/d_s ((D - cA)^-1 is symmetric, Lemma 2's B)."""
    g, G = GRAPHS[12], uploaded[12]
    rp, _ = g.numpy()
    d = np.diff(rp).astype(float)
    s, t = 5, 2900
    es = np.zeros(g.n); es[s] = 1
    et = np.zeros(g.n); et[t] = 1
    a, _ = solve(pkg, G, es, 0.85, 1e-13)
    b, _ = solve(pkg, G, et, 0.85, 1e-13)
    assert abs(a[t] / d[t] - b[s] / d[s]) < 1e-12 * max(a[t] / d[t], 1e-300) + 1e-15


def test_truncation_with_a_negative_entry(pkg):
    """At c = 0.95 the degree-2 truncation's constant term c_0/2 - c_2 is
    negative, so on K_50 with one seed pibar after M = 2 rounds is negative at
    the seed.  The device path matches the oracle there in both
    normalisations (the divide-by-sum uses the signed sum)."""
    g = ci.complete(50)
    G = upload(pkg, g)
    rp, cx = g.numpy()
    p = np.zeros(50); p[0] = 1.0
    assert O.cpaa(rp, cx, p, 0.95, 2, normalize=1).min() < -1e-4
    for norm in (0, 1):
        ref = O.cpaa(rp, cx, p, 0.95, 2, normalize=norm)
        for prec in ("F64", "DF64", "F32"):
            pi, info = solve(pkg, G, p, 0.95, fixed_rounds=2, normalize=norm,
                             precision=getattr(pkg, "CPAA_" + prec))
            assert info.rounds == 2
            err = np.abs(pi - ref).sum()
            if prec == "F32":
                assert err / np.abs(ref).sum() <= 1e-6, (norm, err)
            else:
                assert err <= 1e-12, (prec, norm, err)


def test_single_vertex_self_loop(pkg):
    G = upload(pkg, ci.from_edges(1, [(0, 0)], name="one"))
    pi, info = solve(pkg, G, np.ones(1), 0.85, 1e-10)
    assert pi[0] == pytest.approx(1.0, abs=1e-15)


def test_invalid_arguments(pkg, uploaded):
    G = uploaded[12]
    n = GRAPHS[12].n
    p = np.full(n, 1.0 / n)
    bad = p.copy(); bad[3] = -bad[3]
    with pytest.raises(pkg.CpaaError):
        solve(pkg, G, bad, 0.85)
    with pytest.raises(pkg.CpaaError):
        solve(pkg, G, 2 * p, 0.85)
    nan = p.copy(); nan[0] = np.nan
    with pytest.raises(pkg.CpaaError):
        solve(pkg, G, nan, 0.85)
    for c in (0.0, 1.0, -0.5, 1.5):
        with pytest.raises(pkg.CpaaError):
            solve(pkg, G, p, c)
    with pytest.raises(pkg.CpaaError):
        solve(pkg, G, p, 0.85, tol=0.0)
    # status is ENOTCONV when the bound asks for more than max_rounds
    pd = torch.as_tensor(p).cuda()
    out = torch.empty_like(pd)
    info = G.solve(pd, 0.85, 1e-12, out, max_rounds=5, raise_notconv=False)
    assert info.rounds == 5


def test_invalid_graphs(pkg):
    def mk(n, rp, cx, validate=True):
        return pkg.Graph(torch.tensor(rp, dtype=torch.int32).cuda(),
                         torch.tensor(cx, dtype=torch.int32).cuda(), n=n, validate=validate)
    with pytest.raises(pkg.CpaaError):      # directed: 0->1 without 1->0
        mk(2, [0, 1, 2], [1, 1])
    with pytest.raises(pkg.CpaaError):      # vertex 1 has degree 0
        mk(3, [0, 1, 1, 2], [2, 0])
    with pytest.raises(pkg.CpaaError):      # column out of range
        mk(2, [0, 1, 2], [1, 5])
    with pytest.raises(pkg.CpaaError):      # unsorted row
        mk(3, [0, 2, 3, 4], [2, 1, 0, 0])
    with pytest.raises(pkg.CpaaError):      # row_ptr[n] != nnz
        pkg.cpaa_graph_create(2, 3, torch.tensor([0, 1, 2], dtype=torch.int32).cuda(),
                              torch.tensor([1, 0, 0], dtype=torch.int32).cuda())


def test_invalid_graphs_default_flags(pkg):
    """With the default flags (no CPAA_GRAPH_VALIDATE) an asymmetric CSR, an
    unsorted row and a column >= n or < 0 are rejected with CPAA_EINVAL
    (Sec. 2.1: A symmetric; the remark closing Sec. 3), with the offending
    count in the message; host and device inputs alike."""
    import re
    cases = [(2, [0, 1, 2], [1, 1], r"[1-9]\d* entr\(ies\) without a mirror"),   # 0 -> 1, no 1 -> 0
             (3, [0, 2, 3, 4], [1, 2, 0, 1], r"2 entr\(ies\) without a mirror"),  # 0-2 and 2-1 unmatched
             (2, [0, 1, 2], [1, 2], r"^.*: 1 column\(s\) out of range"),           # column n
             (2, [0, 1, 2], [1, -1], r"^.*: 1 column\(s\) out of range"),          # negative column
             (3, [0, 2, 3, 4], [2, 1, 0, 0], r"[1-9]\d* unsorted")]
    for n, rp, cx, msg in cases:
        for dev in (False, True):
            r = torch.tensor(rp, dtype=torch.int32)
            c = torch.tensor(cx, dtype=torch.int32)
            if dev:
                r, c = r.cuda(), c.cuda()
            with pytest.raises(pkg.CpaaError) as ei:
                pkg.cpaa_graph_create(n, len(cx), r, c)
            assert ei.value.status == pkg.CPAA_EINVAL
            assert re.search(msg, str(ei.value)), str(ei.value)


def test_out_of_range_column_trusted(pkg):
    """CPAA_GRAPH_TRUSTED skips the order and symmetry checks, never the column
    range: the relabelling pass counts the bad entry (it is not used as an
    index) and the graph is rejected; a valid graph created trusted solves
    like a checked one."""
    for cx in ([1, 2], [1, -7], [1, 1 << 30]):
        with pytest.raises(pkg.CpaaError) as ei:
            pkg.cpaa_graph_create(2, 2, torch.tensor([0, 1, 2], dtype=torch.int32).cuda(),
                                  torch.tensor(cx, dtype=torch.int32).cuda(), pkg.CPAA_GRAPH_TRUSTED)
        assert ei.value.status == pkg.CPAA_EINVAL
        assert "out of range" in str(ei.value)
    g = ci.chung_lu(3000, 20000, seed=11)
    G1 = upload(pkg, g, validate=True)
    G2 = upload(pkg, g, validate=False)
    p = np.zeros(g.n)
    p[[1, 2000]] = 0.5
    a, ia = solve(pkg, G1, p, 0.85)
    b, ib = solve(pkg, G2, p, 0.85)
    assert ia.rounds == ib.rounds and np.array_equal(a, b)
    G1.close()
    G2.close()


def test_batch_columns_equal_single(pkg, uploaded):
    g, G = GRAPHS[13], uploaded[13]
    B = 5
    seeds = ci.seed_vectors(g.n, B, seed=3)
    P = ci.seed_dense(g.n, seeds)
    cs = np.array([0.5, 0.85, 0.95, 0.85, 0.7])
    for prec in (pkg.CPAA_F64, pkg.CPAA_F32, pkg.CPAA_DF64, pkg.CPAA_BF16):
        Pd = torch.as_tensor(P).cuda()
        PI = torch.empty_like(Pd)
        infos = G.solve_batch(B, Pd, cs, 1e-7, PI, precision=prec)
        torch.cuda.synchronize()
        for b in range(B):
            single, info = solve(pkg, G, P[b], cs[b], 1e-7, precision=prec)
            assert infos[b].rounds == info.rounds
            assert np.array_equal(PI[b].cpu().numpy(), single)


@pytest.mark.parametrize("prec", ["F32", "BF16", "DF64"])
def test_deferred_accumulation_every_round_count(pkg, uploaded, prec):
    """The single-vector FP32, BF16 and DF64 solves add a term c_k y_k one
    round late, from the stored y_k (deferred accumulation); tiles of two do
    not.  For every round count from 1 to 9 (odd counts end on a term that may
    not be deferred) the two agree bit for bit, and both match the oracle."""
    P = getattr(pkg, "CPAA_" + prec)
    tol = {"F32": 1e-6, "BF16": 5e-2, "DF64": 1e-12}[prec]
    for gi in (12, 13, 14):
        g, G = GRAPHS[gi], uploaded[gi]
        rp, cx = g.numpy()
        p = ci.seed_dense(g.n, ci.seed_vectors(g.n, 1, seed=21 + gi))[0]
        Pd = torch.as_tensor(np.stack([p, p])).cuda()
        for M in range(1, 10):
            single, info = solve(pkg, G, p, 0.85, fixed_rounds=M, precision=P)
            assert info.rounds == M
            PI = torch.empty_like(Pd)
            G.solve_batch(2, Pd, np.full(2, 0.85), 0.0, PI, precision=P, fixed_rounds=M, batch_width=2)
            torch.cuda.synchronize()
            assert np.array_equal(PI[0].cpu().numpy(), single), (gi, M)
            assert np.array_equal(PI[1].cpu().numpy(), single), (gi, M)
            ref = O.cpaa(rp, cx, p, 0.85, M)
            assert np.abs(single - ref).sum() / np.abs(ref).sum() <= tol, (gi, M)


def test_batch_on_fresh_graph(pkg):
    """A batch as the very first solve on a graph (no earlier single solve has
    set up the workspace), with the automatic tile width."""
    g = ci.chung_lu(50000, 600000, seed=77)
    G = upload(pkg, g)
    B = 20
    P = ci.seed_dense(g.n, ci.seed_vectors(g.n, B, seed=8))
    Pd = torch.as_tensor(P).cuda()
    PI = torch.empty_like(Pd)
    infos = G.solve_batch(B, Pd, np.full(B, 0.85), 1e-6, PI, precision=pkg.CPAA_F32)
    torch.cuda.synchronize()
    rp, cx = g.numpy()
    for b in (0, 7, 19):
        ref = O.cpaa(rp, cx, P[b], 0.85, infos[b].rounds)
        assert np.abs(PI[b].cpu().numpy() - ref).sum() / np.abs(ref).sum() <= 1e-6
    G.close()


@pytest.mark.parametrize("gi", [0, 3, 12, 13, 14, 16], ids=lambda i: GRAPHS[i].name)
def test_power_method_matches_oracle(pkg, uploaded, gi):
    """The power-method baseline on the same kernels against the oracle's power
    method for the same rounds (FP64 L1 <= 1e-12), and its rigorous rounds."""
    g, G = GRAPHS[gi], uploaded[gi]
    rp, cx = g.numpy()
    p = _p_variants(g.n)["ramp"]
    pd = torch.as_tensor(p).cuda()
    out = torch.empty_like(pd)
    for T in (1, 2, 7, 30):
        G.power_solve(pd, 0.85, 0.0, out, fixed_rounds=T, normalize=1)
        torch.cuda.synchronize()
        ref, _ = O.power(rp, cx, p, 0.85, rounds=T)
        assert np.abs(out.cpu().numpy() - ref).sum() <= 1e-12, (g.name, T)
    info = G.power_solve(pd, 0.85, 1e-8, out)
    torch.cuda.synchronize()
    T = next(t for t in range(1, 1000) if 2 * 0.85 ** t < 1e-8)
    assert info.rounds == T
    if g.n <= 2500:
        truth = O.lapack_pagerank(rp, cx, p, 0.85)
        assert np.abs(out.cpu().numpy() - truth).sum() <= 1e-8
    outdf = torch.empty_like(pd)
    G.power_solve(pd, 0.85, 0.0, outdf, fixed_rounds=30, normalize=1, precision=pkg.CPAA_DF64)
    torch.cuda.synchronize()
    ref, _ = O.power(rp, cx, p, 0.85, rounds=30)
    assert np.abs(outdf.cpu().numpy() - ref).sum() <= 1e-12, (g.name, "DF64")
    out32 = torch.empty_like(pd)
    G.power_solve(pd, 0.85, 1e-6, out32, precision=pkg.CPAA_F32)
    torch.cuda.synchronize()
    ref, _ = O.power(rp, cx, p, 0.85, rounds=next(t for t in range(1, 1000) if 2 * 0.85 ** t < 1e-6))
    assert np.abs(out32.cpu().numpy() - ref).sum() / np.abs(ref).sum() <= 1e-6


def test_round_graph_cache_across_keys_and_workspace_growth(pkg):
    """The captured round sequences are keyed by every launch value: alternating
    round counts, dampings and precisions, and a batch that grows the workspace
    in between, all give the oracle's result."""
    g = ci.chung_lu(20000, 150000, seed=41)
    G = upload(pkg, g)
    rp, cx = g.numpy()
    p = _p_variants(g.n)["ramp"]
    seq = [(10, 0.85, "F64"), (20, 0.85, "F64"), (10, 0.5, "F64"), (10, 0.85, "F32"), (10, 0.85, "F64")]
    for i, (M, c, prec) in enumerate(seq):
        if i == 3:  # grow the workspace (wider tile, more rounds) between solves
            P = ci.seed_dense(g.n, ci.seed_vectors(g.n, 16, seed=2))
            Pd = torch.as_tensor(P).cuda()
            PI = torch.empty_like(Pd)
            G.solve_batch(16, Pd, np.full(16, 0.85), 0.0, PI, fixed_rounds=40, precision=pkg.CPAA_F32,
                          batch_width=16)
            torch.cuda.synchronize()
        pi, info = solve(pkg, G, p, c, fixed_rounds=M, precision=getattr(pkg, "CPAA_" + prec))
        ref = O.cpaa(rp, cx, p, c, M)
        err = np.abs(pi - ref).sum()
        assert info.rounds == M
        assert err <= (1e-12 if prec == "F64" else 1e-6 * np.abs(ref).sum()), (i, err)
    G.close()


def test_layout_thresholds(pkg, uploaded):
    """cpaa_graph_layout reports the tiling the thresholds give: on the small
    boundary graphs a hub threshold of 64 and 512-entry hub tiles, hub rows
    cut into ceil(degree / 512) tiles, every entry in a hub row or a chunk."""
    for g, G in zip(GRAPHS, uploaded):
        lay = G.layout()
        rp, _ = g.numpy()
        deg = np.diff(rp)
        assert lay["hub_degree"] == 64 if g.nnz < 64 * 4096 else lay["hub_degree"] == min(4096, g.nnz // 4096)
        assert lay["hub_tile"] == max(512, 2 * lay["hub_degree"])
        hub = deg[deg > lay["hub_degree"]]
        assert lay["hub_rows"] == hub.size
        assert lay["hub_entries"] == hub.sum()
        assert lay["hub_tiles"] == int(np.sum((hub + lay["hub_tile"] - 1) // lay["hub_tile"]))
        rest = g.n - hub.size
        assert lay["chunks"] == (rest + 31) // 32
        assert lay["sell_entries"] >= deg.sum() - hub.sum()
        assert 0 <= lay["long_chunks"] <= lay["chunks"]
