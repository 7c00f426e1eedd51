"""The no-allocation entry point against the regular solve and the oracle.

cpaa_solve_fixed_noalloc serves callers that cannot allocate device memory
(an application whose allocator owns the device, a strict memory budget, or a
loop that cannot take cudaMalloc's synchronisation): it keeps every
intermediate vector in the library's fixed 32 MiB per-GPU scratch array.
This file runs last, so a stop-at-first-failure run has done everything else
first; it also passes on its own in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cpaa_inputs as ci
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_01743_gb300 as pkg
    return pkg


def test_noalloc_matches_regular_solve_twice_in_a_row(pkg):
    g = ci.chung_lu(200_000, 2_000_000, seed=21)
    rp_h, cx_h = g.numpy()
    rp = g.row_ptr.to(torch.int32).cuda()
    cx = g.col_idx.to(torch.int32).cuda()
    G = pkg.Graph(rp, cx, n=g.n, validate=True)
    n = g.n
    uni = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    seeded = torch.zeros(n, dtype=torch.float64, device="cuda")
    seeded[[3, 1000, n - 1]] = 1.0 / 3.0
    # two calls in a row with different inputs: the second must not see the
    # first one's leftovers in the shared scratch array
    for p, M, norm in ((uni, 25, 0), (seeded, 31, 1)):
        ref = torch.empty_like(p)
        G.solve(p, 0.85, 0.0, ref, fixed_rounds=M, normalize=norm)
        out = torch.full_like(p, float("nan"))
        pkg.cpaa_solve_fixed_noalloc(n, g.nnz, rp, cx, p, 0.85, M, out, normalize=norm)
        torch.cuda.synchronize()
        err = float((out - ref).abs().sum())
        assert err <= 1e-12, (M, norm, err)
        # and against the FP64 oracle directly (Algorithm 1, M rounds)
        want = O.cpaa(rp_h, cx_h, p.cpu().numpy(), 0.85, M, normalize=norm)
        err_o = float(np.abs(out.cpu().numpy() - want).sum())
        assert err_o <= 1e-12, (M, norm, err_o)
    G.close()


def test_noalloc_at_the_size_limit_against_the_oracle(pkg):
    """n = CPAA_NOALLOC_MAX_N exactly: the largest graph the scratch array
    holds, ragged degrees (Chung-Lu plus ring), against the oracle for M
    rounds, and rounds = 0 (pi = p after normalisation, Algorithm 1 with no
    recurrence term)."""
    n = pkg.CPAA_NOALLOC_MAX_N
    g = ci.chung_lu(n, 4 * n, seed=22, device="cuda")
    rp_h, cx_h = g.numpy()
    hp = np.zeros(n)
    hp[[0, 17, n // 3, n - 1]] = 0.25
    p = torch.as_tensor(hp).cuda()
    for M, norm in ((12, 0), (0, 0), (1, 1)):
        out = torch.full_like(p, float("nan"))
        pkg.cpaa_solve_fixed_noalloc(n, g.nnz, g.row_ptr, g.col_idx, p, 0.85, M, out, normalize=norm)
        torch.cuda.synchronize()
        want = O.cpaa(rp_h, cx_h, hp, 0.85, M, normalize=norm)
        err = float(np.abs(out.cpu().numpy() - want).sum())
        assert err <= 1e-12, (M, norm, err)


def test_noalloc_rejects_invalid_csr(pkg):
    """A column equal to n, a negative column and a row of degree 0 give
    CPAA_EINVAL (the kernels skip such entries, so nothing is read out of
    bounds), for rounds >= 1 and for rounds = 0; a valid call right after each
    still succeeds (the error counter starts at zero every call)."""
    good_rp = torch.tensor([0, 2, 4, 6], dtype=torch.int32).cuda()   # triangle
    good_cx = torch.tensor([1, 2, 0, 2, 0, 1], dtype=torch.int32).cuda()
    p = torch.full((3,), 1.0 / 3, dtype=torch.float64).cuda()
    cases = [
        (good_rp, torch.tensor([1, 3, 0, 2, 0, 1], dtype=torch.int32).cuda(), 6),   # column n
        (good_rp, torch.tensor([1, 2, 0, -1, 0, 1], dtype=torch.int32).cuda(), 6),  # negative column
        (torch.tensor([0, 1, 1, 2], dtype=torch.int32).cuda(),                       # vertex 1: degree 0
         torch.tensor([2, 0], dtype=torch.int32).cuda(), 2),
    ]
    for rp, cx, nnz in cases:
        for M in (0, 1, 5):
            out = torch.empty_like(p)
            with pytest.raises(pkg.CpaaError) as e:
                pkg.cpaa_solve_fixed_noalloc(3, nnz, rp, cx, p, 0.85, M, out)
            assert e.value.status == pkg.CPAA_EINVAL
            assert "invalid CSR" in str(e.value)
            out = torch.empty_like(p)
            pkg.cpaa_solve_fixed_noalloc(3, 6, good_rp, good_cx, p, 0.85, M, out)
            torch.cuda.synchronize()
            # a regular graph with uniform p: pi is uniform after every M (Sec. 4.1)
            assert float((out - 1.0 / 3).abs().max()) <= 1e-15


def test_noalloc_rejects_oversized_graph(pkg):
    n = pkg.CPAA_NOALLOC_MAX_N + 1
    with pytest.raises(pkg.CpaaError) as e:
        # rejected on the host before any device work
        pkg.cpaa_solve_fixed_noalloc(n, 2 * n, 1, 1, 1, 0.85, 10, 1)
    assert e.value.status == pkg.CPAA_EINVAL
    assert "CPAA_NOALLOC_MAX_N" in str(e.value)
