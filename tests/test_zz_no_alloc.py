"""The no-allocation entry point against the regular one.

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

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_01743_gb300 as pkg
    return pkg


def test_noalloc_matches_regular_solve_twice_in_a_row(pkg):
    g = ci.chung_lu(200_000, 2_000_000, seed=21)
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
    G.close()


def test_noalloc_rejects_oversized_graph(pkg):
    n = pkg.CPAA_NOALLOC_MAX_N + 1
    with pytest.raises(pkg.CpaaError) as e:
        # rejected on the host before any device work
        pkg.cpaa_solve_fixed_noalloc(n, 2 * n, 1, 1, 1, 0.85, 10, 1)
    assert e.value.status == pkg.CPAA_EINVAL
    assert "CPAA_NOALLOC_MAX_N" in str(e.value)
