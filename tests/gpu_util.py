"""Helpers shared by the GPU tests (no test functions here)."""
import numpy as np
import torch

import cpaa_inputs as ci


def upload(pkg, g, validate=True):
    return pkg.Graph(g.row_ptr.to(torch.int32).cuda(), g.col_idx.to(torch.int32).cuda(), n=g.n,
                     validate=validate)


def solve(pkg, G, p, c, tol=1e-8, **kw):
    pd = torch.as_tensor(np.ascontiguousarray(p), dtype=torch.float64).cuda()
    pi = torch.empty_like(pd)
    info = G.solve(pd, c, tol, pi, **kw)
    torch.cuda.synchronize()
    return pi.cpu().numpy(), info


def boundary_graphs():
    """Graphs that put rows on every side of the tiling thresholds plus ragged
    general graphs.  On graphs this small the hub threshold is 64 and a hub
    tile holds 512 entries, so the star centres (degree n - 1) fall on both
    sides of four and eight tiles (2048 and 4096 entries); the larger graphs of
    the full-size tests use the 4096 threshold and 8192-entry tiles."""
    gs = [ci.star(2046), ci.star(2047), ci.star(2048), ci.star(2049), ci.star(4097),
          ci.star(4098), ci.star(4099), ci.star(9999), ci.path(2), ci.cycle(3),
          ci.complete(70), ci.complete_bipartite(3, 3000),
          ci.chung_lu(3000, 20000, seed=11), ci.chung_lu(60000, 1500000, seed=12),
          ci.grid_deleted(40, 75, seed=3), ci.random_small(1000, 3000, seed=5)]
    # two hubs joined by a path, plus self-loops on a few vertices
    e = [(0, j) for j in range(2, 2600)] + [(1, j) for j in range(1300, 5200)] + \
        [(j, j + 1) for j in range(5200, 5300)] + [(5199, 5200), (7, 7), (5300, 5300)]
    gs.append(ci.from_edges(5301, e, name="two_hubs_loops"))
    return gs
