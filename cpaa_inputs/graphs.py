"""Seeded undirected graphs as symmetric CSR (int32 row_ptr / col_idx).

Every generator returns a ``Csr`` whose rows list each neighbour once, in
ascending order, with no self-loops (unless a caller builds one on purpose
with ``from_edges``).  The same seed gives the same graph on CPU and on CUDA.

Workload recipes (the paper's own datasets are not available; these stand in):
* ``chung_lu``: weights w_i = (i+1)^(-1/(gamma-1)); draw E endpoint pairs
  i.i.d. from categorical(w) by inverse CDF on 53-bit counter-based integers;
  drop self-loops and duplicates; add the ring (i, i+1 mod n) so every vertex
  has degree >= 2.  Vertex ids stay in weight order (hubs first).  With
  ``distinct=True``, E counts distinct edges instead of draws: the graph keeps
  the first E distinct non-loop pairs in draw order (draws continue until E
  are found), then adds the ring.
* ``grid_deleted``: a rows x cols 4-neighbour lattice; every vertex but the
  corner (0,0) keeps one edge to its upper or left neighbour (chosen by a
  hashed bit), which forms a spanning tree; a seeded uniform sample of the
  remaining edges, of size ``round(frac * all edges)``, is deleted.
"""
from dataclasses import dataclass
import itertools

import numpy as np
import torch

from . import rng


@dataclass
class Csr:
    n: int
    row_ptr: torch.Tensor   # int32 [n+1]
    col_idx: torch.Tensor   # int32 [nnz]
    name: str = ""

    @property
    def nnz(self):
        return int(self.col_idx.numel())

    def numpy(self):
        return (self.row_ptr.cpu().numpy().astype(np.int32),
                self.col_idx.cpu().numpy().astype(np.int32))

    def to(self, device):
        return Csr(self.n, self.row_ptr.to(device), self.col_idx.to(device), self.name)


def _csr_from_undirected_keys(n, keys, device, name):
    """keys: unique int64 min*n+max of undirected edges (u < v or loops u == v)."""
    a = keys // n
    b = keys % n
    loop = a == b
    rows = torch.cat([a, b[~loop]])
    cols = torch.cat([b, a[~loop]])
    del a, b
    k2 = rows * n + cols
    del rows, cols
    k2, _ = torch.sort(k2)
    rows = k2 // n
    counts = torch.bincount(rows, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    if int(row_ptr[-1]) >= 2 ** 31:
        raise ValueError("graph too large for int32 CSR")
    col_idx = (k2 % n).to(torch.int32)
    return Csr(n, row_ptr.to(torch.int32), col_idx, name)


def from_edges(n, edges, device="cpu", name="edges"):
    """Symmetric CSR from an undirected edge list [(u, v), ...]; duplicates merge."""
    e = torch.as_tensor(np.asarray(edges, dtype=np.int64).reshape(-1, 2), device=device)
    u = torch.minimum(e[:, 0], e[:, 1])
    v = torch.maximum(e[:, 0], e[:, 1])
    keys = torch.unique(u * n + v)
    return _csr_from_undirected_keys(n, keys, device, name)


def _chung_lu_keys(n, cum_t, seed, start, stop, device):
    """Keys min * n + max of draws [start, stop), self-loops dropped, in draw order."""
    idx = rng.arange(start, stop, device)
    r1 = rng.u53(seed, 0, idx)
    r2 = rng.u53(seed, 1, idx)
    u = torch.searchsorted(cum_t, r1, right=True)
    v = torch.searchsorted(cum_t, r2, right=True)
    del r1, r2, idx
    keep = u != v
    u, v = u[keep], v[keep]
    return torch.minimum(u, v) * n + torch.maximum(u, v)


def chung_lu(n, edges, gamma=2.1, seed=0, ring=True, device="cpu", chunk=1 << 25, distinct=False):
    """Chung-Lu power-law graph (see module docstring)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    w = i ** (-1.0 / (gamma - 1.0))
    cum = np.cumsum(w)
    cum_int = np.floor(cum / cum[-1] * float(2 ** 53)).astype(np.int64)
    cum_int[-1] = 2 ** 53
    cum_t = torch.as_tensor(cum_int, device=device)
    parts = []
    if distinct:
        if edges > n * (n - 1) // 2:
            raise ValueError("more distinct edges than vertex pairs")
        have = torch.empty(0, dtype=torch.int64, device=device)  # kept keys, sorted
        start = 0
        while have.numel() < edges:
            k = _chung_lu_keys(n, cum_t, seed, start, start + chunk, device)
            start += chunk
            if have.numel():
                pos = torch.searchsorted(have, k).clamp_(max=have.numel() - 1)
                k = k[have[pos] != k]
            if k.numel() == 0:
                continue
            # first occurrence of each new key within the chunk, in draw order
            uk, inv = torch.unique(k, return_inverse=True)
            first = torch.full((uk.numel(),), k.numel(), dtype=torch.int64, device=device)
            first.scatter_reduce_(0, inv, torch.arange(k.numel(), device=device), reduce="amin")
            newk = uk[torch.argsort(first)][:edges - have.numel()]
            have, _ = torch.sort(torch.cat([have, newk]))
            del k, uk, inv, first, newk
        parts.append(have)
    else:
        for start in range(0, edges, chunk):
            parts.append(torch.unique(_chung_lu_keys(n, cum_t, seed, start, min(edges, start + chunk), device)))
    if ring and n > 1:
        a = rng.arange(0, n, device)
        b = (a + 1) % n
        lo = torch.minimum(a, b)
        hi = torch.maximum(a, b)
        parts.append(torch.unique(lo * n + hi))
    keys = torch.unique(torch.cat(parts))
    del parts
    return _csr_from_undirected_keys(n, keys, device, "chung_lu(n=%d,E=%d%s,gamma=%g,seed=%d)"
                                     % (n, edges, " distinct" if distinct else "", gamma, seed))


def grid_deleted(rows, cols, frac=0.2, seed=0, device="cpu"):
    """Lattice with a seeded fraction of edges deleted, kept connected."""
    R, C = rows, cols
    n = R * C
    nh = R * (C - 1)          # horizontal edge (r,c)-(r,c+1): id r*(C-1)+c
    nv = (R - 1) * C          # vertical edge (r,c)-(r+1,c):   id nh + r*C + c
    total = nh + nv
    vid = rng.arange(0, n, device)
    r = vid // C
    c = vid % C
    bit = rng.u32(seed, 7, vid) & 1
    use_left = (r == 0) | ((c > 0) & (bit == 1))
    not_root = vid != 0
    left_edge = r * (C - 1) + (c - 1)
    up_edge = nh + (r - 1) * C + c
    tree_ids = torch.where(use_left, left_edge, up_edge)[not_root]
    in_tree = torch.zeros(total, dtype=torch.bool, device=device)
    in_tree[tree_ids] = True
    eid = rng.arange(0, total, device)
    cand = eid[~in_tree]
    ndel = int(round(frac * total))
    if ndel > cand.numel():
        raise ValueError("cannot delete that many edges and stay connected")
    key = rng.u53(seed, 8, cand)
    order = torch.argsort(key)
    deleted = torch.zeros(total, dtype=torch.bool, device=device)
    deleted[cand[order[:ndel]]] = True
    keep = eid[~deleted]
    is_h = keep < nh
    hr = keep // (C - 1)
    hc = keep % (C - 1)
    vk = keep - nh
    vr = vk // C
    vc = vk % C
    a = torch.where(is_h, hr * C + hc, vr * C + vc)
    b = torch.where(is_h, hr * C + hc + 1, (vr + 1) * C + vc)
    keys, _ = torch.sort(torch.minimum(a, b) * n + torch.maximum(a, b))
    return _csr_from_undirected_keys(n, keys, device, "grid(%dx%d,del=%g,seed=%d)"
                                     % (R, C, frac, seed))


def with_self_loops(g):
    """The same graph with a self-loop added on every vertex that lacks one
    (rows stay ascending; a loop is one entry of its row)."""
    n = g.n
    dev = g.row_ptr.device
    rp = g.row_ptr.to(torch.int64)
    rows = torch.repeat_interleave(torch.arange(n, device=dev), rp[1:] - rp[:-1])
    keys = torch.cat([rows * n + g.col_idx.to(torch.int64), torch.arange(n, device=dev) * (n + 1)])
    keys = torch.unique(keys)
    r = keys // n
    counts = torch.bincount(r, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return Csr(n, row_ptr.to(torch.int32), (keys % n).to(torch.int32), g.name + "+loops")


def shuffled(g, seed=0):
    """The same graph with its vertex ids permuted by a seeded random
    permutation (rows re-sorted, columns ascending): a stand-in for inputs whose
    ids carry no degree or locality order."""
    n = g.n
    dev = g.row_ptr.device
    vid = rng.arange(0, n, dev)
    order = torch.argsort(rng.u53(seed, 9, vid))      # new id -> old id
    new_of = torch.empty_like(order)
    new_of[order] = vid                                # old id -> new id
    rp = g.row_ptr.to(torch.int64)
    deg = rp[1:] - rp[:-1]
    rows = torch.repeat_interleave(vid, deg)
    a = new_of[rows]
    b = new_of[g.col_idx.to(torch.int64)]
    del rows
    keys = a * n + b
    del a, b
    keys, _ = torch.sort(keys)
    r = keys // n
    counts = torch.bincount(r, minlength=n)
    del r
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts, 0)
    col_idx = (keys % n).to(torch.int32)
    return Csr(n, row_ptr.to(torch.int32), col_idx, g.name + "_shuffled(%d)" % seed)


# -- small graphs with known structure (test fixtures) ------------------------

def star(L, device="cpu"):
    """K_{1,L}: centre 0, leaves 1..L."""
    return from_edges(L + 1, [(0, j) for j in range(1, L + 1)], device, "star(%d)" % L)


def cycle(n, device="cpu"):
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], device, "cycle(%d)" % n)


def path(n, device="cpu"):
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], device, "path(%d)" % n)


def complete(n, device="cpu"):
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], device,
                      "complete(%d)" % n)


def complete_bipartite(a, b, device="cpu"):
    """K_{a,b}: side X = 0..a-1, side Y = a..a+b-1."""
    return from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)], device,
                      "K(%d,%d)" % (a, b))


def circulant(n, offsets, device="cpu"):
    """Regular graph: i ~ i +- s (mod n) for s in offsets."""
    e = [(i, (i + s) % n) for i in range(n) for s in offsets]
    return from_edges(n, e, device, "circulant(%d,%s)" % (n, list(offsets)))


def random_small(n, m, seed=0, device="cpu"):
    """Ring plus m extra seeded uniform edges (no isolated vertices)."""
    idx = rng.arange(0, m, "cpu")
    u = (rng.u32(seed, 11, idx) % n).numpy()
    v = (rng.u32(seed, 12, idx) % n).numpy()
    e = [(i, (i + 1) % n) for i in range(n)] + [(int(a), int(b)) for a, b in zip(u, v) if a != b]
    return from_edges(n, e, device, "random_small(%d,%d,%d)" % (n, m, seed))


def all_graphs(n):
    """Every labelled simple graph on n vertices with no isolated vertex."""
    pairs = list(itertools.combinations(range(n), 2))
    out = []
    for mask in range(1, 1 << len(pairs)):
        e = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        deg = [0] * n
        for a, b in e:
            deg[a] += 1
            deg[b] += 1
        if min(deg) > 0:
            out.append(from_edges(n, e, "cpu", "g%d_%d" % (n, mask)))
    return out
