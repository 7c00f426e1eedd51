"""Seeded personalization vectors.

``seed_vectors``: for each query draw k ~ U{1..max_seeds}, then k distinct
vertices uniformly; the vector puts 1/k on each seed.
"""
import numpy as np
import torch

from . import rng


def uniform_p(n, dtype=torch.float64, device="cpu"):
    return torch.full((n,), 1.0 / n, dtype=dtype, device=device)


def seed_vectors(n, count, max_seeds=16, seed=0):
    """List of (seeds int32 array, weights float64 array) per query."""
    out = []
    for q in range(count):
        base = torch.tensor([q], dtype=torch.int64)
        k = int(rng.u32(seed, 21, base)[0] % max_seeds) + 1
        chosen = []
        j = 0
        while len(chosen) < k:
            cand = int(rng.u32(seed, 22 + q % 1024, torch.tensor([q * 4096 + j]))[0] % n)
            j += 1
            if cand not in chosen:
                chosen.append(cand)
        out.append((np.array(chosen, dtype=np.int32), np.full(k, 1.0 / k)))
    return out


def seed_dense(n, seeds_list, dtype=np.float64):
    """Column-major n x B dense matrix from seed lists (column b = query b)."""
    B = len(seeds_list)
    P = np.zeros((B, n), dtype=dtype)
    for b, (s, w) in enumerate(seeds_list):
        P[b, s] = w
    return P
