"""Counter-based random numbers in plain integer tensor arithmetic.

The generator is Chris Wellons' "lowbias32" integer hash (xorshift-multiply
finaliser, constants 0x7feb352d and 0x846ca68b) applied to a counter mixed with
a key derived from (seed, stream).  Every operation is on int64 tensors holding
values below 2^32, and every product is split into 16-bit halves so that no
intermediate exceeds 2^63: the stream is bit-identical on CPU and CUDA.
"""
import torch

M32 = 0xFFFFFFFF


def _mul32(x, k):
    """(x * k) mod 2^32 for an int64 tensor x < 2^32 and a 32-bit constant k."""
    lo = x * (k & 0xFFFF)
    hi = (x * (k >> 16)) & 0xFFFF
    return (lo + (hi << 16)) & M32


def hash32(x):
    """lowbias32 of an int64 tensor of values in [0, 2^32)."""
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B)
    x = x ^ (x >> 16)
    return x


def _key(seed, stream):
    k = torch.tensor([(int(seed) * 0x9E3779B9 + int(stream) * 0x85EBCA6B + 0x6A09E667) & M32],
                     dtype=torch.int64)
    return int(hash32(hash32(k))[0])


def u32(seed, stream, idx):
    """Uniform 32-bit integers for counters ``idx`` (int64 tensor, values < 2^32)."""
    k = _key(seed, stream)
    return hash32(hash32(idx ^ k) ^ 0x9E3779B9)


def u53(seed, stream, idx):
    """Uniform integers in [0, 2^53) (two 32-bit draws from streams 2s, 2s+1)."""
    a = u32(seed, 2 * stream, idx)
    b = u32(seed, 2 * stream + 1, idx)
    return (a << 21) | (b >> 11)


def arange(start, stop, device):
    return torch.arange(start, stop, dtype=torch.int64, device=device)
