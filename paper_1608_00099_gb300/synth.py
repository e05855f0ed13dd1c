"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module generates inputs only.  It holds none of the tensor method's
arithmetic (no embedding, products or moments): it draws shapes and values so
that the CPU oracle and the GPU kernels can be fed identical bits.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in its counter form: output i of seed s
is mix64(s + (i + 1) * GOLDEN_GAMMA).  It is pure 64-bit integer arithmetic,
so U(0,1) draws are identical on every host (x86_64 and aarch64 alike).
N(0,1) draws use Box-Muller through numpy's log/sqrt/cos, which may differ in
the last ulp between hosts; such values are regenerated per run and never
stored as golden data.

Workloads (shapes, seeds and value laws) follow the five synthetic
configurations the build measures; the tensor shapes come from the paper's own
style of benchmark (copy into a larger zero-padded tensor, products over the
shared tuples, tuple-weighted sums; Section 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = 1.0 / float(1 << 53)

# seed of configuration k is 1000 + k
SEED_BASE = 1000

# numpy reduces uint64 arithmetic modulo 2**64 for arrays; scalar overflow
# warnings are silenced where scalars are mixed in.


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream of `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """U[0,1) doubles: top 53 bits of each SplitMix64 output times 2**-53."""
    out = np.empty(count, dtype=np.float64)
    for off in range(0, count, chunk):
        n = min(chunk, count - off)
        z = splitmix64(seed, start + off, n)
        out[off:off + n] = (z >> np.uint64(11)).astype(np.float64) * _TWO_M53
    return out


def normal01(seed: int, count: int) -> np.ndarray:
    """N(0,1) doubles by Box-Muller on pairs of SplitMix64 uniforms."""
    npairs = (count + 1) // 2
    z = splitmix64(seed, 0, 2 * npairs)
    u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * _TWO_M53  # (0, 1]
    u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * _TWO_M53          # [0, 1)
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * math.pi * u2
    out = np.empty(2 * npairs, dtype=np.float64)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    return out[:count]


def randint_inclusive(seed: int, count: int, lo: int, hi: int, start: int = 0) -> np.ndarray:
    """Integers uniform on {lo..hi} by multiply-shift of the top 32 bits."""
    z = splitmix64(seed, start, count)
    top = (z >> np.uint64(32)).astype(np.uint64)
    span = np.uint64(hi - lo + 1)
    with np.errstate(over="ignore"):
        r = (top * span) >> np.uint64(32)
    return (r.astype(np.int64) + lo)


def normalise(u: np.ndarray) -> np.ndarray:
    """u / sum(u) in float64 with an exactly rounded sum (math.fsum)."""
    s = math.fsum(u.tolist()) if u.size <= (1 << 22) else float(np.sum(u, dtype=np.float64))
    return u / s


# ---------------------------------------------------------------- storage dtypes

def to_storage(a64: np.ndarray, dtype: str):
    """Round float64 values to a storage dtype with torch (IEEE RN-even).

    Returns a torch CPU tensor.  float64 -> bfloat16 goes through float32 in
    torch, which is a double rounding; callers that need single rounding pass
    values already exact in float32 or use the oracle's rounding instead.
    """
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a64))
    if dtype == "f64":
        return t.clone()
    if dtype == "f32":
        return t.to(torch.float32)
    if dtype == "bf16":
        return t.to(torch.float32).to(torch.bfloat16)
    if dtype == "f16":
        return t.to(torch.float16)
    raise ValueError(dtype)


# ---------------------------------------------------------------- configurations

@dataclass
class EmbedProductMoment:
    """One 'embed x -> y_embed, product y_prod *= x, moment of p' workload."""
    name: str
    dtype: str
    xshape: tuple
    embed_shape: tuple
    prod_shape: tuple
    seed: int
    x_law: str = "uniform"      # "uniform" or "normal"
    p_normalised: bool = True   # moment input p = x / sum(x)
    notes: str = ""

    def x_values(self) -> np.ndarray:
        n = int(np.prod(self.xshape))
        if self.x_law == "normal":
            return normal01(self.seed, n)
        return uniform01(self.seed, n)

    def yprod_values(self) -> np.ndarray:
        # the product destination is an independent U(0,1) tensor (seed + 500)
        return uniform01(self.seed + 500, int(np.prod(self.prod_shape)))


def config_embed_small() -> EmbedProductMoment:
    """Embed FP64 d=6: x (8,)*6 ~ N(0,1) into zero y (10,)*6, crop back."""
    return EmbedProductMoment("embed_f64_d6", "f64", (8,) * 6, (10,) * 6, (10,) * 6,
                              SEED_BASE + 1, x_law="normal")


def config_f64_d8() -> EmbedProductMoment:
    """FP64 d=8: x 9^8 U(0,1); embed into (11,10)x4; product with (12,8)x4; moment of x/sum(x)."""
    return EmbedProductMoment("f64_d8", "f64", (9,) * 8, (11, 10) * 4, (12, 8) * 4,
                              SEED_BASE + 2)


def config_f32_d24() -> EmbedProductMoment:
    """FP32 d=24: x all-2 U(0,1) into 3^16 x 2^8; product over all-2; moment of x."""
    return EmbedProductMoment("f32_d24", "f32", (2,) * 24, (3,) * 16 + (2,) * 8,
                              (3,) * 16 + (2,) * 8, SEED_BASE + 3, p_normalised=False)


@dataclass
class PrecisionCase:
    """Two d=10 tensors with extents uniform on {3..7}, Dirichlet-like values."""
    pshape: tuple
    qshape: tuple
    p64: np.ndarray
    q64: np.ndarray


def config_precision(seed: int = SEED_BASE + 4, d: int = 10, lo: int = 3, hi: int = 7,
                     normalised: bool = True) -> PrecisionCase:
    ext = randint_inclusive(seed, 2 * d, lo, hi)
    pshape = tuple(int(v) for v in ext[:d])
    qshape = tuple(int(v) for v in ext[d:])
    up = uniform01(seed + 100, int(np.prod(pshape)))
    uq = uniform01(seed + 200, int(np.prod(qshape)))
    if normalised:
        up, uq = normalise(up), normalise(uq)
    return PrecisionCase(pshape, qshape, up, uq)


@dataclass
class BatchPair:
    xshape: tuple
    yshape: tuple


def config_batch_shapes(npairs: int = 4096, seed: int = SEED_BASE + 5,
                        rank_lo: int = 2, rank_hi: int = 10, ext_lo: int = 2,
                        ext_hi: int = 32, cap_log2: int = 22) -> list:
    """Pair shapes: rank r ~ U{2..10}; y extents E_i ~ U{2..min(32, floor(2^(22/r)))}
    (so |y| <= 2^22 by construction); x extents e_i ~ U{2..E_i}."""
    pairs = []
    ctr = 0
    ranks = randint_inclusive(seed, npairs, rank_lo, rank_hi)
    for r in ranks:
        r = int(r)
        cap = min(ext_hi, int(math.floor(2.0 ** (cap_log2 / r) + 1e-9)))
        E = randint_inclusive(seed + 1, r, ext_lo, cap, start=ctr)
        ctr += r
        ys = [int(v) for v in E]
        xs = [int(randint_inclusive(seed + 2, 1, ext_lo, e, start=ctr + i)[0]) for i, e in enumerate(ys)]
        ctr += r
        pairs.append(BatchPair(tuple(xs), tuple(ys)))
    return pairs


def batch_x_values(pairs: list, seed: int = SEED_BASE + 5) -> list:
    out, start = [], 0
    for pr in pairs:
        n = int(np.prod(pr.xshape))
        out.append(uniform01(seed + 7, n, start=start))
        start += n
    return out
