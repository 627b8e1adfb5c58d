"""Seeded synthetic SIFT-shaped inputs, shared by the oracle, the tests and the bench.

This module holds none of the search method's arithmetic.  It only draws
integer-valued D-dimensional points (coordinates in [0, 255], like SIFT
descriptors) from a Gaussian mixture, using a counter-based generator so that
any point can be produced on its own, on the host (here, numpy) or on the device
(``synthdata/csrc/synth.cu``), with identical bytes.

Generator
---------
Counter-based SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  SplitMix64 advances a 64-bit state by the
golden-ratio increment GAMMA and returns ``mix64(state)``.  Output number c of a
generator seeded with s is therefore ``mix64(s + (c + 1) * GAMMA)``, which is
what :func:`draw` computes directly from the counter

    ctr = (stream << 48) | (n << 8) | w      stream < 2^16, n < 2^40, w < 2^8

with ``s = mix64(seed)``.

Mixture (all tables are integers, so no libm runs per point)
-------------------------------------------------------------
Points have low intrinsic dimension, like SIFT: a component mean plus a shared
F = 16 factor latent term plus small per-dimension noise, clipped to [0, 255].

Parameter stream ``PARAM_STREAM``; counter n = c for component c:
  * latent scale sigma_c = 3 + (word0 >> 32) % 4                in [3, 6]
  * weight W_c = 2^20 + (word1 >> 43)                            in [2^20, 3*2^20)
  * mean mu_c[d] = min(255, 12*g + ((word(2+d) >> 16) % 24)), where g is the
    number of consecutive low-order one bits of word(2+d) (capped at 8), a
    Geometric(1/2) draw: SIFT-like mass near zero with a long tail.  (For
    d >= 254 the word is word(2 + d mod 254) of counter c + 2^38 * floor(d / 254),
    so that w stays below 2^8.)
  * cum[c] = floor(2^32 * sum_{c'<=c} W_c' / sum W)              (cum[-1] = 2^32)
and counter n = 2^39 + d for the shared loadings B[d][f] = (word f >> 32) % 7 - 3.

Point n of a stream:
  * component c = first index with cum[c] > (word0 >> 32)
  * 16 + D Irwin-Hall(4) draws: the 32-bit halves of words 1 .. 8 + D/2 in order
    (low half first) are split into four bytes b0..b3 and z = b0+b1+b2+b3 - 510
    (standard deviation ~147.8); the first 16 are the latent factors l_f, the
    next D the noise e_d.
  * x[d] = clamp(mu_c[d] + floor((sigma_c * sum_f B[d][f] l_f + 8 e_d + 83) / 166), 0, 255)
    (integer arithmetic; floor((a + 83) / 166) rounds a / 166 half up).

Streams: 0 = base points, 1 = learn (training) points, 2 = queries.
"""

from __future__ import annotations

import dataclasses

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

STREAM_BASE = 0
STREAM_LEARN = 1
STREAM_QUERY = 2
PARAM_STREAM = 0xFFFF

_U64 = np.uint64


def mix64(z):
    """SplitMix64 output function on a numpy uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=_U64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _U64(MIX1)
        z = (z ^ (z >> _U64(27))) * _U64(MIX2)
        z = z ^ (z >> _U64(31))
    return z


def mix64_int(z: int) -> int:
    """Scalar SplitMix64 output function on a Python int."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def splitmix64_sequence(seed: int, count: int) -> list[int]:
    """The plain SplitMix64 sequence: state += GAMMA; yield mix64(state)."""
    out, s = [], seed & MASK64
    for _ in range(count):
        s = (s + GAMMA) & MASK64
        out.append(mix64_int(s))
    return out


def draw(seed: int, stream: int, n, w):
    """Counter-based SplitMix64 word for (stream, n, w); n and w broadcast."""
    n = np.asarray(n, dtype=_U64)
    w = np.asarray(w, dtype=_U64)
    ctr = (_U64(stream) << _U64(48)) | (n << _U64(8)) | w
    with np.errstate(over="ignore"):
        state = _U64(mix64_int(seed)) + (ctr + _U64(1)) * _U64(GAMMA)
    return mix64(state)


N_FACTORS = 16
SCALE = 166
NOISE = 8


@dataclasses.dataclass(frozen=True)
class Mixture:
    seed: int
    dim: int
    n_comp: int
    mu: np.ndarray      # (n_comp, dim) int32 in [0, 255]
    sigma: np.ndarray   # (n_comp,) int32 latent scale in [3, 6]
    cum: np.ndarray     # (n_comp,) uint64 thresholds, last == 2^32
    B: np.ndarray       # (dim, N_FACTORS) int32 loadings in [-3, 3]


def make_mixture(seed: int, n_comp: int, dim: int = 128) -> Mixture:
    if dim % 2 or 1 + N_FACTORS // 2 + dim // 2 > 255:
        raise ValueError("dim must be even and at most 492")
    c = np.arange(n_comp, dtype=_U64)
    w0 = draw(seed, PARAM_STREAM, c, 0)
    w1 = draw(seed, PARAM_STREAM, c, 1)
    sigma = (3 + (w0 >> _U64(32)) % _U64(4)).astype(np.int32)
    weight = [int(x) for x in ((1 << 20) + (w1 >> _U64(43)))]
    total = sum(weight)
    cum, run = np.empty(n_comp, dtype=_U64), 0
    for i in range(n_comp):
        run += weight[i]
        cum[i] = (run << 32) // total
    dd = np.arange(dim, dtype=_U64)
    wd = draw(seed, PARAM_STREAM, c[:, None] + (dd[None, :] // _U64(254)) * (_U64(1) << _U64(38)),
              _U64(2) + dd[None, :] % _U64(254))
    g = np.zeros(wd.shape, dtype=np.int32)
    alive = np.ones(wd.shape, dtype=bool)
    for b in range(8):
        alive &= ((wd >> _U64(b)) & _U64(1)) == _U64(1)
        g += alive
    mu = np.minimum(255, 12 * g + ((wd >> _U64(16)) % _U64(24)).astype(np.int32)).astype(np.int32)
    wb = draw(seed, PARAM_STREAM, (_U64(1) << _U64(39)) + np.arange(dim, dtype=_U64)[:, None],
              np.arange(N_FACTORS, dtype=_U64)[None, :])
    B = ((wb >> _U64(32)) % _U64(7)).astype(np.int32) - 3
    return Mixture(seed=seed, dim=dim, n_comp=n_comp, mu=mu, sigma=sigma, cum=cum, B=B)


def points(mix: Mixture, stream: int, start: int, count: int, out: np.ndarray | None = None) -> np.ndarray:
    """Points start .. start+count-1 of a stream, as an (count, dim) uint8 array."""
    if out is None:
        out = np.empty((count, mix.dim), dtype=np.uint8)
    chunk = 1 << 15
    nwords = N_FACTORS // 2 + mix.dim // 2
    widx = 1 + np.arange(nwords, dtype=_U64)
    Bt = mix.B.T.astype(np.int64)
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        n = np.arange(start + s, start + e, dtype=_U64)
        comp = np.searchsorted(mix.cum, draw(mix.seed, stream, n, 0) >> _U64(32), side="right")
        words = draw(mix.seed, stream, n[:, None], widx[None, :])
        # little-endian byte view: bytes 0..3 of a word are its low 32-bit half
        b = words.astype("<u8", copy=False).view(np.uint8).reshape(e - s, N_FACTORS + mix.dim, 4)
        z = b.sum(axis=2, dtype=np.int64) - 510
        a = mix.sigma[comp].astype(np.int64)[:, None] * (z[:, :N_FACTORS] @ Bt) + NOISE * z[:, N_FACTORS:]
        x = mix.mu[comp].astype(np.int64) + (a + SCALE // 2) // SCALE
        out[s:e] = np.clip(x, 0, 255).astype(np.uint8)
    return out


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape of one synthetic workload (sizes only; no method arithmetic)."""
    name: str
    n_base: int
    n_learn: int
    n_query: int
    n_comp: int
    T: int            # coarse codewords per half (T^2 cells)
    M: int            # PQ sub-quantizers
    L: tuple          # candidate budgets
    k: int            # results per query
    kmeans_iters: int = 10
    dim: int = 128
    seed: int = 1234


# Configurations of the paper-shaped workloads (SIFT-shaped, D = 128).
TINY = Workload("tiny-100k-T64-M8", n_base=100_000, n_learn=20_000, n_query=100,
                n_comp=64, T=64, M=8, L=(10_000,), k=100)
SIFT10M = Workload("sift10m-T1024-M8", n_base=10_000_000, n_learn=1_024_000, n_query=10_000,
                   n_comp=1024, T=1024, M=8, L=(1_000, 10_000, 100_000), k=100)
# 100M points with M = 16 (the precision-variant shape), 100M points with M = 8
# (uneven budgets, local codebooks) and 1B points (the serving shape).
SIFT100M_M16 = Workload("sift100m-T1024-M16", n_base=100_000_000, n_learn=1_024_000, n_query=10_000,
                        n_comp=1024, T=1024, M=16, L=(30_000,), k=100)
SIFT100M = Workload("sift100m-T1024-M8", n_base=100_000_000, n_learn=1_024_000, n_query=10_000,
                    n_comp=1024, T=1024, M=8, L=(1_000, 100_000), k=100)
SIFT1B = Workload("sift1b-T1024-M8", n_base=1_000_000_000, n_learn=1_024_000, n_query=10_000,
                  n_comp=4096, T=1024, M=8, L=(1_000, 10_000, 100_000), k=100)
# GIST-shaped (D = 384, 8-byte codes, T = 1024 as for GIST50M): the same generator in 384
# dimensions; and a small case of the same shape for parity tests.
GIST50M = Workload("gist50m-T1024-M8", n_base=50_000_000, n_learn=1_024_000, n_query=10_000,
                   n_comp=1024, T=1024, M=8, L=(10_000, 30_000, 100_000), k=100, dim=384)
TINY_GIST = Workload("tiny-gist-50k-T32-M8", n_base=50_000, n_learn=20_000, n_query=30,
                     n_comp=64, T=32, M=8, L=(5_000,), k=50, dim=384, kmeans_iters=4)
WORKLOADS = {w.name: w for w in (TINY, SIFT10M, SIFT100M_M16, SIFT100M, SIFT1B, GIST50M, TINY_GIST)}
