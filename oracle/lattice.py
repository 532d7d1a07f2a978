"""Simplex-lattice geometry in FP64 (test infrastructure only; see ``oracle``).

Restates, in the paper's order and notation:

* Eq. 2 (coordinate skew) and Eq. 3 (unskew), Sec. 2.2 (a), (d) and Sec. 4.1;
* the per-level resolution and the scale adjustment S_n = sqrt(n+1), Sec. 5.1,
  plus the optional equal-memory level factor (n+1)^((n-1)/(2n)), Sec. 5.2;
* the simplicial subdivision: floor, sort the fractional parts in decreasing
  order keeping their indices, walk +1 along the sorted axes (Sec. 2.2 b,
  Sec. 4.2, Remark 2);
* the barycentric weights w_1 = 1 - s_1, w_k = s_{k-1} - s_k, w_{n+1} = s_n on the
  sorted fractional parts s (Sec. 4.3, from the proof of Theorem 1);
* the vertex hash of Sec. 5 (a) (each vertex's integer coordinates are hashed).

Readings where the paper is silent:

* Level resolution N_l = floor(base * growth^l), the Instant-NGP rule the
  backbone of Sec. 5 uses; no +0.5 offset; the point is used as given.
* The adjustment scale S_n of Sec. 5.1 is read as dividing the level-scaled
  input by S_n = sqrt(n+1) *before* the skew, so that the skewed image of the
  unit cube fits the lattice box [0, N_l]^n.  (Pinned by the memory-usage
  figure of Sec. 5.2, see tests.)
* Ties between equal fractional parts are broken by the lower axis index
  first (a stable descending sort).  Every tie order gives the same
  interpolated value; the rule only fixes which zero-weight vertex is listed.
* The skewed, scaled coordinate that feeds the floor is formed in IEEE binary32
  with one rounding per operation in this order: p_i = x_i*s, sigma = ((p_1 +
  p_2) + p_3) + ..., t = F*sigma, q_i = p_i + t.  Index parity with the GPU is
  conditioned on this binary32 value; everything after it is FP64 here.
* Optional dense indexing of coarse levels (``INDEX_DENSE_COARSE``; Instant-NGP
  stores a level directly when its lattice fits the table, the paper hashes every
  level): the vertices of points in [0,1]^n have coordinates 0..B-1 per axis with
  B = floor(top) + 2, top = s_l sqrt(n+1) (simplex: q_i <= s_l (1 + n F_n)) or N_l
  (grid), evaluated from the binary32 scale with a 2^-20 relative margin so that a
  rounded-up binary32 coordinate stays inside; a level with B^n <= T stores vertex v
  at sum_i v_i B^i (uint32 arithmetic, then modulo T), other levels hash.
* Hash: XOR over axes of (uint32 v_i * pi_i) modulo T (a power of two), with
  pi = (1, 2654435761, 805459861) for the first three axes (Instant-NGP's
  spatial hash, which the paper's backbone uses) and, for axes 4 and 5,
  the smallest primes not below frac(sqrt(5))*2^32 and frac(sqrt(7))*2^32.
  Parity of the hash is pinned only by hand-derived slot values.
"""
from __future__ import annotations

import math

import numpy as np

#: hash multipliers per axis (see module docstring for their origin)
HASH_PRIMES = (1, 2654435761, 805459861, 1013904263, 2773480771)

RES_RAW = 0
RES_EQUAL_MEM = 1

INDEX_HASH = 0
INDEX_DENSE_COARSE = 1


# --------------------------------------------------------------------------
# Eq. 2 / Eq. 3
# --------------------------------------------------------------------------
def skew_factor(n: int) -> float:
    """F_n = (sqrt(n+1) - 1) / n  (Eq. 2)."""
    return (math.sqrt(n + 1.0) - 1.0) / n


def unskew_factor(n: int) -> float:
    """G_n = (1 - 1/sqrt(n+1)) / n  (Eq. 3)."""
    return (1.0 - 1.0 / math.sqrt(n + 1.0)) / n


def skew(x: np.ndarray) -> np.ndarray:
    """x' = x + F_n * (sum_i x_i) * 1  (Eq. 2), FP64, last axis is the dimension."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[-1]
    return x + skew_factor(n) * np.sum(x, axis=-1, keepdims=True)


def unskew(xp: np.ndarray) -> np.ndarray:
    """x = x' - G_n * (sum_i x'_i) * 1  (Eq. 3), FP64."""
    xp = np.asarray(xp, dtype=np.float64)
    n = xp.shape[-1]
    return xp - unskew_factor(n) * np.sum(xp, axis=-1, keepdims=True)


# --------------------------------------------------------------------------
# Sec. 5.1 / 5.2: per-level scales
# --------------------------------------------------------------------------
def level_resolutions(n_levels: int, base_res: float, growth: float) -> list[int]:
    """N_l = floor(base * growth^l), l = 0..L-1 (Instant-NGP's rule; the paper is silent)."""
    return [int(math.floor(base_res * growth ** l)) for l in range(n_levels)]


def equal_memory_factor(n: int) -> float:
    """(n+1)^((n-1)/(2n)): level multiplier that keeps the touched lattice the
    same size as the 2^n grid's at equal table memory (Sec. 5.2, last paragraph)."""
    return (n + 1.0) ** ((n - 1.0) / (2.0 * n))


def simplex_level_scales_fp64(n: int, n_levels: int, base_res: float, growth: float,
                              res_mode: int = RES_RAW) -> list[float]:
    """Input multiplier per level before the skew: N_l * m / S_n with S_n = sqrt(n+1) (Sec. 5.1)."""
    m = 1.0 if res_mode == RES_RAW else equal_memory_factor(n)
    return [N * m / math.sqrt(n + 1.0) for N in level_resolutions(n_levels, base_res, growth)]


def simplex_level_scales_fp32(n, n_levels, base_res, growth, res_mode=RES_RAW) -> np.ndarray:
    """The same scales rounded once to binary32 (the value the binary32 skew multiplies by)."""
    return np.array(simplex_level_scales_fp64(n, n_levels, base_res, growth, res_mode), dtype=np.float32)


def grid_level_scales_fp32(n_levels, base_res, growth) -> np.ndarray:
    """The 2^n grid multiplies the input by N_l directly (Algorithm 1 on the level lattice)."""
    return np.array(level_resolutions(n_levels, base_res, growth), dtype=np.float32)


# --------------------------------------------------------------------------
# binary32 scale + skew (the one step whose rounding is fixed, see docstring)
# --------------------------------------------------------------------------
def scaled_skewed_fp32(x: np.ndarray, scale: np.float32) -> np.ndarray:
    """q = skew(x * scale) evaluated in binary32, one rounding per operation (Sec. 5.1, Eq. 2).

    ``x`` is [P, n] binary32; returns binary32 [P, n].
    """
    x = np.asarray(x, dtype=np.float32)
    n = x.shape[1]
    F = np.float32(skew_factor(n))
    p = x * np.float32(scale)
    sigma = p[:, 0].copy()
    for i in range(1, n):
        sigma = sigma + p[:, i]
    t = F * sigma
    return p + t[:, None]


# --------------------------------------------------------------------------
# Sec. 2.2 (b), Sec. 4.2, Remark 2: simplicial subdivision
# --------------------------------------------------------------------------
def subdivide(q: np.ndarray):
    """Floor the skewed coordinate and order its fractional parts in decreasing order.

    Returns (c, order, f): c = floor(q) as int64 [P, n] (the base vertex v_1),
    f = q - c in FP64 [P, n], and order [P, n] = the axis indices sorted so that
    f[order[0]] >= f[order[1]] >= ... (equal values keep the lower index first).
    """
    q = np.asarray(q, dtype=np.float64)
    c = np.floor(q)
    f = q - c
    order = np.argsort(-f, axis=1, kind="stable")
    return c.astype(np.int64), order, f


def simplex_vertices(c: np.ndarray, order: np.ndarray) -> np.ndarray:
    """Remark 2 / Sec. 4.2: v_1 = c and v_{k+1} = v_k + e_{order[k]}; returns int64 [P, n+1, n]."""
    P, n = c.shape
    V = np.empty((P, n + 1, n), dtype=np.int64)
    V[:, 0] = c
    rows = np.arange(P)
    for k in range(n):
        V[:, k + 1] = V[:, k]
        V[rows, k + 1, order[:, k]] += 1
    return V


def barycentric_weights(f: np.ndarray, order: np.ndarray) -> np.ndarray:
    """Sec. 4.3: with s the fractional parts sorted in decreasing order,
    w_1 = 1 - s_1, w_k = s_{k-1} - s_k (k = 2..n), w_{n+1} = s_n.  FP64 [P, n+1]."""
    s = np.take_along_axis(np.asarray(f, dtype=np.float64), order, axis=1)
    P, n = s.shape
    w = np.empty((P, n + 1), dtype=np.float64)
    w[:, 0] = 1.0 - s[:, 0]
    for k in range(1, n):
        w[:, k] = s[:, k - 1] - s[:, k]
    w[:, n] = s[:, n - 1]
    return w


# --------------------------------------------------------------------------
# Sec. 5 (a): vertex hash
# --------------------------------------------------------------------------
def hash_slot(v: np.ndarray, log2_T: int) -> np.ndarray:
    """Slot of integer vertex v (int64 [..., n]) in a table of T = 2^log2_T entries.

    (XOR over i of (v_i mod 2^32) * pi_i mod 2^32) mod T, evaluated with
    exact integer arithmetic on uint64.
    """
    v = np.asarray(v, dtype=np.int64)
    n = v.shape[-1]
    if n > len(HASH_PRIMES):
        raise ValueError("no hash multiplier for dimension %d" % n)
    mask32 = np.uint64(0xFFFFFFFF)
    h = np.zeros(v.shape[:-1], dtype=np.uint64)
    for i in range(n):
        vi = v[..., i].astype(np.uint64) & mask32          # two's complement mod 2^32
        h ^= (vi * np.uint64(HASH_PRIMES[i])) & mask32     # product < 2^64: exact
    return (h & np.uint64((1 << log2_T) - 1)).astype(np.int64)


# --------------------------------------------------------------------------
# optional direct (collision-free) indexing of the coarse levels
# --------------------------------------------------------------------------
def dense_box_width(kind: str, n: int, scale_fp32) -> int:
    """Number of lattice coordinates per axis that the vertices of points in [0,1]^n take."""
    top = float(scale_fp32) * (math.sqrt(n + 1.0) if kind == "simplex" else 1.0)
    return int(math.floor(top * (1.0 + 2.0 ** -20))) + 2


def level_box_widths(kind: str, n: int, scales, log2_T: int, index_mode: int) -> list[int]:
    """Per level: the box width B if that level is stored directly (B^n <= T), else 0 (hashed)."""
    out = []
    for s in scales:
        B = dense_box_width(kind, n, s) if index_mode == INDEX_DENSE_COARSE else 0
        out.append(B if B and B ** n <= (1 << log2_T) else 0)
    return out


def dense_slot(v: np.ndarray, width: int, log2_T: int) -> np.ndarray:
    """(sum_i (v_i mod 2^32) * width^i mod 2^32) mod T, exact on uint64."""
    v = np.asarray(v, dtype=np.int64)
    mask32 = np.uint64(0xFFFFFFFF)
    h = np.zeros(v.shape[:-1], dtype=np.uint64)
    stride = 1
    for i in range(v.shape[-1]):
        vi = v[..., i].astype(np.uint64) & mask32
        h = (h + ((vi * np.uint64(stride % (1 << 32))) & mask32)) & mask32
        stride *= width
    return (h & np.uint64((1 << log2_T) - 1)).astype(np.int64)


def slot_of(v: np.ndarray, log2_T: int, width: int = 0) -> np.ndarray:
    """Table slot of vertex v: direct index for a stored level (width > 0), else the hash."""
    return dense_slot(v, width, log2_T) if width else hash_slot(v, log2_T)
