"""Multiresolution encodings in FP64 (test infrastructure only; see ``oracle``).

* ``simplex_encode`` / ``simplex_encode_bwd``: the paper's pipeline of Sec. 5,
  steps (a) hash the simplex vertices at L levels, (b) look up the feature
  vectors of table H_l, (c) barycentric interpolation (Sec. 4.3), (d) concatenate
  the levels; (e) the backward pass accumulates the loss gradient into the
  looked-up entries.
* ``grid_encode`` / ``grid_encode_bwd``: the baseline the paper compares
  against (Instant-NGP's 2^n-vertex grid), interpolated by repeated linear
  interpolation one axis at a time as in Algorithm 1 (trilinear interpolation
  by recursion on the dimension), with the same hash and tables.

Tables are [L, T, F] arrays of any float dtype (the values are upcast to FP64);
the output layout is [P, L*F] with level-major feature groups.  The first
level-scaling step is evaluated in binary32 (see ``lattice``), everything after
the floor is FP64.

Parity pins: the simplex path is pinned by weights >= 0, sum 1, exact
reconstruction of the point, agreement with a brute-force point-in-simplex
search, exact interpolation of affine fields and the memory-usage figure of
Sec. 5.2; the grid path by exact interpolation of multilinear fields.  The
backward passes are pinned by adjointness and by exact finite differences
(both encodings are linear in the tables).  The input gradients
(``simplex_encode_dx`` / ``grid_encode_dx``) are pinned by the exact gradient of
affine (simplex) and multilinear (grid) fields and by central differences of the
forward pass inside one cell.  ``simplex_encode_fp64`` / ``grid_encode_fp64`` evaluate the level
scaling and skew in FP64 from x (no binary32 step): pinned by the same affine / multilinear
exactness and by agreement with the binary32-conditioned paths within the quantisation bound.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import lattice


def _level_params(kind, n, n_levels, base_res, growth, res_mode):
    if kind == "simplex":
        return lattice.simplex_level_scales_fp32(n, n_levels, base_res, growth, res_mode)
    return lattice.grid_level_scales_fp32(n_levels, base_res, growth)


def _widths(kind, n, scales, log2_T, index_mode):
    return lattice.level_box_widths(kind, n, scales, log2_T, index_mode)


# --------------------------------------------------------------------------
# simplex encoding, Sec. 5 (a)-(d)
# --------------------------------------------------------------------------
def simplex_level_vertices(x32: np.ndarray, level_scale: np.float32, log2_T: int, width: int = 0):
    """Steps (a) for one level: returns (slots int64 [P, n+1], weights FP64 [P, n+1],
    vertices int64 [P, n+1, n])."""
    q = lattice.scaled_skewed_fp32(x32, level_scale)
    c, order, f = lattice.subdivide(q)
    V = lattice.simplex_vertices(c, order)
    w = lattice.barycentric_weights(f, order)
    slots = lattice.slot_of(V, log2_T, width)
    return slots, w, V


def simplex_encode(x32, tables, *, base_res, growth, res_mode=lattice.RES_RAW, with_denominator=False,
                   index_mode=lattice.INDEX_HASH):
    """Forward simplex encoding of points ``x32`` ([P, n], binary32) with tables [L, T, F].

    Returns FP64 [P, L*F]; with ``with_denominator`` also returns sum_k |w_k H_k|
    per output, the scale against which a relative tolerance is measured.
    """
    x32 = np.asarray(x32, dtype=np.float32)
    P, n = x32.shape
    L, T, F = tables.shape
    log2_T = int(T).bit_length() - 1
    scales = _level_params("simplex", n, L, base_res, growth, res_mode)
    widths = _widths("simplex", n, scales, log2_T, index_mode)
    out = np.zeros((P, L * F), dtype=np.float64)
    den = np.zeros((P, L * F), dtype=np.float64)
    for l in range(L):
        slots, w, _ = simplex_level_vertices(x32, scales[l], log2_T, widths[l])
        H = np.asarray(tables[l], dtype=np.float64)[slots]            # (b) lookup [P, n+1, F]
        out[:, l * F:(l + 1) * F] = np.einsum("pk,pkf->pf", w, H)      # (c) interpolate, (d) concat
        den[:, l * F:(l + 1) * F] = np.einsum("pk,pkf->pf", np.abs(w), np.abs(H))
    return (out, den) if with_denominator else out


def simplex_encode_fp64(x, tables, *, base_res, growth, res_mode=lattice.RES_RAW):
    """The forward simplex encoding with the level scale and the skew of Eq. 2 evaluated in FP64
    from x (FP64 multipliers N_l m / sqrt(n+1)), instead of from the binary32 skewed coordinate
    ``simplex_encode`` conditions on; hashed levels only.  Everything else is ``simplex_encode``'s.

    Its difference from ``simplex_encode`` is the binary32 quantisation of the skewed coordinate
    (reported beside the parity results, not a parity gate), and it is an exactly piecewise-linear
    function of x, so that its central differences give the input gradient in FP64.
    """
    x = np.asarray(x, dtype=np.float64)
    P, n = x.shape
    L, T, F = tables.shape
    log2_T = int(T).bit_length() - 1
    scales = lattice.simplex_level_scales_fp64(n, L, base_res, growth, res_mode)
    out = np.zeros((P, L * F), dtype=np.float64)
    for l in range(L):
        q = lattice.skew(x * scales[l])
        c, order, f = lattice.subdivide(q)
        slots = lattice.slot_of(lattice.simplex_vertices(c, order), log2_T)
        w = lattice.barycentric_weights(f, order)
        out[:, l * F:(l + 1) * F] = np.einsum("pk,pkf->pf", w, np.asarray(tables[l], dtype=np.float64)[slots])
    return out


def simplex_encode_bwd(x32, dout, *, n_levels, log2_T, n_features, base_res, growth,
                       res_mode=lattice.RES_RAW, levels=None, with_denominator=False,
                       index_mode=lattice.INDEX_HASH):
    """Step (e): dH_l[slot(v_k)][f] += w_k * dout[p][l*F + f], FP64.

    Returns a dict level -> FP64 [T, F] gradient (only the levels asked for), and
    with ``with_denominator`` a second dict of sum |w_k * dout| per entry.
    """
    x32 = np.asarray(x32, dtype=np.float32)
    dout = np.asarray(dout, dtype=np.float64)
    P, n = x32.shape
    F = n_features
    T = 1 << log2_T
    scales = _level_params("simplex", n, n_levels, base_res, growth, res_mode)
    widths = _widths("simplex", n, scales, log2_T, index_mode)
    grads, dens = {}, {}
    for l in (range(n_levels) if levels is None else levels):
        slots, w, _ = simplex_level_vertices(x32, scales[l], log2_T, widths[l])
        terms = w[:, :, None] * dout[:, None, l * F:(l + 1) * F]       # [P, n+1, F]
        g = np.zeros((T, F), dtype=np.float64)
        np.add.at(g, slots.ravel(), terms.reshape(-1, F))
        grads[l] = g
        if with_denominator:
            a = np.zeros((T, F), dtype=np.float64)
            np.add.at(a, slots.ravel(), np.abs(terms).reshape(-1, F))
            dens[l] = a
    return (grads, dens) if with_denominator else grads


def simplex_encode_dx(x32, tables, dout, *, base_res, growth, res_mode=lattice.RES_RAW, with_denominator=False,
                      index_mode=lattice.INDEX_HASH):
    """Gradient of sum_p,j dout[p][j] * out[p][j] with respect to the points, FP64 [P, n].

    Inside one simplex the output is affine in the fractional parts: by the weights of
    Sec. 4.3, moving f along axis order[k] shifts weight from vertex v_k to v_{k+1}, so
    d out / d q_order[k] = H(v_{k+1}) - H(v_k).  The skew of Eq. 2 (q = p + F_n sum p) is
    symmetric, so d/dp_j = g_j + F_n sum_i g_i, and p = x s_l gives the factor s_l.  The
    constants are the binary32 s_l and F_n of the forward pass.  Where the point lies on a
    face (tied fractional parts) the derivative is the one-sided value of the forward
    pass's simplex.  With ``with_denominator`` also returns the sum of the magnitudes of
    the terms (the scale of the rounding error of any evaluation order).
    """
    x32 = np.asarray(x32, dtype=np.float32)
    dout = np.asarray(dout, dtype=np.float64)
    P, n = x32.shape
    L, T, F = tables.shape
    log2_T = int(T).bit_length() - 1
    scales = _level_params("simplex", n, L, base_res, growth, res_mode)
    widths = _widths("simplex", n, scales, log2_T, index_mode)
    Fn = float(np.float32(lattice.skew_factor(n)))
    dx = np.zeros((P, n))
    den = np.zeros((P, n))
    rows = np.arange(P)
    for l in range(L):
        q = lattice.scaled_skewed_fp32(x32, scales[l])
        c, order, _ = lattice.subdivide(q)
        V = lattice.simplex_vertices(c, order)
        H = np.asarray(tables[l], dtype=np.float64)[lattice.slot_of(V, log2_T, widths[l])]   # [P, n+1, F]
        dl = dout[:, l * F:(l + 1) * F]
        g = np.zeros((P, n))
        a = np.zeros((P, n))
        for k in range(n):
            diff = H[:, k + 1] - H[:, k]                                    # [P, F]
            g[rows, order[:, k]] = np.einsum("pf,pf->p", dl, diff)
            a[rows, order[:, k]] = np.einsum("pf,pf->p", np.abs(dl), np.abs(H[:, k + 1]) + np.abs(H[:, k]))
        s = float(scales[l])
        dx += s * (g + Fn * g.sum(axis=1, keepdims=True))
        den += s * (a + Fn * a.sum(axis=1, keepdims=True))
    return (dx, den) if with_denominator else dx


# --------------------------------------------------------------------------
# 2^n grid comparator, Algorithm 1
# --------------------------------------------------------------------------
def grid_level_cell(x32, level_res: np.float32):
    """p = x * N_l in binary32, c = floor(p), f = p - c (FP64)."""
    p = np.asarray(x32, dtype=np.float32) * np.float32(level_res)
    p = p.astype(np.float64)
    c = np.floor(p)
    return c.astype(np.int64), p - c


def _corner_offsets(n):
    """All b in {0,1}^n, in the order of a C-ordered [2]*n array (axis 0 slowest)."""
    return np.array(list(itertools.product((0, 1), repeat=n)), dtype=np.int64)


def grid_level_corner_weights(f: np.ndarray) -> np.ndarray:
    """Weight of every corner as the adjoint of the axis-by-axis linear interpolation.

    Runs the recursion of Algorithm 1 backwards: a unit output is split by
    (1 - f_i, f_i) along each axis in turn, giving [P, 2^n] weights in the
    corner order of ``_corner_offsets``.
    """
    P, n = f.shape
    w = np.ones((P, 1))
    for i in range(n):                       # split along axes 0..n-1 (axis 0 slowest)
        lo = w * (1.0 - f[:, i])[:, None]
        hi = w * f[:, i][:, None]
        w = np.stack([lo, hi], axis=2).reshape(P, -1)
    return w


def grid_encode(x32, tables, *, base_res, growth, index_mode=lattice.INDEX_HASH):
    """Forward 2^n grid encoding, [P, L*F] FP64.

    Per level: look up the 2^n corner values, then (Algorithm 1) interpolate
    linearly along the last remaining axis and recurse on the others until a
    single value is left.
    """
    x32 = np.asarray(x32, dtype=np.float32)
    P, n = x32.shape
    L, T, F = tables.shape
    log2_T = int(T).bit_length() - 1
    res = _level_params("grid", n, L, base_res, growth, None)
    widths = _widths("grid", n, res, log2_T, index_mode)
    offs = _corner_offsets(n)
    out = np.zeros((P, L * F), dtype=np.float64)
    for l in range(L):
        c, f = grid_level_cell(x32, res[l])
        corners = c[:, None, :] + offs[None, :, :]                       # [P, 2^n, n]
        vals = np.asarray(tables[l], dtype=np.float64)[lattice.slot_of(corners, log2_T, widths[l])]
        vals = vals.reshape((P,) + (2,) * n + (F,))
        for i in reversed(range(n)):                                   # lerp along axis i
            t = f[:, i].reshape((P,) + (1,) * i + (1,))
            v0 = np.take(vals, 0, axis=1 + i)
            v1 = np.take(vals, 1, axis=1 + i)
            vals = v0 * (1.0 - t) + v1 * t
        out[:, l * F:(l + 1) * F] = vals.reshape(P, F)
    return out


def grid_encode_fp64(x, tables, *, base_res, growth):
    """``grid_encode`` with p = x N_l in FP64 (instead of binary32), hashed levels only: the
    comparator's FP64 forward, exactly multilinear in x inside a cell (see ``simplex_encode_fp64``)."""
    x = np.asarray(x, dtype=np.float64)
    P, n = x.shape
    L, T, F = tables.shape
    log2_T = int(T).bit_length() - 1
    res = lattice.level_resolutions(L, base_res, growth)
    offs = _corner_offsets(n)
    out = np.zeros((P, L * F), dtype=np.float64)
    for l in range(L):
        p = x * float(res[l])
        c = np.floor(p)
        f = p - c
        corners = c.astype(np.int64)[:, None, :] + offs[None, :, :]
        vals = np.asarray(tables[l], dtype=np.float64)[lattice.slot_of(corners, log2_T)]
        out[:, l * F:(l + 1) * F] = np.einsum("pk,pkf->pf", grid_level_corner_weights(f), vals)
    return out


def grid_encode_bwd(x32, dout, *, n_levels, log2_T, n_features, base_res, growth, levels=None,
                    index_mode=lattice.INDEX_HASH):
    """Backward of ``grid_encode``: dH_l[slot(c+b)] += w_b * dout, FP64 dict level -> [T, F]."""
    x32 = np.asarray(x32, dtype=np.float32)
    dout = np.asarray(dout, dtype=np.float64)
    P, n = x32.shape
    F = n_features
    T = 1 << log2_T
    res = _level_params("grid", n, n_levels, base_res, growth, None)
    widths = _widths("grid", n, res, log2_T, index_mode)
    offs = _corner_offsets(n)
    grads = {}
    for l in (range(n_levels) if levels is None else levels):
        c, f = grid_level_cell(x32, res[l])
        w = grid_level_corner_weights(f)                                 # [P, 2^n]
        slots = lattice.slot_of(c[:, None, :] + offs[None, :, :], log2_T, widths[l])
        terms = w[:, :, None] * dout[:, None, l * F:(l + 1) * F]
        g = np.zeros((T, F), dtype=np.float64)
        np.add.at(g, slots.ravel(), terms.reshape(-1, F))
        grads[l] = g
    return grads


def grid_level_corner_weight_derivatives(f: np.ndarray, axis: int) -> np.ndarray:
    """d w_b / d f_axis for every corner b (same order as ``grid_level_corner_weights``): the
    factor of the differentiated axis becomes -1 (lower corner) or +1 (upper corner)."""
    P, n = f.shape
    w = np.ones((P, 1))
    for i in range(n):
        lo = w * ((-1.0 + 0.0 * f[:, i]) if i == axis else (1.0 - f[:, i]))[:, None]
        hi = w * ((1.0 + 0.0 * f[:, i]) if i == axis else f[:, i])[:, None]
        w = np.stack([lo, hi], axis=2).reshape(P, -1)
    return w


def grid_encode_dx(x32, tables, dout, *, base_res, growth, with_denominator=False, index_mode=lattice.INDEX_HASH):
    """Gradient of sum dout * out of ``grid_encode`` with respect to the points, FP64 [P, n]:
    the derivative of the n-linear weights along each axis, times N_l (p = x N_l)."""
    x32 = np.asarray(x32, dtype=np.float32)
    dout = np.asarray(dout, dtype=np.float64)
    P, n = x32.shape
    L, T, F = tables.shape
    log2_T = int(T).bit_length() - 1
    res = _level_params("grid", n, L, base_res, growth, None)
    widths = _widths("grid", n, res, log2_T, index_mode)
    offs = _corner_offsets(n)
    dx = np.zeros((P, n))
    den = np.zeros((P, n))
    for l in range(L):
        c, f = grid_level_cell(x32, res[l])
        H = np.asarray(tables[l], dtype=np.float64)[lattice.slot_of(c[:, None, :] + offs[None, :, :], log2_T,
                                                                      widths[l])]
        dl = dout[:, l * F:(l + 1) * F]
        proj = np.einsum("pf,pbf->pb", dl, H)                                # [P, 2^n]
        aproj = np.einsum("pf,pbf->pb", np.abs(dl), np.abs(H))
        for j in range(n):
            dw = grid_level_corner_weight_derivatives(f, j)
            dx[:, j] += float(res[l]) * np.einsum("pb,pb->p", dw, proj)
            den[:, j] += float(res[l]) * np.einsum("pb,pb->p", np.abs(dw), aproj)
    return (dx, den) if with_denominator else dx


def grid_level_vertices(x32, level_res, log2_T, width=0):
    """Slots int64 [P, 2^n] and weights FP64 [P, 2^n] of one grid level."""
    c, f = grid_level_cell(x32, level_res)
    offs = _corner_offsets(c.shape[1])
    return lattice.slot_of(c[:, None, :] + offs[None, :, :], log2_T, width), grid_level_corner_weights(f)
