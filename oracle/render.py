"""Volumetric rendering with the encodings in FP64 (test infrastructure only; see ``oracle``).

Sec. 6.2 renders a ray's colour by Eq. 5, C(r) = int T(t) sigma(r(t)) c(r(t), d) dt with
T(t) = exp(-int sigma), querying the field at discrete samples along the ray and compositing
them.  The paper does not print the discretisation, the sampling or the networks; the readings
taken here (NeRF's quadrature and Instant-NGP's field layout, the systems Sec. 6.2 builds on):

* Samples: S points per ray at the midpoints of S equal segments of [t_near, t_far]:
  delta = (t_far - t_near) / S, t_i = t_near + (i + 1/2) delta, x_i = o + t_i d.  These are
  evaluated in binary32 with one rounding per operation in exactly this order (the point the
  lattice sees must be the same on every implementation), then used as given.
* Quadrature of Eq. 5 for a field that is constant on each segment (exact for such fields):
  alpha_i = 1 - exp(-sigma_i delta), T_i = prod_{j<i} (1 - alpha_j) = exp(-sum_{j<i} sigma_j delta),
  C = sum_i T_i alpha_i c_i; the remaining transmittance T_S is returned (black background).
* Field: the encoding of x_i feeds a density network (n_in -> 64 -> 16, one hidden layer); its
  first output is the log-density, sigma = exp(min(v_0, 15)); all 16 outputs, followed by the 16
  real spherical harmonics of degree <= 3 of the ray direction, feed a colour network
  (32 -> 64 -> 64 -> 3) whose outputs pass a logistic sigmoid.
* Real spherical harmonics (l = 0..3, m = -l..l, l-major): the orthonormal real basis
  sqrt(2) (-1)^m Im Y_l^|m| (m < 0), Y_l^0, sqrt(2) (-1)^m Re Y_l^m (m > 0) of the complex
  harmonics with the Condon-Shortley phase, written out as polynomials of the unit vector.

Parity pins (tests): the compositing equals the closed form of Eq. 5 for piecewise-constant
media; the harmonics equal scipy's complex harmonics through the real-basis relation and are
orthonormal on the sphere; every sample lies on its ray inside [t_near, t_far].  The gradients
(``composite_bwd``, ``render_l2_grads``) equal central differences of the forward functions and,
for a homogeneous medium, the derivative of its closed form.
"""
from __future__ import annotations

import math

import numpy as np

from . import encoding, mlp

DENSITY_LOGIT_MAX = 15.0


def ray_samples_fp32(o, d, t_near, t_far, S: int):
    """Sample points [R*S, 3] (binary32, ray-major) and segment lengths delta [R] (binary32)."""
    o = np.asarray(o, dtype=np.float32)
    d = np.asarray(d, dtype=np.float32)
    tn = np.asarray(t_near, dtype=np.float32)
    tf = np.asarray(t_far, dtype=np.float32)
    delta = (tf - tn) / np.float32(S)                                       # one rounding
    k = (np.arange(S, dtype=np.float32) + np.float32(0.5))                 # exact
    t = tn[:, None] + k[None, :] * delta[:, None]                          # [R, S], mul then add
    x = o[:, None, :] + t[:, :, None] * d[:, None, :]                      # [R, S, 3]
    return x.reshape(-1, 3).astype(np.float32), delta


def sh_basis(dirs) -> np.ndarray:
    """Real spherical harmonics of degree 0..3 of unit vectors, FP64 [P, 16] (l-major, m = -l..l)."""
    v = np.asarray(dirs, dtype=np.float64)
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    pi = math.pi
    out = np.empty((v.shape[0], 16))
    out[:, 0] = 0.5 * math.sqrt(1.0 / pi)
    c1 = math.sqrt(3.0 / (4.0 * pi))
    out[:, 1], out[:, 2], out[:, 3] = c1 * y, c1 * z, c1 * x
    c2 = 0.5 * math.sqrt(15.0 / pi)
    out[:, 4] = c2 * x * y
    out[:, 5] = c2 * y * z
    out[:, 6] = 0.25 * math.sqrt(5.0 / pi) * (3.0 * z * z - 1.0)
    out[:, 7] = c2 * x * z
    out[:, 8] = 0.5 * c2 * (x * x - y * y)
    a3 = 0.25 * math.sqrt(35.0 / (2.0 * pi))
    b3 = 0.5 * math.sqrt(105.0 / pi)
    c3 = 0.25 * math.sqrt(21.0 / (2.0 * pi))
    out[:, 9] = a3 * y * (3.0 * x * x - y * y)
    out[:, 10] = b3 * x * y * z
    out[:, 11] = c3 * y * (5.0 * z * z - 1.0)
    out[:, 12] = 0.25 * math.sqrt(7.0 / pi) * (5.0 * z ** 3 - 3.0 * z)
    out[:, 13] = c3 * x * (5.0 * z * z - 1.0)
    out[:, 14] = 0.5 * b3 * z * (x * x - y * y)
    out[:, 15] = a3 * x * (x * x - 3.0 * y * y)
    return out


def composite(sigma, rgb, delta):
    """Eq. 5 on piecewise-constant segments, one sample after the other.

    sigma [R, S] >= 0, rgb [R, S, 3], delta [R]; returns (C [R, 3], T_final [R], weights [R, S])."""
    sigma = np.asarray(sigma, dtype=np.float64)
    rgb = np.asarray(rgb, dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64)
    R, S = sigma.shape
    C = np.zeros((R, 3))
    T = np.ones(R)
    w = np.zeros((R, S))
    for i in range(S):
        # alpha = 1 - exp(-sigma delta) and the factor 1 - alpha = exp(-sigma delta) (Eq. 5's
        # T = exp(-integral of sigma)) are formed without cancellation: expm1 and exp directly
        alpha = -np.expm1(-sigma[:, i] * delta)
        w[:, i] = T * alpha
        C += w[:, i, None] * rgb[:, i]
        T = T * np.exp(-sigma[:, i] * delta)
    return C, T, w


def composite_bwd(sigma, rgb, delta, dC):
    """Gradients of sum(dC * C) of ``composite`` with respect to sigma [R, S] and rgb [R, S, 3].

    From Eq. 5's quadrature: sigma_k enters alpha_k (d alpha_k / d sigma_k = delta (1 - alpha_k)) and
    every later transmittance (d T_i / d sigma_k = -delta T_i for i > k), so
    dC/dsigma_k = delta (T_{k+1} c_k - sum_{i>k} w_i c_i) and dC/dc_k = w_k.  Written out per sample
    with the suffix sums accumulated from the far end of the ray."""
    sigma = np.asarray(sigma, dtype=np.float64)
    rgb = np.asarray(rgb, dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64)
    dC = np.asarray(dC, dtype=np.float64)
    R, S = sigma.shape
    _, T, w = composite(sigma, rgb, delta)
    Tk = np.ones((R, S + 1))                                  # T_0 .. T_S
    for i in range(S):
        Tk[:, i + 1] = Tk[:, i] * np.exp(-sigma[:, i] * delta)
    dsigma = np.zeros((R, S))
    suffix = np.zeros((R, 3))                                 # sum_{i>k} w_i c_i
    for k in range(S - 1, -1, -1):
        dsigma[:, k] = delta * np.einsum("rc,rc->r", dC, Tk[:, k + 1, None] * rgb[:, k] - suffix)
        suffix += w[:, k, None] * rgb[:, k]
    drgb = w[:, :, None] * dC[:, None, :]
    return dsigma, drgb


def density_from_logit(v):
    return np.exp(np.minimum(np.asarray(v, dtype=np.float64), DENSITY_LOGIT_MAX))


def sigmoid(v):
    return 1.0 / (1.0 + np.exp(-np.asarray(v, dtype=np.float64)))


def render_l2_grads(o, d, t_near, t_far, S, tables, W_density, W_color, target, *, kind, base_res, growth,
                    index_mode=0):
    """Loss mean((C - target)^2) over rays and channels of ``render`` and its gradients with respect to
    the tables ({level: [T, F]}) and both networks' weights, by the chain rule through Eq. 5, the
    sigmoid, the colour network, the field head (sigma = exp(min(v_0, 15)): d sigma / d v_0 = sigma
    below the clamp, 0 above; the harmonics take no gradient), the density network and the encoding."""
    C, _, it = render(o, d, t_near, t_far, S, tables, W_density, W_color, kind=kind, base_res=base_res,
                      growth=growth, index_mode=index_mode)
    R = C.shape[0]
    target = np.asarray(target, dtype=np.float64)
    loss = float(np.mean((C - target) ** 2))
    dC = 2.0 * (C - target) / C.size
    rgb = sigmoid(it["logits"])
    dsigma, drgb = composite_bwd(it["sigma"].reshape(R, S), rgb.reshape(R, S, 3), it["delta"], dC)
    dlogits = drgb.reshape(-1, 3) * rgb * (1.0 - rgb)
    _, acts_c = mlp.mlp_forward(W_color, it["color_in"])
    dWc, dcin = mlp.mlp_backward(W_color, acts_c, dlogits)
    dv = dcin[:, :16].copy()
    h0 = it["density_out"][:, 0]
    dv[:, 0] += dsigma.reshape(-1) * np.where(h0 < DENSITY_LOGIT_MAX, it["sigma"], 0.0)
    _, acts_d = mlp.mlp_forward(W_density, it["enc"])
    dWd, denc = mlp.mlp_backward(W_density, acts_d, dv)
    L, T, F = np.asarray(tables).shape
    bwd = encoding.simplex_encode_bwd if kind == "simplex" else encoding.grid_encode_bwd
    gt = bwd(it["x"], denc, n_levels=L, log2_T=int(T).bit_length() - 1, n_features=F, base_res=base_res,
             growth=growth, index_mode=index_mode)
    return loss, gt, dWd, dWc, dict(it, C=C, dC=dC, dsigma=dsigma, dlogits=dlogits, dv=dv, denc=denc)


def render(o, d, t_near, t_far, S, tables, W_density, W_color, *, kind, base_res, growth, index_mode=0):
    """Full forward render: samples -> encoding -> density network -> (sigma, 16 features) ->
    [features, SH(d)] -> colour network -> sigmoid -> Eq. 5.  Returns (C, T_final, intermediates)."""
    x, delta = ray_samples_fp32(o, d, t_near, t_far, S)
    R = len(delta)
    enc_fn = encoding.simplex_encode if kind == "simplex" else encoding.grid_encode
    e = enc_fn(x, tables, base_res=base_res, growth=growth, index_mode=index_mode)
    h, _ = mlp.mlp_forward(W_density, e)                                   # [R*S, 16]
    sigma = density_from_logit(h[:, 0])
    sh = np.repeat(sh_basis(d), S, axis=0)
    c_in = np.concatenate([h, sh], axis=1)
    logits, _ = mlp.mlp_forward(W_color, c_in)
    rgb = sigmoid(logits)
    C, Tf, w = composite(sigma.reshape(R, S), rgb.reshape(R, S, 3), delta)
    return C, Tf, dict(x=x, delta=delta, enc=e, density_out=h, sigma=sigma, color_in=c_in, logits=logits, w=w)
