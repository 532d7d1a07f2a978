"""Volumetric rendering with the simplex (or grid) encoding, Sec. 6.2 (Eq. 5).

A ``Renderer`` renders a batch of rays through the library's kernels only:

1. ``sxe_vr_samples``   -- S midpoint samples per ray in [t_near, t_far];
2. ``sxe_encode_fwd``   -- the multiresolution encoding of every sample (Sec. 5 a-d);
3. ``sxe_vr_field_mlp`` -- density network (encoding -> 64 -> 16), sigma = exp(min(v_0, 15)),
                           colour input [v, SH(d)] and colour network (32 -> 64 -> 64 -> 3) in
                           one kernel;
4. ``sxe_vr_composite`` -- sigmoid colours composited front to back (Eq. 5).

With ``fused=False`` step 3 is three launches (``sxe_mlp_fwd``, ``sxe_vr_field``,
``sxe_mlp_fwd``) with the same results; with ``keep_intermediates`` the fused step is
``sxe_vr_field_mlp_saved``, which also writes the density outputs and the colour input that a
training step's backward reads.  All buffers are allocated once for the largest ray batch and
reused; every launch is asynchronous on one stream.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .api import Encoder, Mlp, _need, _ptr, _stream, torch_dtype

_VR_DTYPES = {"f16": L.SXE_F16, "bf16": L.SXE_BF16}


class Renderer:
    """Renders rays of a field = (encoder, density network, colour network)."""

    def __init__(self, encoder: Encoder, max_rays: int, n_samples: int, *, dtype: str = "f16", device="cuda",
                 fused: bool = True, keep_intermediates: bool = False):
        if encoder.d != 3:
            raise ValueError("volumetric rendering needs a 3-D encoder")
        if encoder.out_dtype != dtype:
            raise ValueError("encoder output dtype %s != network dtype %s" % (encoder.out_dtype, dtype))
        self.enc, self.S, self.max_rays, self.dtype, self.fused = encoder, n_samples, max_rays, dtype, fused
        self.keep = bool(keep_intermediates)
        self.density = Mlp(encoder.n_out, 16, n_hidden=1, dtype=dtype)
        self.color = Mlp(32, 3, n_hidden=2, dtype=dtype)
        dev = torch.device(device)
        P = max_rays * n_samples
        self.x = torch.empty((P, 3), dtype=torch.float32, device=dev)
        self.delta = torch.empty((max_rays,), dtype=torch.float32, device=dev)
        self.enc_out = torch.empty((P, encoder.n_out), dtype=torch_dtype(dtype), device=dev)
        self.dens_out = torch.empty((P, 16), dtype=torch.float32, device=dev)
        self.sigma = torch.empty((P,), dtype=torch.float32, device=dev)
        self.color_in = torch.empty((P, 32), dtype=torch_dtype(dtype), device=dev)
        self.logits = torch.empty((P, 3), dtype=torch.float32, device=dev)

    def init_weights(self, seed: int):
        """He-uniform weights of both networks in the network dtype (device tensors)."""
        dev = self.x.device
        Wd = torch.from_numpy(self.density.init_weights(seed)).to(dev).to(torch_dtype(self.dtype))
        Wc = torch.from_numpy(self.color.init_weights(seed + 1)).to(dev).to(torch_dtype(self.dtype))
        return Wd, Wc

    def render(self, origins, dirs, t_near, t_far, tables, W_density, W_color, color=None, transmittance=None,
               weights=None, stream=None):
        """Colours [R, 3] (and optionally the remaining transmittance [R] and sample weights [R*S])."""
        R = origins.shape[0]
        if R > self.max_rays:
            raise ValueError("batch of %d rays > max_rays %d" % (R, self.max_rays))
        S = self.S
        P = R * S
        for t, name, shape in ((origins, "origins", (R, 3)), (dirs, "dirs", (R, 3)), (t_near, "t_near", (R,)),
                               (t_far, "t_far", (R,))):
            _need(t, torch.float32, name, shape)
        if color is None:
            color = torch.empty((R, 3), dtype=torch.float32, device=origins.device)
        _need(color, torch.float32, "color", (R, 3))
        if transmittance is not None:
            _need(transmittance, torch.float32, "transmittance", (R,))
        if weights is not None:
            _need(weights, torch.float32, "weights", (P,))
        st = _stream(stream)
        lib = L.lib()
        x = self.x[:P]
        L.check(lib.sxe_vr_samples(_ptr(origins), _ptr(dirs), _ptr(t_near), _ptr(t_far), R, S, _ptr(x),
                                   _ptr(self.delta), st), "sxe_vr_samples")
        self.enc.encode_fwd(x, tables, self.enc_out[:P], stream=stream)
        if self.fused:
            for W, m, nm in ((W_density, self.density, "W_density"), (W_color, self.color, "W_color")):
                _need(W, torch_dtype(self.dtype), nm, (m.n_params,))
            if self.keep:
                L.check(lib.sxe_vr_field_mlp_saved(ctypes.byref(self.density.desc), _ptr(W_density),
                                                   ctypes.byref(self.color.desc), _ptr(W_color), _ptr(self.enc_out),
                                                   _ptr(dirs), R, S, _ptr(self.sigma), _ptr(self.logits),
                                                   _ptr(self.dens_out), _ptr(self.color_in), st),
                        "sxe_vr_field_mlp_saved")
            else:
                L.check(lib.sxe_vr_field_mlp(ctypes.byref(self.density.desc), _ptr(W_density),
                                             ctypes.byref(self.color.desc), _ptr(W_color), _ptr(self.enc_out),
                                             _ptr(dirs), R, S, _ptr(self.sigma), _ptr(self.logits), st),
                        "sxe_vr_field_mlp")
        else:
            self.density.mlp_fwd(W_density, self.enc_out[:P], out=self.dens_out[:P], stream=stream)
            L.check(lib.sxe_vr_field(_ptr(self.dens_out), _ptr(dirs), R, S, _VR_DTYPES[self.dtype],
                                     _ptr(self.sigma), _ptr(self.color_in), st), "sxe_vr_field")
            self.color.mlp_fwd(W_color, self.color_in[:P], out=self.logits[:P], stream=stream)
        L.check(lib.sxe_vr_composite(_ptr(self.sigma), _ptr(self.logits), _ptr(self.delta), R, S, _ptr(color),
                                     _ptr(transmittance), _ptr(weights), st), "sxe_vr_composite")
        return color

    @property
    def n_launches(self) -> int:
        return 4 if self.fused else 6


class VolumeTrainer:
    """Trains a field (hash tables + density and colour networks) from ray colours (Sec. 6.2): one
    ``step(rays, target)`` renders the rays, takes the mean squared colour error, back-propagates
    it through the compositing (``sxe_vr_composite_bwd``), the colour network, the field head
    (``sxe_vr_field_bwd``), the density network and the encoding, and takes Adam steps on the table
    entries that received a gradient and on both networks.  Every step runs in the library's
    kernels; the step count lives on the device."""

    def __init__(self, encoder: Encoder, max_rays: int, n_samples: int, *, dtype: str = "f16", seed: int = 0,
                 device="cuda", table_init: float = 1e-4, lr: float = 1e-2, betas=(0.9, 0.99), eps: float = 1e-15,
                 table_layout: str = "auto", split_coarse="auto"):
        from . import synth
        from .api import Adam
        from .trainer import TableState, choose_table_layout, default_loss_scale
        self.enc, self.R, self.S = encoder, max_rays, n_samples
        # the fused field, keeping the density outputs and colour input the backward reads
        self.rr = Renderer(encoder, max_rays, n_samples, dtype=dtype, device=device, fused=True,
                           keep_intermediates=True)
        dev = self.rr.x.device
        F, n_entries = encoder.n_features, encoder.n_levels * encoder.T
        vals = synth.uniform_tables(encoder.n_levels, encoder.T, F, seed, dtype="f32", scale=table_init)[0]
        init = torch.from_numpy(vals.reshape(n_entries, F)).to(dev)
        self.tab = TableState(encoder, init, choose_table_layout(encoder, dev, table_layout), dev,
                              split_coarse=split_coarse)
        self.tables = self.tab.tables
        self.nets = []
        for k, m in enumerate((self.rr.density, self.rr.color)):
            W = torch.from_numpy(m.init_weights(seed + 1 + k)).to(dev)
            self.nets.append(dict(mlp=m, W=W, W_lowp=W.to(torch_dtype(dtype)), m=torch.zeros_like(W),
                                  v=torch.zeros_like(W), dW=torch.zeros_like(W), ws=m.workspace(max_rays * n_samples, dev)))
        P = max_rays * n_samples
        self.color = torch.empty((max_rays, 3), dtype=torch.float32, device=dev)
        self.dcolor = torch.empty_like(self.color)
        self.sq_sum = torch.zeros((1,), dtype=torch.float32, device=dev)
        self.dsigma = torch.empty((P,), dtype=torch.float32, device=dev)
        self.dlogits = torch.empty((P, 3), dtype=torch.float32, device=dev)
        self.dcin = torch.empty((P, 32), dtype=torch.float32, device=dev)
        self.dv = torch.empty((P, 16), dtype=torch.float32, device=dev)
        self.denc = torch.empty((P, encoder.n_out), dtype=torch.float32, device=dev)
        self.loss_scale = default_loss_scale(max_rays, 3)
        self.adam_tables = Adam(lr, betas[0], betas[1], eps, skip_zero_grad=True)
        self.adam_nets = Adam(lr, betas[0], betas[1], eps, skip_zero_grad=False)
        self.t = 0
        self.t_dev = torch.zeros((1,), dtype=torch.int64, device=dev)
        self.corrections = torch.zeros((2,), dtype=torch.float32, device=dev)
        self._n_rays = 0

    def gradients(self, origins, dirs, t_near, t_far, target, stream=None) -> None:
        """Forward render, loss and every gradient (table gradients in the state records' gradient
        fields, touched entries marked; network gradients in nets[k]['dW'])."""
        from .api import loss_l2
        R, S, F = origins.shape[0], self.S, self.enc.n_features
        P = R * S
        rr, st = self.rr, _stream(stream)
        dens, col = self.nets
        rr.render(origins, dirs, t_near, t_far, self.tables, dens["W_lowp"], col["W_lowp"], color=self.color[:R],
                  stream=stream)
        self.sq_sum.zero_()
        _need(target, torch.float32, "target", (R, 3))
        loss_l2(self.color[:R], target, self.dcolor[:R], self.sq_sum, stream=stream)
        L.check(L.lib().sxe_vr_composite_bwd(_ptr(rr.sigma), _ptr(rr.logits), _ptr(rr.delta), _ptr(self.color),
                                             _ptr(self.dcolor), R, S, _ptr(self.dsigma), _ptr(self.dlogits), st),
                "sxe_vr_composite_bwd")
        col["mlp"].mlp_bwd(col["W_lowp"], rr.color_in[:P], self.dlogits[:P], col["dW"], din=self.dcin[:P],
                           loss_scale=self.loss_scale, workspace=col["ws"], stream=stream)
        L.check(L.lib().sxe_vr_field_bwd(_ptr(self.dcin), _ptr(self.dsigma), _ptr(rr.sigma), _ptr(rr.dens_out), R, S,
                                         _ptr(self.dv), st), "sxe_vr_field_bwd")
        dens["mlp"].mlp_bwd(dens["W_lowp"], rr.enc_out[:P], self.dv[:P], dens["dW"], din=self.denc[:P],
                            loss_scale=self.loss_scale, workspace=dens["ws"], stream=stream)
        self.tab.backward(rr.x[:P], self.denc[:P], stream=stream)
        self._n_rays = R

    def step(self, origins, dirs, t_near, t_far, target, stream=None) -> None:
        """One optimisation step on a batch of rays and their target colours [R, 3]."""
        self.t += 1
        self.adam_tables.advance(self.t_dev, self.corrections, stream=stream)
        self.gradients(origins, dirs, t_near, t_far, target, stream=stream)
        self.tab.adam(self.adam_tables, self.corrections, stream=stream)
        for n in self.nets:
            self.adam_nets.step_dev(self.corrections, n["W"], n["m"], n["v"], n["dW"], lowp=n["W_lowp"], stream=stream)

    def loss(self) -> float:
        """Mean squared colour error of the last step (synchronises)."""
        return float(self.sq_sum.item()) / (self._n_rays * 3)

    def table_grads(self) -> torch.Tensor:
        """Table gradient of the last ``gradients`` call, [L, T, F] (before the Adam step)."""
        return self.tab.grads()


def vr_samples(origins, dirs, t_near, t_far, n_samples: int, stream=None):
    """``sxe_vr_samples`` alone: (x [R*S, 3], delta [R])."""
    R = origins.shape[0]
    x = torch.empty((R * n_samples, 3), dtype=torch.float32, device=origins.device)
    delta = torch.empty((R,), dtype=torch.float32, device=origins.device)
    L.check(L.lib().sxe_vr_samples(_ptr(origins), _ptr(dirs), _ptr(t_near), _ptr(t_far), R, n_samples, _ptr(x),
                                   _ptr(delta), _stream(stream)), "sxe_vr_samples")
    return x, delta


def vr_field(density_out, dirs, n_samples: int, dtype: str = "f16", stream=None):
    """``sxe_vr_field`` alone: (sigma [P], color_in [P, 32])."""
    P = density_out.shape[0]
    _need(density_out, torch.float32, "density_out", (P, 16))
    sigma = torch.empty((P,), dtype=torch.float32, device=density_out.device)
    cin = torch.empty((P, 32), dtype=torch_dtype(dtype), device=density_out.device)
    L.check(L.lib().sxe_vr_field(_ptr(density_out), _ptr(dirs), dirs.shape[0], n_samples, _VR_DTYPES[dtype],
                                 _ptr(sigma), _ptr(cin), _stream(stream)), "sxe_vr_field")
    return sigma, cin


def vr_composite(sigma, logits, delta, n_samples: int, with_weights: bool = False, stream=None):
    """``sxe_vr_composite`` alone: (color [R, 3], transmittance [R], weights [P] or None)."""
    R = delta.shape[0]
    color = torch.empty((R, 3), dtype=torch.float32, device=sigma.device)
    trans = torch.empty((R,), dtype=torch.float32, device=sigma.device)
    w = torch.empty((R * n_samples,), dtype=torch.float32, device=sigma.device) if with_weights else None
    L.check(L.lib().sxe_vr_composite(_ptr(sigma), _ptr(logits), _ptr(delta), R, n_samples, _ptr(color), _ptr(trans),
                                     _ptr(w), _stream(stream)), "sxe_vr_composite")
    return color, trans, w


def _main(argv=None):
    """Render seeded camera rays through a random field and print the time per render:
    ``python -m paper_2311_15439_gb300.render --rays 65536 --samples 64 --kind simplex``;
    with ``--train``, the time per training step (``VolumeTrainer.step``) towards seeded uniform
    target colours."""
    import argparse
    from . import synth
    ap = argparse.ArgumentParser(description=_main.__doc__)
    ap.add_argument("--rays", type=int, default=1 << 16)
    ap.add_argument("--samples", type=int, default=64)
    ap.add_argument("--kind", default="simplex", choices=["simplex", "grid"])
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--repeat", type=int, default=5)
    ap.add_argument("--unfused", action="store_true", help="the field as three launches")
    ap.add_argument("--train", action="store_true", help="time training steps instead of renders")
    a = ap.parse_args(argv)
    enc = Encoder(3, 16, 2, 19, 16.0, 1.38, kind=a.kind, table_dtype="f16")
    if a.train:
        vt = VolumeTrainer(enc, a.rays, a.samples, seed=63)
        rays = [torch.from_numpy(v).cuda() for v in synth.camera_rays(a.rays, 60)]
        target = torch.from_numpy(synth.rng(64).random((a.rays, 3)).astype("float32")).cuda()
        for _ in range(a.warmup):
            vt.step(*rays, target)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        for _ in range(a.repeat):
            vt.step(*rays, target)
        e.record()
        torch.cuda.synchronize()
        print("train %s: %d rays x %d samples: %.3f ms per step, loss %.4g" %
              (a.kind, a.rays, a.samples, s.elapsed_time(e) / a.repeat, vt.loss()))
        return
    rr = Renderer(enc, a.rays, a.samples, dtype="f16", fused=not a.unfused)
    _, store = synth.uniform_tables(16, 1 << 19, 2, 61, dtype="f16", scale=1.0)
    tab = torch.from_numpy(store).cuda()
    Wd, Wc = rr.init_weights(62)
    rays = [torch.from_numpy(v).cuda() for v in synth.camera_rays(a.rays, 60)]
    for _ in range(a.warmup):
        rr.render(*rays, tab, Wd, Wc)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(a.repeat):
        rr.render(*rays, tab, Wd, Wc)
    e.record()
    torch.cuda.synchronize()
    print("render %s: %d rays x %d samples: %.3f ms" % (a.kind, a.rays, a.samples, s.elapsed_time(e) / a.repeat))


if __name__ == "__main__":
    _main()
