"""Python binding of libsimplexenc: the C-ABI entry points with tensor arguments.

Every method checks that its tensors live on the GPU, are contiguous and have the
expected dtype, then passes their device pointers and the current CUDA stream to the
library.  No arithmetic of the method happens here: PyTorch only provides device
memory and streams.  Names follow the C functions (``sxe_encode_fwd`` ->
``Encoder.encode_fwd`` and so on).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib as L

_DTYPES = {"f32": (L.SXE_F32, torch.float32), "f16": (L.SXE_F16, torch.float16),
           "bf16": (L.SXE_BF16, torch.bfloat16)}
_KINDS = {"simplex": L.SXE_SIMPLEX, "grid": L.SXE_GRID}
_RES = {"raw": L.SXE_RES_RAW, "equal_mem": L.SXE_RES_EQUAL_MEM}
_INDEX = {"hash": L.SXE_INDEX_HASH, "dense_coarse": L.SXE_INDEX_DENSE_COARSE}


def torch_dtype(name: str) -> torch.dtype:
    return _DTYPES[name][1]


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t):
    return None if t is None else t.data_ptr()


def _need(t: torch.Tensor, dtype: torch.dtype, name: str, shape=None) -> None:
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (the library has no CPU path)" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))


class Encoder:
    """Multiresolution simplex (or 2^d grid) hash encoding, ``sxe_encoder_*`` / ``sxe_encode_*``."""

    def __init__(self, d: int, n_levels: int, n_features: int, log2_T: int, base_res: float, growth: float,
                 kind: str = "simplex", res_mode: str = "raw", table_dtype: str = "f16", out_dtype: str | None = None,
                 index_mode: str = "hash"):
        self.d, self.n_levels, self.n_features, self.log2_T = d, n_levels, n_features, log2_T
        self.base_res, self.growth, self.kind, self.res_mode = base_res, growth, kind, res_mode
        self.index_mode = index_mode
        self.table_dtype = table_dtype
        self.out_dtype = out_dtype or table_dtype
        self.T = 1 << log2_T
        self.n_out = n_levels * n_features
        self.n_vertices = d + 1 if kind == "simplex" else (1 << d)
        desc = L.EncodingDesc(d, n_levels, n_features, log2_T, float(base_res), float(growth), _KINDS[kind],
                              _RES[res_mode], _DTYPES[table_dtype][0], _DTYPES[self.out_dtype][0],
                              _INDEX[index_mode])
        h = ctypes.c_void_p()
        L.check(L.lib().sxe_encoder_create(ctypes.byref(desc), ctypes.byref(h)), "sxe_encoder_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            L.lib().sxe_encoder_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def table_shape(self):
        return (self.n_levels, self.T, self.n_features)

    def level_params(self):
        """(binary32 per-level multipliers, int32 level resolutions N_l) as numpy arrays."""
        s = np.zeros(self.n_levels, dtype=np.float32)
        r = np.zeros(self.n_levels, dtype=np.int32)
        L.check(L.lib().sxe_encoder_level_params(self._h, s.ctypes.data, r.ctypes.data), "sxe_encoder_level_params")
        return s, r

    def level_index(self):
        """int32 box width B per level for directly indexed levels, 0 for hashed ones."""
        w = np.zeros(self.n_levels, dtype=np.int32)
        L.check(L.lib().sxe_encoder_level_index(self._h, w.ctypes.data), "sxe_encoder_level_index")
        return w

    def encode_fwd(self, x: torch.Tensor, tables: torch.Tensor, out: torch.Tensor | None = None, stream=None,
                   touched: torch.Tensor | None = None):
        """``sxe_encode_fwd``; with ``touched`` (int32 bitmap of L*T bits) ``sxe_encode_fwd_marked``."""
        P = x.shape[0]
        _need(x, torch.float32, "x", (P, self.d))
        _need(tables, torch_dtype(self.table_dtype), "tables", self.table_shape())
        if out is None:
            out = torch.empty((P, self.n_out), dtype=torch_dtype(self.out_dtype), device=x.device)
        _need(out, torch_dtype(self.out_dtype), "out", (P, self.n_out))
        if touched is None:
            L.check(L.lib().sxe_encode_fwd(self._h, _ptr(x), P, _ptr(tables), _ptr(out), _stream(stream)),
                    "sxe_encode_fwd")
        else:
            _need(touched, torch.int32, "touched", ((self.n_levels * self.T + 31) // 32,))
            L.check(L.lib().sxe_encode_fwd_marked(self._h, _ptr(x), P, _ptr(tables), _ptr(out), _ptr(touched),
                                                  _stream(stream)), "sxe_encode_fwd_marked")
        return out

    def encode_bwd(self, x: torch.Tensor, dout: torch.Tensor, grad: torch.Tensor, grad_stride: int | None = None,
                   touched: torch.Tensor | None = None, grad_offset: int = 0, levels: tuple[int, int] | None = None,
                   stream=None):
        """grad += d(out)/d(tables)^T dout.  ``grad`` is a float32 tensor; entry (l, slot) starts at
        float ``grad_offset + (l*T + slot) * grad_stride`` (default stride F: a dense [L, T, F] array).
        ``levels = (begin, end)`` restricts the terms to those levels (``sxe_encode_bwd_levels``)."""
        P = x.shape[0]
        _need(x, torch.float32, "x", (P, self.d))
        _need(dout, torch.float32, "dout", (P, self.n_out))
        stride = self.n_features if grad_stride is None else grad_stride
        _need(grad, torch.float32, "grad")
        if grad.numel() < grad_offset + (self.n_levels * self.T - 1) * stride + self.n_features:
            raise ValueError("grad is too small for the table layout")
        if touched is not None:
            _need(touched, torch.int32, "touched")
            if touched.numel() * 32 < self.n_levels * self.T:
                raise ValueError("touched bitmap too small")
        gp = grad.data_ptr() + 4 * grad_offset
        if levels is None:
            L.check(L.lib().sxe_encode_bwd(self._h, _ptr(x), P, _ptr(dout), gp, stride, _ptr(touched),
                                           _stream(stream)), "sxe_encode_bwd")
        else:
            L.check(L.lib().sxe_encode_bwd_levels(self._h, _ptr(x), P, _ptr(dout), gp, stride, _ptr(touched),
                                                  int(levels[0]), int(levels[1]), _stream(stream)),
                    "sxe_encode_bwd_levels")
        return grad

    def set_bwd_aggregation(self, on: bool) -> None:
        """Warp-level sums of the backward terms that land in the same table entry
        (``sxe_encoder_set_bwd_aggregation``): for batches whose consecutive points are spatially
        coherent, such as the samples along rays."""
        L.check(L.lib().sxe_encoder_set_bwd_aggregation(self._h, 1 if on else 0), "sxe_encoder_set_bwd_aggregation")

    def set_fwd_order(self, order: str) -> None:
        """Work-item order of the forward encoding (``sxe_encoder_set_fwd_order``): "auto"
        (level-major where the tables exceed L2 but one level's fits), "point" or "level"; the
        outputs are the same bit for bit."""
        code = {"auto": L.SXE_FWD_ORDER_AUTO, "point": L.SXE_FWD_ORDER_POINT_MAJOR,
                "level": L.SXE_FWD_ORDER_LEVEL_MAJOR}[order]
        L.check(L.lib().sxe_encoder_set_fwd_order(self._h, code), "sxe_encoder_set_fwd_order")

    def bwd_kernel_count(self, n_points: int, levels: tuple[int, int] | None = None) -> int:
        """Kernels one ``encode_bwd`` call launches for this many points (0, 1 or 2)."""
        if levels is None:
            return int(L.lib().sxe_encode_bwd_kernel_count(self._h, n_points))
        return int(L.lib().sxe_encode_bwd_levels_kernel_count(self._h, n_points, int(levels[0]), int(levels[1])))

    def bwd_coarse_levels(self, n_points: int) -> int:
        """Leading levels whose backward is summed per block in shared memory for this many points
        (their own kernel; ``encode_bwd(levels=(0, n))`` and ``levels=(n, L)`` may run on two streams)."""
        return int(L.lib().sxe_encode_bwd_coarse_levels(self._h, n_points))

    def encode_bwd_input(self, x: torch.Tensor, tables: torch.Tensor, dout: torch.Tensor,
                         dx: torch.Tensor | None = None, stream=None):
        """dx += d(out)/dx^T dout (``sxe_encode_bwd_input``); returns dx [P, d] float32."""
        P = x.shape[0]
        _need(x, torch.float32, "x", (P, self.d))
        _need(tables, torch_dtype(self.table_dtype), "tables", self.table_shape())
        _need(dout, torch.float32, "dout", (P, self.n_out))
        if dx is None:
            dx = torch.zeros((P, self.d), dtype=torch.float32, device=x.device)
        _need(dx, torch.float32, "dx", (P, self.d))
        L.check(L.lib().sxe_encode_bwd_input(self._h, _ptr(x), P, _ptr(tables), _ptr(dout), _ptr(dx),
                                             _stream(stream)), "sxe_encode_bwd_input")
        return dx

    def encode_plain_fwd(self, x: torch.Tensor, tables: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """Plain binary32 comparator path (``sxe_encode_plain_fwd``)."""
        P = x.shape[0]
        _need(x, torch.float32, "x", (P, self.d))
        _need(tables, torch.float32, "tables", self.table_shape())
        if out is None:
            out = torch.empty((P, self.n_out), dtype=torch.float32, device=x.device)
        _need(out, torch.float32, "out", (P, self.n_out))
        L.check(L.lib().sxe_encode_plain_fwd(self._h, _ptr(x), P, _ptr(tables), _ptr(out), _stream(stream)),
                "sxe_encode_plain_fwd")
        return out

    def encode_plain_bwd(self, x: torch.Tensor, dout: torch.Tensor, grad: torch.Tensor, stream=None):
        """Plain binary32 comparator path (``sxe_encode_plain_bwd``); grad is a dense [L, T, F] array."""
        P = x.shape[0]
        _need(x, torch.float32, "x", (P, self.d))
        _need(dout, torch.float32, "dout", (P, self.n_out))
        _need(grad, torch.float32, "grad", self.table_shape())
        L.check(L.lib().sxe_encode_plain_bwd(self._h, _ptr(x), P, _ptr(dout), _ptr(grad), _stream(stream)),
                "sxe_encode_plain_bwd")
        return grad

    def encode_vertices(self, x: torch.Tensor, stream=None):
        """(slots int32 [P, L, V], weights float32 [P, L, V])."""
        P = x.shape[0]
        _need(x, torch.float32, "x", (P, self.d))
        slots = torch.empty((P, self.n_levels, self.n_vertices), dtype=torch.int32, device=x.device)
        w = torch.empty((P, self.n_levels, self.n_vertices), dtype=torch.float32, device=x.device)
        L.check(L.lib().sxe_encode_vertices(self._h, _ptr(x), P, _ptr(slots), _ptr(w), _stream(stream)),
                "sxe_encode_vertices")
        return slots, w


class Mlp:
    """Fully fused 64-wide ReLU network, ``sxe_mlp_*``."""

    def __init__(self, n_in: int, n_out: int, n_hidden: int = 2, width: int = 64, dtype: str = "f16"):
        self.n_in, self.n_out, self.n_hidden, self.width, self.dtype = n_in, n_out, n_hidden, width, dtype
        self.desc = L.MlpDesc(n_in, width, n_hidden, n_out, _DTYPES[dtype][0])
        self.n_params = int(L.lib().sxe_mlp_n_params(ctypes.byref(self.desc)))
        self.shapes = [(width, n_in)] + [(width, width)] * (n_hidden - 1) + [(n_out, width)]

    def init_weights(self, seed: int) -> np.ndarray:
        """He-uniform binary32 weights (host), layout of the C ABI."""
        g = np.random.Generator(np.random.PCG64(seed))
        parts = [g.uniform(-math.sqrt(6.0 / fi), math.sqrt(6.0 / fi), size=(fo, fi)) for fo, fi in self.shapes]
        return np.concatenate([p.ravel() for p in parts]).astype(np.float32)

    def split(self, flat):
        """View a flat weight vector as the list of [fan_out, fan_in] matrices."""
        out, o = [], 0
        for fo, fi in self.shapes:
            out.append(flat[o:o + fo * fi].reshape(fo, fi))
            o += fo * fi
        return out

    def workspace_bytes(self, P: int) -> int:
        return int(L.lib().sxe_mlp_bwd_workspace_bytes(ctypes.byref(self.desc), P))

    def workspace(self, P: int, device) -> torch.Tensor:
        return torch.empty(max(1, self.workspace_bytes(P) // 4), dtype=torch.float32, device=device)

    def mlp_fwd(self, W: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None, act: torch.Tensor | None = None,
                stream=None):
        dt = torch_dtype(self.dtype)
        P = x.shape[0]
        _need(W, dt, "weights", (self.n_params,))
        _need(x, dt, "in", (P, self.n_in))
        if out is None:
            out = torch.empty((P, self.n_out), dtype=torch.float32, device=x.device)
        _need(out, torch.float32, "out", (P, self.n_out))
        if act is not None:
            _need(act, dt, "act", (self.n_hidden, P, self.width))
        L.check(L.lib().sxe_mlp_fwd(ctypes.byref(self.desc), _ptr(W), _ptr(x), P, _ptr(out), _ptr(act),
                                    _stream(stream)), "sxe_mlp_fwd")
        return out

    def mlp_bwd(self, W, x, dout, dW, din=None, loss_scale: float = 1.0, workspace=None, stream=None):
        dt = torch_dtype(self.dtype)
        P = x.shape[0]
        _need(W, dt, "weights", (self.n_params,))
        _need(x, dt, "in", (P, self.n_in))
        _need(dout, torch.float32, "dout", (P, self.n_out))
        _need(dW, torch.float32, "dweights", (self.n_params,))
        if din is not None:
            _need(din, torch.float32, "din", (P, self.n_in))
        ws = workspace if workspace is not None else self.workspace(P, x.device)
        L.check(L.lib().sxe_mlp_bwd(ctypes.byref(self.desc), _ptr(W), _ptr(x), _ptr(dout), float(loss_scale), P,
                                    _ptr(din), _ptr(dW), _ptr(ws), ws.numel() * 4, _stream(stream)), "sxe_mlp_bwd")
        return dW

    def mlp_train_l2(self, W, x, target, dW, sq_sum, din=None, loss_scale: float = 1.0, workspace=None, stream=None):
        dt = torch_dtype(self.dtype)
        P = x.shape[0]
        _need(W, dt, "weights", (self.n_params,))
        _need(x, dt, "in", (P, self.n_in))
        _need(target, torch.float32, "target", (P, self.n_out))
        _need(dW, torch.float32, "dweights", (self.n_params,))
        _need(sq_sum, torch.float32, "sq_sum", (1,))
        if din is not None:
            _need(din, torch.float32, "din", (P, self.n_in))
        ws = workspace if workspace is not None else self.workspace(P, x.device)
        L.check(L.lib().sxe_mlp_train_l2(ctypes.byref(self.desc), _ptr(W), _ptr(x), _ptr(target), float(loss_scale),
                                         P, _ptr(din), _ptr(dW), _ptr(sq_sum), _ptr(ws), ws.numel() * 4,
                                         _stream(stream)), "sxe_mlp_train_l2")
        return dW

    def mlp_train_l2_part(self, W, x, target, dW, sq_sum, batch_points: int, din=None, loss_scale: float = 1.0,
                          workspace=None, stream=None):
        """``sxe_mlp_train_l2_part``: the L2 pass on one part (x, target) of a batch of ``batch_points``
        points; the gradient is normalised by the whole batch and accumulated into dW."""
        dt = torch_dtype(self.dtype)
        P = x.shape[0]
        _need(W, dt, "weights", (self.n_params,))
        _need(x, dt, "in", (P, self.n_in))
        _need(target, torch.float32, "target", (P, self.n_out))
        _need(dW, torch.float32, "dweights", (self.n_params,))
        _need(sq_sum, torch.float32, "sq_sum", (1,))
        if din is not None:
            _need(din, torch.float32, "din", (P, self.n_in))
        ws = workspace if workspace is not None else self.workspace(P, x.device)
        L.check(L.lib().sxe_mlp_train_l2_part(ctypes.byref(self.desc), _ptr(W), _ptr(x), _ptr(target),
                                              float(loss_scale), P, int(batch_points), _ptr(din), _ptr(dW),
                                              _ptr(sq_sum), _ptr(ws), ws.numel() * 4, _stream(stream)),
                "sxe_mlp_train_l2_part")
        return dW

    def mlp_train_l2_grouped(self, W, x, target, dW, sq_sum, din, din_group: int, loss_scale: float = 1.0,
                             workspace=None, stream=None):
        """``sxe_mlp_train_l2_grouped``: din written as [n_in / g, P, g]."""
        dt = torch_dtype(self.dtype)
        P = x.shape[0]
        _need(W, dt, "weights", (self.n_params,))
        _need(x, dt, "in", (P, self.n_in))
        _need(target, torch.float32, "target", (P, self.n_out))
        _need(dW, torch.float32, "dweights", (self.n_params,))
        _need(sq_sum, torch.float32, "sq_sum", (1,))
        _need(din, torch.float32, "din", (self.n_in // din_group, P, din_group))
        ws = workspace if workspace is not None else self.workspace(P, x.device)
        L.check(L.lib().sxe_mlp_train_l2_grouped(ctypes.byref(self.desc), _ptr(W), _ptr(x), _ptr(target),
                                                 float(loss_scale), P, _ptr(din), int(din_group), _ptr(dW),
                                                 _ptr(sq_sum), _ptr(ws), ws.numel() * 4, _stream(stream)),
                "sxe_mlp_train_l2_grouped")
        return dW

    def mlp_train_l2_static(self, W, x, target, dW, sq_sum, din=None, loss_scale: float = 1.0, stream=None):
        """``sxe_mlp_train_l2_static``: the same computation without a workspace argument, for
        callers that cannot allocate device memory (the library's own fixed scratch is used)."""
        dt = torch_dtype(self.dtype)
        P = x.shape[0]
        _need(W, dt, "weights", (self.n_params,))
        _need(x, dt, "in", (P, self.n_in))
        _need(target, torch.float32, "target", (P, self.n_out))
        _need(dW, torch.float32, "dweights", (self.n_params,))
        _need(sq_sum, torch.float32, "sq_sum", (1,))
        if din is not None:
            _need(din, torch.float32, "din", (P, self.n_in))
        L.check(L.lib().sxe_mlp_train_l2_static(ctypes.byref(self.desc), _ptr(W), _ptr(x), _ptr(target),
                                                float(loss_scale), P, _ptr(din), _ptr(dW), _ptr(sq_sum),
                                                _stream(stream)), "sxe_mlp_train_l2_static")
        return dW


def loss_l2(y, target, dy, sq_sum, stream=None):
    P, n_out = y.shape
    for t, n in ((y, "y"), (target, "target"), (dy, "dy")):
        _need(t, torch.float32, n, (P, n_out))
    _need(sq_sum, torch.float32, "sq_sum", (1,))
    L.check(L.lib().sxe_loss_l2(_ptr(y), _ptr(target), P, n_out, _ptr(dy), _ptr(sq_sum), _stream(stream)),
            "sxe_loss_l2")


class Adam:
    """Adam hyper-parameters and the ``sxe_step`` / ``sxe_step_touched`` updates."""

    def __init__(self, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15, skip_zero_grad=False):
        self.desc = L.AdamDesc(lr, beta1, beta2, eps, int(skip_zero_grad))

    def step(self, t: int, param, m, v, grad, lowp=None, stream=None):
        n = param.numel()
        for x, nm in ((param, "param"), (m, "m"), (v, "v"), (grad, "grad")):
            _need(x, torch.float32, nm)
            if x.numel() != n:
                raise ValueError("%s has %d elements, expected %d" % (nm, x.numel(), n))
        ldt = L.SXE_F32
        if lowp is not None:
            ldt = {torch.float32: L.SXE_F32, torch.float16: L.SXE_F16, torch.bfloat16: L.SXE_BF16}[lowp.dtype]
            if not lowp.is_cuda or not lowp.is_contiguous() or lowp.numel() != n:
                raise ValueError("lowp must be a contiguous CUDA tensor with %d elements" % n)
        L.check(L.lib().sxe_step(ctypes.byref(self.desc), int(t), n, _ptr(param), _ptr(m), _ptr(v), _ptr(grad),
                                 _ptr(lowp), ldt, _stream(stream)), "sxe_step")

    def advance(self, t_dev: torch.Tensor, corrections: torch.Tensor, stream=None):
        """Device step counter: t_dev += 1 (int64 [1]) and corrections = bias corrections (float32 [2])."""
        _need(t_dev, torch.int64, "t", (1,))
        _need(corrections, torch.float32, "corrections", (2,))
        L.check(L.lib().sxe_adam_advance(ctypes.byref(self.desc), _ptr(t_dev), _ptr(corrections), _stream(stream)),
                "sxe_adam_advance")

    def step_dev(self, corrections, param, m, v, grad, lowp=None, stream=None):
        """``step`` with the bias corrections read from device memory (``advance``)."""
        n = param.numel()
        _need(corrections, torch.float32, "corrections", (2,))
        for x, nm in ((param, "param"), (m, "m"), (v, "v"), (grad, "grad")):
            _need(x, torch.float32, nm)
            if x.numel() != n:
                raise ValueError("%s has %d elements, expected %d" % (nm, x.numel(), n))
        ldt = L.SXE_F32
        if lowp is not None:
            ldt = {torch.float32: L.SXE_F32, torch.float16: L.SXE_F16, torch.bfloat16: L.SXE_BF16}[lowp.dtype]
            if not lowp.is_cuda or not lowp.is_contiguous() or lowp.numel() != n:
                raise ValueError("lowp must be a contiguous CUDA tensor with %d elements" % n)
        L.check(L.lib().sxe_step_dev(ctypes.byref(self.desc), _ptr(corrections), n, _ptr(param), _ptr(m), _ptr(v),
                                     _ptr(grad), _ptr(lowp), ldt, _stream(stream)), "sxe_step_dev")

    def step_touched_dev(self, corrections, state, touched, table_lowp, n_features: int, stream=None):
        """``step_touched`` with the bias corrections read from device memory (``advance``)."""
        F = n_features
        _need(corrections, torch.float32, "corrections", (2,))
        _need(state, torch.float32, "state")
        _need(touched, torch.int32, "touched")
        n_entries = table_lowp.numel() // F
        if state.numel() != 4 * F * n_entries or touched.numel() * 32 < n_entries:
            raise ValueError("state / touched sizes do not match the table")
        ldt = {torch.float32: L.SXE_F32, torch.float16: L.SXE_F16, torch.bfloat16: L.SXE_BF16}[table_lowp.dtype]
        if not table_lowp.is_cuda or not table_lowp.is_contiguous():
            raise ValueError("table_lowp must be a contiguous CUDA tensor")
        L.check(L.lib().sxe_step_touched_dev(ctypes.byref(self.desc), _ptr(corrections), n_entries, F, _ptr(state),
                                             _ptr(touched), _ptr(table_lowp), ldt, _stream(stream)),
                "sxe_step_touched_dev")

    def step_touched(self, t: int, state, touched, table_lowp, n_features: int, stream=None):
        F = n_features
        _need(state, torch.float32, "state")
        _need(touched, torch.int32, "touched")
        n_entries = table_lowp.numel() // F
        if state.numel() != 4 * F * n_entries or touched.numel() * 32 < n_entries:
            raise ValueError("state / touched sizes do not match the table")
        ldt = {torch.float32: L.SXE_F32, torch.float16: L.SXE_F16, torch.bfloat16: L.SXE_BF16}[table_lowp.dtype]
        if not table_lowp.is_cuda or not table_lowp.is_contiguous():
            raise ValueError("table_lowp must be a contiguous CUDA tensor")
        L.check(L.lib().sxe_step_touched(ctypes.byref(self.desc), int(t), n_entries, F, _ptr(state), _ptr(touched),
                                         _ptr(table_lowp), ldt, _stream(stream)), "sxe_step_touched")


def version() -> str:
    return L.lib().sxe_version().decode()
