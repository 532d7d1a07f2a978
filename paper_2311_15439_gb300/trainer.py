"""Training step of the image-fitting and SDF-style workloads (Sec. 6.1 of arXiv 2311.15439).

One ``step(x, target)`` runs, on the caller's stream and entirely in libsimplexenc
kernels:

1. ``sxe_encode_fwd_strided`` -- multiresolution encoding of the batch, gathering the
                                 low-precision table values from the state records (Sec. 5 a-d);
2. ``sxe_mlp_train_l2``       -- network forward, L2 loss, network backward, dL/d(encoding)
                                 (Sec. 5 d-e);
3. ``sxe_table_step``         -- per level: scatter-add of dL/d(encoding) into an L2-resident
                                 scratch, then Adam (zero-gradient skip rule) on the touched
                                 entries, refreshing their low-precision copies (Sec. 5 e);
4. ``sxe_step``               -- Adam on the network weights, refreshing their fp16 copy.

Table state in HBM: one record of 4F binary32 words per entry {param[F], m[F], v[F],
low-precision copy of param}, entries ordered [level][slot] (32 bytes = one DRAM sector
for F = 2); a [T][F] binary32 scratch and an L*T-bit touched bitmap, both zero between steps.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import synth
from .api import Adam, Encoder, Mlp, torch_dtype


def default_loss_scale(P: int, n_out: int) -> float:
    """Power of two near P*n_out/2 so that the scaled L2 gradient 2 r / (P n_out) is O(r)."""
    return float(2.0 ** max(0, math.floor(math.log2(max(1.0, P * n_out / 2.0)))))


def pack_records(values: np.ndarray, table_dtype: str) -> np.ndarray:
    """State records {param, m = 0, v = 0, low-precision copy} for binary32 parameters [n, F]."""
    n, F = values.shape
    rec = np.zeros((n, 4 * F), dtype=np.float32)
    rec[:, :F] = values
    if table_dtype == "f32":
        rec[:, 3 * F:] = values
    else:
        bits = values.astype(np.float16).view(np.uint16) if table_dtype == "f16" else synth.fp32_to_bf16_bits(values)
        rec.view(np.uint16)[:, 6 * F:7 * F] = bits
    return rec


class Trainer:
    def __init__(self, encoder: Encoder, mlp: Mlp, batch: int, *, seed: int = 0, device="cuda",
                 table_init: float = 1e-4, lr: float = 1e-2, betas=(0.9, 0.99), eps: float = 1e-15):
        if mlp.n_in != encoder.n_out:
            raise ValueError("network input %d != encoding width %d" % (mlp.n_in, encoder.n_out))
        self.enc, self.mlp, self.P = encoder, mlp, batch
        self.device = torch.device(device)
        F = encoder.n_features
        n_entries = encoder.n_levels * encoder.T
        # seeded host values U(-table_init, table_init), so any checker can regenerate them
        vals = synth.uniform_tables(encoder.n_levels, encoder.T, F, seed, dtype="f32", scale=table_init)[0]
        self.state = torch.from_numpy(pack_records(vals.reshape(n_entries, F), encoder.table_dtype)).to(self.device)
        del vals
        self.scratch = torch.zeros((encoder.T, F), dtype=torch.float32, device=self.device)
        self.touched = torch.zeros(((n_entries + 31) // 32,), dtype=torch.int32, device=self.device)
        W0 = torch.from_numpy(mlp.init_weights(seed + 1)).to(self.device)
        self.W = W0.clone()
        self.W_lowp = W0.to(torch_dtype(mlp.dtype))
        self.mW = torch.zeros_like(W0)
        self.vW = torch.zeros_like(W0)
        self.dW = torch.zeros_like(W0)
        self.enc_out = torch.empty((batch, encoder.n_out), dtype=torch_dtype(encoder.out_dtype), device=self.device)
        self.d_enc = torch.empty((batch, encoder.n_out), dtype=torch.float32, device=self.device)
        self.sq_sum = torch.zeros((1,), dtype=torch.float32, device=self.device)
        self.ws = mlp.workspace(batch, self.device)
        self.loss_scale = default_loss_scale(batch, mlp.n_out)
        self.adam_tables = Adam(lr, betas[0], betas[1], eps, skip_zero_grad=True)
        self.adam_mlp = Adam(lr, betas[0], betas[1], eps, skip_zero_grad=False)
        self.t = 0

    @property
    def n_launches_per_step(self) -> int:
        # encode, network train + its partial reduction, 2 per level for the tables, network Adam
        return 4 + 2 * self.enc.n_levels

    def forward_and_grads(self, x: torch.Tensor, target: torch.Tensor, stream=None) -> None:
        """Encode and run the network with its L2 loss and backward pass (stages 1-2)."""
        self.enc.encode_fwd_records(x, self.state, self.enc_out, stream=stream)
        self.mlp.mlp_train_l2(self.W_lowp, self.enc_out, target, self.dW, self.sq_sum, din=self.d_enc,
                              loss_scale=self.loss_scale, workspace=self.ws, stream=stream)

    def apply_updates(self, x: torch.Tensor, stream=None) -> None:
        """Table update and network Adam step (stages 3-4)."""
        self.enc.table_step(self.adam_tables, self.t, x, self.d_enc, self.state, self.scratch, self.touched,
                            stream=stream)
        self.adam_mlp.step(self.t, self.W, self.mW, self.vW, self.dW, lowp=self.W_lowp, stream=stream)

    def step(self, x: torch.Tensor, target: torch.Tensor, stream=None) -> None:
        """One optimisation step on batch (x [P, d] float32, target [P, n_out] float32); asynchronous."""
        self.t += 1
        self.forward_and_grads(x, target, stream)
        self.apply_updates(x, stream)

    def loss(self) -> float:
        """Mean squared error of the last step (synchronises)."""
        return float(self.sq_sum.item()) / (self.P * self.mlp.n_out)

    def table_params(self) -> torch.Tensor:
        """binary32 master table parameters as [L*T, F] (a view)."""
        return self.state[:, :self.enc.n_features]

    def table_lowp(self) -> torch.Tensor:
        """The low-precision table copy as a dense [L, T, F] tensor (copied out of the records)."""
        F = self.enc.n_features
        dt = torch_dtype(self.enc.table_dtype)
        low = self.state[:, 3 * F:].contiguous().view(dt)[:, :F]
        return low.reshape(self.enc.table_shape()).contiguous()
