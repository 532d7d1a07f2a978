"""Training step of the image-fitting and SDF-style workloads (Sec. 6.1 of arXiv 2311.15439).

One ``step(x, target)`` runs, on the caller's stream and entirely in libsimplexenc
kernels:

1. ``sxe_encode_fwd``           -- multiresolution encoding of the batch from the dense
                                   low-precision tables (Sec. 5 a-d);
2. ``sxe_mlp_train_l2_grouped`` -- network forward, L2 loss, network backward; dL/d(encoding)
                                   written level-major [L][P][F] (Sec. 5 d-e);
3. ``sxe_table_step``           -- scatter of dL/d(encoding) into the tables and Adam with the
                                   zero-gradient skip rule on the touched entries, refreshing the
                                   low-precision tables (Sec. 5 e);
4. ``sxe_step``                 -- Adam on the network weights, refreshing their fp16 copy.

Table state in HBM: one record of 4F binary32 words per entry {param[F], m[F], v[F], grad[F]},
entries ordered [level][slot] (32 bytes = one DRAM sector for F = 2); a dense [L][T][F]
low-precision copy for the forward gathers; a [T][F] binary32 scratch and an L*T-bit touched
bitmap, both zero between steps.
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


def pack_records(values: np.ndarray) -> np.ndarray:
    """State records {param, m = 0, v = 0, grad = 0} for binary32 parameters [n, F]."""
    n, F = values.shape
    rec = np.zeros((n, 4 * F), dtype=np.float32)
    rec[:, :F] = values
    return rec


def lowp_copy(values: np.ndarray, table_dtype: str):
    """The table-dtype rounding of binary32 values as a torch tensor (host)."""
    if table_dtype == "f32":
        return torch.from_numpy(values.copy())
    if table_dtype == "f16":
        return torch.from_numpy(values.astype(np.float16))
    return torch.from_numpy(synth.fp32_to_bf16_bits(values).view(np.int16)).view(torch.bfloat16)


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
        self.state = torch.from_numpy(pack_records(vals.reshape(n_entries, F))).to(self.device)
        self.tables = lowp_copy(vals, encoder.table_dtype).to(self.device)
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
        self.d_enc = torch.empty((encoder.n_levels, batch, F), dtype=torch.float32, device=self.device)
        self.sq_sum = torch.zeros((1,), dtype=torch.float32, device=self.device)
        self.ws = mlp.workspace(batch, self.device)
        self.loss_scale = default_loss_scale(batch, mlp.n_out)
        self.adam_tables = Adam(lr, betas[0], betas[1], eps, skip_zero_grad=True)
        self.adam_mlp = Adam(lr, betas[0], betas[1], eps, skip_zero_grad=False)
        self.t = 0

    @property
    def n_launches_per_step(self) -> int:
        # encode, network train + its partial reduction, table step, network Adam
        lc = sum(1 for N in self.enc.level_params()[1] if (int(N) + 2.0) ** self.enc.d <= self.enc.T / 4.0)
        table = (2 if lc > 0 else 0) + 2 * (self.enc.n_levels - lc)
        return 4 + table

    def forward_and_grads(self, x: torch.Tensor, target: torch.Tensor, stream=None) -> None:
        """Encode and run the network with its L2 loss and backward pass (stages 1-2)."""
        self.enc.encode_fwd(x, self.tables, self.enc_out, stream=stream)
        self.mlp.mlp_train_l2_grouped(self.W_lowp, self.enc_out, target, self.dW, self.sq_sum, self.d_enc,
                                      self.enc.n_features, loss_scale=self.loss_scale, workspace=self.ws,
                                      stream=stream)

    def apply_updates(self, x: torch.Tensor, stream=None) -> None:
        """Table update and network Adam step (stages 3-4)."""
        self.enc.table_step(self.adam_tables, self.t, x, self.d_enc, self.state, self.tables, self.scratch,
                            self.touched, stream=stream)
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
        """The dense low-precision tables the forward pass reads, [L, T, F]."""
        return self.tables

    def d_enc_rows(self) -> torch.Tensor:
        """dL/d(encoding) of the last step in the [P, L*F] layout of ``sxe_encode_bwd``."""
        return self.d_enc.permute(1, 0, 2).reshape(self.P, -1).contiguous()
