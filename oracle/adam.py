"""Adam update in FP64 (test infrastructure only; see ``oracle``).

The paper trains tables and network with a gradient optimiser but does not
name it; its backbone (Instant-NGP) uses Adam and skips the update of every
hash-table entry whose gradient is exactly zero, so untouched entries keep
their parameter and moments.  This module restates Adam (Kingma & Ba,
Algorithm 1: bias-corrected first and second moments) with that skip rule as
an option.  Parity pin: an independent library Adam on the entries that take
a step.
"""
from __future__ import annotations

import numpy as np


def adam_step(theta, grad, m, v, t, *, lr, beta1, beta2, eps, skip_zero_grad):
    """One Adam step at 1-based step count ``t``; returns new (theta, m, v) as FP64 arrays."""
    theta = np.asarray(theta, dtype=np.float64).copy()
    g = np.asarray(grad, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64).copy()
    v = np.asarray(v, dtype=np.float64).copy()
    take = (g != 0.0) if skip_zero_grad else np.ones(g.shape, dtype=bool)
    m_new = beta1 * m + (1.0 - beta1) * g
    v_new = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m_new / (1.0 - beta1 ** t)
    v_hat = v_new / (1.0 - beta2 ** t)
    theta_new = theta - lr * m_hat / (np.sqrt(v_hat) + eps)
    theta[take] = theta_new[take]
    m[take] = m_new[take]
    v[take] = v_new[take]
    return theta, m, v
