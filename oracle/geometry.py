"""Brute-force and closed-form geometry used only to pin the oracle (test infrastructure only).

* ``kuhn_simplex``: the n+1 vertices of S_pi (Remark 2).
* ``barycentric_solve``: barycentric coordinates of a point in a simplex by a
  dense linear solve (the system of the proof of Theorem 1).
* ``containing_permutations``: every permutation pi whose S_pi contains the
  point, found by trying all n! of them (Theorem 5).
* ``unskewed_edge_lengths``: edge lengths of a Kuhn simplex after the unskew
  of Eq. 3 (Lemma 4 states their closed form).
* ``parallelepiped_volume``: |det| of the unskewed lattice cell scaled by
  S_n = sqrt(n+1) (Sec. 5.2).
* ``touched_vertex_count``: how many vertices of the (N+1)^n lattice box get a
  positive weight from some point of the unit cube, decided exactly by a
  linear program per vertex (Sec. 5.2, memory-usage figure).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import lattice


def kuhn_simplex(perm) -> np.ndarray:
    """Remark 2: v_1 = 0 and v_{i+1} = v_i + e_{perm[i]}; returns int64 [n+1, n]."""
    n = len(perm)
    V = np.zeros((n + 1, n), dtype=np.int64)
    for i, axis in enumerate(perm):
        V[i + 1] = V[i]
        V[i + 1, axis] = 1
    return V


def barycentric_solve(V: np.ndarray, x: np.ndarray) -> np.ndarray:
    """lambda with [1 ... 1; v_1 ... v_{n+1}] lambda = [1; x] (proof of Theorem 1)."""
    V = np.asarray(V, dtype=np.float64)
    n = V.shape[1]
    A = np.vstack([np.ones(n + 1), V.T])
    b = np.concatenate([[1.0], np.asarray(x, dtype=np.float64)])
    return np.linalg.solve(A, b)


def containing_permutations(x, tol=1e-12):
    """All permutations pi with x in S_pi (all barycentric coordinates >= -tol)."""
    n = len(x)
    hits = []
    for perm in itertools.permutations(range(n)):
        lam = barycentric_solve(kuhn_simplex(perm), x)
        if np.all(lam >= -tol):
            hits.append(perm)
    return hits


def unskewed_edge_lengths(perm) -> np.ndarray:
    """Sorted lengths of the n(n+1)/2 edges of S_pi mapped back by Eq. 3."""
    V = lattice.unskew(kuhn_simplex(perm).astype(np.float64))
    d = [np.linalg.norm(V[i] - V[j]) for i, j in itertools.combinations(range(len(V)), 2)]
    return np.sort(np.array(d))


def parallelepiped_volume(n: int) -> float:
    """|det(unskew(S_n I))|: volume, in the original space, of the lattice cell
    spanned by S_n e_1 ... S_n e_n of the skewed space (Sec. 5.2)."""
    S = math.sqrt(n + 1.0)
    M = lattice.unskew(S * np.eye(n))          # rows are the unskewed edge vectors
    return abs(float(np.linalg.det(M)))


def vertex_hat_weight(q: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Weight that vertex v receives at skewed point q in the Kuhn triangulation,
    written as the standard closed form of its piecewise-linear hat function:
    max(0, 1 - (max(0, max_i y_i) - min(0, min_i y_i))) with y = q - v."""
    y = np.asarray(q, dtype=np.float64) - np.asarray(v, dtype=np.float64)
    hi = np.maximum(0.0, y.max(axis=-1))
    lo = np.minimum(0.0, y.min(axis=-1))
    return np.maximum(0.0, 1.0 - (hi - lo))


def touched_vertex_count(n: int, N: int, margin: float = 1e-9) -> int:
    """Number of lattice vertices v in [0, N]^n whose hat function is positive
    somewhere on skew(s [0,1]^n), s = N / sqrt(n+1) (Sec. 5.1 scale).

    For each v solve: maximise delta over u in [0, s]^n with y = skew(u) - v and
    y_i <= 1 - delta, -y_i <= 1 - delta, y_i - y_j <= 1 - delta; v is touched iff
    the optimum delta exceeds ``margin``.
    """
    from scipy.optimize import linprog

    s = N / math.sqrt(n + 1.0)
    F = lattice.skew_factor(n)
    # q = (I + F 11^T) u
    K = np.eye(n) + F * np.ones((n, n))
    rows, rhs_const = [], []
    for i in range(n):
        rows.append(np.concatenate([K[i], [1.0]]));  rhs_const.append((i, +1))   # y_i + delta <= 1
        rows.append(np.concatenate([-K[i], [1.0]])); rhs_const.append((i, -1))   # -y_i + delta <= 1
    pair_rows = []
    for i in range(n):
        for j in range(n):
            if i != j:
                r = np.zeros(n + 1)
                r[i], r[j], r[n] = 1.0, -1.0, 1.0                                    # u_i - u_j - (v_i - v_j) + delta <= 1
                pair_rows.append((r, i, j))
    A = np.array(rows + [r for r, _, _ in pair_rows])
    c = np.zeros(n + 1)
    c[n] = -1.0
    bounds = [(0.0, s)] * n + [(None, 1.0)]
    count = 0
    for v in itertools.product(range(N + 1), repeat=n):
        v = np.array(v, dtype=np.float64)
        b = [1.0 + sign * v[i] for i, sign in rhs_const]
        b += [1.0 + v[i] - v[j] for _, i, j in pair_rows]
        res = linprog(c, A_ub=A, b_ub=np.array(b), bounds=bounds, method="highs")
        if res.status == 0 and -res.fun > margin:
            count += 1
    return count
