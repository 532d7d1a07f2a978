"""Pins of the oracle's lattice geometry against what the paper and mathematics fix (CPU only)."""
import itertools
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import geometry, lattice
from paper_2311_15439_gb300 import synth


@pytest.mark.parametrize("n", range(2, 8))
def test_unskew_inverts_skew(n):
    """Eq. 3 inverts Eq. 2 (Sec. 2.2 d: unskewing recovers the original coordinate)."""
    x = synth.rng(n).standard_normal((500, n)) * 50
    back = lattice.unskew(lattice.skew(x))
    assert np.max(np.abs(back - x)) <= 1e-13 * np.max(np.abs(x))
    fwd = lattice.skew(lattice.unskew(x))
    assert np.max(np.abs(fwd - x)) <= 1e-13 * np.max(np.abs(x))


@pytest.mark.parametrize("n", range(2, 8))
def test_skew_maps_diagonal_corner(n):
    """Sec. 5.1: after the skew the corner 1 becomes sqrt(n+1) * 1."""
    y = lattice.skew(np.ones((1, n)))
    np.testing.assert_allclose(y, math.sqrt(n + 1) * np.ones((1, n)), rtol=1e-15)


@pytest.mark.parametrize("n", range(2, 8))
def test_skew_equalises_diagonal(n):
    """Sec. 2.2 a: seen in the original space, the lattice corner 1 is as far from the
    origin as the lattice corner e_1 (the cube is squashed along its main diagonal)."""
    a = lattice.unskew(np.eye(n)[:1])
    b = lattice.unskew(np.ones((1, n)))
    assert np.linalg.norm(b) == pytest.approx(np.linalg.norm(a), rel=1e-14)


def test_2d_cells_are_equilateral():
    """Sec. 4.1: in two dimensions the skew turns each Kuhn simplex into an equilateral triangle."""
    for perm in itertools.permutations(range(2)):
        e = geometry.unskewed_edge_lengths(perm)
        np.testing.assert_allclose(e, e[0], rtol=1e-14)


def test_3d_edge_ratio():
    """Sec. 4.1: a 3-D cell has 4 edges of one length and 2 of another, ratio sqrt(3)/2."""
    for perm in itertools.permutations(range(3)):
        e = geometry.unskewed_edge_lengths(perm)
        short, long_ = e[:4], e[4:]
        np.testing.assert_allclose(short, short[0], rtol=1e-14)
        np.testing.assert_allclose(long_, long_[0], rtol=1e-14)
        assert short[0] / long_[0] == pytest.approx(math.sqrt(3) / 2, rel=1e-14)


@pytest.mark.parametrize("n", range(2, 7))
def test_lemma4_edge_lengths(n):
    """Lemma 4: every unskewed S_pi has n+1-k edges of length
    sqrt(k (1 - k G)^2 + (n - k)(k G)^2), k = 1..n (so all S'_pi are congruent)."""
    G = (1 - 1 / math.sqrt(n + 1)) / n
    want = []
    for k in range(1, n + 1):
        want += [math.sqrt(k * (1 - k * G) ** 2 + (n - k) * (k * G) ** 2)] * (n + 1 - k)
    want = np.sort(want)
    perms = list(itertools.permutations(range(n)))
    for perm in perms[:: max(1, len(perms) // 24)]:
        np.testing.assert_allclose(geometry.unskewed_edge_lengths(perm), want, rtol=1e-13)


@pytest.mark.parametrize("n", range(2, 7))
def test_theorem3_kuhn_edges(n):
    """Theorem 3: before the skew every S_pi has n+1-k edges of length sqrt(k)."""
    want = np.sort(sum([[math.sqrt(k)] * (n + 1 - k) for k in range(1, n + 1)], []))
    for perm in list(itertools.permutations(range(n)))[:24]:
        V = geometry.kuhn_simplex(perm).astype(float)
        d = np.sort([np.linalg.norm(V[i] - V[j]) for i, j in itertools.combinations(range(n + 1), 2)])
        np.testing.assert_allclose(d, want, rtol=1e-14)


def test_theoretical_memory_usage_figure():
    """Sec. 5.2 figure: 100 / V with V = |det(unskew(S_n I))| = (n+1)^((n-1)/2)."""
    for n, pct in read_golden("theoretical_memory_usage.txt"):
        n = int(n)
        assert 100.0 / geometry.parallelepiped_volume(n) == pytest.approx(float(pct), abs=6e-5)


def test_equal_memory_factor_keeps_touched_volume():
    """Sec. 5.2: scaling every level by m = (n+1)^((n-1)/(2n)) makes the touched simplex lattice of
    the unit cube, (m N)^n / V vertices with V the parallelepiped volume, as large as the grid's N^n:
    m^n equals V = |det(unskew(S_n I))| computed from the skew matrices."""
    for n in range(2, 8):
        assert lattice.equal_memory_factor(n) ** n == pytest.approx(geometry.parallelepiped_volume(n), rel=1e-12)


@pytest.mark.parametrize("n", range(2, 8))
def test_weights_reconstruct_point(n):
    """Theorem 1 / Sec. 4.3: weights are >= 0, sum to 1 and reproduce the skewed point."""
    q = synth.rng(10 + n).uniform(-3, 40, size=(2000, n))
    c, order, f = lattice.subdivide(q)
    V = lattice.simplex_vertices(c, order)
    w = lattice.barycentric_weights(f, order)
    assert np.all(w >= 0)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    rec = np.einsum("pk,pkn->pn", w, V.astype(float))
    np.testing.assert_allclose(rec, q, rtol=0, atol=1e-12)
    # Remark 2: the walk starts at floor(q) and ends at floor(q) + 1
    assert np.array_equal(V[:, 0], c) and np.array_equal(V[:, -1], c + 1)


@pytest.mark.parametrize("n", range(2, 6))
def test_weights_equal_hat_functions(n):
    """Every vertex of the cell gets the closed-form Kuhn hat-function value:
    listed vertices get the oracle's weight, all other cell corners get 0."""
    q = synth.rng(20 + n).uniform(0, 9, size=(400, n))
    c, order, f = lattice.subdivide(q)
    V = lattice.simplex_vertices(c, order)
    w = lattice.barycentric_weights(f, order)
    for k in range(n + 1):
        np.testing.assert_allclose(geometry.vertex_hat_weight(q, V[:, k]), w[:, k], atol=1e-13)
    for b in itertools.product((0, 1), repeat=n):
        corner = c + np.array(b)
        hat = geometry.vertex_hat_weight(q, corner)
        in_simplex = np.all(V == corner[:, None, :], axis=2).any(axis=1)
        assert np.all(hat[~in_simplex] <= 1e-13)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_subdivision_matches_brute_force(n):
    """Theorem 5 / Remark 2: the sorted-order simplex is the one (of n!) that contains
    the point, and its weights are the barycentric solve's coordinates."""
    g = synth.rng(30 + n)
    f = g.random((150, n))
    for p in range(len(f)):
        q = f[p:p + 1]
        c, order, ff = lattice.subdivide(q)
        assert np.all(c == 0)
        perm = tuple(order[0])
        hits = geometry.containing_permutations(q[0])
        assert hits == [perm]                      # interior point: exactly one simplex
        lam = geometry.barycentric_solve(geometry.kuhn_simplex(perm), q[0])
        np.testing.assert_allclose(lam, lattice.barycentric_weights(ff, order)[0], atol=1e-12)


def test_subdivision_on_ties():
    """Points on shared faces: the chosen simplex still contains the point and the
    tie rule (lower axis first) fixes the listed vertex order."""
    q = np.array([[0.5, 0.5, 0.2], [0.3, 0.3, 0.3], [0.0, 0.7, 0.7], [0.25, 0.0, 0.25]])
    c, order, f = lattice.subdivide(q)
    assert order.tolist() == [[0, 1, 2], [0, 1, 2], [1, 2, 0], [0, 2, 1]]
    for p in range(len(q)):
        assert tuple(order[p]) in geometry.containing_permutations(q[p])


def test_memory_usage_figure_exact():
    """Sec. 5.2 figure "Actual memory usage": the exact count of lattice vertices that the
    scaled (N / sqrt(n+1)) and skewed unit cube touches equals the paper's sampled figure
    at every point where the paper's sampling was dense enough (n = 2, N <= 32;
    n = 3, N <= 8; n = 4, N <= 4)."""
    golden = {(int(n), int(N)): float(p) for n, N, p in read_golden("memory_usage_by_level.txt")}
    for n, N in [(2, 2), (2, 4), (2, 8), (2, 16), (2, 32), (3, 2), (3, 4), (3, 8), (4, 2), (4, 4)]:
        count = geometry.touched_vertex_count(n, N)
        assert 100.0 * count / (N + 1) ** n == pytest.approx(golden[(n, N)], abs=6e-5), (n, N, count)


@pytest.mark.parametrize("n,N", [(2, 8), (2, 16), (3, 4)])
def test_memory_usage_by_subdivision(n, N):
    """The oracle's own subdivision, run on a dense sample of the unit cube, touches
    (with positive weight) exactly the lattice vertices the figure counts."""
    golden = {(int(a), int(b)): float(p) for a, b, p in read_golden("memory_usage_by_level.txt")}
    S = {2: 700, 3: 90}[n]
    g1 = (np.arange(S) + 0.5) / S
    x = np.stack(np.meshgrid(*([g1] * n), indexing="ij"), -1).reshape(-1, n)
    q = lattice.skew(x * (N / math.sqrt(n + 1)))
    c, order, f = lattice.subdivide(q)
    V = lattice.simplex_vertices(c, order)
    w = lattice.barycentric_weights(f, order)
    touched = np.unique(V[w > 0], axis=0)
    assert touched.min() >= 0 and touched.max() <= N            # stays inside [0, N]^n
    assert 100.0 * len(touched) / (N + 1) ** n == pytest.approx(golden[(n, N)], abs=6e-5)


def test_level_resolutions():
    for row in read_golden("level_resolutions.txt"):
        base, growth, L = float(row[0]), float(row[1]), int(row[2])
        assert lattice.level_resolutions(L, base, growth) == [int(v) for v in row[3:]]


def test_vertex_counts_figure():
    """Sec. 6.3 vertex-count figure: n+1 simplex vertices vs 2^n grid corners."""
    from oracle import encoding
    for n, s, g in read_golden("vertex_counts.txt"):
        n = int(n)
        x = synth.uniform_points(4, n, 1)
        q = lattice.scaled_skewed_fp32(x, np.float32(7.5))
        c, order, f = lattice.subdivide(q)
        assert lattice.simplex_vertices(c, order).shape[1] == int(s)
        _, f2 = encoding.grid_level_cell(x, np.float32(7))
        assert encoding.grid_level_corner_weights(f2).shape[1] == int(g)


def test_fp32_skew_matches_fp64_closely():
    """The binary32 scale+skew stays within a few ulps of the FP64 value (the
    quantisation the index parity is conditioned on is small)."""
    for n in range(2, 6):
        x = synth.uniform_points(10000, n, 5)
        for s in (9.2, 302.7, 3.0e5):
            q32 = lattice.scaled_skewed_fp32(x, np.float32(s)).astype(np.float64)
            q64 = lattice.skew(x.astype(np.float64) * float(np.float32(s)))
            assert np.max(np.abs(q32 - q64) / np.maximum(q64, 1e-30)) < (n + 2) * 2.0 ** -23


def test_hash_special_cases():
    """Hash: axis 0 has multiplier 1, so a vertex (a, 0, ..., 0) lands in slot a mod T;
    negative coordinates wrap as two's complement; slots stay inside the table."""
    for n in range(2, 6):
        for T in (10, 14, 19, 22):
            a = np.array([0, 1, 5, (1 << T) - 1, 1 << T, (1 << T) + 3, 123456789])
            v = np.zeros((len(a), n), dtype=np.int64)
            v[:, 0] = a
            assert np.array_equal(lattice.hash_slot(v, T), a % (1 << T))
            v[:, 0] = -1
            assert np.all(lattice.hash_slot(v, T) == (1 << T) - 1)
        # the published multipliers: a unit vertex e_i lands in slot pi_i mod T; the axes combine by
        # XOR, so (1, 1) lands in pi_2 XOR 1 = pi_2 - 1 (pi_2 odd) and (2, 3) in (3 pi_2 mod 2^32) XOR 2
        # = 3668339987 XOR 2 = 3668339985 (its two low bits are 11); all mod T = 2^19 here
        e = np.eye(n, dtype=np.int64)
        assert lattice.hash_slot(e, 19).tolist() == [p % (1 << 19) for p in (1, 2654435761, 805459861,
                                                                             1013904263, 2773480771)[:n]]
        pair = np.zeros((2, n), dtype=np.int64)
        pair[0, :2], pair[1, :2] = (1, 1), (2, 3)
        assert lattice.hash_slot(pair, 19).tolist() == [489904, 421137]
        big = synth.rng(n).integers(-2**31, 2**31 - 1, size=(1000, n))
        s = lattice.hash_slot(big, 19)
        assert s.min() >= 0 and s.max() < (1 << 19)


@pytest.mark.parametrize("n", range(2, 6))
def test_hash_uniformity(n):
    """A dense block of lattice vertices spreads evenly over the table (chi-square)."""
    log2_T = 10
    side = {2: 256, 3: 40, 4: 16, 5: 10}[n]
    v = np.stack(np.meshgrid(*([np.arange(side)] * n), indexing="ij"), -1).reshape(-1, n)
    counts = np.bincount(lattice.hash_slot(v, log2_T), minlength=1 << log2_T)
    expected = len(v) / (1 << log2_T)
    chi2 = np.sum((counts - expected) ** 2 / expected)
    dof = (1 << log2_T) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)
