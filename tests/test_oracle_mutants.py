"""Planted mistakes in the oracle, each of which one of its pins must catch (CPU only).

Every case takes the source of one oracle function, makes one textual change that stands for a
plausible slip (a dropped term, a wrong sign or index, a transposed operand, an off-by-one), runs
the changed function in place of the original and requires at least one of the listed pin tests
to fail.  The change must match the source exactly once, so a later edit of the oracle that
removes the target text fails here instead of silently turning the case into a no-op.
"""
import functools
import inspect
import textwrap

import pytest

from oracle import adam, encoding, geometry, lattice, mlp, render

import test_oracle_encoding as TE
import test_oracle_lattice as TL
import test_oracle_render as TR


def _mutant(module, name, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert src.count(old) == 1, f"{module.__name__}.{name}: target {old!r} found {src.count(old)} times"
    ns = dict(module.__dict__)
    exec(compile(src.replace(old, new), f"<planted mistake in {module.__name__}.{name}>", "exec"), ns)
    return ns[name]


P = functools.partial

# (module, function, original text, planted text, pins that must catch it)
CASES = {
    # Eq. 2 / Eq. 3 and the scale of Sec. 5.1
    "skew factor over n+1": (lattice, "skew_factor", "- 1.0) / n", "- 1.0) / (n + 1)",
                             [P(TL.test_unskew_inverts_skew, 3), P(TL.test_skew_maps_diagonal_corner, 3)]),
    "unskew factor sign": (lattice, "unskew_factor", "(1.0 - 1.0 / math.sqrt", "(1.0 + 1.0 / math.sqrt",
                           [P(TL.test_unskew_inverts_skew, 3)]),
    "binary32 skew subtracts": (lattice, "scaled_skewed_fp32", "return p + t[:, None]", "return p - t[:, None]",
                                [TL.test_fp32_skew_matches_fp64_closely]),
    "level scale times sqrt(n+1)": (lattice, "simplex_level_scales_fp64", "/ math.sqrt(n + 1.0)",
                                    "* math.sqrt(n + 1.0)", [P(TE.test_simplex_reproduces_affine_fields, 2)]),
    "equal-memory exponent": (lattice, "equal_memory_factor", "((n - 1.0) / (2.0 * n))", "((n - 1.0) / n)",
                              [TL.test_equal_memory_factor_keeps_touched_volume]),
    "level resolution off by one": (lattice, "level_resolutions", "growth ** l", "growth ** (l + 1)",
                                    [TL.test_level_resolutions]),
    # Sec. 4.2 subdivision and Sec. 4.3 weights
    "fractions sorted ascending": (lattice, "subdivide", "np.argsort(-f,", "np.argsort(f,",
                                   [P(TL.test_subdivision_matches_brute_force, 3)]),
    "vertex steps along unpermuted axis": (lattice, "simplex_vertices", "k + 1, order[:, k]] += 1",
                                           "k + 1, k] += 1", [P(TL.test_subdivision_matches_brute_force, 3),
                                                             P(TE.test_simplex_reproduces_affine_fields, 3),
                                                             P(TL.test_memory_usage_by_subdivision, 2, 8)]),
    "first weight from last fraction": (lattice, "barycentric_weights", "w[:, 0] = 1.0 - s[:, 0]",
                                        "w[:, 0] = 1.0 - s[:, n - 1]", [P(TL.test_weights_reconstruct_point, 3)]),
    "weight difference sign": (lattice, "barycentric_weights", "s[:, k - 1] - s[:, k]", "s[:, k] - s[:, k - 1]",
                               [P(TL.test_weights_reconstruct_point, 3)]),
    # geometry used by the pins (Remark 2, Theorem 1's proof, Sec. 5.1-5.2, Kuhn hat functions)
    "Kuhn vertex steps along the unpermuted axis": (geometry, "kuhn_simplex", "V[i + 1, axis] = 1", "V[i + 1, i] = 1",
                                                    [P(TL.test_subdivision_matches_brute_force, 3)]),
    "barycentric solve without the partition of unity": (geometry, "barycentric_solve", "np.concatenate([[1.0],",
                                                         "np.concatenate([[0.0],",
                                                         [P(TL.test_subdivision_matches_brute_force, 3)]),
    "cell volume without the scale adjustment": (geometry, "parallelepiped_volume", "S = math.sqrt(n + 1.0)",
                                                 "S = 1.0", [TL.test_theoretical_memory_usage_figure]),
    "hat function adds the one-sided extents": (geometry, "vertex_hat_weight", "1.0 - (hi - lo)", "1.0 - (hi + lo)",
                                                [P(TL.test_weights_equal_hat_functions, 3)]),
    "touched count at the unadjusted scale": (geometry, "touched_vertex_count", "s = N / math.sqrt(n + 1.0)",
                                              "s = N / math.sqrt(n)", [TL.test_memory_usage_figure_exact]),
    # Sec. 5 (a) hash and the direct coarse indexing
    "hash axes added": (lattice, "hash_slot", "h ^= (vi", "h += (vi", [TL.test_hash_special_cases]),
    "hash multiplier of the next axis": (lattice, "hash_slot", "HASH_PRIMES[i]", "HASH_PRIMES[(i + 1) % n]",
                                         [TL.test_hash_special_cases]),
    "box one coordinate short": (lattice, "dense_box_width", "))) + 2", "))) + 1",
                                 [P(TE.test_dense_box_holds_every_vertex, "simplex", 2)]),
    "dense stride off by one": (lattice, "dense_slot", "stride *= width", "stride *= width - 1",
                                [P(TE.test_dense_slots_are_a_bijection_of_the_box, 3)]),
    "dense levels strictly smaller": (lattice, "level_box_widths", "B ** n <= (1", "B ** n < (1",
                                      [TE.test_dense_levels_are_exactly_those_that_fit]),
    # Sec. 5 (b)-(e) encodings
    "weights reversed in the interpolation": (encoding, "simplex_encode", '"pk,pkf->pf", w, H)',
                                              '"pk,pkf->pf", w[:, ::-1], H)',
                                              [P(TE.test_simplex_reproduces_affine_fields, 3)]),
    "lookup in level 0's table": (encoding, "simplex_encode", "np.asarray(tables[l], dtype=np.float64)[slots]",
                                  "np.asarray(tables[0], dtype=np.float64)[slots]",
                                  [P(TE.test_simplex_reproduces_affine_fields, 3)]),
    "level scale of the next level": (encoding, "simplex_encode", "simplex_level_vertices(x32, scales[l],",
                                      "simplex_level_vertices(x32, scales[min(l + 1, L - 1)],",
                                      [P(TE.test_simplex_reproduces_affine_fields, 3),
                                       P(TE.test_backward_is_adjoint_of_forward, "simplex", 3)]),
    "backward scatters reversed weights": (encoding, "simplex_encode_bwd", "w[:, :, None] * dout",
                                           "w[:, ::-1, None] * dout",
                                           [P(TE.test_backward_is_adjoint_of_forward, "simplex", 3)]),
    "backward reads level 0's gradient": (encoding, "simplex_encode_bwd", "dout[:, None, l * F:(l + 1) * F]",
                                          "dout[:, None, 0:F]",
                                          [P(TE.test_backward_is_adjoint_of_forward, "simplex", 3)]),
    "grid corner weight transposed": (encoding, "grid_level_corner_weights", "np.stack([lo, hi], axis=2)",
                                      "np.stack([lo, hi], axis=1)", [P(TE.test_grid_weights_are_products, 3)]),
    "grid lerp swapped": (encoding, "grid_encode", "v0 * (1.0 - t) + v1 * t", "v0 * t + v1 * (1.0 - t)",
                          [P(TE.test_grid_reproduces_multilinear_fields, 3)]),
    "grid lookup in level 0's table": (encoding, "grid_encode", "np.asarray(tables[l], dtype=np.float64)",
                                       "np.asarray(tables[0], dtype=np.float64)",
                                       [P(TE.test_grid_reproduces_multilinear_fields, 3)]),
    "grid cell at level 0's resolution": (encoding, "grid_encode", "grid_level_cell(x32, res[l])",
                                          "grid_level_cell(x32, res[0])",
                                          [P(TE.test_grid_reproduces_multilinear_fields, 3),
                                           P(TE.test_backward_is_adjoint_of_forward, "grid", 3)]),
    # the FP64 forward paths (scale and skew in FP64)
    "FP64 path without the skew": (encoding, "simplex_encode_fp64", "q = lattice.skew(x * scales[l])",
                                   "q = x * scales[l]",
                                   [P(TE.test_fp64_paths_reproduce_affine_and_multilinear_fields, 2),
                                    P(TE.test_fp64_paths_agree_with_binary32_conditioned_paths, "simplex", 2)]),
    "FP64 path at the next level's scale": (encoding, "simplex_encode_fp64", "x * scales[l]",
                                            "x * scales[min(l + 1, L - 1)]",
                                            [P(TE.test_fp64_paths_reproduce_affine_and_multilinear_fields, 3),
                                             P(TE.test_fp64_paths_agree_with_binary32_conditioned_paths, "simplex", 3)]),
    "FP64 grid weights of the floor's complement": (encoding, "grid_encode_fp64", "f = p - c", "f = 1.0 - (p - c)",
                                                    [P(TE.test_fp64_paths_reproduce_affine_and_multilinear_fields, 2),
                                                     P(TE.test_fp64_central_differences_equal_the_input_gradient,
                                                       "grid", 2)]),
    "grid backward reversed corners": (encoding, "grid_encode_bwd", "w[:, :, None] * dout",
                                       "w[:, ::-1, None] * dout",
                                       [P(TE.test_backward_is_adjoint_of_forward, "grid", 3)]),
    # input gradient (chain rule through Sec. 4.3, Eq. 2 and the level scale)
    "dx drops the skew term": (encoding, "simplex_encode_dx", "s * (g + Fn * g.sum(axis=1, keepdims=True))",
                               "s * g", [P(TE.test_simplex_dx_of_affine_field, 3)]),
    "dx vertex difference sign": (encoding, "simplex_encode_dx", "diff = H[:, k + 1] - H[:, k]",
                                  "diff = H[:, k] - H[:, k + 1]", [P(TE.test_simplex_dx_of_affine_field, 3)]),
    "dx difference from the base vertex": (encoding, "simplex_encode_dx", "diff = H[:, k + 1] - H[:, k]",
                                           "diff = H[:, k + 1] - H[:, 0]",
                                           [P(TE.test_simplex_dx_of_affine_field, 3)]),
    "dx unpermuted axis": (encoding, "simplex_encode_dx", "g[rows, order[:, k]] =", "g[rows, k] =",
                           [P(TE.test_simplex_dx_of_affine_field, 3)]),
    "dx without the level scale": (encoding, "simplex_encode_dx", "s = float(scales[l])", "s = 1.0",
                                   [P(TE.test_simplex_dx_of_affine_field, 3)]),
    "grid dx without the resolution": (encoding, "grid_encode_dx", 'dx[:, j] += float(res[l]) * np.einsum',
                                       "dx[:, j] += np.einsum", [P(TE.test_grid_dx_of_multilinear_field, 3)]),
    "grid dx lower-corner sign": (encoding, "grid_level_corner_weight_derivatives", "(-1.0 + 0.0 * f",
                                  "(1.0 + 0.0 * f", [P(TE.test_grid_dx_of_multilinear_field, 3)]),
    # network, loss, optimiser
    "relu replaced by abs": (mlp, "mlp_forward", "np.maximum(z, 0.0)", "np.abs(z)",
                             [TE.test_mlp_matches_independent_autograd, TE.test_mlp_hand_example]),
    "relu derivative dropped": (mlp, "mlp_backward", "delta * (acts[i] > 0.0)", "delta * 1.0",
                                [TE.test_mlp_finite_differences, TE.test_mlp_matches_independent_autograd]),
    "relu mask includes zeros": (mlp, "mlp_backward", "(acts[i] > 0.0)", "(acts[i] >= 0.0)",
                                 [TE.test_mlp_finite_differences]),
    "loss gradient over rows only": (mlp, "l2_loss", "2.0 * r / r.size", "2.0 * r / len(r)",
                                     [TE.test_l2_loss_closed_form]),
    "loss residual sign flipped in the square": (mlp, "l2_loss", "float(np.mean(r * r))", "float(np.mean(r * np.abs(r)))",
                                                  [TE.test_l2_loss_closed_form]),
    "loss as a sum": (mlp, "l2_loss", "float(np.mean(r * r))", "float(np.sum(r * r))", [TE.test_l2_loss_closed_form]),
    "adam second-moment correction with beta1": (adam, "adam_step", "(1.0 - beta2 ** t)", "(1.0 - beta1 ** t)",
                                                 [TE.test_adam_matches_library_and_skips_zero_grads]),
    "adam first-moment correction with beta2": (adam, "adam_step", "m_new / (1.0 - beta1 ** t)",
                                                "m_new / (1.0 - beta2 ** t)",
                                                [TE.test_adam_matches_library_and_skips_zero_grads]),
    "adam second moment of the raw gradient": (adam, "adam_step", "(1.0 - beta2) * g * g", "(1.0 - beta2) * np.abs(g)",
                                               [TE.test_adam_matches_library_and_skips_zero_grads]),
    "adam first moment without the decay": (adam, "adam_step", "m_new = beta1 * m +", "m_new = m +",
                                            [TE.test_adam_matches_library_and_skips_zero_grads]),
    "adam epsilon inside the root": (adam, "adam_step", "np.sqrt(v_hat) + eps", "np.sqrt(v_hat + eps)",
                                     [TE.test_adam_matches_library_and_skips_zero_grads]),
    "adam skips negative gradients": (adam, "adam_step", "(g != 0.0)", "(g > 0.0)",
                                      [TE.test_adam_matches_library_and_skips_zero_grads]),
    # volumetric rendering (Sec. 6.2, Eq. 5)
    "weights without transmittance": (render, "composite", "w[:, i] = T * alpha", "w[:, i] = alpha",
                                      [TR.test_composite_equals_eq5_for_homogeneous_media]),
    "opacity as the transmittance factor": (render, "composite", "alpha = -np.expm1(-sigma[:, i] * delta)",
                                            "alpha = np.exp(-sigma[:, i] * delta)",
                                            [TR.test_composite_equals_eq5_for_homogeneous_media]),
    "opacity without delta": (render, "composite", "alpha = -np.expm1(-sigma[:, i] * delta)",
                              "alpha = -np.expm1(-sigma[:, i])",
                              [TR.test_composite_equals_eq5_for_homogeneous_media]),
    "transmittance without delta": (render, "composite", "T = T * np.exp(-sigma[:, i] * delta)",
                                    "T = T * np.exp(-sigma[:, i])",
                                    [TR.test_composite_equals_eq5_for_homogeneous_media]),
    "samples at left endpoints": (render, "ray_samples_fp32", "+ np.float32(0.5))", "+ np.float32(0.0))",
                                  [TR.test_samples_lie_on_their_rays_in_order]),
    "harmonic axes swapped": (render, "sh_basis", "c1 * y, c1 * z, c1 * x", "c1 * x, c1 * z, c1 * y",
                              [TR.test_sh_equals_scipy_real_basis]),
    "harmonic l=2 m=0 constant sign": (render, "sh_basis", "(3.0 * z * z - 1.0)", "(3.0 * z * z + 1.0)",
                                       [TR.test_sh_equals_scipy_real_basis, TR.test_sh_orthonormal_on_the_sphere]),
    "harmonic l=2 xy term on yz": (render, "sh_basis", "out[:, 4] = c2 * x * y", "out[:, 4] = c2 * y * z",
                                   [TR.test_sh_equals_scipy_real_basis, TR.test_sh_orthonormal_on_the_sphere]),
    "harmonic l=3 m=-1 constant sign": (render, "sh_basis", "out[:, 11] = c3 * y * (5.0 * z * z - 1.0)",
                                        "out[:, 11] = c3 * y * (5.0 * z * z + 1.0)",
                                        [TR.test_sh_equals_scipy_real_basis, TR.test_sh_orthonormal_on_the_sphere]),
    "harmonic l=3 xyz normalisation": (render, "sh_basis", "out[:, 10] = b3 * x * y * z",
                                       "out[:, 10] = c3 * x * y * z",
                                       [TR.test_sh_equals_scipy_real_basis, TR.test_sh_orthonormal_on_the_sphere]),
    "compositing gradient with T_k": (render, "composite_bwd", "Tk[:, k + 1, None] * rgb[:, k]",
                                      "Tk[:, k, None] * rgb[:, k]",
                                      [TR.test_composite_bwd_matches_central_differences,
                                       TR.test_composite_bwd_homogeneous_closed_form]),
    "compositing gradient suffix sign": (render, "composite_bwd", "* rgb[:, k] - suffix)", "* rgb[:, k] + suffix)",
                                         [TR.test_composite_bwd_matches_central_differences]),
    "render loss drops the density chain factor": (render, "render_l2_grads", 'DENSITY_LOGIT_MAX, it["sigma"], 0.0)',
                                                   "DENSITY_LOGIT_MAX, 1.0, 0.0)",
                                                   [TR.test_render_l2_grads_match_central_differences]),
    "render loss drops the sigmoid derivative": (render, "render_l2_grads", "rgb * (1.0 - rgb)", "rgb",
                                                 [TR.test_render_l2_grads_match_central_differences]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_planted_mistake_is_caught(case, monkeypatch):
    module, name, old, new, pins = CASES[case]
    monkeypatch.setattr(module, name, _mutant(module, name, old, new))
    caught = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught.append(pin)
    assert caught, f"no pin caught the planted mistake {case!r}"


def test_unchanged_oracle_passes_the_same_pins():
    """The pins the cases rely on pass on the oracle as it stands (so a caught case is the plant's doing)."""
    seen = set()
    for _, _, _, _, pins in CASES.values():
        for pin in pins:
            key = (pin.func.__name__, pin.args) if isinstance(pin, functools.partial) else (pin.__name__, ())
            if key not in seen:
                seen.add(key)
                pin()
