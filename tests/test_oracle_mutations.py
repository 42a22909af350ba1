"""Planted mistakes in the oracle must fail its pins.

The pins in ``tests/test_oracle_*.py`` are meant to be chosen so that a
plausible mistake anywhere in the oracle (a dropped term or factor, a flipped
sign, a swapped index or operand, a wrong constant) fails at least one of them.
This file checks that, case by case: each case plants one such mistake in the
oracle and runs the pin that should catch it, which must then fail.

Mistakes in the C part are planted in a copy of ``oracle/hcgs_oracle.c``,
built with gcc into a temporary library that the oracle loads for the
duration of the case; mistakes in the Python part by re-executing one oracle
function's source with one expression changed.  The oracle is restored after
every case.  CPU only: nothing here touches the CUDA path or a GPU.
"""
import inspect
import subprocess
import textwrap

import pytest

import oracle
import test_oracle_asm as A
import test_oracle_densify as D
import test_oracle_grad as GR
import test_oracle_objective as OB
import test_oracle_raster as R
import test_oracle_rho_dense as RD


def _plant_c(monkeypatch, tmp_path, old, new):
    src = open(oracle._SRC).read()
    assert old in src, "mutation site not found: " + old
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(src.replace(old, new, 1))  # the first occurrence in the file
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    monkeypatch.setattr(oracle, "build", lambda: str(so))
    monkeypatch.setattr(oracle, "_SO", str(so))
    monkeypatch.setattr(oracle, "_lib", None)


def _plant_py(monkeypatch, name, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(oracle, name)))
    assert old in src, "mutation site not found: " + old
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new, 1), "<mutant of oracle.%s>" % name, "exec"), ns)
    monkeypatch.setattr(oracle, name, ns[name])


# (what is wrong, original expression, planted expression, the pin that must fail)
C_CASES = [
    ("depth key compared in FP64 instead of rounded to FP32",
     "const float di = (float)g_sort_depth[i], dj = (float)g_sort_depth[j];",
     "const double di = g_sort_depth[i], dj = g_sort_depth[j];", R.test_depth_key_is_rounded_once_to_fp32),
    ("depth key ignored (index order only)", "if (di < dj) return -1;\n    if (di > dj) return 1;",
     "", R.test_depth_key_is_rounded_once_to_fp32),
    ("transmittance update 1 + alpha", "T *= (1.0 - a);", "T *= (1.0 + a);", R.test_weights_sum_to_one_minus_T),
    ("transmittance update in the golden pixel", "T *= (1.0 - a);", "T *= (1.0 - 0.5 * a);",
     R.test_three_gaussians_golden_fixture),
    ("alpha_min doubled", "if (a < amin) continue;", "if (a < 2.0 * amin) continue;",
     R.test_reduces_to_textbook_alpha_blending),
    ("stop threshold ten times T_eps", "if (T < teps) break;", "if (T < 10.0 * teps) break;",
     R.test_thresholds_alpha_min_and_stop_after_add),
    ("exponent without the 1/2", "double power = 0.5 * (", "double power = 1.0 * (", R.test_single_gaussian_closed_form),
    ("exponent cross term sign", "+ 2.0 * conic[1] * dx * dy +", "- 2.0 * conic[1] * dx * dy +",
     R.test_rotated_gaussian_closed_form),
    ("conic off-diagonal sign", "P->conic[1] = -P->cov[1] / P->det;", "P->conic[1] = P->cov[1] / P->det;",
     R.test_rotated_gaussian_closed_form),
    ("Jacobian x-z entry sign", "P->J[2] = -fx * P->tcx / (tz * tz);", "P->J[2] = fx * P->tcx / (tz * tz);",
     R.test_projection_matches_numerical_jacobian),
    ("Sigma = R^T S^2 R (transposed rotation)", "P->R[3 * i + k] * P->s[k] * P->s[k] * P->R[3 * j + k]",
     "P->R[3 * k + i] * P->s[k] * P->s[k] * P->R[3 * k + j]", R.test_projection_matches_numerical_jacobian),
    ("rotation matrix entry sign", "R[1] = 2 * (x * y - w * z);", "R[1] = 2 * (x * y + w * z);",
     R.test_projection_matches_numerical_jacobian),
    ("quaternion not normalised", "P->qn[i] = quat[i] / P->qnorm;", "P->qn[i] = quat[i];",
     R.test_projection_matches_numerical_jacobian),
    ("opacity sigmoid sign", "P->opac = 1.0 / (1.0 + exp(-logit));", "P->opac = 1.0 / (1.0 + exp(logit));",
     R.test_single_gaussian_closed_form),
    ("principal point swapped", "P->mu[0] = fx * P->t[0] / tz + cx;", "P->mu[0] = fx * P->t[0] / tz + cy;",
     R.test_projection_matches_numerical_jacobian),
    ("dilation dropped", "P->cov[0] = c2[0] + opt[O_DIL];", "P->cov[0] = c2[0];",
     R.test_dilation_adds_to_the_2d_covariance),
    ("Jacobian clamp not applied", "if (rx > limx) { P->tcx = limx * tz; P->clx = 1; }",
     "if (rx > limx) { P->tcx = P->t[0]; P->clx = 1; }", R.test_jacobian_clamp_closed_form),
    ("adjoint: suffix term S / (1 - alpha) dropped", "double dUr = wr * Tk - S[2 * c] / (1.0 - a);",
     "double dUr = wr * Tk;", GR.test_fd_exact_preset),
    ("adjoint: factor 1/2 of dL/dA", "g_conic[3 * n] += 0.5 * dx * dx * dLdpower;",
     "g_conic[3 * n] += dx * dx * dLdpower;", GR.test_fd_exact_preset),
    ("adjoint: mean gradient cross term sign", "double gmx = -dLdpower * (K3[0] * dx + K3[1] * dy);",
     "double gmx = -dLdpower * (K3[0] * dx - K3[1] * dy);", GR.test_fd_exact_preset),
    ("adjoint: opacity factor", "double dLdo = dLda * G;", "double dLdo = dLda * G * G;", GR.test_fd_exact_preset),
    ("projection adjoint: d J / d t_z factor 2", "gt[2] += GJ[2] * 2.0 * fx * tx / (tz * tz * tz)",
     "gt[2] += GJ[2] * fx * tx / (tz * tz * tz)", GR.test_fd_exact_preset),
    ("straight-through rule without the softmax", "gpl[(size_t)L * n + a] += drho * exp((r[a] - mx) / tau) / Z;",
     "gpl[(size_t)L * n + a] += drho;", GR.test_ste_plane_logit_gradient),
    ("dense plane-weight gradient without the opacity", "vg[K] = opac[n] * G;", "vg[K] = G;",
     RD.test_dense_gradient_matches_finite_differences),
    ("support box too small", "double k = 2.0 * log(P.opac / opt[O_AMIN]);",
     "double k = 0.5 * log(P.opac / opt[O_AMIN]);", R.test_reduces_to_textbook_alpha_blending),
    ("support box axes swapped", "double rx = sqrt(k * P.cov[0]) + 1e-9, ry = sqrt(k * P.cov[2]) + 1e-9;",
     "double rx = sqrt(k * P.cov[2]) + 1e-9, ry = sqrt(k * P.cov[0]) + 1e-9;",
     R.test_reduces_to_textbook_alpha_blending),
    ("back-to-front order not reversed", "if (order == 1)", "if (order == 2)", R.test_three_gaussians_golden_fixture),
    ("dense plane-weight gradient: suffix sign", "double Sr = pre[2 * c] - vP[(size_t)k * 32 + 2 * c];",
     "double Sr = vP[(size_t)k * 32 + 2 * c] - pre[2 * c];", RD.test_dense_gradient_matches_finite_differences),
    ("quaternion adjoint without the normalisation's projection",
     "gq[4 * n + k] += (gqn[k] - P.qn[k] * dot) / P.qnorm;", "gq[4 * n + k] += gqn[k] / P.qnorm;",
     GR.test_fd_exact_preset),
    ("rotation adjoint entry sign", "gqn[0] = 2 * (-z * GR[1] + y * GR[2]", "gqn[0] = 2 * (z * GR[1] + y * GR[2]",
     GR.test_fd_exact_preset),
    ("log-scale adjoint without the exp chain factor", "gls[3 * n + j] += gs * P.s[j];",
     "gls[3 * n + j] += gs;", GR.test_fd_exact_preset),
    ("opacity logit adjoint without the sigmoid derivative", "gol[n] += g_opac[n] * o * (1.0 - o);",
     "gol[n] += g_opac[n] * o;", GR.test_fd_exact_preset),
    ("phase adjoint sign", "gph[C * n + c] += am * (-gr * sin(ph) + gi * cos(ph));",
     "gph[C * n + c] += am * (gr * sin(ph) + gi * cos(ph));", GR.test_fd_exact_preset),
    ("alpha_max clamp not applied", "if (a > amax) { a = amax; *clamped = 1; }",
     "if (0) { a = amax; *clamped = 1; }", R.test_alpha_max_clamp_and_its_flat_adjoint),
    ("clamped alpha not flat in the adjoint", "if (kcl[k]) continue; /* alpha = alpha_max: flat in o G */",
     "/* (planted: the clamp's flatness dropped) */", R.test_alpha_max_clamp_and_its_flat_adjoint),
    ("near-plane cull at z > 0", "if (!(P->t[2] >= opt[O_NEAR])) { P->valid = 0; return; }",
     "if (!(P->t[2] > 0)) { P->valid = 0; return; }", R.test_near_plane_cull),
    ("plane argmax ties keep the highest index", "if (logits[l] > logits[best]) best = l;",
     "if (logits[l] >= logits[best]) best = l;", GR.test_ste_plane_logit_gradient),
    ("adjoint suffix accumulated without T", "S[2 * c] += wr * a * Tk;", "S[2 * c] += wr * a;",
     GR.test_fd_exact_preset),
    ("support radius from 1.5 ln(o / alpha_min)", "double k = 2.0 * log(P.opac / opt[O_AMIN]);",
     "double k = 1.5 * log(P.opac / opt[O_AMIN]);", R.test_reduces_to_textbook_alpha_blending),
    ("equal depths visited by descending index", "return (i > j) - (i < j);", "return (i < j) - (i > j);",
     R.test_equal_depths_visit_in_index_order),
    ("adjoint's replay stops at ten times T_eps", "T *= (1.0 - a);\n                        if (T < teps) break;",
     "T *= (1.0 - a);\n                        if (T < 10.0 * teps) break;", R.test_stop_rule_in_the_adjoint),
]


@pytest.mark.parametrize("what,old,new,pin", C_CASES, ids=[c[0] for c in C_CASES])
def test_c_mistake_fails_its_pin(monkeypatch, tmp_path, what, old, new, pin):
    _plant_c(monkeypatch, tmp_path, old, new)
    with pytest.raises(AssertionError):
        pin()


PY_CASES = [
    ("FFT-order frequencies", "frequencies", "k < (n + 1) // 2", "k < n // 2", A.test_frequencies_fft_order),
    ("transfer function phase without 2", "transfer_function", "phase = 2.0 * np.pi * z",
     "phase = np.pi * z", A.test_transfer_function_values),
    ("evanescent bins not cut", "transfer_function", "return np.where(inside, np.exp(1j * phase), 0.0)",
     "return np.exp(1j * phase)", A.test_transfer_function_values),
    ("band limit without its factor 2", "transfer_function", "np.sqrt((2.0 * dux * z) ** 2 + 1.0)",
     "np.sqrt((dux * z) ** 2 + 1.0)", A.test_band_limit_is_the_unaliased_phase_region),
    ("propagation with the conjugate kernel", "propagate", "return np.fft.ifft2(Hz * np.fft.fft2(u))",
     "return np.fft.ifft2(np.conj(Hz) * np.fft.fft2(u))", lambda: A.test_gaussian_beam_fresnel(5e-3)),
    ("plane sum keeps only the last plane", "propagate_planes", "P[c] += propagate(", "P[c] = propagate(",
     A.test_plane_sum_matches_frequency_domain_sum),
    ("adjoint propagation without the conjugate", "propagate_planes_adjoint", "np.conj(Hz) * G", "Hz * G",
     A.test_adjoint_dot_product),
    ("inverse propagation towards +Z", "inverse_propagate", "-plane_z[l]", "plane_z[l]",
     A.test_inverse_propagation_and_loss),
    ("loss gradient factor", "focal_stack_loss", "gV = (4.0 / n)", "gV = (2.0 / n)", A.test_inverse_propagation_and_loss),
    ("zero embedding in the corner", "zero_pad", "out[..., H // 2:H // 2 + H, W // 2:W // 2 + W] = u",
     "out[..., :H, :W] = u", A.test_zero_padding_is_the_embedding_done_by_hand),
    ("SSIM window width", "ssim_window", "g = np.exp(-(x * x) / (2.0 * sigma * sigma))",
     "g = np.exp(-(x * x) / (3.0 * sigma * sigma))", OB.test_ssim_map_matches_brute_force_window_sums),
    ("SSIM gradient sign of the variance term", "ssim_grad", "d_xx = -S / d", "d_xx = S / d",
     OB.test_ssim_gradient_finite_differences),
    ("reconstruction loss without the mask term", "paper_loss_intensities",
     "w = 1.0 + np.asarray(M, dtype=np.float64)[:, None] + I_gt * I_gt", "w = 1.0 + I_gt * I_gt",
     OB.test_recon_loss_weights_reduce_to_scaled_plain_loss),
    ("Adan step without the (1 - a2) on v", "adan_step", "(m + beta2 * v)", "(m + v)",
     OB.test_adan_matches_the_algorithm_in_its_authors_notation),
    ("Adan n from g alone", "adan_step", "u = g + beta2 * dg", "u = g",
     OB.test_adan_matches_the_algorithm_in_its_authors_notation),
    ("cosine schedule without the 1/2", "cosine_lr", "(1.0 + math.cos(math.pi * t / total)) / 2.0",
     "(1.0 + math.cos(math.pi * t / total))", OB.test_cosine_schedule_endpoints),
    ("phase-only gradient takes the real part", "phase_only_loss", "return loss, np.imag(np.conj(Pphi) * gP)",
     "return loss, np.real(np.conj(Pphi) * gP)", OB.test_phase_only_loss_vanishes_at_a_phase_only_target),
    ("Philox round permutation", "philox4x32_10", "c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0",
     "c0, c1, c2, c3 = hi0 ^ c1 ^ k0, lo1, hi1 ^ c3 ^ k1, lo0", D.test_philox_known_answers),
    ("Box-Muller radius", "philox_normals", "r = np.sqrt(-2.0 * np.log(u))", "r = np.sqrt(-np.log(u))",
     D.test_philox_normals_are_standard_normal),
    ("uniforms without the half-cell offset", "uniform_of_words", "astype(np.float64) + 0.5)", "astype(np.float64) + 0.0)",
     D.test_uniform_map_is_the_open_interval_symmetric_about_one_half),
    ("uniforms offset by a whole cell", "uniform_of_words", "astype(np.float64) + 0.5)", "astype(np.float64) + 1.0)",
     D.test_uniform_map_is_the_open_interval_symmetric_about_one_half),
    ("densification: small Gaussians split", "densify_actions",
     'act[dens & (smax <= f(o["split_scale"]))] = CLONE', 'act[dens & (smax <= f(o["split_scale"]))] = SPLIT',
     D.test_actions_follow_the_thresholds),
    ("split children grow", "densify", "out[k].append(p[k][n] - shrink)", "out[k].append(p[k][n] + shrink)",
     D.test_densify_counts_order_and_copies),
    ("split children drawn with R^T", "densify", "p[k][n] + R @ (s * z[n, child, :3])",
     "p[k][n] + R.T @ (s * z[n, child, :3])", D.test_split_children_are_draws_from_the_parent),
    ("densification statistic in pixels along x", "densify_accumulate", "g[:, 0] * (W / 2.0)", "g[:, 0] * W",
     D.test_accumulate_uses_ndc_gradient_norm_of_visible_gaussians),
    ("Adam without bias correction", "adam_step", "mh = m / (1 - beta1 ** step)", "mh = m",
     GR.test_adam_first_step_closed_form),
    ("network activation not a ReLU", "mlp_forward", "h = np.maximum(z, 0.0)", "h = np.abs(z)",
     GR.test_mlp_reverse_mode),
    ("network adjoint without the ReLU mask", "mlp_backward", "g = g * (z > 0)", "g = g",
     GR.test_mlp_reverse_mode),
    ("bfloat16 rounding without ties to even", "round_bf16", "u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16",
     "u = (u + 0x8000) >> 16 << 16", GR.test_bf16_rounding_matches_torch),
    ("Adam second moment of g, not g^2", "adam_step", "v = beta2 * v + (1 - beta2) * g * g",
     "v = beta2 * v + (1 - beta2) * g", GR.test_adam_first_step_closed_form),
    ("paper loss gradient through |V|^2 halved", "paper_loss", "gV = 2.0 * gI * V", "gV = gI * V",
     OB.test_paper_loss_gradient_finite_differences),
    ("phase-only objective compares the real part twice", "phase_only_loss",
     "X = np.stack([Uphi.real, Uphi.imag])", "X = np.stack([Uphi.real, Uphi.real])",
     OB.test_phase_only_loss_without_ssim_is_the_field_mse),
    ("inverse-propagation adjoint without the conjugate", "inverse_propagate_adjoint",
     "r = np.fft.ifft2(np.conj(Hm) * np.fft.fft2(g))", "r = np.fft.ifft2(Hm * np.fft.fft2(g))",
     OB.test_paper_loss_gradient_finite_differences),
    ("clone copy without the phase-noise scale", "densify", 'o["phase_noise"] * z[n, 0, 3:]', "z[n, 0, 3:]",
     D.test_densify_counts_order_and_copies),
    ("straight-through weights without the temperature", "ste_softmax", "/ tau", "/ 1.0",
     RD.test_ste_weights_are_the_tempered_softmax),
    ("split log-scale shift by ln 2", "densify", 'shrink = np.log(o["split_shrink"])', "shrink = np.log(2.0)",
     D.test_densify_counts_order_and_copies),
    ("crop window off by one column", "crop", "return u[..., H // 2:H // 2 + H, W // 2:W // 2 + W]",
     "return u[..., H // 2:H // 2 + H, W // 2 + 1:W // 2 + 1 + W]", A.test_zero_padding_is_the_embedding_done_by_hand),
    ("band limit along y from the x spacing", "transfer_function",
     "lim_y = 1.0 / (wavelength * np.sqrt((2.0 * duy * z) ** 2 + 1.0))",
     "lim_y = 1.0 / (wavelength * np.sqrt((2.0 * dux * z) ** 2 + 1.0))", A.test_band_limit_applies_per_axis),
    ("SSIM gradient normalised over planes only", "paper_loss_intensities",
     "g[l, c] -= lam / (L * C) * ssim_grad", "g[l, c] -= lam / L * ssim_grad",
     OB.test_paper_loss_is_a_mean_over_planes_and_channels),
    ("SSIM loss normalised over planes only", "paper_loss_intensities",
     "loss += lam * (1.0 - s_sum / (L * C))", "loss += lam * (1.0 - s_sum / L)",
     OB.test_paper_loss_is_a_mean_over_planes_and_channels),
]


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # a mutant may take the sqrt of a negative number
@pytest.mark.parametrize("what,name,old,new,pin", PY_CASES, ids=[c[0] for c in PY_CASES])
def test_python_mistake_fails_its_pin(monkeypatch, what, name, old, new, pin):
    _plant_py(monkeypatch, name, old, new)
    with pytest.raises(AssertionError):
        pin()


def test_unmutated_oracle_passes_the_same_pins():
    # the pins above fail because of the planted mistake, not on their own
    for pin in {c[-1] for c in C_CASES + PY_CASES}:
        pin()
