"""Planted mistakes: the oracle's pins must catch the mistakes they claim to (CPU only).

Each case below takes a copy of the oracle's source, substitutes one plausible mistake (a
flipped sign, a dropped term or factor, a transposed index, another formula for a step of
Algorithm 1) and runs the named pins against that copy; every named pin must fail.  The C
oracle's copies are compiled into libraries of their own (the same gcc command as the
oracle's build) and put in place of the oracle's library for one test; the network
reference's copies are executed as a module of their own.  The oracle's files are never
modified, and an unmodified copy, built the same way, passes every pin used here.

A substitution site that no longer appears exactly once in the source fails the build of
the copies: the mistake list follows the source it plants into.
"""
import os
import subprocess
import sys

import pytest

import oracle
from oracle import orc as O
from tests import test_cnn_oracle as TC
from tests import test_oracle as T0
from tests import test_oracle_subpixel as T2
from tests import test_oracle_variants as T1

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# pins of the C oracle, by name (one parameter set each)
PINS = {
    "fft_bruteforce": lambda: T0.test_fft_matches_bruteforce_dft(oracle, 4),
    "fft_numpy": lambda: T0.test_fft_matches_numpy(oracle, 64),
    "fft_closed_forms": lambda: T0.test_fft_closed_forms(oracle),
    "parseval": lambda: T0.test_parseval_and_inverse(oracle),
    "adjoint_dot": lambda: T0.test_adjoint_dot_tests(oracle),
    "dense_operator": lambda: T0.test_forward_adjoint_against_dense_matrix(oracle),
    "illumination": lambda: T0.test_illumination_map_by_counting(oracle),
    "finite_differences": lambda: T0.test_gradient_finite_differences(oracle, "random"),
    "objective_bruteforce": lambda: T0.test_objective_and_gradient_against_bruteforce(oracle),
    "truth_stationary": lambda: T0.test_noise_free_truth_is_stationary(oracle),
    "cg_scalar_golden": lambda: T0.test_cg_hand_derived_scalar_case(oracle),
    "cg_bruteforce": lambda: T0.test_cg_against_bruteforce(oracle),
    "cg_termination_strict": lambda: T0.test_cg_termination_parameter_against_bruteforce(oracle, -5e3),
    "cg_termination_loose": lambda: T0.test_cg_termination_parameter_against_bruteforce(oracle, 3e4),
    "cg_invariants": lambda: T0.test_cg_invariants(oracle),
    "ls_bruteforce": lambda: T1.test_ls_objective_and_gradient_against_bruteforce(oracle),
    "ls_eps_zero": lambda: T1.test_ls_at_eps_zero_is_the_amplitude_misfit(oracle),
    "ls_finite_differences": lambda: T1.test_ls_gradient_finite_differences(oracle, "random"),
    "ls_scalar_golden": lambda: T1.test_ls_hand_derived_scalar_cg(oracle),
    "gd_scalar_golden": lambda: T1.test_gd_hand_derived_scalar(oracle),
    "gd_bruteforce": lambda: T1.test_gd_against_bruteforce(oracle, "ml"),
    "gd_decreases": lambda: T1.test_gd_small_step_decreases(oracle),
    "warm_scalar_golden": lambda: T1.test_warm_hand_derived_scalar_cg(oracle),
    "warm_bruteforce": lambda: T1.test_warm_cg_against_bruteforce(oracle),
    "shift_integer_roll": lambda: T2.test_integer_shift_is_circular_roll(3, -2),
    "shift_plane_wave": lambda: T2.test_plane_wave_shifts_by_its_phase(-5, 2),
    "shift_band_limited": lambda: T2.test_band_limited_function_is_evaluated_between_samples(),
    "shift_nyquist": lambda: T2.test_nyquist_rows_take_cos_pi_delta(),
    "shift_real_stays_real": lambda: T2.test_real_probe_stays_real(),
    "subpixel_adjoint_dot": lambda: T2.test_subpixel_adjoint_dot(),
    "subpixel_finite_differences": lambda: T2.test_subpixel_gradient_finite_difference(),
    "per_position_dense": lambda: T2.test_per_position_probes_against_the_dense_restatement(),
    "threaded_paths": lambda: T0.test_threaded_paths_against_bruteforce(oracle, 3),
    "swept_shapes": lambda: T0.test_operators_objective_gradient_swept_against_bruteforce(oracle, 11, 7, 4, 12, 35,
                                                                                           "ml"),
}

# (name, text of the oracle's C source, replacement, pins that must fail)
C_MISTAKES = [
    ("dft_kernel_sign", "double a = -2.0 * ORC_PI * (double)j / (double)n;",
     "double a = 2.0 * ORC_PI * (double)j / (double)n;", ["fft_bruteforce", "fft_closed_forms", "fft_numpy"]),
    ("dft_not_unitary", "double s = 1.0 / (double)P;", "double s = 1.0 / sqrt((double)P);",
     ["parseval", "fft_bruteforce"]),
    ("dft_rows_transformed_twice", "for (int c = 0; c < P; c++) fft1(x + c, P, P, sign, tw);",
     "for (int c = 0; c < P; c++) fft1(x + (long)c * P, P, 1, sign, tw);", ["fft_bruteforce", "fft_numpy"]),
    ("inverse_dft_without_conj", "if (sign > 0) w = conj(w);", "(void)sign;",
     ["fft_bruteforce", "parseval", "adjoint_dot"]),
    ("probe_transposed_in_Q", "e[(long)y * P + x] = p[(long)y * P + x] * psi",
     "e[(long)y * P + x] = p[(long)x * P + y] * psi", ["dense_operator", "adjoint_dot", "swept_shapes"]),
    ("QH_without_conj", "+= conj(p[(long)y * P + x]) * w[(long)y * P + x];", "+= p[(long)y * P + x] * w[(long)y * P + x];",
     ["adjoint_dot", "dense_operator", "finite_differences"]),
    ("QH_patch_rows_flipped", "acc[(long)(r + y) * W + (c + x)] +=", "acc[(long)(r + (P - 1 - y)) * W + (c + x)] +=",
     ["adjoint_dot", "illumination", "finite_differences"]),
    ("per_position_probe_ignored",
     "p += (long)k * ps;\n    for (int y = 0; y < P; y++)\n        for (int x = 0; x < P; x++)\n            e[",
     "for (int y = 0; y < P; y++)\n        for (int x = 0; x < P; x++)\n            e[",
     ["subpixel_adjoint_dot", "subpixel_finite_differences", "per_position_dense"]),
    ("threaded_scatter_drops_last_buffer", "for (int t = 0; t < T; t++) {\n        const cplx *b = bufs",
     "for (int t = 0; t + 1 < T; t++) {\n        const cplx *b = bufs", ["threaded_paths", "adjoint_dot"]),
    ("threaded_chunks_overlap", "long k0 = (long)K * t / T, k1 = (long)K * (t + 1) / T;",
     "long k0 = (long)K * t / T, k1 = (long)K * (t + 1) / T + (t + 1 < T);", ["threaded_paths"]),
    ("objective_partials_miss_the_last_pattern", "for (int k = 0; k < K; k++) s += fpart[k];\n    *F = s;",
     "for (int k = 0; k + 1 < K; k++) s += fpart[k];\n    *F = s;", ["threaded_paths", "cg_bruteforce"]),
    ("objective_without_intensity_term", "return a - d * log(a + eps);", "return -d * log(a + eps);",
     ["finite_differences", "objective_bruteforce", "truth_stationary"]),
    ("objective_without_eps", "return a - d * log(a + eps);", "return a - d * log(a + 0.0 * eps);",
     ["finite_differences", "objective_bruteforce"]),
    ("objective_drops_pixels_without_counts", "if (!(d > 0.0)) return a;\n    if (est == ORC_EST_LS) return a - 2.0",
     "if (!(d > 0.0)) return 0.0;\n    if (est == ORC_EST_LS) return a - 2.0",
     ["finite_differences", "objective_bruteforce", "ls_bruteforce"]),
    ("residual_sign", "return u - (d / (a + eps)) * u;", "return u + (d / (a + eps)) * u;",
     ["finite_differences", "objective_bruteforce", "truth_stationary"]),
    ("residual_without_eps", "return u - (d / (a + eps)) * u;", "return u - (d / (a + 1e-300)) * u;",
     ["finite_differences", "objective_bruteforce"]),
    ("gradient_factor_two", "return u - (d / (a + eps)) * u;", "return 2.0 * (u - (d / (a + eps)) * u);",
     ["finite_differences", "cg_scalar_golden"]),
    ("ls_objective_factor", "return a - 2.0 * sqrt(d) * sqrt(a + eps) + d;", "return a - sqrt(d) * sqrt(a + eps) + d;",
     ["ls_bruteforce", "ls_eps_zero", "ls_finite_differences"]),
    ("ls_residual_of_the_ml_estimator", "return u - (sqrt(d) / sqrt(a + eps)) * u;", "return u - (d / (a + eps)) * u;",
     ["ls_bruteforce", "ls_finite_differences", "ls_scalar_golden"]),
    ("fletcher_reeves_for_dai_yuan", "den += creal(eta[i]) * creal(dg) + cimag(eta[i]) * cimag(dg);",
     "den += creal(g_prev[i]) * creal(g_prev[i]) + cimag(g_prev[i]) * cimag(g_prev[i]);",
     ["cg_scalar_golden", "cg_bruteforce"]),
    ("polak_ribiere_numerator", "double num = re_dot(g, g, n);", "double num = re_dot(g, g, n) - re_dot(g, g_prev, n);",
     ["cg_scalar_golden", "cg_bruteforce"]),
    ("direction_sign", "eta[i] = -g[i] + alpha * eta[i];", "eta[i] = -g[i] - alpha * eta[i];",
     ["cg_scalar_golden", "cg_bruteforce"]),
    ("previous_gradient_not_kept", "memcpy(g_prev, g, sizeof(cplx) * n);", "(void)g_prev;",
     ["cg_scalar_golden", "cg_bruteforce", "cg_invariants"]),
    ("first_trial_at_gamma0", "double gam = opts->gamma0, Ft = 0.0;", "double gam = opts->gamma0 / opts->tau, Ft = 0.0;",
     ["cg_scalar_golden", "cg_bruteforce", "cg_invariants"]),
    ("termination_term_sign", "ok = (Ft <= Fm + gam * opts->t);", "ok = (Ft <= Fm - gam * opts->t);",
     ["cg_termination_strict", "cg_termination_loose"]),
    ("termination_term_dropped", "ok = (Ft <= Fm + gam * opts->t);", "ok = (Ft <= Fm);",
     ["cg_termination_strict", "cg_termination_loose"]),
    ("warm_start_at_previous_step", "gam = gam_prev / opts->tau;", "gam = gam_prev;",
     ["warm_scalar_golden", "warm_bruteforce"]),
    ("gradient_ascent", "psi[i] -= opts->gd_step * g[i];", "psi[i] += opts->gd_step * g[i];",
     ["gd_scalar_golden", "gd_bruteforce", "gd_decreases"]),
    ("shift_phase_sign", "fy[j] = cexp(-2.0 * ORC_PI * I * (double)kappa * dy / (double)P);",
     "fy[j] = cexp(2.0 * ORC_PI * I * (double)kappa * dy / (double)P);",
     ["shift_integer_roll", "shift_plane_wave", "shift_band_limited"]),
    ("shift_nyquist_complex", "fy[j] = cos(ORC_PI * dy);", "fy[j] = cexp(-ORC_PI * I * dy);",
     ["shift_nyquist", "shift_real_stays_real"]),
    ("shift_unsigned_frequency", "int kappa = j < P / 2 ? j : j - P;", "int kappa = j;",
     ["shift_plane_wave", "shift_band_limited", "shift_real_stays_real"]),
]

# (name, text of oracle/cnn.py, replacement, pins of tests/test_cnn_oracle.py that must fail)
CNN_MISTAKES = [
    ("convolution_for_correlation", 'z += np.einsum("oc,bcyx->boyx", W[:, :, dy, dx], patch)',
     'z += np.einsum("oc,bcyx->boyx", W[:, :, 2 - dy, 2 - dx], patch)',
     ["test_conv_matches_scipy_correlate", "test_gradients_finite_differences"]),
    ("input_gradient_kernel_flipped", 'np.einsum("oc,boyx->bcyx", W[:, :, dy, dx], dz)',
     'np.einsum("oc,boyx->bcyx", W[:, :, 2 - dy, 2 - dx], dz)', ["test_gradients_finite_differences"]),
    ("bias_gradient_of_one_sample", "db = dz.sum(axis=(0, 2, 3))", "db = dz[0].sum(axis=(1, 2))",
     ["test_gradients_finite_differences"]),
    ("gelu_derivative_term_dropped", "return _Phi(z) + z * _phi(z)", "return _Phi(z)",
     ["test_gelu_closed_form_and_derivative", "test_gradients_finite_differences"]),
    ("gelu_tanh_approximation", "return z * _Phi(z)",
     "return z * 0.5 * (1.0 + np.tanh(0.7978845608 * (z + 0.044715 * z ** 3)))",
     ["test_gelu_closed_form_and_derivative"]),
    ("amplitude_head_scale_dropped", "damp * 0.2 * s0 * (1 - s0)", "damp * s0 * (1 - s0)",
     ["test_gradients_finite_differences"]),
    ("phase_gradient_sign", "dph = 2.0 * np.real(np.conj(r) * 1j * o)", "dph = 2.0 * np.real(np.conj(r) * -1j * o)",
     ["test_gradients_finite_differences"]),
    ("loss_not_averaged_over_batch", "norm = B * w.sum()", "norm = w.sum()",
     ["test_zero_network_predicts_centre_of_ranges"]),
    ("amplitude_range", "amp = 0.8 + 0.2 * s0", "amp = 0.8 + 0.1 * s0",
     ["test_zero_network_predicts_centre_of_ranges"]),
    ("adam_without_bias_correction", 'mh = state["m"][j] / (1 - b1**t)', 'mh = state["m"][j]',
     ["test_adam_first_step_is_signed_learning_rate", "test_adam_constant_gradient_second_step"]),
    ("adam_second_moment_of_abs", "(1 - b2) * g * g", "(1 - b2) * np.abs(g)",
     ["test_adam_first_step_is_signed_learning_rate", "test_adam_constant_gradient_second_step"]),
    ("adam_eps_inside_root", "np.sqrt(vh) + eps", "np.sqrt(vh + eps)", ["test_adam_first_step_with_eps"]),
    ("features_not_centred",
     "np.roll(np.log1p(np.sqrt(np.maximum(d, 0.0))), (P // 2, P // 2), axis=(-2, -1))",
     "np.log1p(np.sqrt(np.maximum(d, 0.0)))", ["test_features_centre_zero_frequency"]),
    ("features_of_counts", "np.log1p(np.sqrt(np.maximum(d, 0.0)))", "np.log1p(np.maximum(d, 0.0))",
     ["test_features_centre_zero_frequency"]),
    ("stitch_weight", "den[r:r + P, c:c + P] += w", "den[r:r + P, c:c + P] += np.sqrt(w)",
     ["test_stitch_constant_patches"]),
    ("stitch_uncovered_zero", "out = np.ones((H, W), np.complex128)", "out = np.zeros((H, W), np.complex128)",
     ["test_stitch_constant_patches"]),
]


def _planted(src, old, new, name):
    n = src.count(old)
    assert n == 1, f"site of {name!r} found {n} times in the oracle's source"
    return src.replace(old, new)


@pytest.fixture(scope="module")
def c_libs(tmp_path_factory):
    """name -> library path: an unmodified copy and one copy per planted mistake, compiled
    in parallel with the oracle's own gcc command."""
    src = open(os.path.join(ROOT, "oracle", "orc.c")).read()
    out = tmp_path_factory.mktemp("planted")
    jobs = []
    for name, old, new, _ in [("unmodified", None, None, None)] + C_MISTAKES:
        text = src if old is None else _planted(src, old, new, name)
        c, so = out / f"{name}.c", out / f"{name}.so"
        c.write_text(text)
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", str(c), "-o", str(so), "-lm"]
        jobs.append((name, str(so), subprocess.Popen(cmd)))
    failed = [name for name, _, p in jobs if p.wait() != 0]
    assert not failed, f"copies that did not compile: {failed}"
    return {name: so for name, so, _ in jobs}


def _use_library(monkeypatch, path):
    monkeypatch.setattr(O, "build", lambda force=False: path)
    monkeypatch.setattr(O, "_lib", None)
    O._get()


def test_unmodified_copy_passes_every_pin(c_libs, monkeypatch):
    _use_library(monkeypatch, c_libs["unmodified"])
    for pin in sorted({p for m in C_MISTAKES for p in m[3]}):
        PINS[pin]()


@pytest.mark.parametrize("name,old,new,pins", C_MISTAKES, ids=[m[0] for m in C_MISTAKES])
def test_planted_mistake_is_caught(c_libs, monkeypatch, name, old, new, pins):
    _use_library(monkeypatch, c_libs[name])
    for pin in pins:
        with pytest.raises(AssertionError):
            PINS[pin]()


def _cnn_copy(src):
    mod = type(sys)("cnn_planted")
    exec(compile(src, "cnn_planted.py", "exec"), mod.__dict__)
    return mod


def test_unmodified_network_copy_passes_every_pin(monkeypatch):
    src = open(os.path.join(ROOT, "oracle", "cnn.py")).read()
    monkeypatch.setattr(TC, "cnn", _cnn_copy(src))
    for pin in sorted({p for m in CNN_MISTAKES for p in m[3]}):
        getattr(TC, pin)()


@pytest.mark.filterwarnings("ignore::RuntimeWarning")
@pytest.mark.parametrize("name,old,new,pins", CNN_MISTAKES, ids=[m[0] for m in CNN_MISTAKES])
def test_planted_network_mistake_is_caught(monkeypatch, name, old, new, pins):
    src = open(os.path.join(ROOT, "oracle", "cnn.py")).read()
    monkeypatch.setattr(TC, "cnn", _cnn_copy(_planted(src, old, new, name)))
    for pin in pins:
        with pytest.raises(AssertionError):
            getattr(TC, pin)()
