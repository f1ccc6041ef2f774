"""The oracle's pins must catch plausible mistakes: each case plants one mistake in a
temporary copy of the oracle source (CPU only), rebuilds it, and checks that at least one
pin of ``test_oracle_pins`` fails against the mutant."""
import importlib
import os
import subprocess
import tempfile

import pytest

import tests.test_oracle_pins as pins

MUTANTS = {
    # attached segment weight without the triangle-area ratio
    "drop_area_ratio": ("T g = fabs(dot(nprev, din)) * fabs(dot(n, din)) * area / r2;",
                        "T g = fabs(dot(nprev, din)) * fabs(dot(n, din)) / r2;",
                        ["test_attached_gradient_unbiased_for_derivative_of_expected_image"]),
    # sensor importance with cos^2 instead of cos^3 of the camera angle
    "importance_cos2": ("T geo = cosc * T(K) / (dist2 * cc * cc * cc);",
                        "T geo = cosc * T(K) / (dist2 * cc * cc);",
                        ["test_primal_closed_form_area_light_over_plane"]),
    # emitted flux without the pi of the cosine-weighted direction pdf
    "emitter_no_pi": ("beta[c] = Le[c] * T(A_L * PI);", "beta[c] = Le[c] * T(A_L);",
                      ["test_primal_closed_form_area_light_over_plane"]),
    # p-polarised Fresnel amplitude with a flipped sign inside
    "fresnel_rp": ("T rp = (ci - eta * ct) / (ci + eta * ct);", "T rp = (ci + eta * ct) / (ci + eta * ct);",
                   ["test_dielectric_fresnel_and_snell"]),
    # tent filter taps swapped (splat lands on the wrong side of the pixel centre)
    "tent_swap": ("T wx[2] = {T(1.0) - fx, fx}, wy[2] = {T(1.0) - fy, fy};",
                  "T wx[2] = {fx, T(1.0) - fx}, wy[2] = {fy, T(1.0) - fy};",
                  ["test_primal_reciprocity_with_path_tracer", "test_primal_closed_form_area_light_over_plane"]),
    # LRB-3 restatement: subtract the vertex's own contribution before its splat gradient
    "lrb3_order": ("for (int c = 0; c < 3; ++c) { wsplat[c] = Pw[3 * ci + c]; rem[c] -= Pw[3 * ci + c]; }",
                   "for (int c = 0; c < 3; ++c) { rem[c] -= Pw[3 * ci + c]; wsplat[c] = 0; }",
                   ["test_lrb3_restatement_equals_naive_ad_per_seed"]),
    # reservoir replacement probability w/Omega replaced by w/(Omega+w)
    "reservoir_prob": ("if (u[i] < w[i] / Om) { R = (int)i; wR = w[i]; }",
                       "if (u[i] < w[i] / (Om + w[i])) { R = (int)i; wR = w[i]; }",
                       ["test_reservoir_selection_pmf_and_unbiasedness"]),
    # Russian roulette without the 1/q weight of the surviving paths
    "rr_no_weight": ("if (rand4(seed, n, (uint32_t)d, 2).u[0] < rr_q) P.v.back().rr = 1.0 / rr_q;",
                     "if (rand4(seed, n, (uint32_t)d, 2).u[0] < rr_q) P.v.back().rr = 1.0;",
                     ["test_russian_roulette_unbiased_and_exact"]),
    # Gaussian filter without the cut at the radius (weights jump to zero there)
    "gauss_no_cut": ("const double inv_c = 1.0 / gauss_norm(), cut = std::exp(-4.5);",
                     "const double inv_c = 1.0 / gauss_norm(), cut = 0.0;",
                     ["test_gaussian_filter_definition_and_flux"]),
    # bidirectional weights: the light-tracer side's density ratio without the pi of its film density
    "bidir_ratio_pi": ("const double pfilm = c.geo * N * PI / ((double)sc.s->W * (double)sc.s->H);",
                       "const double pfilm = c.geo * N / ((double)sc.s->W * (double)sc.s->H);",
                       ["test_bidirectional_estimator_unbiased_and_exact"]),
    # bidirectional weights: the camera side's next-event density without the cosine at the emitter
    "bidir_nee_cos": ("const double pf0 = dot(v.ns, wn) * -dot(nL, wn) / (PI * dl * dl);",
                      "const double pf0 = dot(v.ns, wn) / (PI * dl * dl);",
                      ["test_bidirectional_estimator_unbiased_and_exact"]),
    # Philox key schedule with a wrong Weyl increment (still a good generator: only the
    # published known-answer vectors tell it apart)
    "philox_weyl": ("    k1 += 0xBB67AE85u;\n", "    k1 += 0xBB67AE87u;\n", ["test_philox_known_answer_vectors"]),
    # attached slide: intersection parameter with the wrong sign
    "slide_sign": ("T tt = dot(o - xprev, n) / dot(din, n);", "T tt = dot(xprev - o, n) / dot(din, n);",
                   ["test_attached_height_gradient_vs_frozen_central_differences"]),
    # ResLRB restatement: the winner's adjoint without the reservoir weight Omega/omega_R
    "reslrb_no_weight": ("for (int c = 0; c < 3; ++c) { rem[c] = Pw[3 * P.R + c] * P.res_w;",
                         "for (int c = 0; c < 3; ++c) { rem[c] = Pw[3 * P.R + c];",
                         ["test_reslrb_restatement_equals_ad_of_reservoir_estimator"]),
    # literal transport: the remainder contracted with the transposed inverse Jacobian
    "literal_inv_transpose": ("for (int k = 0; k < 4; ++k) aloc[c] += Arem[k] * inv[k][c];",
                              "for (int k = 0; k < 4; ++k) aloc[c] += Arem[k] * inv[c][k];",
                              ["test_literal_attached_variant_exact_on_first_chains_and_unbiased_with_noise"]),
    # Gauss-Jordan inverse without the final division by the pivots
    "inverse_no_pivot": ("for (int j = 0; j < 4; ++j) inv[i][j] = m[i][j + 4] / m[i][i];",
                         "for (int j = 0; j < 4; ++j) inv[i][j] = m[i][j + 4];",
                         ["test_literal_attached_variant_exact_on_first_chains_and_unbiased_with_noise"]),
    # Jacobian noise on one film axis only (the product stays singular)
    "literal_noise_one_axis": ("          Jj[3][1] = eps;\n", "          Jj[3][1] = 0.0;\n",
                               ["test_literal_attached_variant_exact_on_first_chains_and_unbiased_with_noise"]),
    # network backward: hidden-layer adjoint through the transposed weights
    "mlp_w2_transpose": ("a += dz2[j] * M.W2(i, j);", "a += dz2[j] * M.W2(j, i);",
                         ["test_mlp_oracle_gradient_vs_central_differences"]),
    # network backward: first ReLU's derivative dropped
    "mlp_relu_mask": ("const double dz1 = z1[i] > 0 ? dh1[i] : 0.0;", "const double dz1 = dh1[i];",
                      ["test_mlp_oracle_gradient_vs_central_differences"]),
    # Snell's law with the relative index inverted (entering and leaving swapped)
    "snell_eta_swap": ("T eta = entering ? T(1.0 / ior) : T(ior);", "T eta = entering ? T(ior) : T(1.0 / ior);",
                       ["test_dielectric_fresnel_and_snell"]),
    # refracted direction with the normal component's sign flipped
    "refract_sign": ("refr = din * eta + ns * (eta * ci - ct);", "refr = din * eta + ns * (eta * ci + ct);",
                     ["test_dielectric_fresnel_and_snell"]),
    # diffuse bounce that continues the path without the albedo in its throughput
    "bounce_no_albedo": ("      for (int c = 0; c < 3; ++c) beta[c] = beta[c] * rho[c];\n", "\n",
                         ["test_primal_reciprocity_with_path_tracer",
                          "test_detached_albedo_gradient_vs_central_differences"]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_detect_planted_mistake(oracle, name):
    old, new, tests = MUTANTS[name]
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found: {name}"
    tmpdir = tempfile.mkdtemp(prefix="lt_mut_")
    cpp = os.path.join(tmpdir, "mut.cpp")
    so = os.path.join(tmpdir, "libmut.so")
    open(cpp, "w").write(src.replace(old, new))
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-pthread",
                           "-Wno-dangling-pointer", "-o", so, cpp])
    mod = importlib.import_module("oracle.oracle")
    saved_lib, saved_path = mod._lib, mod.LIB
    failed = []
    try:
        mod._lib, mod.LIB = None, so
        for t in tests:
            fn = getattr(pins, t)
            kwargs = {}
            if t == "test_attached_height_gradient_vs_frozen_central_differences":
                kwargs["which"] = "slab"
            try:
                fn(mod, **kwargs)
            except (AssertionError, ValueError, FloatingPointError):
                failed.append(t)
    finally:
        mod._lib, mod.LIB = saved_lib, saved_path
    assert failed, f"no pin caught mutant {name}"
