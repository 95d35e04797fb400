"""The oracle's pins have teeth: each plausible mistake planted in a copy of
the oracle source (a dropped term, a wrong sign, a wrong index, a swapped
operand) makes at least one pin fail.  Mistakes are planted on the CPU only,
in a temporary build of ``oracle/soma_oracle.c``; no GPU code is involved."""
import functools
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_philox as PH
from tests import test_oracle_pins as PIN
from tests import test_oracle_topology as TOPO
from tests import test_oracle_types as TYPES
from tests import test_oracle_learned_bf16 as BF16
from tests import test_oracle_golden as GOLD

SRC = os.path.join(os.path.dirname(oracle.__file__), "soma_oracle.c")

# (id, original text, planted text, pin that must fail)
MUTANTS = [
    ("field_sign", "(w_t[c_new] - w_t[c_old])", "(w_t[c_old] - w_t[c_new])",
     lambda L: PIN.check_two_particle_balance_brute_force(0, L)),
    ("field_type_swapped", "const double* w_t = or_is_B(s, chain, i) ? wB : wA;\n  if (s->n_types",
     "const double* w_t = or_is_B(s, chain, i) ? wA : wB;\n  if (s->n_types",
     lambda L: PIN.check_two_particle_balance_brute_force(0, L)),
    ("bond_half_strength", "dEb += s->K_b * (d_new - d_old);", "dEb += 0.5 * s->K_b * (d_new - d_old);",
     PIN.check_ideal_chain_relaxes_to_gaussian_statistics),
    ("metropolis_sign", "(lnu < -dE)", "(lnu < dE)",
     PIN.check_ideal_chain_relaxes_to_gaussian_statistics),
    ("one_sided_bonds", "  if (i + 1u < s->N) out[k++] = i + 1u;\n", "",
     PIN.check_ideal_chain_relaxes_to_gaussian_statistics),
    ("chi_sign", "      a = comp - 0.5 * chi0 * (phiA - phiB);", "      a = comp + 0.5 * chi0 * (phiA - phiB);",
     PIN.check_fields_closed_forms),
    ("kappa_dropped_minus_one", "kappa0 * (phiA + phiB - 1.0)", "kappa0 * (phiA + phiB)",
     PIN.check_fields_closed_forms),
    ("energy_pair_counted_twice", "0.25 * s->chiN * df * df", "0.5 * s->chiN * df * df",
     PIN.check_fields_are_the_energy_derivative),
    ("type_boundary", "  return i >= s->N_A;\n}", "  return i > s->N_A;\n}",
     PIN.check_histogram_matches_numpy_binning_with_edge_cases),
    ("truncate_not_floor", "long long f = (long long)floor(p[d]);", "long long f = (long long)(p[d]);",
     PIN.check_histogram_matches_numpy_binning_with_edge_cases),
    ("cell_axes_swapped", "return ((uint64_t)c[2] * s->grid[1] + (uint64_t)c[1]) * s->grid[0] + (uint64_t)c[0];",
     "return ((uint64_t)c[0] * s->grid[1] + (uint64_t)c[1]) * s->grid[2] + (uint64_t)c[2];",
     PIN.check_histogram_matches_numpy_binning_with_edge_cases),
    ("init_sigma_N", "s->Re / sqrt(3.0 * (double)(N - 1))", "s->Re / sqrt(3.0 * (double)N)",
     PIN.check_init_bond_and_end_to_end_statistics),
    ("init_cos_only", "return (j % 2u == 0u) ? rad * cos(th) : rad * sin(th);", "return rad * cos(th);",
     PIN.check_init_bond_and_end_to_end_statistics),
    ("philox_multipliers_swapped", "uint64_t p0 = M0 * (uint64_t)c0;", "uint64_t p0 = M1 * (uint64_t)c0;",
     lambda L: PH.check_philox_matches_curand_host_generator(1, L)),
    ("philox_key_bump_late", "if (round > 0) { k0 += W0; k1 += W1; }", "if (round > 1) { k0 += W0; k1 += W1; }",
     lambda L: PH.check_philox_matches_curand_host_generator(1, L)),
    ("sq_wrong_axis", "(double)m[3 * q + 1] * cy / s->grid[1]", "(double)m[3 * q + 1] * cy / s->grid[0]",
     PIN.check_structure_factor_matches_numpy_fft),
    ("bond_energy_observable", "      b2 += bb;\n      Eb += s->K_b * bb;",
     "      b2 += bb;\n      Eb += 2.0 * s->K_b * bb;",
     PIN.check_observables_hand_values),
    ("smc_reverse_density_dropped", "const double log_alpha = -dE - rev / (4.0 * A) + fwd / (4.0 * A);",
     "const double log_alpha = -dE;",
     lambda L: PIN.check_two_particle_balance_brute_force(0, L, move=1)),
    ("smc_field_gradient_sign", "F[d] -= 0.5 * (w_t[or_cell_shift(s, c, d, +1)] - w_t[or_cell_shift(s, c, d, -1)]);",
     "F[d] += 0.5 * (w_t[or_cell_shift(s, c, d, +1)] - w_t[or_cell_shift(s, c, d, -1)]);",
     PIN.check_smc_force_direction),
    ("smc_bond_force_sign", "F[d] -= 2.0 * s->K_b * (r[d] - rn[d]);", "F[d] += 2.0 * s->K_b * (r[d] - rn[d]);",
     PIN.check_smc_force_direction),
    ("learned_reverse_density_dropped",
     "const double log_alpha = -dE + or_log_q(s, o_rev, r_new, r_old) - or_log_q(s, o, r_old, r_new);",
     "const double log_alpha = -dE;",
     lambda L: PIN.check_two_particle_balance_brute_force(0, L, move=2)),
    ("esjd_gradient_bond_sign", "g_rp[d] += cl * (-2.0 * s->K_b * (rp[d] - rn[d]));",
     "g_rp[d] += cl * (2.0 * s->K_b * (rp[d] - rn[d]));",
     PIN.check_esjd_gradient_matches_finite_differences),
    ("esjd_gradient_logscale_term", "dls += cl * 3.0;", "dls += cl * 2.0;",
     PIN.check_esjd_gradient_matches_finite_differences),
    ("mlp_second_bias_dropped", "double a = W[L_B2 + j];", "double a = 0.0;",
     PIN.check_mlp_forward_closed_form),
    ("mlp_first_layer_transposed", "a += W[L_W1 + 12 * j + k] * x[k];",
     "a += W[L_W1 + 32 * k + j] * x[k];", PIN.check_mlp_forward_closed_form),
    ("feature_prev_bond_reversed", "feat[0] = r[0] - x[n]; feat[1] = r[1] - y[n]; feat[2] = r[2] - z[n];",
     "feat[0] = x[n] - r[0]; feat[1] = y[n] - r[1]; feat[2] = z[n] - r[2];",
     PIN.check_learned_features_hand_values),
    ("gradient_interpolation_reversed", "g[d] = (1.0 - t) * lo + t * hi;", "g[d] = t * lo + (1.0 - t) * hi;",
     PIN.check_learned_features_hand_values),
    ("molecule_choice_half",
     "const uint32_t i = (uint32_t)(((uint64_t)(w[3] & 0xFFu) * or_length(s, chain)) >> 8);",
     "const uint32_t i = (uint32_t)(((uint64_t)(w[3] & 0xFFu) * or_length(s, chain)) >> 9);",
     PIN.check_molecule_iteration_attempts),
    ("k1_coupling_sign", "      a = comp + chi0 * phiB;", "      a = comp - chi0 * phiB;",
     functools.partial(PIN.check_fields_are_the_energy_derivative, hamiltonian=1)),
    ("external_types_swapped", "if (s->ext) { a += s->ext[c]; b += s->ext[cells + c]; }",
     "if (s->ext) { a += s->ext[cells + c]; b += s->ext[c]; }",
     functools.partial(PIN.check_fields_are_the_energy_derivative, external=True)),
    ("forbidden_cells_ignored", "if (s->forbidden && s->forbidden[c]) { a = INFINITY; b = INFINITY; }",
     "", PIN.check_walls_and_external_field_balance),
    ("architecture_bits_reversed", "if (s->seq && s->arch) return (int)((s->seq[s->arch[chain]] >> i) & 1u);",
     "if (s->seq && s->arch) return (int)((s->seq[s->arch[chain]] >> (s->N - 1 - i)) & 1u);",
     PIN.check_architecture_mixture),
    ("sort_key_axis", "for (int d = 0; d < 3; ++d) key |= ((b[d] >> bit) & 1u) << (3 * bit + d);",
     "for (int d = 0; d < 3; ++d) key |= ((b[2 - d] >> bit) & 1u) << (3 * bit + d);",
     PIN.check_sort_chains_is_a_spatial_permutation),
    # molecular architectures (Sec. 3.2.1) and independent sets (Sec. 3.1.2)
    ("topo_offset_sign", "const int32_t off = (int32_t)w >> 5;", "const int32_t off = -((int32_t)w >> 5);",
     TOPO.check_architecture_words_decode),
    ("topo_type_byte", "return topo[start + 1u + i] & 0xFFu;", "return (topo[start + 1u + i] >> 24) & 0xFFu;",
     TOPO.check_architecture_words_decode),
    ("topo_first_bond_only", "if (w & 1u) break;", "if ((w & 1u) || k >= 1u) break;",
     TOPO.check_architecture_words_decode),
    ("topo_types_ignored",
     "if (s->topo && s->arch) return or_topo_type(s->topo, s->topo_start[s->arch[chain]], i) == 1u;",
     "if (s->topo && s->arch) return i >= s->N_A;", TOPO.check_linear_topology_is_the_linear_chain),
    ("sets_see_later_partners", "if (partners[b] < i) taken |= 1u << set_of[partners[b]];",
     "if (partners[b] != i) taken |= 1u << set_of[partners[b]];", TOPO.check_sets_hand_values),
    ("set_shuffle_cyclic", "const uint32_t j = (h * (k + 1u)) >> 16;", "const uint32_t j = (h * k) >> 16;",
     TOPO.check_set_order_is_a_uniform_permutation),
    ("set_order_ignored", "if (s->topo_set[(uint64_t)a * N + i] != order[k]) continue;",
     "if (s->topo_set[(uint64_t)a * N + i] != k) continue;", TOPO.check_linear_topology_is_the_linear_chain),
    ("two_set_rule_reversed", "order[0] = first;\n    order[1] = 1u - first;",
     "order[0] = 1u - first;\n    order[1] = first;", TOPO.check_linear_topology_is_the_linear_chain),
    ("topo_bond_counted_twice", "if (j <= i) continue;", "if (j == i) continue;",
     TOPO.check_topology_observables_hand_values),
    ("trial_rounded_twice", "r_new[d] = (double)fmaf(s->a32, (float)or_uniform_sym(w[d]), pos[d]);",
     "r_new[d] = (double)(float)(r_old[d] + (double)(float)((double)s->a32 * or_uniform_sym(w[d])));",
     PIN.check_sweep_moves_follow_the_draws),
    # the BF16 reading of the learned proposal's network
    ("bf16_inputs_not_rounded", "xb[k] = or_round_bf16((float)x[k]);", "xb[k] = x[k];",
     BF16.check_bf16_network_closed_form),
    ("bf16_weights_not_rounded", "static double or_wbf(const double* W, int k) { return or_round_bf16((float)W[k]); }",
     "static double or_wbf(const double* W, int k) { return W[k]; }", BF16.check_bf16_network_closed_form),
    ("bf16_first_hidden_not_rounded", "h1[j] = a > 0.0 ? or_round_bf16((float)a) : 0.0;",
     "h1[j] = a > 0.0 ? a : 0.0;", BF16.check_bf16_network_closed_form),
    ("bf16_second_hidden_not_rounded", "h2[j] = a > 0.0 ? or_round_bf16((float)a) : 0.0;",
     "h2[j] = a > 0.0 ? a : 0.0;", BF16.check_bf16_network_closed_form),
    ("bf16_reverse_density_in_fp64", "or_mlp_bf16_run(s->mlp, f, T, o_rev, NULL, &slack);",
     "or_mlp_forward(s->mlp, f, o_rev);", BF16.check_bf16_move_uses_the_bf16_network),
    ("bf16_slack_inner_boundary_only", "for (int k = -1; k <= 1; ++k) {", "for (int k = 0; k <= 0; ++k) {",
     BF16.check_bf16_slack_values),
    # molecules of several lengths
    ("blend_histogram_counts_absent_slots", "const uint32_t n_k = or_length(s, k);",
     "const uint32_t n_k = s->N;", TOPO.check_blend_histogram_and_density),
    ("blend_end_to_end_to_last_slot", "const uint32_t last = or_length(s, k) - 1u;",
     "const uint32_t last = s->N - 1u;", TOPO.check_blend_ideal_statistics),
    ("blend_sq_over_all_slots", "  const double M = or_particles(s);",
     "  const double M = (double)s->n_chains * (double)s->N;", TOPO.check_blend_histogram_and_density),
    ("smc_acceptance_from_the_angle_word", "(w1[1] & 0xFFu) << 8 | (w1[2] & 0xFFu) << 16) << 8;",
     "(w1[1] & 0xFFu) << 8 | (w1[3] & 0xFFu) << 16) << 8;", PIN.check_smc_moves_follow_the_draws),
    ("smc_normals_paired_wrongly", "double u1 = or_uniform_open(w1[2 * p]), u2 = or_uniform_open(w1[2 * p + 1]);\n    double rad = sqrt(-2.0 * log(u1)), th = 2.0 * M_PI * u2;\n    xi[2 * p] = rad * cos(th);\n    xi[2 * p + 1] = rad * sin(th);\n  }\n  const double A = s->a * s->a / 6.0;",
     "double u1 = or_uniform_open(w1[p]), u2 = or_uniform_open(w1[p + 2]);\n    double rad = sqrt(-2.0 * log(u1)), th = 2.0 * M_PI * u2;\n    xi[2 * p] = rad * cos(th);\n    xi[2 * p + 1] = rad * sin(th);\n  }\n  const double A = s->a * s->a / 6.0;",
     PIN.check_smc_moves_follow_the_draws),
    ("density_counts_bonds", "s->rho_cell = (double)n_chains * (double)N / cells;",
     "s->rho_cell = (double)n_chains * (double)(N - 1) / cells;", GOLD.check_printed_systems),
    # smart Monte Carlo on molecules of any architecture and type
    ("smc_force_linear_on_architectures", "  const uint32_t n_fpart = or_partners(s, chain, i, fpart);",
     "  uint32_t n_fpart = 0;\n  if (i > 0) fpart[n_fpart++] = i - 1u;\n"
     "  if (i + 1u < s->N) fpart[n_fpart++] = i + 1u;", TOPO.check_smc_force_follows_the_architecture),
    ("smc_bond_energy_linear_on_architectures", "  const uint32_t n_epart = or_partners(s, chain, i, epart);",
     "  uint32_t n_epart = 0;\n  if (i > 0) epart[n_epart++] = i - 1u;\n"
     "  if (i + 1u < s->N) epart[n_epart++] = i + 1u;",
     lambda L: TOPO.check_ideal_star_and_ring_closed_forms(L, move=1)),
    ("smc_architectures_take_uniform_moves", "          if (s->move == 1)\n            or_move_smc(",
     "          if (0)\n            or_move_smc(",
     lambda L: TOPO.check_linear_topology_is_the_linear_chain(L, 0, 1)),
    ("smc_types_field_plane", "? s->w_types[or_type(s, chain, i)]\n", "? s->w_types[0]\n",
     lambda L: TYPES.check_two_types_equal_the_AB_path(L, 0, 1)),
    # n_t particle types
    ("types_K0_sign", "else v = v - 0.5 * chi0 * (phi[i] - phi[k]);",
     "else v = v + 0.5 * chi0 * (phi[i] - phi[k]);",
     lambda L: TYPES.check_type_fields_are_the_energy_derivative(L, 0)),
    ("types_K1_own_density", "if (s->hamiltonian == 1) v = v + chi0 * phi[k];",
     "if (s->hamiltonian == 1) v = v + chi0 * phi[i];", lambda L: TYPES.check_two_types_equal_the_AB_path(L, 1)),
    ("types_kappa_minus_one", "const double comp = kappa0 * (total - 1.0);",
     "const double comp = kappa0 * total;", lambda L: TYPES.check_type_fields_are_the_energy_derivative(L, 1)),
    ("types_energy_pair_weight", "else k -= 0.25 * chi * (phi[i] - phi[j]) * (phi[i] - phi[j]);",
     "else k -= 0.5 * chi * (phi[i] - phi[j]) * (phi[i] - phi[j]);",
     lambda L: TYPES.check_type_fields_are_the_energy_derivative(L, 0)),
    ("types_sweep_plane", "if (s->n_types && s->w_types) w_t = s->w_types[or_type(s, chain, i)];",
     "if (s->n_types && s->w_types) w_t = s->w_types[0];", TYPES.check_identical_types_collapse_under_K1),
    ("types_histogram_plane", "n[(uint64_t)or_type(s, k, i) * cells + or_cell(s, x[m], y[m], z[m])] += 1u;",
     "n[(uint64_t)(or_type(s, k, i) & 1u) * cells + or_cell(s, x[m], y[m], z[m])] += 1u;",
     TYPES.check_type_histogram_matches_numpy),
]


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


@pytest.mark.parametrize("mid,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(oracle_lib, mutant_dir, mid, old, new, pin):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {mid} not found exactly once"
    path_c = mutant_dir / f"{mid}.c"
    path_c.write_text(src.replace(old, new))
    hdr = os.path.join(os.path.dirname(SRC), "soma_oracle.h")
    so = mutant_dir / f"lib{mid}.so"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    f"-I{os.path.dirname(hdr)}", "-o", str(so), str(path_c), "-lm"], check=True)
    L = oracle.load(str(so))
    with pytest.raises(AssertionError):
        pin(L)
