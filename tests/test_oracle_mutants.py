"""Planted mistakes in the oracle: each case builds a copy of the oracle with
one plausible error (a wrong sign, swapped weights, a transposed operand, a
dropped term) and runs the pins that cover that part against it; at least
one of them must fail.  The mistakes exist only in temporary builds (the C
oracle) or in modified copies loaded for one test (the network's Python
reference); the oracle itself is untouched."""
import pytest

from oracle import oracle as orc
from tests import test_oracle_alg as alg
from tests import test_oracle_prox as prox
from tests import test_oracle_twa as twa
from tests import test_oracle_user as usr

# (name, exact source text, replacement, pins that must catch it)
MUTANTS = [
    ("radius reward sign",
     "x[0] = n[0] + p[0] / rho[0];", "x[0] = n[0] - p[0] / rho[0];",
     [(prox.test_radius_rewards, dict(rho=r)) for r in (0.5, 1.0, 3.0)]),
    ("area reward with rho + 1 in the denominator",
     "x[0] = (rho[0] * n[0]) / (rho[0] - 1.0);", "x[0] = (rho[0] * n[0]) / (rho[0] + 1.0);",
     [(prox.test_radius_rewards, dict(rho=3.0))]),
    ("disk pair: radii moved up",
     "x[2] = n[2] - tr1;", "x[2] = n[2] + tr1;",
     [(prox.test_pack_pair_matches_bruteforce, dict(seed=s)) for s in range(4)]),
    ("disk pair: shares by rho instead of 1 / rho",
     "double wc1 = 1.0 / rho[0], wr1 = 1.0 / rho[2];", "double wc1 = rho[0], wr1 = rho[2];",
     [(prox.test_pack_pair_matches_bruteforce, dict(seed=s)) for s in range(4)]),
    ("L2 factor: lambda subtracted",
     "x[j] = (rho[j] * n[j]) / (rho[j] + p[0]);", "x[j] = (rho[j] * n[j]) / (rho[j] - p[0]);",
     [(prox.test_svm_l2_and_quad, dict(lam=l)) for l in (1.0, 5.0)]),
    ("quadratic cost: q in the numerator",
     "x[j] = (rho[j] * n[j]) / (p[j] + rho[j]);", "x[j] = (p[j] * n[j]) / (p[j] + rho[j]);",
     [(prox.test_svm_l2_and_quad, dict(lam=1.0))]),
    ("box: upper violations clamped to the lower bound",
     "if (v > hi) v = hi;", "if (v > hi) v = lo;",
     [(prox.test_box_and_fix, {})]),
    ("dual residual without rho",
     "double s = g->rho[e] * (g->z[b] - g->zprev[b]);", "double s = (g->z[b] - g->zprev[b]);",
     [(alg.test_two_factor_weighted_rho_and_alpha_by_hand, {})]),
    ("primal residual against the previous z",
     "double r = g->x[e] - g->z[b];", "double r = g->x[e] - g->zprev[b];",
     [(alg.test_residual_definition_and_stop_rule, {}), (alg.test_two_factor_weighted_rho_and_alpha_by_hand, {})]),
    ("m-update with u subtracted",
     "for (int64_t e = 0; e < E; ++e) g->m[e] = g->x[e] + g->u[e];",
     "for (int64_t e = 0; e < E; ++e) g->m[e] = g->x[e] - g->u[e];",
     [(alg.test_two_factor_weighted_rho_and_alpha_by_hand, {}), (alg.test_alg1_equals_alg2_scalar_consensus, {})]),
    ("n-update with u added",
     "for (int64_t e = 0; e < E; ++e) g->n[e] = g->z[g->ez[e]] - g->u[e];",
     "for (int64_t e = 0; e < E; ++e) g->n[e] = g->z[g->ez[e]] + g->u[e];",
     [(alg.test_two_factor_weighted_rho_and_alpha_by_hand, {}), (alg.test_residual_definition_and_stop_rule, {})]),
    ("stop rule on the primal residual alone",
     "if (rpri <= tol_pri && rdual <= tol_dual) break;", "if (rpri <= tol_pri) break;",
     [(alg.test_residual_definition_and_stop_rule, {})]),
    ("stop rule on the dual residual alone",
     "if (rpri <= tol_pri && rdual <= tol_dual) break;", "if (rdual <= tol_dual) break;",
     [(alg.test_residual_definition_and_stop_rule, {})]),
    ("wall weights swapped",
     "double wc = 1.0 / rho[0], wr = 1.0 / rho[2];", "double wc = 1.0 / rho[2], wr = 1.0 / rho[0];",
     [(prox.test_pack_wall_matches_bruteforce, dict(seed=s)) for s in range(10)]),
    ("dynamics with B transposed",
     "M[i * nvv + nx + j] = B[i * nu + j];", "M[i * nvv + nx + j] = B[j * nx + i];",
     [(alg.test_mpc_inactive_box_is_lqr, {}), (alg.test_mpc_horizon_pendulum_is_lqr, {})]),
    ("hinge step not clipped at c",
     "if (gam > c) gam = c;", "",
     [(prox.test_svm_hinge_matches_bruteforce, dict(seed=s)) for s in range(10)]),
    ("z-update without the rho weights",
     "double S = 0.0, R = 0.0;\n                for (int64_t k = g->row[b]; k < g->row[b + 1]; ++k) {\n"
     "                    int64_t e = g->col[k];\n                    S += g->rho[e] * g->m[e];",
     "double S = 0.0, R = 0.0;\n                for (int64_t k = g->row[b]; k < g->row[b + 1]; ++k) {\n"
     "                    int64_t e = g->col[k];\n                    S += g->m[e];",
     [(alg.test_alg1_equals_alg2_scalar_consensus, {}), (alg.test_alg1_equals_alg2_mpc_without_box, {})]),
    ("u-update with the wrong sign",
     "g->u[e] = g->u[e] + g->alpha[e] * (g->x[e] - g->z[g->ez[e]]);",
     "g->u[e] = g->u[e] - g->alpha[e] * (g->x[e] - g->z[g->ez[e]]);",
     [(alg.test_alg1_equals_alg2_scalar_consensus, {}), (alg.test_mpc_inactive_box_is_lqr, {})]),
    ("margin: y dropped from the b update",
     "x[d] = n[d] + (lam * y) / rho[d];", "x[d] = n[d] + lam / rho[d];",
     [(prox.test_svm_margin_matches_bruteforce, dict(seed=s)) for s in range(10)]),
    ("minimal error: threshold with the wrong sign",
     "const double v = n[j] - p[0] / rho[j];", "const double v = n[j] + p[0] / rho[j];",
     [(prox.test_svm_slack_matches_bruteforce, dict(lam=l)) for l in (0.0, 0.3, 2.0)]),
    ("equality: weights swapped",
     "const double v = (rho[j] * n[j] + rho[d + j] * n[d + j]) / (rho[j] + rho[d + j]);",
     "const double v = (rho[d + j] * n[j] + rho[j] * n[d + j]) / (rho[j] + rho[d + j]);",
     [(prox.test_equal_matches_constrained_minimiser, {})]),
    ("u-update ignores alpha",
     "g->u[e] = g->u[e] + g->alpha[e] * (g->x[e] - g->z[g->ez[e]]);",
     "g->u[e] = g->u[e] + (g->x[e] - g->z[g->ez[e]]);",
     [(alg.test_two_factor_weighted_rho_and_alpha_by_hand, {}),
      (alg.test_weighted_dual_sum_decays_by_one_minus_alpha, {})]),
    ("z-update as an unweighted mean",
     "S += g->rho[e] * g->m[e];\n                    R += g->rho[e];\n                }",
     "S += g->m[e];\n                    R += 1.0;\n                }",
     [(alg.test_two_factor_weighted_rho_and_alpha_by_hand, {})]),
    ("three weights: infinite weight treated as standard",
     "if (g->cls[e] == OW_INF) {", "if (0) {",
     [(twa.test_infinite_weight_decides_z, {})]),
    ("three weights: zero-weight messages averaged",
     "if (g->cls[e] == OW_STD) {\n                            Ss", "if (1) {\n                            Ss",
     [(twa.test_inactive_box_by_hand, {})]),
    ("three weights: u not reset on non-standard edges",
     "g->cls[e] == OW_STD ? g->u[e] + g->alpha[e] * (g->x[e] - g->z[g->ez[e]]) : 0.0",
     "g->u[e] + g->alpha[e] * (g->x[e] - g->z[g->ez[e]])",
     [(twa.test_inactive_box_by_hand, {}), (twa.test_infinite_weight_decides_z, {})]),
    ("user operator given the first factor's parameters",
     "g->params + f->par0, g->x + f->edge0, g->uctx[k]", "g->params, g->x + f->edge0, g->uctx[k]",
     [(usr.test_operator_sees_its_messages_in_creation_order, {})]
     + [(usr.test_user_lasso_converges_to_the_closed_form, dict(seed=s)) for s in (1, 2, 3)]),
    ("user operator given the first edges' rho",
     "g->ufn[k](f->arity, g->n + f->edge0, g->rho + f->edge0,", "g->ufn[k](f->arity, g->n + f->edge0, g->rho,",
     [(usr.test_operator_sees_its_messages_in_creation_order, {}),
      (usr.test_user_operators_restating_builtins_match_bit_for_bit, {})]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new, pins):
    src = orc.source_text()
    assert src.count(old) == 1, "the planted line must match the oracle source exactly once"
    lib = orc.build_variant(src.replace(old, new), str(tmp_path / "libmutant.so"))
    failed = []
    with orc.using_build(lib):
        for pin, kw in pins:
            try:
                pin(**kw)
            except Exception as e:   # an assertion, or a solver the mistake derailed
                failed.append("%s(%s): %s" % (pin.__name__, kw, type(e).__name__))
    assert failed, "no pin caught the planted mistake '%s'" % name


# Planted mistakes in the warm-start network's FP64 reference
# (oracle/mlp_oracle.py): each is loaded as a modified copy of the module in
# place of the real one inside tests/test_oracle_mlp.py, whose pins must
# then fail.
MLP_MUTANTS = [
    ("loss gradient without the factor 2", "dY = 2.0 * D / n", "dY = D / n",
     ["test_gradients_match_finite_differences"]),
    ("second hidden layer masked by the first layer's activations",
     'dH2 = r((dYq @ f["W3q"]) * (f["H2"] > 0))', 'dH2 = r((dYq @ f["W3q"]) * (f["H1"] > 0))',
     ["test_gradients_match_finite_differences"]),
    ("W2 gradient against the wrong activations", 'gW2 = dH2.T @ f["H1"]', 'gW2 = dH2.T @ f["H2"]',
     ["test_gradients_match_finite_differences"]),
    ("Adam without bias correction", "mh = m / (1 - b1 ** step)", "mh = m",
     ["test_adam_closed_form_first_step"]),
    ("bfloat16 by truncation", "u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u = u & 0xFFFF0000",
     ["test_bf16_rounding"]),
]


@pytest.mark.parametrize("name,old,new,pins", MLP_MUTANTS, ids=[m[0] for m in MLP_MUTANTS])
def test_planted_mlp_mistake_fails_a_pin(monkeypatch, name, old, new, pins):
    import types

    from oracle import mlp_oracle
    from tests import test_oracle_mlp as mlp_pins
    with open(mlp_oracle.__file__) as fh:
        src = fh.read()
    assert src.count(old) == 1, "the planted line must match the module source exactly once"
    mutant = types.ModuleType("mlp_oracle_mutant")
    exec(compile(src.replace(old, new), "mlp_oracle_mutant", "exec"), mutant.__dict__)
    monkeypatch.setattr(mlp_pins, "mo", mutant)
    failed = []
    for pin in pins:
        try:
            getattr(mlp_pins, pin)()
        except Exception as e:   # an assertion, or arithmetic the mistake derailed
            failed.append("%s: %s" % (pin, type(e).__name__))
    assert failed, "no pin caught the planted mistake '%s'" % name
