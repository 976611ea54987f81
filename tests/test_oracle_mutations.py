"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake (a dropped term, a wrong sign or index, a
transposed operand, a wrong constant) in a copy of spg_oracle.c, builds it
on the CPU and runs the quick pins of test_oracle_pins.py against it: at
least one must fail. No GPU is involved.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_readings as readings

SRC = os.path.join(os.path.dirname(oracle.__file__), "spg_oracle.c")

MUTATIONS = {
    "D^T without the first-plane gate": ("if (has_diff(p, c, na)) s += ua[v];", "s += ua[v];"),
    "backward difference taken forward": (
        "d = x[v] - x[at_axis(p, xx, y, z, a, wrapc(c, -1, na))];",
        "d = x[at_axis(p, xx, y, z, a, wrapc(c, 1, na))] - x[v];"),
    "y neighbour taken along x": ("if (a == 1) return AT(p, xx, c, z);", "if (a == 1) return AT(p, c, y, z);"),
    "first-plane difference not zeroed (wraps around)": ("return p->forward ? c + 1 <= na - 1 : c >= 1;",
                                                         "return p->forward ? c + 1 <= na - 1 : c >= 0;"),
    "TV weight dropped from the gradient": ("double om = (omtv && !p->post_div) ? omtv[v] : 1.0;",
                                              "double om = 1.0;"),
    "periodic D^T without the wrap-around term": (
        "if (p->periodic || c + 1 <= na - 1) s -= ua[at_axis(p, xx, y, z, a, wrapc(c, 1, na))];",
        "if (c + 1 <= na - 1) s -= ua[at_axis(p, xx, y, z, a, wrapc(c, 1, na))];"),
    "forward-difference D^T with the wrong sign": ("if (has_diff(p, c, na)) s -= ua[v];",
                                                   "if (has_diff(p, c, na)) s += ua[v];"),
    "post-divergence weight applied twice": ("for (long long v = 0; v < (long long)n; v++) out[v] *= omtv[v];",
                                             "for (long long v = 0; v < (long long)n; v++) out[v] *= omtv[v] * omtv[v];"),
    "Huber offset mu instead of mu/2": ("return s - 0.5 * mu;", "return s - mu;"),
    "Huber gradient not clipped to the unit ball": ("double d = s > mu ? s : mu;", "double d = mu;"),
    "soft-threshold shrinks by 2t": ("return z > 0.0 ? z - t : z + t;", "return z > 0.0 ? z - 2.0 * t : z + 2.0 * t;"),
    "gradient step with the wrong sign": ("xnext[v] = orc_soft(y[v] - tau * g[v]", "xnext[v] = orc_soft(y[v] + tau * g[v]"),
    "lambda_tv dropped from grad f": ("out[v] = w[v] * (x[v] - b[v]) + p->lambda_tv * out[v];",
                                      "out[v] = w[v] * (x[v] - b[v]) + out[v];"),
    "data term without the 1/2": ("sd += 0.5 * w[v] * r * r;", "sd += w[v] * r * r;"),
    "om1 ignored in the objective's l1 sum": ("sl += (om1 ? om1[v] : 1.0) * fabs(x[v]);",
                                              "sl += fabs(x[v]);"),
    "omtv ignored in the objective's TV sum": ("st += (omtv ? omtv[v] : 1.0) * orc_huber(",
                                               "st += 1.0 * orc_huber("),
    "lambda_l1 dropped from the objective": ("out[1] = p->lambda_l1 * sl;", "out[1] = sl;"),
    "TV weight built from eps instead of eps_tv": ("omtv[v] = p->eps_tv / (gn + p->eps_tv);",
                                                   "omtv[v] = p->eps / (gn + p->eps);"),
    "l1 weight ignored in the prox": ("tau * p->lambda_l1 * (om1 ? om1[v] : 1.0));\n    free(y);",
                                      "tau * p->lambda_l1);\n    free(y);"),
    "extrapolation divides by t_k": ("beta[k] = momentum == 0 ? (t - 1.0) / tn : 0.0;",
                                     "beta[k] = momentum == 0 ? (t - 1.0) / t : 0.0;"),
    "extrapolation with the wrong sign": ("y[v] = xk[v] + beta * (xk[v] - xkm1[v]);",
                                          "y[v] = xk[v] - beta * (xk[v] - xkm1[v]);"),
    "adjoint drops the (1 + beta) factor": ("a_cur[v] += (1.0 + beta[k]) * ybar;", "a_cur[v] += ybar;"),
    "adjoint Hessian projection with the wrong sign": ("h0 = (q0 - e0 * eq) / s;", "h0 = (q0 + e0 * eq) / s;"),
    "adjoint of w uses b - y": ("gw[v] += -tau * (y[v] - b[v]) * m[v];", "gw[v] += tau * (y[v] - b[v]) * m[v];"),
    "restart test with the wrong sign": ("if (p->restart && restart_dot(p, x, xprev, xnext, beta[km]) > 0.0)",
                                         "if (p->restart && restart_dot(p, x, xprev, xnext, beta[km]) < 0.0)"),
    "Lipschitz bound with |D|^2 <= 4": ("return m + 12.0 * p->lambda_tv * max_omtv / p->mu",
                                         "return m + 4.0 * p->lambda_tv * max_omtv / p->mu"),
    "certificate with grad f(y) - grad f(x+)": ("double r = gx[v] - gy[v] + (y[v] - xplus[v]) / tau;",
                                               "double r = gy[v] - gx[v] + (y[v] - xplus[v]) / tau;"),
    "certificate without the 1/tau": ("double r = gx[v] - gy[v] + (y[v] - xplus[v]) / tau;",
                                      "double r = gx[v] - gy[v] + (y[v] - xplus[v]);"),
    "gamma term without its factor 2 in the gradient": ("out[v] += 2.0 * p->gamma * (x[v] - p->anchor[v]);",
                                                        "out[v] += p->gamma * (x[v] - p->anchor[v]);"),
}

QUICK = [
    pins.test_soft_threshold_table,
    pins.test_huber_table,
    pins.test_grad_hand_example,
    lambda o: pins.test_grad_matches_kronecker_matrix(o, (3, 4, 5)),
    lambda o: pins.test_adjoint_identity(o, (5, 7, 9)),
    pins.test_constant_has_zero_gradient_and_tv,
    pins.test_tv_of_ramp_and_spike,
    pins.test_objective_hand_example,
    lambda o: pins.test_objective_parts_match_sparse_evaluation(o, (4, 5, 6)),
    pins.test_reweight_spike,
    pins.test_lipschitz_bound_holds,
    pins.test_lipschitz_bound_is_valid_and_tight,
    pins.test_grad_f_matches_finite_difference_of_objective,
    pins.test_data_only_closed_form,
    pins.test_beta_table,
    pins.test_no_regularisation_converges_to_b,
    pins.test_tv_1d_reducible_matches_newton,
    pins.test_ista_is_monotone,
    pins.test_fista_rate_bound,
    pins.test_4cubed_optimality_lbfgs_kkt,
    pins.test_adjoint_identity_of_one_linear_step,
    pins.test_adjoint_matches_central_differences,
    pins.test_gradient_restart_converges_faster,
    pins.test_gamma_term_folds_into_data_and_weight,
    pins.test_certificate_is_the_norm_of_a_subgradient,
    lambda o: readings.test_div_is_the_adjoint_of_grad("forward", "neumann", (5, 7, 9)),
    lambda o: readings.test_div_is_the_adjoint_of_grad("backward", "periodic", (5, 7, 9)),
    lambda o: readings.test_div_is_the_adjoint_of_grad("forward", "periodic", (5, 7, 9)),
    lambda o: readings.test_forward_differences_are_reversed_backward_ones(),
    lambda o: readings.test_tv_weight_inside_is_a_gradient_and_post_div_is_not(),
]


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="orc_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, workdir):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {name}"
    mut = src.replace(old, new)
    tag = "".join(c if c.isalnum() else "_" for c in name)
    csrc = os.path.join(workdir, f"{tag}.c")
    lib = os.path.join(workdir, f"lib{tag}.so")
    with open(csrc, "w") as f:
        f.write(mut)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", csrc, "-o", lib, "-lm"])
    caught = None
    with oracle.using_library(lib):
        for pin in QUICK:
            try:
                pin(oracle)
            except Exception as e:  # a failing pin (assertion or a numerical blow-up)
                caught = f"{getattr(pin, '__name__', 'pin')}: {type(e).__name__}"
                break
    assert caught is not None, f"no pin caught: {name}"
