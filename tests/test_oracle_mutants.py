"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a flipped
sign, a wrong power of s, a dropped softening term, a swapped index, a wrong
kick factor, a wrong adjoint term, a wrong expansion term or traversal
rule of the fast multipole method, a splitting or sending rule of the
parallel tree code), builds it, swaps it in for the real
oracle, and runs the pins of test_oracle_pins.py against it: at least one pin
must fail.  The real oracle is restored afterwards.  Only the oracle (CPU)
is mutated.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle_bh as bhpins
import test_oracle_fmm as fmmpins
import test_oracle_let as letpins
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "nbody_oracle.c")

MUTANTS = {
    "sign of d": ("double dx = x[3 * j] - xi;", "double dx = xi - x[3 * j];"),
    "power of s": ("double inv_s3 = 1.0 / (s2 * sqrt(s2));\n        ax",
                   "double inv_s3 = 1.0 / s2;\n        ax"),
    "softening dropped": ("dz * dz + eps * eps;\n        double inv_s3",
                          "dz * dz;\n        double inv_s3"),
    "mass index": ("ax += m[j] * dx * inv_s3;", "ax += m[i] * dx * inv_s3;"),
    "self pair kept": ("        if (j == i) continue;\n        double dx",
                       "        double dx"),
    "G dropped": ("out[0] = G * ax;", "out[0] = ax;"),
    "potential power": ("s += m[j] / sqrt(dx * dx + dy * dy + dz * dz + eps * eps);",
                        "s += m[j] / (dx * dx + dy * dy + dz * dz + eps * eps);"),
    "kinetic factor": ("ek += 0.5 * m[i] *", "ek += m[i] *"),
    "first kick": ("for (int64_t k = 0; k < 3 * n; ++k) v[k] += 0.5 * dt * acc[k];\n"
                   "        for (int64_t k = 0; k < 3 * n; ++k) x[k] += dt * v[k];",
                   "for (int64_t k = 0; k < 3 * n; ++k) v[k] += dt * acc[k];\n"
                   "        for (int64_t k = 0; k < 3 * n; ++k) x[k] += dt * v[k];"),
    "vjp dyadic sign": ("g[c] += w[c] * inv_s3 - 3.0 * d[c] * dw * inv_s5;",
                        "g[c] += w[c] * inv_s3 + 3.0 * d[c] * dw * inv_s5;"),
    "vjp w swapped": ("w[c] = m[k] * lam[3 * j + c] - m[j] * lam[3 * k + c];",
                      "w[c] = m[j] * lam[3 * j + c] - m[k] * lam[3 * k + c];"),
    "vjp mass sign": ("gmk += -ld * inv_s3;", "gmk += ld * inv_s3;"),
    "adjoint drift": ("for (size_t k = 0; k < per; ++k) lv[k] += dt * lx[k];",
                      "for (size_t k = 0; k < per; ++k) lv[k] += 0.5 * dt * lx[k];"),
    "bh acceptance inverted": ("if (!(d2 >= crit2[nd->level])) all = 0;",
                               "if (!(d2 <= crit2[nd->level])) all = 0;"),
    "bh centre of mass": ("nd->com[c] = M > 0.0 ? s[c] / M : 0.0;", "nd->com[c] = s[c];"),
    "bh cell mass": ("double w = nd->M / (s2 * sqrt(s2));", "double w = 1.0 / (s2 * sqrt(s2));"),
    "bh octant shift": ("while (e < end && (t->key[e] >> shift) == cp) ++e;",
                        "while (e < end && (t->key[e] >> (shift + 3)) == cp) ++e;"),
    "bh key axis": ("key0[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);",
                    "key0[i] = spread10(q[0]) | (spread10(q[0]) << 1) | (spread10(q[2]) << 2);"),
    "fmm derivative factor": ("if (q2 >= 0) v += (double)(n[c] - 1) * T[(m + 1) * nt + q2];",
                              "if (q2 >= 0) v += (double)(n[c]) * T[(m + 1) * nt + q2];"),
    "fmm derivative sign": ("T[m * nt] = -(double)(2 * m - 1) * T[(m - 1) * nt] / s2;",
                            "T[m * nt] = (double)(2 * m - 1) * T[(m - 1) * nt] / s2;"),
    "fmm moment sign": ("double y = -(xj[c] - z[c]);", "double y = xj[c] - z[c];"),
    "fmm moment factorial": ("pw[2][B->mi[q][2]] * B->inv_fact[q];", "pw[2][B->mi[q][2]];"),
    "fmm truncation": ("if (n[0] + n[1] + n[2] > p - kk) break;",
                       "if (n[0] + n[1] + n[2] > p - kk - 1) break;"),
    "fmm gradient axis": ("a[1] += L[fmm_slot(k[0], k[1] + 1, k[2])] * w;",
                          "a[1] += L[fmm_slot(k[0] + 1, k[1], k[2])] * w;"),
    "fmm separation inverted": ("return (double)d2 >= T->crit", "return (double)d2 < T->crit"),
    "fmm ancestors skipped": ("for (int64_t an = a; an >= 0; an = parent[an]) {\n                double u[3];",
                              "for (int64_t an = a; an >= 0; an = -1) {\n                double u[3];"),
    "fmm equal cells not split": ("if (nb->child[o] >= 0) fmm_push(&down, (int32_t)nb->child[o]);",
                                  "if (nb->child[o] >= 0) fmm_push(&down, (int32_t)b);"),
    "fmm octant skipped": ("if (nb->child[o] >= 0) fmm_leaf_visit(T, a, nb->child[o]);",
                           "if (nb->child[o] >= 0 && o > 0) fmm_leaf_visit(T, a, nb->child[o]);"),
    "fmm centre at corner": ("z[id][c] = P.box_lo[c] + cell * ((double)ic[c] + 0.5);",
                             "z[id][c] = P.box_lo[c] + cell * (double)ic[c];"),
    "fmm inscribed radius": ("T.crit[la][lb] = 0.75 * s * s / (theta * theta);",
                             "T.crit[la][lb] = 0.25 * s * s / (theta * theta);"),
    "orb shortest axis": ("if (hi[c] - lo[c] > hi[axis] - lo[axis]) axis = c;",
                          "if (hi[c] - lo[c] < hi[axis] - lo[axis]) axis = c;"),
    "orb halves regardless of p": ("int64_t k = cnt * (int64_t)p_lo / p;", "int64_t k = cnt / 2;"),
    "sharded remote trees skipped": ("for (int q = 0; q < P; ++q) {\n                int s = q == 0",
                                     "for (int q = 0; q < 1; ++q) {\n                int s = q == 0"),
    "sharded self pair by local index": ("if (sid[j] == tid[k]) continue;",
                                         "if (j == k) continue;"),
    "sharded cell not covering its bodies": ("cov += nd->end - nd->start;", "cov += 1;"),
    "sharded cell mass": ("double wc = nd->M / (s2 * sqrt(s2));",
                          "double wc = 1.0 / (s2 * sqrt(s2));"),
    "let near box corner": ("float aa = nd->lo[c] - bhi[c];", "float aa = nd->lo[c] - blo[c];"),
    "let children not sent": ("if (nd->child[o] >= 0) kind[nd->child[o]] = -1;",
                              "if (nd->child[o] >= 0) kind[nd->child[o]] = 0;"),
}

PINS = [
    pins.test_two_body_closed_form, pins.test_two_body_zero_softening,
    pins.test_equilateral_triangle, pins.test_newton_third_law,
    pins.test_power_of_two_scaling_is_exact, pins.test_monopole_far_field,
    pins.test_force_is_minus_gradient_of_potential, pins.test_energy_closed_forms,
    pins.test_circular_orbit_phase_error_is_second_order,
    pins.test_kepler_orbit_zero_softening, pins.test_time_reversibility,
    pins.test_force_vjp_central_differences, pins.test_kdk_grad_central_differences,
    lambda: bhpins.test_theta_zero_is_the_direct_sum(8, 32), bhpins.test_error_falls_with_theta,
    bhpins.test_far_cluster_is_its_monopole, bhpins.test_tree_counts_and_cost,
    fmmpins.test_derivatives_closed_forms, lambda: fmmpins.test_derivatives_finite_differences(0.4),
    fmmpins.test_derivatives_harmonic_without_softening,
    lambda: fmmpins.test_expansion_order_of_accuracy(0.3),
    fmmpins.test_expansion_converges_to_the_direct_sum,
    lambda: fmmpins.test_theta_zero_is_the_direct_sum(16, 6),
    lambda: fmmpins.test_every_body_meets_every_other_once(0.6),
    fmmpins.test_power_of_two_scaling_is_exact, fmmpins.test_error_falls_with_theta_and_order,
    fmmpins.test_far_cluster_through_expansions_only,
    lambda: letpins.test_orb_equal_counts_and_bisecting_planes(5, 1000),
    letpins.test_orb_follows_the_bodies,
    lambda: letpins.test_one_processor_is_the_tree_code(0.5, 32),
    lambda: letpins.test_theta_zero_is_the_direct_sum(3),
    lambda: letpins.test_every_body_is_met_once(0.5, 4),
    lambda: letpins.test_let_holds_everything_a_remote_body_meets(0.7),
    letpins.test_let_of_a_far_destination_is_the_root_alone,
]


def _build_mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                    "-shared", str(path), "-o", str(so), "-lm"], check=True)
    return oracle._bind(ctypes.CDLL(str(so)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    mutant = _build_mutant(tmp_path, old, new)
    real = oracle._load()
    caught = []
    try:
        oracle._lib = mutant
        for pin in PINS:
            try:
                with __import__("warnings").catch_warnings():
                    __import__("warnings").simplefilter("ignore")
                    pin()
            except (AssertionError, FloatingPointError, ValueError):
                caught.append(getattr(pin, "__name__", "pin"))
    finally:
        oracle._lib = real
    assert caught, f"no pin caught the mutant '{name}'"


def test_unmutated_copy_passes_every_pin(tmp_path):
    real = oracle._load()
    copy = _build_mutant(tmp_path, "int oracle_threads(void)", "int oracle_threads(void)")
    try:
        oracle._lib = copy
        for pin in PINS:
            pin()
    finally:
        oracle._lib = real
