"""Each pin must be able to fail: plant one plausible mistake at a time in a copy of
the oracle (the C part compiled separately, on the CPU; the Python solvers of Sec. 5.1-5.2
re-executed from their mutated source) and check that at least one pin rejects it."""
import inspect
import textwrap

import pytest

import oracle
from tests import test_oracle_pins as P

MUTATIONS = {
    "transposed outer product X (x) W": ("s += X[j * p + m] * W[j * p + c];",
                                         "s += X[j * p + c] * W[j * p + m];"),
    "dropped d2W0/dr2 term of element 3": ("if (a == 2) v += f2 * rx * rx;", "if (a == 2) v += 0 * rx * rx;"),
    "wrong sign of a d2W0/dr2 term, order 3": ("if (a == 3) v += f3 * rx * rx * rx + f2 * 3 * rx * rxx;",
                                               "if (a == 3) v += f3 * rx * rx * rx - f2 * 3 * rx * rxx;"),
    "minimum image shifted the wrong way": ("if (dx > halfL[0]) dx -= L[0];", "if (dx > halfL[0]) dx += L[0];"),
    "h-scaling exponent off by one": ("for (int t = 0; t < a + b; t++) s /= hi;",
                                      "for (int t = 0; t < a + b - 1; t++) s /= hi;"),
    "factorial dropped from X": ("for (int t = 1; t <= a; t++) v = v * x / (real)t;",
                                 "for (int t = 1; t <= a; t++) v = v * x;"),
    "binomial dropped in the |r| recurrence": ("rhs -= binom(a, a2) * binom(b, b2) * dr[a2][b2] * dr[a - a2][b - b2];",
                                               "rhs -= binom(a, a2) * dr[a2][b2] * dr[a - a2][b - b2];"),
    "f_j instead of f_j - f_i": ("s += ((real)f[col[e]] - (real)f[i]) * (real)w[e * n_ops + d];",
                                 "s += ((real)f[col[e]]) * (real)w[e * n_ops + d];"),
    "RK4 stage weight": ("(k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i])", "(k1[i] + k2[i] + 2 * k3[i] + k4[i])"),
    "truncation rule ignored (W'' kept at order 4)": ("        } else if (n == 3) {",
                                                      "        } else if (n == 4) { v += f2 * rx * rx * rx * rx;\n        } else if (n == 3) {"),
    "stencil radius h instead of 2h": ("double R = 2.0 * h[i];", "double R = h[i];"),
    "dw0 form keeps the d2W0/dr2 terms": ("if (rbf_form & ORC_ABF_DW0_ONLY) f2 = f3 = 0;",
                                          "if (rbf_form & ORC_ABF_DW0_ONLY) f3 = 0;"),
    "Burgers advection with the wrong sign": (
        "real fu = -(u[i] * op_sum(row_ptr, col, w, n_ops, 0, u, i) + v[i] * op_sum(row_ptr, col, w, n_ops, 1, u, i));",
        "real fu = (u[i] * op_sum(row_ptr, col, w, n_ops, 0, u, i) + v[i] * op_sum(row_ptr, col, w, n_ops, 1, u, i));"),
    "Burgers advection of u by u only (v term dropped)": (
        "real fu = -(u[i] * op_sum(row_ptr, col, w, n_ops, 0, u, i) + v[i] * op_sum(row_ptr, col, w, n_ops, 1, u, i));",
        "real fu = -(u[i] * op_sum(row_ptr, col, w, n_ops, 0, u, i));"),
    "Burgers viscous term on the wrong operator": (
        "fu += (real)beta[d] * op_sum(row_ptr, col, w, n_ops, d, u, i);",
        "fu += (real)beta[d] * op_sum(row_ptr, col, w, n_ops, d - 1, u, i);"),
}

PINS = [
    lambda: P.test_abfs_match_printed_forms("wendland_c2"),
    lambda: P.test_abfs_match_printed_forms("cone"),
    P.test_r_derivatives_vs_sympy,
    P.test_x_vector_printed,
    P.test_neighbours_vs_kdtree,
    P.test_lattice_parity_zeros,
    P.test_assembly_and_solve_vs_lapack,
    lambda: P.test_polynomial_reproduction(4, 1.6, "quadratic", 1e-11),
    lambda: P.test_polynomial_reproduction(6, 2.0, "wendland_c2", 1e-9),
    P.test_rk4_linear_system_is_taylor_polynomial,
    P.test_abfs_truncated_high_orders_vs_sympy,
    lambda: P.test_abfs_dw0_form_is_the_printed_dW0_bracket("quadratic"),
    lambda: P.test_laplacian_noise_limits_dw0_form(4, 2.0, 1.0),
    P.test_burgers_quick_convergence,
    P.test_burgers_2d_convergence,
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, name
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "mutant.so"))
    monkeypatch.setitem(oracle._LIBS, "f64", lib)
    caught = []
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            caught.append(pin)
        except Exception:  # a crash (e.g. a bad stencil size) also rejects the mutant
            caught.append(pin)
    assert caught, f"no pin caught: {name}"


# the global matrix, the steady state and the direct solve (oracle/__init__.py): (function, old, new)
PY_MUTATIONS = {
    "global matrix diagonal with the wrong sign": ("operator_matrix", "return (A - sp.diags(", "return (A + sp.diags("),
    "global matrix transposed (w_ij for w_ji)": (
        "operator_matrix", "(wb, (node, np.asarray(col, dtype=np.int64)))",
        "(wb, (np.asarray(col, dtype=np.int64), node))"),
    "beta ignored (first operator only)": (
        "operator_matrix", "wb = np.asarray(w, dtype=np.float64) @ np.asarray(beta, dtype=np.float64)",
        "wb = np.asarray(w, dtype=np.float64)[:, 0]"),
    "steady state with the boundary term's sign flipped": ("steady_state", "-(A[I][:, B] @ u[B])",
                                                            "(A[I][:, B] @ u[B])"),
    "steady state from the transposed interior block": ("steady_state", "spl.spsolve(A[I][:, I].tocsc()",
                                                        "spl.spsolve(A[I][:, I].T.tocsc()"),
    "Dirichlet rows ignored": ("solve_operator", "for i in np.nonzero(np.asarray(dirichlet))[0]:",
                               "for i in np.nonzero(np.asarray(dirichlet))[0][:0]:"),
    "operator index ignored": ("solve_operator", "beta[op] = 1.0", "beta[0] = 1.0"),
    "Neumann row diagonal on the ghost instead of its parent": (
        "solve_operator", "row[pb] = row.get(pb, 0.0) - total", "row[gi] = row.get(gi, 0.0) - total"),
    "Neumann row without the normal's y component": (
        "solve_operator", "c = nx * w[e, op_x] + ny * w[e, op_y]", "c = nx * w[e, op_x]"),
    "Neumann row with the x and y operators swapped": (
        "solve_operator", "c = nx * w[e, op_x] + ny * w[e, op_y]", "c = nx * w[e, op_y] + ny * w[e, op_x]"),
    "Neumann ghost rows left out": ("solve_operator", "for g in range(len(ghost)):", "for g in range(0):"),
}

PY_PINS = [  # cheapest first; the first pin that fails ends the search
    P.test_poisson_neumann_ghost_rows_reproduce_polynomials,
    P.test_global_matrix_and_direct_solve_vs_apply,
    P.test_heat_frozen_rk4_reaches_the_steady_state,
    lambda: P.test_heat_steady_state_table(2),
    P.test_poisson_periodic_even_order_pattern,
]


def _mutated(func, old, new):
    src = textwrap.dedent(inspect.getsource(func))
    assert src.count(old) == 1, (func.__name__, old)
    ns = dict(func.__globals__)
    exec(compile(src.replace(old, new), f"<mutant {func.__name__}>", "exec"), ns)
    return ns[func.__name__]


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_planted_mistake_in_the_python_solvers_is_caught(name, monkeypatch):
    fname, old, new = PY_MUTATIONS[name]
    monkeypatch.setattr(oracle, fname, _mutated(getattr(oracle, fname), old, new))
    for pin in PY_PINS:
        try:
            pin()
        except Exception:  # an assertion, or a failed solve of a singular system
            return
    pytest.fail(f"no pin caught: {name}")
