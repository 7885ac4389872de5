"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each compares it with values
the paper prints, an independent library (sympy, scipy, LAPACK), a closed-form
identity, or a property (exact polynomial reproduction, convergence order,
symmetry, exact power-of-two scaling) that a dropped term, wrong sign or index,
or transposed operand would break.
"""
import math
import os

import numpy as np
import pytest

import labfm_synth as S
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _paper_numbers():
    out = {}
    with open(os.path.join(GOLD, "paper_numbers.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = vals
    return out


def _printed_abfs():
    rows = []
    with open(os.path.join(GOLD, "abf_printed_forms.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            e, br, expr = line.split(maxsplit=2)
            rows.append((int(e), br, expr))
    return rows


def _ghost_lattice(n_side, hs, jitter, seed):
    """Noisy Cartesian nodes on [0,1]^2 plus a ghost strip wider than 2h (Sec. 4.1);
    returns (xy, h, indices of the nodes inside the unit square)."""
    s = 1.0 / n_side
    g = int(np.ceil(2 * hs)) + 1
    idx = np.arange(-g, n_side + g)
    ii, jj = np.meshgrid(idx, idx, indexing="xy")
    x = (ii.ravel() + 0.5) * s
    y = (jj.ravel() + 0.5) * s
    u = S.uniform01(seed, 2 * x.size)
    x = x + (2 * u[0::2] - 1) * jitter * s
    y = y + (2 * u[1::2] - 1) * jitter * s
    inner = (ii.ravel() >= 0) & (ii.ravel() < n_side) & (jj.ravel() >= 0) & (jj.ravel() < n_side)
    return np.stack([x, y], 1), np.full(x.size, hs * s), np.nonzero(inner)[0]


BIG = (-100.0, -100.0), (100.0, 100.0)  # a non-periodic box that contains every node


# ------------------------------------------------------------------------ indexing


def test_p_sequence_printed():
    nums = _paper_numbers()
    printed = [int(v) for v in nums["p_of_k"]]
    assert [oracle.p_of_k(k) for k in range(1, 7)] == printed
    # the same rule continues to k = 8 (p = 44, the order-8 system size)
    assert oracle.p_of_k(7) == 35 and oracle.p_of_k(8) == 44


def test_x_vector_printed():
    """First ten entries of X as printed in Sec. 2: x, y, x^2/2, xy, y^2/2, x^3/6, ..."""
    nums = _paper_numbers()
    x, y = 0.7, -1.3
    X = oracle.monomials(x, y, 4)
    for e, spec in enumerate(nums["x_vector"]):
        a, b, div = (int(t) for t in spec.split(","))
        assert X[e] == pytest.approx(x ** a * y ** b / div, rel=1e-15)


def test_c_vectors_and_hyperviscosity_positions():
    """C^x, C^y, C^L (Sec. 2) and the nabla^4 / nabla^6 element positions (Sec. 4.2)."""
    nums = _paper_numbers()

    def nz(c):
        return [int(i) + 1 for i in np.nonzero(c)[0]]

    assert nz(S.op_c_vector("dx", 4)) == [int(v) for v in nums["c_x"]]
    assert nz(S.op_c_vector("dy", 4)) == [int(v) for v in nums["c_y"]]
    assert nz(S.op_c_vector("lap", 4)) == [int(v) for v in nums["c_lap"]]
    c4 = S.op_c_vector("lap2", 4)
    assert nz(c4) == [int(v) for v in nums["hv_nabla4_elements"]]
    assert list(c4[np.nonzero(c4)[0]]) == [float(v) for v in nums["hv_nabla4_coeffs"]]
    c6 = S.op_c_vector("lap3", 6)
    assert nz(c6) == [int(v) for v in nums["hv_nabla6_elements"]]
    assert list(c6[np.nonzero(c6)[0]]) == [float(v) for v in nums["hv_nabla6_coeffs"]]
    # nabla^8 continues the rule: elements 36..44 step 2 with binomial(4, t)
    c8 = S.op_c_vector("lap4", 8)
    assert nz(c8) == [36, 38, 40, 42, 44]
    assert list(c8[np.nonzero(c8)[0]]) == [1.0, 4.0, 6.0, 4.0, 1.0]
    with pytest.raises(ValueError):
        S.op_c_vector("lap4", 6)  # only up to nabla^k (Sec. 4.2)


# ------------------------------------------------------------------------ RBFs


def _sympy_kernels():
    sp = pytest.importorskip("sympy")
    q = sp.symbols("q", positive=True)
    pi = sp.pi
    return sp, q, {
        "cone": sp.Rational(3, 4) / pi * (1 - q / 2),
        "quadratic": sp.Rational(3, 16) / pi * (q - 2) ** 2,
        "wendland_c2": sp.Rational(7, 4) / pi * (1 - q / 2) ** 4 * (1 + 2 * q),
        "wendland_c6": sp.Rational(78, 28) / pi * (1 - q / 2) ** 8
        * (4 * q ** 3 + sp.Rational(25, 4) * q ** 2 + 4 * q + 1),
        "gaussian": 9 / pi * sp.exp(-9 * q ** 2),
    }


@pytest.mark.parametrize("rbf", ["cone", "quadratic", "wendland_c2", "wendland_c6", "gaussian"])
def test_rbf_derivatives_vs_sympy(rbf):
    """W0 and its first three q-derivatives against symbolic differentiation of the
    kernels as printed (Sec. 3.2, Appendix A; Wendland C2 from its standard form)."""
    sp, q, ker = _sympy_kernels()
    expr = ker[rbf]
    ders = [expr, sp.diff(expr, q), sp.diff(expr, q, 2), sp.diff(expr, q, 3)]
    fns = [sp.lambdify(q, d, "math") for d in ders]
    for qv in (0.05, 0.37, 0.9, 1.31, 1.77, 1.995):
        d = oracle.rbf_derivs(rbf, qv)
        for m in range(4):
            ref = fns[m](qv)
            assert d[m] == pytest.approx(ref, rel=1e-12, abs=1e-14), (rbf, qv, m)


def test_cone_slope_printed():
    nums = _paper_numbers()
    assert oracle.rbf_derivs("cone", 0.8)[1] == pytest.approx(float(nums["cone_dW0dq"][0]), rel=1e-15)


@pytest.mark.parametrize("rbf,expected", [("cone", 1.0), ("wendland_c2", 1.0), ("wendland_c6", 1.0),
                                          ("gaussian", 1.0), ("quadratic", 0.5)])
def test_rbf_normalisation(rbf, expected):
    """2 pi int_0^2 q W0(q) dq = 1 and W0(2) = 0 (Appendix A).  The quadratic kernel as
    printed integrates to 1/2, not 1: a constant factor on W0 cancels in the weights
    (the ABFs and M scale together), so it is used as printed."""
    from scipy.integrate import quad

    val, _ = quad(lambda t: 2 * math.pi * t * oracle.rbf_derivs(rbf, t)[0], 0.0, 2.0,
                  epsabs=1e-14, epsrel=1e-13, limit=400, points=[1.0])
    assert val == pytest.approx(expected, abs=1e-12)
    w2 = oracle.rbf_derivs(rbf, 2.0)[0]
    if rbf == "gaussian":
        assert abs(w2 - float(_paper_numbers()["gaussian_w2"][0])) < 1e-17
    else:
        assert w2 == 0.0


# ------------------------------------------------------------------------ |r| derivatives and ABFs


def test_r_derivatives_vs_sympy():
    """d^(a+b)|r|/dx^a dy^b for a + b <= 8 (the Leibniz recurrence of the oracle)
    against symbolic differentiation."""
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y", real=True)
    r = sp.sqrt(x ** 2 + y ** 2)
    pts = [(0.31, -0.77), (1.2, 0.45), (-0.6, -0.9)]
    for a in range(9):
        for b in range(9 - a):
            if a + b == 0:
                continue
            f = sp.lambdify((x, y), sp.diff(r, x, a, y, b) if b else sp.diff(r, x, a), "math")
            for px, py in pts:
                ref = f(px, py)
                got = oracle.dr(px, py, 8)[a, b]
                assert got == pytest.approx(ref, rel=1e-11, abs=1e-12 * max(1.0, abs(ref))), (a, b)


@pytest.mark.parametrize("rbf", ["cone", "wendland_c2", "quadratic", "gaussian", "wendland_c6"])
def test_abfs_match_printed_forms(rbf):
    """ABF elements 1-14 against the closed forms printed in Sec. 3.2 and Appendix A:
    elements 1-9 carry the dW0/dr, d2W0/dr2 and d3W0/dr3 brackets, elements 10-14
    only the dW0/dr bracket (truncation rule)."""
    rows = _printed_abfs()
    for x, y in [(0.3, 0.5), (-1.1, 0.4), (0.9, -1.2), (-0.2, -0.35)]:
        r = math.hypot(x, y)
        d = oracle.rbf_derivs(rbf, r)
        ref = np.zeros(14)
        for e, br, expr in rows:
            val = eval(expr, {"__builtins__": {}}, {"x": x, "y": y, "r": r})
            ref[e - 1] += {"d1": d[1], "d2": d[2], "d3": d[3]}[br] * val
        got = oracle.abfs(rbf, x, y, 4)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_abfs_truncated_high_orders_vs_sympy():
    """Elements 15-44 are dW0/dr times d^alpha |r| (Appendix A truncation), checked for the
    Wendland C2 kernel against sympy."""
    sp = pytest.importorskip("sympy")
    X, Y = sp.symbols("x y", real=True)
    R = sp.sqrt(X ** 2 + Y ** 2)
    x, y = 0.41, -0.63
    r = math.hypot(x, y)
    d1 = oracle.rbf_derivs("wendland_c2", r)[1]
    got = oracle.abfs("wendland_c2", x, y, 8)
    for e in range(14, 44):
        n = 1
        while S.p_of_k(n) <= e:
            n += 1
        a = n - (e - S.p_of_k(n - 1))
        b = n - a
        ex = sp.diff(R, X, a, Y, b) if (a and b) else (sp.diff(R, X, a) if a else sp.diff(R, Y, b))
        ref = d1 * float(ex.subs({X: x, Y: y}))
        assert got[e] == pytest.approx(ref, rel=1e-10), e


# ------------------------------------------------------------------------ neighbours


def test_neighbours_vs_kdtree():
    """Brute-force stencils (|r_ji| < 2h, j != i, minimum image) against scipy's kd-tree."""
    from scipy.spatial import cKDTree

    for periodic in (True, False):
        ns = S.jittered_lattice(40, 2.2, 8, seed=5, periodic=periodic)
        rp, col = oracle.neighbours(ns.xy, ns.h, periodic)
        tree = cKDTree(ns.xy, boxsize=1.0 if periodic else None)
        ref = tree.query_ball_point(ns.xy, 2 * ns.h[0] * (1 - 1e-12))
        for i in range(ns.n):
            mine = col[rp[i]:rp[i + 1]]
            assert np.all(np.diff(mine) > 0)  # ascending j
            theirs = sorted(j for j in ref[i] if j != i)
            assert list(mine) == theirs, i


def test_large_set_neighbours_equal_the_brute_force():
    """The kd-tree-proposed stencils for large node sets equal the brute force bit for bit:
    periodic and non-periodic jittered lattices, a node set with ghosts outside the unit square,
    a query subset, and a lattice without jitter (nodes exactly 2h apart sit on the strict
    boundary of the predicate)."""
    q = S.neumann_square(21, 2.0, 4, 0.5, seed=21).ns
    cases = [(S.jittered_lattice(40, 2.2, 8, seed=5), None), (S.jittered_lattice(40, 2.2, 8, seed=6, periodic=False), None),
             (q, None), (S.jittered_lattice(32, 2.0, 4, jitter=0.0, seed=1), None),
             (S.jittered_lattice(48, 2.2, 8, jitter=0.1, seed=7), np.arange(0, 48 * 48, 37))]
    for ns, queries in cases:
        rp, col = oracle.neighbours(ns.xy, ns.h, ns.periodic, ns.lo, ns.hi, queries=queries)
        rp2, col2 = oracle.neighbours_large(ns.xy, ns.h, ns.periodic, ns.lo, ns.hi, queries=queries)
        assert np.array_equal(rp, rp2) and np.array_equal(col, col2)


# ------------------------------------------------------------------------ M, solve, weights


def test_lattice_parity_zeros():
    """On an unperturbed lattice M has exact zeros where X_m W_n is odd in x or y
    (Sec. 3.2: orthogonality of odd and even ABFs and monomials)."""
    ns = S.jittered_lattice(32, 2.5, 8, jitter=0.0, seed=1)
    q = np.array([0, 517])
    rp, col = oracle.neighbours(ns.xy, ns.h, True, queries=q)
    C = S.op_c_vector("dx", 8)[None]
    r = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=8, queries=q, rbf="quadratic", want_mhat=True)
    for M in r["mhat"]:
        scale = np.abs(M).max()
        for m in range(44):
            for n in range(44):
                am, bm = _ab(m)
                an, bn = _ab(n)
                if (am + an) % 2 or (bm + bn) % 2:
                    assert abs(M[m, n]) < 1e-13 * scale, (m, n, M[m, n])


def _ab(e):
    n = 1
    while S.p_of_k(n) <= e:
        n += 1
    a = n - (e - S.p_of_k(n - 1))
    return a, n - a


def test_assembly_and_solve_vs_lapack():
    """M = sum_j X_j (outer) W_j recomputed from the oracle's own X and W with numpy, and
    the elimination result against LAPACK's solve of the same system."""
    ns = S.jittered_lattice(32, 1.8, 6, seed=3)
    q = np.array([5, 300, 777])
    rp, col = oracle.neighbours(ns.xy, ns.h, True, queries=q)
    ops = ("dx", "dy", "lap", "lap3")
    C = np.stack([S.op_c_vector(o, 6) for o in ops])
    r = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=6, queries=q, want_mhat=True)
    for t, i in enumerate(q):
        h = ns.h[i]
        js = col[rp[t]:rp[t + 1]]
        d = ns.xy[js] - ns.xy[i]
        d = np.where(d > 0.5, d - 1, np.where(d < -0.5, d + 1, d)) / h
        X = np.stack([oracle.monomials(a, b, 6) for a, b in d])
        W = np.stack([oracle.abfs("wendland_c2", a, b, 6) for a, b in d])
        M = X.T @ W
        np.testing.assert_allclose(r["mhat"][t], M, rtol=1e-12, atol=1e-13 * np.abs(M).max())
        deg = np.array([sum(_ab(e)) for e in range(27)])
        Chat = C[:, :27] * h ** (-deg)[None, :]
        psi = np.linalg.solve(M, Chat.T)
        w = W @ psi
        wo = r["w"][rp[t]:rp[t + 1]]
        np.testing.assert_allclose(wo, w, rtol=0, atol=1e-9 * np.abs(w).max())


def test_power_of_two_scaling_is_exact():
    """Scaling positions, h and the box by 2 leaves rhat unchanged bit for bit, so the
    weights of an l-th derivative scale by exactly 2^-l (Sec. 3.1: w ~ h^-l)."""
    ns = S.jittered_lattice(24, 1.8, 6, seed=4)
    q = np.arange(0, ns.n, 7)
    ops = ("dx", "lap", "lap3")
    C = np.stack([S.op_c_vector(o, 6) for o in ops])
    rp, col = oracle.neighbours(ns.xy, ns.h, True, queries=q)
    a = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=6, queries=q)
    rp2, col2 = oracle.neighbours(2 * ns.xy, 2 * ns.h, True, lo=(0, 0), hi=(2, 2), queries=q)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    b = oracle.build_weights(2 * ns.xy, 2 * ns.h, True, rp2, col2, C, k=6, queries=q, lo=(0, 0), hi=(2, 2))
    for d, l in enumerate((1, 2, 6)):
        assert np.array_equal(b["w"][:, d] * 2.0 ** l, a["w"][:, d])


@pytest.mark.parametrize("k,hs,rbf,tol", [(2, 1.2, "wendland_c2", 1e-11), (3, 1.4, "gaussian", 1e-11),
                                          (4, 1.6, "quadratic", 1e-11), (5, 1.8, "wendland_c6", 1e-10),
                                          (6, 2.0, "wendland_c2", 1e-9), (7, 2.2, "cone", 1e-8),
                                          (8, 2.5, "wendland_c2", 1e-8)])
def test_polynomial_reproduction(k, hs, rbf, tol):
    """Exact reproduction of polynomials up to degree k (Sec. 3.1): for a random polynomial
    of degree k, sum_j (f_j - f_i) w_ji^d equals C^d . D f at node i to rounding.  The
    tolerance is about 100x the measured FP64 floor of each order; a wrong term anywhere
    in X, M, the solve or the h-scaling gives O(1) errors."""
    xy, h, q = _ghost_lattice(12, hs, 0.25, seed=20 + k)
    rp, col = oracle.neighbours(xy, h, False, *BIG, queries=q)
    ops = ["dx", "dy", "lap"] + (["lap2"] if k >= 4 else [])
    C = np.stack([S.op_c_vector(o, k) for o in ops])
    r = oracle.build_weights(xy, h, False, rp, col, C, k=k, queries=q, rbf=rbf, lo=BIG[0], hi=BIG[1])
    assert np.all(r["status"] == 0)
    coef = S.normal01(100 + k, S.p_of_k(k) + 1)
    terms = [(0, 0)] + [_ab(e) for e in range(S.p_of_k(k))]
    cx, cy = 0.37, 0.61

    def poly_d(px, py):
        out = np.zeros(len(xy))
        for c, (a, b) in zip(coef, terms):
            if px > a or py > b:
                continue
            out += c * math.perm(a, px) * math.perm(b, py) * (xy[:, 0] - cx) ** (a - px) * (xy[:, 1] - cy) ** (b - py)
        return out

    f = poly_d(0, 0)
    out = oracle.apply(rp, col, r["w"], f, queries=q)
    exact = {"dx": poly_d(1, 0), "dy": poly_d(0, 1), "lap": poly_d(2, 0) + poly_d(0, 2),
             "lap2": poly_d(4, 0) + 2 * poly_d(2, 2) + poly_d(0, 4)}
    for d, o in enumerate(ops):
        ex = exact[o][q]
        err = np.linalg.norm(out[d] - ex) / np.linalg.norm(ex)
        # nabla^4 weights scale with h^-4: two more orders of the rounding floor
        assert err < (100 * tol if o == "lap2" else tol), (o, err)


def test_p6_order8_exact_to_rounding():
    """Eq. (p6) with k = 8 and conic ABFs, h/dr = 2.5, ghost strip (Sec. 4.1): the degree-8
    test function is reproduced to rounding.  The error is a rounding floor: the long-double
    build of the same oracle cuts it by more than 100x (the paper quotes ~1e-14 for
    gradients and ~1e-13 for Laplacians, which the long-double build reaches), and so does the
    binary128 build (on every host; its inputs and the exact values are doubles)."""
    f = S.p6_field()
    xy, h, q = _ghost_lattice(16, 2.5, 0.25, seed=11)
    rp, col = oracle.neighbours(xy, h, False, *BIG, queries=q)
    ops = ("dx", "dy", "lap")
    C = np.stack([S.op_c_vector(o, 8) for o in ops])
    errs = {}
    for prec in ("f64", "ld", "q"):
        r = oracle.build_weights(xy, h, False, rp, col, C, k=8, queries=q, rbf="cone",
                                 lo=BIG[0], hi=BIG[1], precision=prec)
        out = oracle.apply(rp, col, r["w"], f.value(xy), queries=q, precision=prec)
        errs[prec] = [np.linalg.norm(out[d] - f.deriv(o, xy[q])) / np.linalg.norm(f.deriv(o, xy[q]))
                      for d, o in enumerate(ops)]
    assert max(errs["f64"][:2]) < 1e-10 and errs["f64"][2] < 1e-9, errs
    assert max(errs["ld"][:2]) < 1e-12 and errs["ld"][2] < 1e-11, errs
    if oracle.mant_bits("ld") > 53:
        assert max(errs["ld"]) < max(errs["f64"]) / 30, errs
    assert oracle.mant_bits("q") == 113
    assert max(errs["q"]) < max(errs["f64"]) / 100, errs


def _slopes(errs, hh):
    return [np.polyfit(np.log(hh), np.log(errs[:, d]), 1)[0] for d in range(errs.shape[1])]


@pytest.mark.parametrize("k,hs,grad_min,lap_min", [(2, 2.0, 1.8, 0.8), (4, 2.0, 3.7, 2.7),
                                                   (6, 2.0, 5.5, 4.6), (8, 2.5, 7.3, 6.5)])
def test_convergence_orders(k, hs, grad_min, lap_min):
    """Sec. 4.1 (Fig. glerror, conic ABFs, h/dr = 2, 2.5 for k = 8): the L2-norm error of
    gradients converges with order k and of the Laplacian with order k - 1 on noisy
    Cartesian nodes, here f = sin(2 pi x) cos(2 pi y) on the periodic unit square."""
    f = S.sincos_field()
    ops = ("dx", "dy", "lap")
    C = np.stack([S.op_c_vector(o, k) for o in ops])
    errs, hh = [], []
    for n_side in (24, 32, 48, 64):
        ns = S.jittered_lattice(n_side, hs, k, jitter=0.25, seed=7)
        q = np.arange(0, ns.n, max(1, ns.n // 1000))
        rp, col = oracle.neighbours(ns.xy, ns.h, True, queries=q)
        r = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=k, queries=q, rbf="cone")
        out = oracle.apply(rp, col, r["w"], f.value(ns.xy), queries=q)
        errs.append([np.linalg.norm(out[d] - f.deriv(o, ns.xy[q])) / np.linalg.norm(f.deriv(o, ns.xy[q]))
                     for d, o in enumerate(ops)])
        hh.append(ns.h[0])
    sl = _slopes(np.array(errs), np.array(hh))
    assert sl[0] > grad_min and sl[1] > grad_min and sl[2] > lap_min, sl


@pytest.mark.parametrize("k,hs,grad_min,lap_min", [(2, 2.0, 1.5, 1.5), (4, 3.0, 3.4, 2.6)])
def test_one_sided_stencils_keep_order(k, hs, grad_min, lap_min):
    """Sec. 4.1 / 4.1: at walls without ghost nodes the stencils are one-sided and, with a
    large enough h/dr, keep the interior order up to k = 4 (gradient ~k, Laplacian ~k-1).
    The error measure is the median over the wall band (the typical stencil): a few
    undersampled one-sided stencils dominate an L2 norm there, which the paper's own
    caveat (h/dr must be large enough at the walls) anticipates."""
    f = S.sincos_field(1.0, 0.5)  # derivatives that do not vanish on the wall
    ops = ("dx", "dy", "lap")
    C = np.stack([S.op_c_vector(o, k) for o in ops])
    errs, hh = [], []
    for n_side in (48, 64, 96, 128, 192):
        ns = S.jittered_lattice(n_side, hs, k, jitter=0.1, seed=9, periodic=False)
        x, y = ns.xy[:, 0], ns.xy[:, 1]
        q = np.nonzero((x < 2 * ns.h[0]) & (y > 0.3) & (y < 0.7))[0]
        rp, col = oracle.neighbours(ns.xy, ns.h, False, queries=q)
        r = oracle.build_weights(ns.xy, ns.h, False, rp, col, C, k=k, queries=q, rbf="cone")
        out = oracle.apply(rp, col, r["w"], f.value(ns.xy), queries=q)
        errs.append([np.median(np.abs(out[d] - f.deriv(o, ns.xy[q]))) / np.sqrt(np.mean(f.deriv(o, ns.xy[q]) ** 2))
                     for d, o in enumerate(ops)])
        hh.append(ns.h[0])
    sl = _slopes(np.array(errs), np.array(hh))
    assert min(sl[0], sl[1]) > grad_min and sl[2] > lap_min, sl


def test_sph_limit():
    """k = 1 collapses to SPH (Sec. 2, Sec. 6): on an unperturbed lattice, w^x_ji tends to
    dV dW_ij/dx with the normalised kernel W = W0/h^2, and the gap shrinks with h/dr.  For
    the printed quadratic kernel (which integrates to 1/2) LABFM matches SPH with twice
    that kernel, as the weights do not depend on a constant factor of W0."""
    def gap(rbf, hs, factor):
        ns = S.jittered_lattice(32, hs, 1, jitter=0.0, seed=1)
        q = np.array([100])
        rp, col = oracle.neighbours(ns.xy, ns.h, True, queries=q)
        r = oracle.build_weights(ns.xy, ns.h, True, rp, col, S.op_c_vector("dx", 1)[None], k=1, queries=q, rbf=rbf)
        j = col[rp[0]:rp[1]]
        d = ns.xy[j] - ns.xy[q[0]]
        d = np.where(d > 0.5, d - 1, np.where(d < -0.5, d + 1, d))
        h = ns.h[0]
        qq = np.hypot(d[:, 0], d[:, 1]) / h
        d1 = np.array([oracle.rbf_derivs(rbf, v)[1] for v in qq]) * factor
        wsph = -(ns.s[0] ** 2) * d1 * (d[:, 0] / h) / qq / h ** 3
        w = r["w"][:, 0]
        return np.linalg.norm(w - wsph) / np.linalg.norm(wsph)

    g = [gap("wendland_c2", hs, 1.0) for hs in (1.0, 1.5, 2.5, 4.0)]
    assert all(a > b for a, b in zip(g, g[1:])), g
    assert g[-1] < 1e-4, g
    gq = [gap("quadratic", hs, 2.0) for hs in (1.5, 4.0)]
    assert gq[1] < gq[0] and gq[1] < 1e-2, gq


def test_status_undersampled_and_collinear():
    """Per-node failure is reported, not hidden: a stencil with fewer neighbours than p
    makes M rank deficient (M is a sum of N_i rank-one terms, Eq. disc_form), and a
    stencil whose neighbours are all collinear with i has identically zero y-monomial
    rows; both get a status code and zero weights."""
    # undersampled: fewer neighbours than p -> status 2, zero weights
    xy = np.array([[0.5, 0.5], [0.52, 0.5], [0.5, 0.53], [0.47, 0.49]])
    h = np.full(4, 0.05)
    rp, col = oracle.neighbours(xy, h, False, *BIG, queries=np.array([0]))
    r = oracle.build_weights(xy, h, False, rp, col, S.op_c_vector("dx", 2)[None], k=2,
                             queries=np.array([0]), lo=BIG[0], hi=BIG[1])
    assert r["status"][0] == oracle.ST_UNDERSAMPLED and np.all(r["w"] == 0)
    # collinear: every neighbour on the line y = y_i -> the y-monomial rows of M vanish
    xs = np.linspace(0.3, 0.7, 21)
    xy = np.stack([xs, np.full_like(xs, 0.5)], 1)
    h = np.full(xs.size, 0.06)
    q = np.array([10])
    rp, col = oracle.neighbours(xy, h, False, *BIG, queries=q)
    r = oracle.build_weights(xy, h, False, rp, col, S.op_c_vector("dx", 2)[None], k=2, queries=q,
                             lo=BIG[0], hi=BIG[1])
    assert r["status"][0] == oracle.ST_SINGULAR and np.all(r["w"] == 0)


def test_rk4_linear_system_is_taylor_polynomial():
    """Classical RK4 (Sec. 5.1) on the linear system du/dt = A u advances by the degree-4
    Taylor polynomial of exp(dt A)."""
    ns = S.jittered_lattice(8, 1.4, 2, seed=2)
    rp, col = oracle.neighbours(ns.xy, ns.h, True)
    ops = ("dx", "dy", "lap")
    C = np.stack([S.op_c_vector(o, 2) for o in ops])
    r = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=2)
    beta = np.array([-1.0, -0.5, 1e-3])
    n = ns.n
    A = np.zeros((n, n))
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            wsum = float(r["w"][e] @ beta)
            A[i, col[e]] += wsum
            A[i, i] -= wsum
    u0 = S.sincos_field().value(ns.xy)
    dt = 2e-3
    Z = dt * A
    P = np.eye(n) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    ref = np.linalg.matrix_power(P, 3) @ u0
    got = oracle.rk4(rp, col, r["w"], beta, u0, dt, 3)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    # frozen (Dirichlet) nodes keep their value: du/dt = 0 there, i.e. their rows of A vanish,
    # in every stage -- the step is then the Taylor polynomial of the row-zeroed matrix
    fz = np.zeros(n, dtype=np.uint8)
    fz[::5] = 1
    got2 = oracle.rk4(rp, col, r["w"], beta, u0, dt, 3, frozen=fz)
    assert np.array_equal(got2[::5], u0[::5])
    Zf = Z.copy()
    Zf[fz.astype(bool)] = 0.0
    Pf = np.eye(n) + Zf + Zf @ Zf / 2 + Zf @ Zf @ Zf / 6 + Zf @ Zf @ Zf @ Zf / 24
    np.testing.assert_allclose(got2, np.linalg.matrix_power(Pf, 3) @ u0, rtol=0, atol=1e-13)


# ------------------------------------------------------------------------ ABF forms, stability


@pytest.mark.parametrize("rbf", ["cone", "wendland_c2", "quadratic", "gaussian", "wendland_c6"])
def test_abfs_dw0_form_is_the_printed_dW0_bracket(rbf):
    """abf_form "dw0" (every element truncated to dW0/dr d^alpha|r|): elements 1-14 equal dW0/dr
    times the printed dW0/dr bracket of Sec. 3.2 / Appendix A, for every kernel."""
    rows = [r for r in _printed_abfs() if r[1] == "d1"]
    assert sorted(e for e, _, _ in rows) == list(range(1, 15))
    for x, y in [(0.3, 0.5), (-1.1, 0.4), (0.9, -1.2), (-0.2, -0.35)]:
        r = math.hypot(x, y)
        d1 = oracle.rbf_derivs(rbf, r)[1]
        ref = np.zeros(14)
        for e, _, expr in rows:
            ref[e - 1] = d1 * eval(expr, {"__builtins__": {}}, {"x": x, "y": y, "r": r})
        got = oracle.abfs(rbf, x, y, 4, abf_form="dw0")
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
        # elements >= 10 are the same in both forms
        np.testing.assert_array_equal(oracle.abfs(rbf, x, y, 8, abf_form="dw0")[9:],
                                      oracle.abfs(rbf, x, y, 8)[9:])


def _global_matrix(n, rp, col, w):
    """A with (A f)_i = sum_j (f_j - f_i) w_ji (the global derivative matrix of Sec. 4.2)."""
    A = np.zeros((n, n))
    node = np.repeat(np.arange(n), np.diff(rp))
    np.add.at(A, (node, col), w)
    np.add.at(A, (node, node), -w)
    return A


def _spectrum(k, hdr, rbf, form, jitter, op, seed=5, n_side=21):
    ns = S.jittered_lattice(n_side, hdr, k, jitter=jitter, seed=seed)
    rp, col = oracle.neighbours(ns.xy, ns.h, True)
    w = oracle.build_weights(ns.xy, ns.h, True, rp, col, S.op_c_vector(op, k)[None, :], k=k, rbf=rbf,
                             abf_form=form)["w"][:, 0]
    return np.linalg.eigvals(_global_matrix(ns.n, rp, col, w)), ns.h[0]


def _noise_limits():
    out = []
    with open(os.path.join(GOLD, "paper_numbers.txt")) as fh:
        for line in fh:
            if line.startswith("noise_limit_quadratic"):
                _, k, hdr, lim = line.split()
                out.append((int(k), float(hdr), float(lim)))
    return out


@pytest.mark.parametrize("k,hdr,limit", _noise_limits())
def test_laplacian_noise_limits_dw0_form(k, hdr, limit):
    """Sec. 4.2, Table of noise limits: with the quadratic ABFs the Laplacian has no growing mode
    for noise below the printed limit.  Checked at half the limit (at most 0.5 dr of displacement;
    each coordinate uniform in +-eps/sqrt(2), so no node moves further than eps) on two node sets:
    the largest real part of the spectrum stays at rounding level."""
    eps = min(0.5, limit / 2)
    for seed in (5, 6):
        lam, h = _spectrum(k, hdr, "quadratic", "dw0", eps / math.sqrt(2), "lap", seed=seed)
        assert lam.real.max() * h * h < 1e-10, (seed, lam.real.max() * h * h)
        assert lam.real.min() * h * h < -1.0  # the operator does damp


def test_chain_form_breaks_the_noise_limits():
    """The same points with the chain-rule terms kept in elements 1-9 (Appendix A as printed)
    have modes that grow at rates far above rounding level: the stability results of Sec. 4.2
    are those of the dW0/dr-only form.  (Records why both forms exist.)"""
    for k, hdr, limit in _noise_limits():
        eps = min(0.5, limit / 2)
        lam, h = _spectrum(k, hdr, "quadratic", "chain", eps / math.sqrt(2), "lap")
        assert lam.real.max() * h * h > 0.1, (k, hdr)


def test_convective_spectrum_on_a_regular_lattice():
    """Sec. 4.2 (eigenvalues of the convective operator, regular lattice, h/dr = 2): the
    real parts are at rounding level for the quadratic and Wendland ABFs, larger by orders of
    magnitude (yet small) for the Gaussian, and substantial for the cone, whose dW0/dr does not
    vanish at q = 2.  At h/dr = 2 lattice neighbours sit on the support edge, so only kernels
    whose ABFs vanish there give a skew-symmetric operator."""
    def ratio(rbf, k, form="dw0"):
        lam, _ = _spectrum(k, 2.0, rbf, form, 0.0, "dx")
        return np.abs(lam.real).max() / np.abs(lam).max()
    for k in (2, 4, 6):
        assert ratio("quadratic", k) < 1e-13
        assert ratio("wendland_c2", k) < 1e-13
        assert ratio("wendland_c6", k) < 1e-13
        assert ratio("gaussian", k) < 1e-6
        assert ratio("cone", k) > 1e-2
    assert ratio("gaussian", 6) > 1e3 * ratio("quadratic", 6)
    # the chain-rule form with the quadratic kernel does not have this property (d2W0/dq2 != 0 at q = 2)
    assert ratio("quadratic", 4, form="chain") > 0.1


# ------------------------------------------------------------- heat equation (Sec. 5.1)


def _heat_table():
    rows = {}
    with open(os.path.join(GOLD, "paper_numbers.txt")) as fh:
        for line in fh:
            if line.startswith("heat_steady_l2"):
                _, k, hH, err, rate = line.split()
                rows.setdefault(int(k), []).append((float(hH), float(err), None if rate == "-" else float(rate)))
    return rows


def heat_steady_errors(k, levels, seed):
    """Oracle steady states of the Dirichlet heat problem of Sec. 5.1 (quadratic ABFs in the
    dW0/dr form, h/dr = 2, interior noise eps/dr = 0.5) at the given h/H, as relative L2 errors
    against sinh(pi (1 - y)) sin(pi x) / sinh(pi) over all nodes."""
    field = S.HeatSteadyField()
    errs = []
    for hH in levels:
        ns = S.dirichlet_square(int(round(2.0 / hH)) + 1, 2.0, k, 0.5, seed=seed)
        rp, col = oracle.neighbours(ns.xy, ns.h, False)
        r = oracle.build_weights(ns.xy, ns.h, False, rp, col, S.op_c_vector("lap", k)[None, :], k=k,
                                 rbf="quadratic", abf_form="dw0")
        assert (r["status"] == 0).all()
        u = oracle.steady_state(rp, col, r["w"], [1.0], field.boundary(ns.xy, ns.wall), ns.wall)
        ex = field.value(ns.xy)
        errs.append(np.linalg.norm(u - ex) / np.linalg.norm(ex))
    return np.array(errs)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_heat_steady_state_table(k):
    """Sec. 5.1, Table of steady-state errors (inhomogeneous Dirichlet walls): the oracle's
    errors at h/H = 0.2 ... 0.025 fall at the printed rates (k = 2, 4: each rate within 0.7 of
    the printed one; k = 3, whose printed rates drift from 3.1 to 2.1: each within [2, 3.6])
    and lie within a factor 5 of the printed errors (the node sets are random draws of the same
    distribution, not the paper's; over six draws the rates stay within 0.56 of the printed ones
    and the errors are 1.1-3.8 times the printed ones)."""
    rows = _heat_table()[k][:4]
    levels = [r[0] for r in rows]
    errs = heat_steady_errors(k, levels, seed=100 + k)
    rates = np.log2(errs[:-1] / errs[1:])
    printed = np.array([r[2] for r in rows[1:]])
    if k == 3:
        assert np.all((rates >= 2.0) & (rates <= 3.6)), rates
    else:
        assert np.all(np.abs(rates - printed) <= 0.7), (rates, printed)
    ratio = errs / np.array([r[1] for r in rows])
    assert np.all((ratio > 0.2) & (ratio < 5.0)), ratio


def test_heat_frozen_rk4_reaches_the_steady_state():
    """RK4 with the wall nodes frozen at their prescribed values (Sec. 5.1), run from zero
    interior values to t* = 8 pi^2 t = 100, lands on the sparse direct solution of the same
    semi-discrete steady problem: two independent routes to one answer."""
    k = 4
    ns = S.dirichlet_square(11, 2.0, k, 0.5, seed=104)
    rp, col = oracle.neighbours(ns.xy, ns.h, False)
    w = oracle.build_weights(ns.xy, ns.h, False, rp, col, S.op_c_vector("lap", k)[None, :], k=k,
                             rbf="quadratic", abf_form="dw0")["w"]
    ub = S.HeatSteadyField().boundary(ns.xy, ns.wall)
    uss = oracle.steady_state(rp, col, w, [1.0], ub, ns.wall)
    dt = 0.05 * ns.h[0] ** 2  # Sec. 5.1: 0.05 h^2 / kappa, kappa = 1
    nsteps = int(math.ceil(100.0 / (8.0 * math.pi ** 2) / dt))
    u = oracle.rk4(rp, col, w, np.array([1.0]), ub, dt, nsteps, frozen=ns.wall.astype(np.uint8))
    assert np.array_equal(u[ns.wall], ub[ns.wall])
    assert np.abs(u - uss).max() < 1e-9 * np.abs(uss).max()


# --------------------------------------------------------- Burgers' equation (Sec. 5.3)


def test_cole_solution_solves_burgers():
    """The exact solution used for the periodic Burgers' problem: u(x, 0) = sin(2 pi x), the
    printed truncation (A_n < 1e-16 for n >= 30 at Re = 100), and the PDE
    u_t + u u_x = u_xx / Re itself by central differences at points across the steepening front,
    relative to the size of its terms (the series loses ~7 digits to cancellation near x = 1/2,
    where the denominator is ~e^-2z; the printed decay factor, 4 times smaller, leaves a
    residual of the order of the terms)."""
    sol = S.ColeBurgersSolution(Re=100.0)
    x = np.linspace(0.0, 1.0, 41)
    assert np.abs(sol.u(x, 0.0) - np.sin(2 * np.pi * x)).max() < 1e-9
    assert np.all(sol.An[29:] < 1e-16) and sol.An[0] > 1e-3
    d = 1e-4
    for t in (0.1, 0.3, 0.6):
        xs = np.array([0.05, 0.21, 0.4, 0.47, 0.55, 0.8])
        ut = (sol.u(xs, t + d) - sol.u(xs, t - d)) / (2 * d)
        ux = (sol.u(xs + d, t) - sol.u(xs - d, t)) / (2 * d)
        uxx = (sol.u(xs + d, t) - 2 * sol.u(xs, t) + sol.u(xs - d, t)) / d ** 2
        scale = np.abs(ut) + np.abs(sol.u(xs, t) * ux) + np.abs(uxx / 100.0)
        assert np.all(np.abs(ut + sol.u(xs, t) * ux - uxx / 100.0) <= 1e-3 * scale + 1e-6), t


def _burgers_error(k, nside, T, Re=100.0, eps=0.2, seed=7):
    ns = S.jittered_lattice(nside, 2.0, k, jitter=eps / math.sqrt(2), seed=seed)
    rp, col = oracle.neighbours(ns.xy, ns.h, True)
    C = np.stack([S.op_c_vector(o, k) for o in ("dx", "dy", "lap")])
    w = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=k, rbf="quadratic", abf_form="dw0")["w"]
    h = ns.h[0]
    dt = min(0.2 * h / 1.0, 0.05 * h * h * Re)  # Eq. (tstep), max|u| = 1
    nsteps = int(math.ceil(T / dt))
    u0 = np.sin(2 * np.pi * ns.xy[:, 0])
    u, v = oracle.rk4_burgers(rp, col, w, [0.0, 0.0, 1.0 / Re], u0, np.zeros(ns.n), T / nsteps, nsteps)
    ex = S.ColeBurgersSolution(Re).u(ns.xy[:, 0], T)
    return np.linalg.norm(u - ex) / np.linalg.norm(ex), np.abs(v).max()


def test_burgers_quick_convergence():
    """The periodic Burgers' problem at k = 4 between h/H = 2/41 and 2/81 (t = 0.4): rate 4.06,
    band [3.5, 4.6], and v stays exactly 0 (a cheap form of the pin below)."""
    e1, v1 = _burgers_error(4, 41, 0.4)
    e2, v2 = _burgers_error(4, 81, 0.4)
    rate = math.log(e1 / e2) / math.log(81 / 41)
    assert 3.5 <= rate <= 4.6, (e1, e2, rate)
    assert v1 == 0.0 and v2 == 0.0


def test_cole_hopf_2d_solves_burgers():
    """The two-dimensional Cole-Hopf solution satisfies both components of
    u_t + (u . grad) u = nabla^2 u / Re (central differences, relative to the size of the terms)."""
    sol = S.ColeHopf2DSolution(Re=10.0, a=0.5)
    pts = np.array([[0.1, 0.2], [0.37, 0.61], [0.5, 0.5], [0.83, 0.12], [0.66, 0.9]])
    d, t = 1e-4, 0.1
    ex, ey = np.array([[d, 0.0]]), np.array([[0.0, d]])
    U = lambda p, tt: np.stack(sol.uv(p, tt))  # [2, npts]
    ut = (U(pts, t + d) - U(pts, t - d)) / (2 * d)
    ux = (U(pts + ex, t) - U(pts - ex, t)) / (2 * d)
    uy = (U(pts + ey, t) - U(pts - ey, t)) / (2 * d)
    lap = (U(pts + ex, t) + U(pts - ex, t) + U(pts + ey, t) + U(pts - ey, t) - 4 * U(pts, t)) / d ** 2
    u, v = sol.uv(pts, t)
    res = ut + u * ux + v * uy - lap / 10.0
    scale = np.abs(ut) + np.abs(u * ux) + np.abs(v * uy) + np.abs(lap / 10.0)
    assert np.all(np.abs(res) <= 1e-5 * scale + 1e-9), res
    assert np.abs(u).max() > 0.1 and np.abs(v).max() > 0.1


def _burgers_2d_error(k, nside, T, Re=10.0, eps=0.2, seed=8):
    ns = S.jittered_lattice(nside, 2.0, k, jitter=eps / math.sqrt(2), seed=seed)
    rp, col = oracle.neighbours(ns.xy, ns.h, True)
    C = np.stack([S.op_c_vector(o, k) for o in ("dx", "dy", "lap")])
    w = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=k, rbf="quadratic", abf_form="dw0")["w"]
    sol = S.ColeHopf2DSolution(Re=Re)
    u0, v0 = sol.uv(ns.xy, 0.0)
    h = ns.h[0]
    nsteps = int(math.ceil(T / min(0.2 * h / 1.0, 0.05 * h * h * Re)))
    u, v = oracle.rk4_burgers(rp, col, w, [0.0, 0.0, 1.0 / Re], u0, v0, T / nsteps, nsteps)
    eu, ev = sol.uv(ns.xy, T)
    return math.sqrt(np.sum((u - eu) ** 2 + (v - ev) ** 2) / np.sum(eu ** 2 + ev ** 2))


def test_burgers_2d_convergence():
    """Burgers' equation with both velocity components active (the Cole-Hopf solution above,
    Re = 10, k = 4): RK4 of the oracle's discrete system converges at order ~k between h/H = 2/21
    and 2/41 (t = 0.1), band [3.3, 5] (measured 3.8; 2.0 and 5.6 at k = 2 and 6, and 4.0, 2.0, 6.1
    between 2/41 and 2/81)."""
    e1, e2 = _burgers_2d_error(4, 21, 0.1), _burgers_2d_error(4, 41, 0.1)
    rate = math.log(e1 / e2) / math.log(41 / 21)
    assert 3.3 <= rate <= 5.0, (e1, e2, rate)


def test_burgers_periodic_convergence():
    """Sec. 5.3, periodic Burgers' problem at Re = 100 (quadratic ABFs in the dW0/dr form,
    h/dr = 2, eps/dr = 0.2, RK4 with the time step of Eq. (tstep)): at t = 0.4, as the front
    steepens, the error against Cole's solution falls between h/H = 2/81 and 2/161 at rates near
    k (the paper: between k - 1 and k; measured 2.8, 3.9, 5.7 for k = 2, 4, 6), and v stays 0."""
    bands = {2: (1.5, 3.5), 4: (3.0, 4.8), 6: (5.0, 6.8)}
    for k, (lo, hi) in bands.items():
        e1, v1 = _burgers_error(k, 81, 0.4)
        e2, v2 = _burgers_error(k, 161, 0.4)
        rate = math.log(e1 / e2) / math.log(161 / 81)
        assert lo <= rate <= hi, (k, e1, e2, rate)
        assert v1 == 0.0 and v2 == 0.0


# ------------------------------------------------------------ Poisson's equation (Sec. 5.2)


def poisson_periodic_error(k, nside, hdr, seed=3, eps=0.5):
    """Periodic Poisson problem of Sec. 5.2 (phi = sin 2 pi x sin 2 pi y, quadratic ABFs in the
    dW0/dr form): the global system A^L Phi = F by the oracle's direct solve, with node 0 held
    at its exact value to fix the constant of the periodic null space."""
    ns = S.jittered_lattice(nside, hdr, k, jitter=eps / math.sqrt(2), seed=seed)
    rp, col = oracle.neighbours(ns.xy, ns.h, True)
    w = oracle.build_weights(ns.xy, ns.h, True, rp, col, S.op_c_vector("lap", k)[None, :], k=k, rbf="quadratic",
                             abf_form="dw0")["w"]
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    ex = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    f = -8 * np.pi ** 2 * ex
    dm = np.zeros(ns.n, np.uint8)
    dm[0] = 1
    f[0] = ex[0]
    phi = oracle.solve_operator(rp, col, w, 0, f, dm)
    return np.linalg.norm(phi - ex) / np.linalg.norm(ex)


def test_global_matrix_and_direct_solve_vs_apply():
    """The global matrix of Sec. 5.2 (eq. poisson_system) against the oracle's stencil apply
    (Eq. general_do), an independent code path: (A u)_i = sum_d beta_d sum_j (u_j - u_i) w_ji^d
    for three operators and a random beta; and the direct solve of operator 2 (the Laplacian)
    with two Dirichlet rows satisfies L^2(phi)_i = f_i off those rows (residual through the
    apply) and phi_b = f_b on them.  A transposed matrix, a wrong diagonal, an ignored beta or
    operator index, or dropped Dirichlet rows each fail here."""
    k = 2
    ns = S.jittered_lattice(16, 2.0, k, jitter=0.2, seed=11)
    rp, col = oracle.neighbours(ns.xy, ns.h, True)
    C = np.stack([S.op_c_vector(o, k) for o in ("dx", "dy", "lap")])
    r = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=k, rbf="quadratic", abf_form="dw0")
    assert (r["status"] == 0).all()
    w = r["w"]
    rng = np.random.default_rng(5)
    beta, u = rng.standard_normal(3), rng.standard_normal(ns.n)
    ref = beta @ oracle.apply(rp, col, w, u)
    got = oracle.operator_matrix(rp, col, w, beta) @ u
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    f = rng.standard_normal(ns.n)
    dm = np.zeros(ns.n, np.uint8)
    dm[[0, 37]] = 1
    phi = oracle.solve_operator(rp, col, w, 2, f, dm)
    free = dm == 0
    lap = oracle.apply(rp, col, w, phi)[2]
    assert np.abs(lap[free] - f[free]).max() <= 1e-9 * np.abs(f).max()
    assert np.abs(phi[~free] - f[~free]).max() <= 1e-12 * np.abs(f).max()


def test_poisson_periodic_even_order_pattern():
    """Sec. 5.2, periodic test case: the solution converges at order 2 for k = 2 and 3, 4 for
    k = 4 and 5, and 8 for k = 8 (h/dr = 3 there): odd k gives the order of k - 1.  Rates from
    h/H = 2/20 to 2/80 (overall), noise eps/dr = 0.5; bands from the printed orders (k = 4 reads
    3.3 - 4.8 across node draws, single stencils set the finest errors)."""
    bands = {2: (1.8, 2.3), 3: (1.8, 2.3), 4: (3.3, 5.0), 5: (3.6, 4.4), 8: (7.0, 9.5)}
    for k, (lo, hi) in bands.items():
        hdr = 2.0 if k <= 6 else 3.0
        e20, e80 = poisson_periodic_error(k, 20, hdr), poisson_periodic_error(k, 80, hdr)
        rate = math.log2(e20 / e80) / 2.0
        assert lo <= rate <= hi, (k, e20, e80, rate)


# a polynomial of degree 4 as {(a, b): coefficient of x^a y^b}
NEUMANN_POLY = {(0, 0): 0.3, (1, 0): 1.0, (0, 1): -0.7, (2, 0): 0.5, (1, 1): -1.1, (0, 2): 0.8, (3, 0): 0.2,
                (2, 1): -0.4, (0, 3): 0.6, (4, 0): 0.9, (2, 2): -0.3, (1, 3): 0.5, (0, 4): -0.7}


def _poly_eval(c, x, y, dx=0, dy=0):
    """sum c_ab d^dx/dx d^dy/dy (x^a y^b), by the power rule"""
    out = np.zeros_like(x)
    for (a, b), v in c.items():
        if a < dx or b < dy:
            continue
        fa = math.factorial(a) // math.factorial(a - dx)
        fb = math.factorial(b) // math.factorial(b - dy)
        out = out + v * fa * fb * x ** (a - dx) * y ** (b - dy)
    return out


def neumann_problem(nside, k, field, rbf="quadratic", seed=21):
    """Poisson's equation on the Neumann square (Dirichlet walls at x = 0, 1; Neumann walls with
    ghost nodes at y = 0, 1): the oracle's stencils and weights of (d/dx, d/dy, nabla^2), and the
    right-hand side F for the exact solution `field` = (phi, phi_x, phi_y, lap phi) as functions
    of (x, y): nabla^2 phi in the Poisson rows, phi in the Dirichlet rows, n . grad phi at the
    parent in the ghost rows."""
    q = S.neumann_square(nside, 2.0, k, 0.5, seed=seed)
    ns = q.ns
    rp, col = oracle.neighbours(ns.xy, ns.h, False, ns.lo, ns.hi)
    C = np.stack([S.op_c_vector(o, k) for o in ("dx", "dy", "lap")])
    r = oracle.build_weights(ns.xy, ns.h, False, rp, col, C, k=k, rbf=rbf, abf_form="dw0", lo=ns.lo, hi=ns.hi)
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    phi, phx, phy, lap = field
    ex = phi(x, y)
    f = np.where(q.dirichlet, ex, lap(x, y))
    xb, yb = x[q.parent], y[q.parent]
    f[q.ghost] = q.normal[:, 0] * phx(xb, yb) + q.normal[:, 1] * phy(xb, yb)
    return q, rp, col, r, ex, f


def _neumann_poly_field():
    c = NEUMANN_POLY
    return (lambda x, y: _poly_eval(c, x, y), lambda x, y: _poly_eval(c, x, y, 1, 0),
            lambda x, y: _poly_eval(c, x, y, 0, 1),
            lambda x, y: _poly_eval(c, x, y, 2, 0) + _poly_eval(c, x, y, 0, 2))


def test_poisson_neumann_ghost_rows_reproduce_polynomials():
    """The Neumann ghost-node rows of Sec. 5.2 with k = 4 on a 21^2 square (Dirichlet walls at
    x = 0, 1, Neumann walls at y = 0, 1 with one ghost per wall node): for a polynomial phi of
    degree 4 every local operator is exact (polynomial reproduction, Sec. 3.1), so the exact
    nodal values, ghosts included, satisfy every row of the enlarged system; its solution must
    be phi itself.  A ghost row with its diagonal on the ghost instead of the parent, a normal
    with the wrong sign or a dropped component, or rows left out all break it."""
    q, rp, col, r, ex, f = neumann_problem(21, 4, _neumann_poly_field())
    interior = np.ones(q.ns.n, bool)
    interior[q.ghost] = False
    assert (r["status"][interior] == 0).all()
    phi = oracle.solve_operator(rp, col, r["w"], 2, f, q.dirichlet.astype(np.uint8),
                                neumann=(q.ghost, q.parent, q.normal, 0, 1))
    err = np.abs(phi - ex).max() / np.abs(ex).max()
    assert err < 1e-9, err


def test_poisson_neumann_convergence():
    """Sec. 5.2's Neumann treatment is consistent with the order of the discretisation: for
    phi = sin(2x + 0.3) cos(3y - 0.2) (nonzero normal derivative on both Neumann walls) the
    solution error falls at least as h^(k - 1) from 21^2 to 41^2 nodes at k = 4 (one-sided
    stencils at the walls)."""
    field = (lambda x, y: np.sin(2 * x + 0.3) * np.cos(3 * y - 0.2),
             lambda x, y: 2 * np.cos(2 * x + 0.3) * np.cos(3 * y - 0.2),
             lambda x, y: -3 * np.sin(2 * x + 0.3) * np.sin(3 * y - 0.2),
             lambda x, y: -13 * np.sin(2 * x + 0.3) * np.cos(3 * y - 0.2))
    errs = []
    for nside in (21, 41):
        q, rp, col, r, ex, f = neumann_problem(nside, 4, field)
        phi = oracle.solve_operator(rp, col, r["w"], 2, f, q.dirichlet.astype(np.uint8),
                                    neumann=(q.ghost, q.parent, q.normal, 0, 1))
        keep = np.ones(q.ns.n, bool)
        keep[q.ghost] = False
        errs.append(np.linalg.norm(phi[keep] - ex[keep]) / np.linalg.norm(ex[keep]))
    rate = math.log2(errs[0] / errs[1])
    assert rate >= 3.0, (errs, rate)


def _annulus_table():
    out = {}
    for line in open(os.path.join(GOLD, "paper_numbers.txt")):
        if line.startswith("poisson_annulus_l2"):
            _, k, m, err, rate = line.split()
            out.setdefault(int(k), []).append((int(m), float(err), None if rate == "-" else float(rate)))
    return out


annulus_phi, annulus_source = S.annulus_solution, S.annulus_source


def annulus_problem(m, k, seed=31):
    """The annulus of labfm_synth.annulus_nodes with the oracle's stencils and weights of (d/dx,
    d/dy, nabla^2), and F: the printed source in the Poisson rows, g1 = 0 on the outer circle,
    g2 = cos(3 theta) at the parent of each inner-circle ghost."""
    q = S.annulus_nodes(m, k, seed=seed)
    ns = q.ns
    rp, col = oracle.neighbours_large(ns.xy, ns.h, False, ns.lo, ns.hi)
    C = np.stack([S.op_c_vector(o, k) for o in ("dx", "dy", "lap")])
    r = oracle.build_weights(ns.xy, ns.h, False, rp, col, C, k=k, rbf="quadratic", abf_form="dw0", lo=ns.lo, hi=ns.hi)
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    f = np.where(q.dirichlet, 0.0, annulus_source(x, y))
    f[q.ghost] = np.cos(3 * np.arctan2(y[q.parent], x[q.parent]))
    return q, rp, col, r, annulus_phi(x, y), f


def annulus_error(m, k, seed=31):
    q, rp, col, r, ex, f = annulus_problem(m, k, seed)
    keep = np.ones(q.ns.n, bool)
    keep[q.ghost] = False
    assert (r["status"][keep] == 0).all()
    phi = oracle.solve_operator(rp, col, r["w"], 2, f, q.dirichlet.astype(np.uint8),
                                neumann=(q.ghost, q.parent, q.normal, 0, 1))
    return np.linalg.norm(phi[keep] - ex[keep]) / np.linalg.norm(ex[keep])


def test_annulus_source_is_the_laplacian_of_the_solution():
    """The printed source term of the annular problem is nabla^2 of the printed solution
    (central differences in x and y), and the printed Neumann data cos(3 theta) is its radial
    derivative on the inner circle r = 1/8."""
    rng = np.random.default_rng(3)
    rr, th = rng.uniform(0.13, 0.49, 50), rng.uniform(0, 2 * np.pi, 50)
    x, y, d = rr * np.cos(th), rr * np.sin(th), 1e-4
    lap = (annulus_phi(x + d, y) + annulus_phi(x - d, y) + annulus_phi(x, y + d) + annulus_phi(x, y - d)
           - 4 * annulus_phi(x, y)) / d ** 2
    assert np.abs(lap - annulus_source(x, y)).max() < 1e-5 * np.abs(annulus_source(x, y)).max()
    r0 = 0.125
    dphi = (annulus_phi((r0 + d) * np.cos(th), (r0 + d) * np.sin(th)) -
            annulus_phi((r0 - d) * np.cos(th), (r0 - d) * np.sin(th))) / (2 * d)
    assert np.abs(dphi - np.cos(3 * th)).max() < 1e-6


@pytest.mark.parametrize("k", [2, 3, 4])
def test_poisson_annulus_table(k):
    """Sec. 5.2, Table of the annular Poisson problem (Dirichlet outer circle, Neumann inner
    circle through ghost-node rows, quadratic ABFs, h/dr = 2, nodes built by the paper's shifting
    rule): the oracle's errors at h/H = 2/25, 2/49, 2/97.  k = 2, 3: each error within 25 % of the
    printed one and the last rate within 0.15 of the printed (measured over five node draws:
    errors 0.94-1.05 of the printed, rates 1.97-2.00 against 1.98 and 2.01); k = 4, whose coarse
    levels depend on the draw: the errors at 2/49 and 2/97 within a factor 4 of the printed ones
    and the rate from 2/25 to 2/97 at least 3.5 (printed 4.9)."""
    rows = [r for r in _annulus_table()[k] if r[0] in (25, 49, 97)]
    errs = np.array([annulus_error(m, k) for m, _, _ in rows])
    printed = np.array([e for _, e, _ in rows])
    if k in (2, 3):
        assert np.all(np.abs(errs / printed - 1) <= 0.25), (errs, printed)
        rate = math.log(errs[1] / errs[2]) / math.log(97 / 49)
        assert abs(rate - rows[2][2]) <= 0.15, rate
    else:
        ratio = errs[1:] / printed[1:]
        assert np.all((ratio > 0.25) & (ratio < 4.0)), ratio
        assert math.log(errs[0] / errs[2]) / math.log(97 / 25) >= 3.5, errs
