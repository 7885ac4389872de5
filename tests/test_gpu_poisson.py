"""Implicit solves (Sec. 5.2): labfm_solve's Jacobi-preconditioned BiCGStab on the global operator
matrix against the oracle's sparse direct solve of the same system, periodic (one node fixed) and
with Dirichlet walls, and the even-order convergence pattern of the periodic Poisson problem."""
import math

import numpy as np
import pytest

import labfm_synth as S
import oracle
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1912_06441_gb300 as P

    P.load_library()


def _periodic_problem(k, nside, hdr=2.0, eps=0.5, seed=3, weight_dtype="f64"):
    ns = S.jittered_lattice(nside, hdr, k, jitter=eps / math.sqrt(2), seed=seed)
    L, rp, col, w, status, _ = G.gpu_run(ns, k, ("lap",), rbf="quadratic", abf_form="dw0", weight_dtype=weight_dtype)
    assert (status == 0).all()
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    ex = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    f = -8 * np.pi ** 2 * ex
    dm = np.zeros(ns.n, np.uint8)
    dm[0] = 1
    f[0] = ex[0]
    return ns, L, ex, f, dm


def _gpu_solve(L, f, dm, tol=1e-13, max_iter=20000):
    import torch

    dev = torch.device("cuda", 0)
    phi = torch.zeros(len(f), dtype=torch.float64, device=dev)
    iters, resid = L.solve(0, torch.from_numpy(f).to(dev), phi, torch.from_numpy(dm).to(dev), tol=tol,
                           max_iter=max_iter)
    return phi.cpu().numpy(), iters, resid


def _oracle_solve(ns, k, f, dm):
    rp, col = oracle.neighbours(ns.xy, ns.h, ns.periodic, ns.lo, ns.hi)
    w = oracle.build_weights(ns.xy, ns.h, ns.periodic, rp, col, G.c_matrix(k, ("lap",)), k=k, rbf="quadratic",
                             abf_form="dw0", lo=ns.lo, hi=ns.hi)["w"]
    return oracle.solve_operator(rp, col, w, 0, f, dm)


@pytest.mark.parametrize("weight_dtype", ["f64", "f32"])
def test_poisson_periodic_matches_oracle(weight_dtype):
    """k = 4, 40^2 nodes, node 0 fixed: BiCGStab to a relative residual of 1e-13 equals the
    oracle's direct solution on the oracle's weights to 1e-8 (FP64 weights; FP32 weights change
    the operator by ~1e-7 relative, which the solution follows at 1e-4)."""
    ns, L, ex, f, dm = _periodic_problem(4, 40, weight_dtype=weight_dtype)
    phi, iters, resid = _gpu_solve(L, f, dm)
    assert resid <= 1e-13 and 0 < iters < 20000  # LABFM_OK means the true residual met tol
    ref = _oracle_solve(ns, 4, f, dm)
    tol = 1e-8 if weight_dtype == "f64" else 1e-4
    assert np.abs(phi - ref).max() <= tol * np.abs(ref).max(), np.abs(phi - ref).max()
    assert phi[0] == pytest.approx(ex[0], abs=1e-13)


def test_poisson_dirichlet_walls_matches_oracle():
    """Dirichlet rows (Sec. 5.2): the heat-equation node set with walls (k = 4, 41^2 nodes),
    phi = sin(2 pi x) sin(2 pi y) + x y prescribed on the walls, f = nabla^2 phi inside."""
    k = 4
    ns = S.dirichlet_square(41, 2.0, k, 0.5, seed=304)
    L, rp, col, w, status, _ = G.gpu_run(ns, k, ("lap",), rbf="quadratic", abf_form="dw0")
    assert (status == 0).all()
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    ex = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) + x * y
    f = np.where(ns.wall, ex, -8 * np.pi ** 2 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y))
    dm = ns.wall.astype(np.uint8)
    phi, iters, resid = _gpu_solve(L, f, dm)
    assert resid <= 1e-13
    ref = _oracle_solve(ns, k, f, dm)
    assert np.abs(phi - ref).max() <= 1e-8 * np.abs(ref).max()
    assert np.array_equal(phi[ns.wall], ex[ns.wall])
    assert np.linalg.norm(phi - ex) / np.linalg.norm(ex) < 1e-4  # order-4 one-sided stencils at the walls


def test_poisson_even_order_pattern_on_gpu():
    """The periodic convergence orders of Sec. 5.2 from the GPU solves: 2 for k = 3, 4 for k = 5
    (odd k gives the order of k - 1), between h/H = 2/20 and 2/80."""
    for k, (lo, hi) in {3: (1.8, 2.3), 5: (3.6, 4.4)}.items():
        errs = []
        for nside in (20, 80):
            ns, L, ex, f, dm = _periodic_problem(k, nside)
            phi, _, _ = _gpu_solve(L, f, dm, tol=1e-12)
            errs.append(np.linalg.norm(phi - ex) / np.linalg.norm(ex))
            L.close()
        rate = math.log2(errs[0] / errs[1]) / 2.0
        assert lo <= rate <= hi, (k, errs, rate)


def test_solve_reports_non_convergence_and_bad_arguments():
    import torch

    from paper_1912_06441_gb300 import LabfmError

    ns, L, ex, f, dm = _periodic_problem(4, 24)
    dev = torch.device("cuda", 0)
    phi = torch.zeros(ns.n, dtype=torch.float64, device=dev)
    fd = torch.from_numpy(f).to(dev)
    with pytest.raises(LabfmError) as ei:
        L.solve(0, fd, phi, torch.from_numpy(dm).to(dev), tol=1e-14, max_iter=3)
    assert "NOT_CONVERGED" in str(ei.value) and L.last_solve[0] == 3
    with pytest.raises(LabfmError):
        L.solve(1, fd, phi)  # only one operator was built
    with pytest.raises(LabfmError):
        L.solve(0, fd, fd)  # f and phi the same buffer


def test_solve_selects_the_operator():
    """Weights for (d/dx, d/dy, nabla^2): solving with op = 2 uses the Laplacian's column of the
    interleaved weights (k = 4, 40^2 nodes, node 0 fixed) and equals the oracle's solve."""
    import torch

    k = 4
    ns = S.jittered_lattice(40, 2.0, k, jitter=0.5 / math.sqrt(2), seed=3)
    ops = ("dx", "dy", "lap")
    L, rp, col, w, status, _ = G.gpu_run(ns, k, ops, rbf="quadratic", abf_form="dw0")
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    ex = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    f = -8 * np.pi ** 2 * ex
    dm = np.zeros(ns.n, np.uint8)
    dm[0] = 1
    f[0] = ex[0]
    dev = torch.device("cuda", 0)
    phi = torch.zeros(ns.n, dtype=torch.float64, device=dev)
    L.solve(2, torch.from_numpy(f).to(dev), phi, torch.from_numpy(dm).to(dev), tol=1e-13)
    orp, ocol = oracle.neighbours(ns.xy, ns.h, True)
    ow = oracle.build_weights(ns.xy, ns.h, True, orp, ocol, G.c_matrix(k, ops), k=k, rbf="quadratic",
                              abf_form="dw0")["w"]
    ref = oracle.solve_operator(orp, ocol, ow, 2, f, dm)
    got = phi.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def test_solve_all_dirichlet_rows_is_exact_and_immediate():
    """Degenerate system: every row a Dirichlet row (the identity).  The initial guess takes f
    at those nodes, the residual is exactly zero and the solve returns after no iteration with
    phi == f bit for bit."""
    import torch

    ns, L, ex, f, dm = _periodic_problem(4, 24)
    dev = torch.device("cuda", 0)
    phi = torch.full((ns.n,), 7.0, dtype=torch.float64, device=dev)
    allrows = torch.ones(ns.n, dtype=torch.uint8, device=dev)
    iters, resid = L.solve(0, torch.from_numpy(f).to(dev), phi, allrows, tol=1e-12)
    assert iters == 0 and resid == 0.0
    assert np.array_equal(phi.cpu().numpy(), f)


def _neumann_gpu(nside, field, weight_dtype="f64", tol=1e-13):
    """labfm_solve_neumann on the Neumann square (Dirichlet walls at x = 0, 1; ghost rows for the
    walls y = 0, 1), k = 4, weights of (d/dx, d/dy, nabla^2) built on the GPU, and the oracle's
    direct solve of the same system on the oracle's weights."""
    import torch

    from tests import test_oracle_pins as OP

    k = 4
    q, rp, col, r, ex, f = OP.neumann_problem(nside, k, field)
    L, grp, gcol, w, status, _ = G.gpu_run(q.ns, k, ("dx", "dy", "lap"), rbf="quadratic", abf_form="dw0",
                                           weight_dtype=weight_dtype)
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
    assert np.array_equal(status, r["status"])
    dev = torch.device("cuda", 0)
    phi = torch.zeros(q.ns.n, dtype=torch.float64, device=dev)
    nm = (torch.from_numpy(q.ghost).to(dev), torch.from_numpy(q.parent).to(dev),
          torch.from_numpy(q.normal).to(dev), 0, 1)
    dm = q.dirichlet.astype(np.uint8)
    iters, resid = L.solve(2, torch.from_numpy(f).to(dev), phi, torch.from_numpy(dm).to(dev), tol=tol,
                           max_iter=20000, neumann=nm)
    ref = oracle.solve_operator(rp, col, r["w"], 2, f, dm, neumann=(q.ghost, q.parent, q.normal, 0, 1))
    return q, L, phi.cpu().numpy(), ref, ex, iters, resid


def test_poisson_neumann_ghost_rows_match_oracle():
    """Neumann ghost-node rows (Sec. 5.2) through labfm_solve_neumann: for a polynomial of degree
    4 at k = 4 the GPU solution is the polynomial at every node, ghosts included (each row is
    exact); for phi = sin(2x + 0.3) cos(3y - 0.2) on 41^2 nodes it equals the oracle's direct
    solve of the same system to 1e-8 and meets the prescribed normal derivatives, and the error
    against phi is that of the oracle's solution."""
    from tests import test_oracle_pins as OP

    q, L, phi, ref, ex, iters, resid = _neumann_gpu(21, OP._neumann_poly_field())
    assert resid <= 1e-13 and iters > 0
    assert np.abs(phi - ex).max() <= 1e-9 * np.abs(ex).max()
    assert np.abs(phi - ref).max() <= 1e-9 * np.abs(ex).max()
    L.close()
    field = (lambda x, y: np.sin(2 * x + 0.3) * np.cos(3 * y - 0.2),
             lambda x, y: 2 * np.cos(2 * x + 0.3) * np.cos(3 * y - 0.2),
             lambda x, y: -3 * np.sin(2 * x + 0.3) * np.sin(3 * y - 0.2),
             lambda x, y: -13 * np.sin(2 * x + 0.3) * np.cos(3 * y - 0.2))
    q, L, phi, ref, ex, iters, resid = _neumann_gpu(41, field)
    assert np.abs(phi - ref).max() <= 1e-8 * np.abs(ref).max()
    assert np.array_equal(phi[q.dirichlet], ex[q.dirichlet])
    keep = np.ones(q.ns.n, bool)
    keep[q.ghost] = False
    e_gpu = np.linalg.norm(phi[keep] - ex[keep]) / np.linalg.norm(ex[keep])
    e_ref = np.linalg.norm(ref[keep] - ex[keep]) / np.linalg.norm(ex[keep])
    assert abs(e_gpu - e_ref) <= 1e-3 * e_ref and e_gpu < 1e-5
    # the normal derivative at each Neumann wall node, through the GPU's own d/dx, d/dy apply
    import torch

    d = L.apply(torch.from_numpy(phi).to(torch.device("cuda", 0))).cpu().numpy()
    got = q.normal[:, 0] * d[0, q.parent] + q.normal[:, 1] * d[1, q.parent]
    xb, yb = q.ns.xy[q.parent, 0], q.ns.xy[q.parent, 1]
    want = q.normal[:, 0] * field[1](xb, yb) + q.normal[:, 1] * field[2](xb, yb)
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()


def test_poisson_neumann_f32_weights():
    """The ghost rows from FP32-stored weights (widened to FP64 in the solve): the operator changes
    by ~1e-7 relative, which the solution follows."""
    from tests import test_oracle_pins as OP

    q, L, phi, ref, ex, iters, resid = _neumann_gpu(21, OP._neumann_poly_field(), weight_dtype="f32", tol=1e-12)
    assert np.abs(phi - ref).max() <= 1e-4 * np.abs(ex).max()


def test_solve_neumann_rejects_bad_ghost_rows():
    """Ghost rows that index out of range, repeat a ghost, are their own parent or are also
    Dirichlet rows are argument errors, checked on the device before the iteration."""
    import torch

    from paper_1912_06441_gb300 import LabfmError
    from tests import test_oracle_pins as OP

    k = 4
    q, rp, col, r, ex, f = OP.neumann_problem(11, k, OP._neumann_poly_field())
    L, *_ = G.gpu_run(q.ns, k, ("dx", "dy", "lap"), rbf="quadratic", abf_form="dw0")
    dev = torch.device("cuda", 0)
    fd = torch.from_numpy(f).to(dev)
    dm = torch.from_numpy(q.dirichlet.astype(np.uint8)).to(dev)
    nrm = torch.from_numpy(q.normal).to(dev)
    gh = torch.from_numpy(q.ghost).to(dev)
    pa = torch.from_numpy(q.parent).to(dev)
    bad = {
        "out of range": (gh.clone().fill_(q.ns.n), pa),
        "repeated ghost": (torch.cat([gh[:1], gh[:-1]]), pa),
        "own parent": (gh, gh),
        "Dirichlet ghost": (torch.cat([torch.zeros(1, dtype=torch.int64, device=dev), gh[1:]]), pa),
    }
    for name, (g2, p2) in bad.items():
        phi = torch.zeros(q.ns.n, dtype=torch.float64, device=dev)
        with pytest.raises(LabfmError) as ei:
            L.solve(2, fd, phi, dm, tol=1e-12, neumann=(g2, p2, nrm, 0, 1))
        assert "ERR_ARG" in str(ei.value), name
    phi = torch.zeros(q.ns.n, dtype=torch.float64, device=dev)
    L.solve(2, fd, phi, dm, tol=1e-12, neumann=(gh, pa, nrm, 0, 1))  # the context is still usable
    assert np.abs(phi.cpu().numpy() - ex).max() <= 1e-9 * np.abs(ex).max()


@pytest.mark.parametrize("k", [2, 4])
def test_poisson_annulus_matches_oracle(k):
    """The annular problem of Sec. 5.2 (Dirichlet outer circle, Neumann inner circle by ghost
    rows, quadratic ABFs, h/dr = 2) at h/H = 2/49 and 2/97: labfm_solve_neumann on the GPU's
    weights equals the oracle's direct solve on the oracle's weights to 1e-8, and its error
    against r sin(4 pi r) cos(3 theta) is the oracle's (so the printed table holds for it too)."""
    import torch

    from tests import test_oracle_pins as OP

    dev = torch.device("cuda", 0)
    for m in (49, 97):
        q, rp, col, r, ex, f = OP.annulus_problem(m, k)
        L, grp, gcol, w, status, _ = G.gpu_run(q.ns, k, ("dx", "dy", "lap"), rbf="quadratic", abf_form="dw0")
        assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
        keep = np.ones(q.ns.n, bool)
        keep[q.ghost] = False
        assert (status[keep] == 0).all()
        phi = torch.zeros(q.ns.n, dtype=torch.float64, device=dev)
        nm = (torch.from_numpy(q.ghost).to(dev), torch.from_numpy(q.parent).to(dev),
              torch.from_numpy(q.normal).to(dev), 0, 1)
        L.solve(2, torch.from_numpy(f).to(dev), phi, torch.from_numpy(q.dirichlet.astype(np.uint8)).to(dev),
                tol=1e-13, max_iter=50000, neumann=nm)
        got = phi.cpu().numpy()
        ref = oracle.solve_operator(rp, col, r["w"], 2, f, q.dirichlet.astype(np.uint8),
                                    neumann=(q.ghost, q.parent, q.normal, 0, 1))
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), (m, np.abs(got - ref).max())
        e_gpu = np.linalg.norm(got[keep] - ex[keep]) / np.linalg.norm(ex[keep])
        e_ref = np.linalg.norm(ref[keep] - ex[keep]) / np.linalg.norm(ex[keep])
        assert abs(e_gpu - e_ref) <= 1e-4 * e_ref, (m, e_gpu, e_ref)
        L.close()
