"""Builds with five to eight operators (LABFM_MAX_OPS = 8) at order 8, through every call that
takes the operator count: the weight build (FP64 and tensor-core mixed), the apply (all eight,
and masks selecting five, six and seven, so that the reduce-scatter pads to eight lanes' worth
of operators), the RK4 step and Burgers' equation.

Operators (targets C^d, Sec. 2 and Sec. 4.2): d/dx, d/dy, nabla^2, nabla^4, nabla^6, nabla^8,
d^2/dxdy and d^3/dx^3 on a 40 x 40 jittered periodic lattice (h = 2.2 s, Wendland C2)."""
import numpy as np
import pytest

import labfm_synth as S
import oracle
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

K = 8
NAMED = ("dx", "dy", "lap", "lap2", "lap3", "lap4")


def _c8():
    rows = [S.op_c_vector(o, K) for o in NAMED]
    for a, b in ((1, 1), (3, 0)):
        c = np.zeros(S.p_of_k(K))
        c[S.element_index(a, b)] = 1.0
        rows.append(c)
    return np.stack(rows)


@pytest.fixture(scope="module")
def built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1912_06441_gb300 as P
    from paper_1912_06441_gb300 import Labfm

    P.load_library()
    ns = S.jittered_lattice(40, 2.2, K, seed=31)
    C = _c8()
    dev = torch.device("cuda", 0)
    L = Labfm(0)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
    st = torch.full((ns.n,), -1, dtype=torch.int32, device=dev)
    L.build_weights(C, uniform_order=K, node_status=st)
    rp, col = (t.cpu().numpy() for t in L.get_neighbours())
    w = L.get_weights().cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    q = np.arange(ns.n)
    r64 = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=K, queries=q)
    rld = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=K, queries=q, precision=G.REF_PRECISION)
    return ns, C, L, rp, col, w, r64, rld


def test_eight_operator_weights_match_the_oracle(built):
    ns, C, L, rp, col, w, r64, rld = built
    assert w.shape[1] == 8
    G.assert_weights_parity(w, r64, rld, rp, label="8 ops fp64")


def test_eight_operator_weights_mixed_tc(built):
    ns, C, L, rp, col, w, r64, rld = built
    import torch

    from paper_1912_06441_gb300 import Labfm

    dev = torch.device("cuda", 0)
    M = Labfm(0)
    M.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
    M.build_weights(C, uniform_order=K, precision="mixed_tc")
    G.assert_weights_parity(M.get_weights().cpu().numpy(), r64, rld, rp, label="8 ops mixed_tc")


@pytest.mark.parametrize("mask", [0xFF, 0x1F, 0x3F, 0x7F, 0xB5])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_apply_five_to_eight_operators(built, mask, dtype):
    """The gather-sum of the selected operators on every node against the oracle's sum of the
    same weights: FP64 within two summation orders, FP32 field within a few ulp(float) of
    sum_j (|f_j| + |f_i|) |w_j|."""
    import torch

    ns, C, L, rp, col, w, r64, rld = built
    sel = [d for d in range(8) if mask >> d & 1]
    f = S.fourier_field(n_modes=8, kmax=4, seed=3).value(ns.xy)
    dev = torch.device("cuda", 0)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    out = L.apply(torch.from_numpy(f).to(dev, tdt), op_mask=mask).cpu().numpy().astype(np.float64)
    assert out.shape == (len(sel), ns.n)
    ref = oracle.apply(rp, col, w[:, sel], f)
    if dtype == "f64":
        absterm = np.abs(f[col] - np.repeat(f, np.diff(rp)))[:, None] * np.abs(w[:, sel])
        bound = np.add.reduceat(absterm, rp[:-1], axis=0).T
        assert np.all(np.abs(out - ref) <= 1e-14 * bound + 1e-300)
    else:
        absterm = (np.abs(f[col]) + np.abs(np.repeat(f, np.diff(rp))))[:, None] * np.abs(w[:, sel])
        bound = np.add.reduceat(absterm, rp[:-1], axis=0).T
        assert np.all(np.abs(out - ref) <= 8 * 2.0 ** -24 * bound + 2.0 ** -24 * np.abs(ref))


def _beta(h):
    """Advection, a little diffusion, damping hyperviscosities of orders 4, 6 and 8, and small
    cross terms, each weighted by h^m so that no operator dominates."""
    return np.array([-1.0, -0.5, 1e-2, -1e-3 * h ** 3, 2e-5 * h ** 5, -4e-7 * h ** 7, 5e-2 * h, 5e-3 * h ** 2])


def _stable_dt(L, beta, n):
    """0.2 / rho, rho the spectral radius of u -> sum_d beta_d L^d u by power iteration through
    labfm_apply: every eigenvalue then has |lambda dt| <= 0.2, so a few RK4 steps stay bounded
    (noisy order-8 stencils carry eigenvalues far beyond the Fourier symbol's)."""
    import torch

    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(1)
    v = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
    b = torch.tensor(beta, dtype=torch.float64, device=dev)[:, None]
    rho = 0.0
    for _ in range(60):
        v = v / v.norm()
        v = (b * L.apply(v)).sum(0)
        rho = float(v.norm())
    return 0.2 / rho


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rk4_eight_operators(built, dtype):
    """Five RK4 steps of du/dt = sum_d beta_d L^d u with all eight operators combined into one
    weight per entry, against the oracle's RK4 on the same weights."""
    import torch

    ns, C, L, rp, col, w, r64, rld = built
    beta = _beta(ns.h[0])
    dt = _stable_dt(L, beta, ns.n)
    u0 = S.sincos_field().value(ns.xy)
    dev = torch.device("cuda", 0)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u = torch.from_numpy(u0).to(dev, tdt)
    L.step(beta, u, dt, 5)
    got = u.cpu().numpy().astype(np.float64)
    ref = oracle.rk4(rp, col, w, beta, u0.astype(np.float64 if dtype == "f64" else np.float32), dt, 5)
    inc = np.abs(ref - u0).max()  # what the steps changed (dt is small: ~5e-5 here)
    if dtype == "f64":
        # two summation orders of the same stage sums: far below the increment
        assert np.abs(got - ref).max() <= 1e-9 * inc, (np.abs(got - ref).max(), inc)
    else:
        # float field and combined weights: a few ulp(float) of |u| per step
        assert np.abs(got - ref).max() <= 16 * 2.0 ** -24 * np.abs(ref).max(), (np.abs(got - ref).max(), inc)


def test_burgers_eight_operators(built):
    """Burgers' equation with d/dx, d/dy as operators 0 and 1 and six linear operators, five steps
    against the oracle's RK4 of the same system on the same weights."""
    import torch

    ns, C, L, rp, col, w, r64, rld = built
    h = ns.h[0]
    beta = _beta(h)
    dt = _stable_dt(L, beta, ns.n)  # with unit advection: the fields below stay under 0.5
    beta[:2] = 0.0
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    u0 = 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    v0 = 0.25 * np.cos(2 * np.pi * x) * np.sin(4 * np.pi * y)
    dev = torch.device("cuda", 0)
    u = torch.from_numpy(u0).to(dev)
    v = torch.from_numpy(v0).to(dev)
    L.step_burgers(beta, u, v, dt, 5)
    ru, rv = oracle.rk4_burgers(rp, col, w, beta, u0, v0, dt, 5)
    inc = max(np.abs(ru - u0).max(), np.abs(rv - v0).max())
    assert np.abs(u.cpu().numpy() - ru).max() <= 1e-9 * inc
    assert np.abs(v.cpu().numpy() - rv).max() <= 1e-9 * inc
