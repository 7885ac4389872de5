"""Parity at the full sizes of the benchmark workloads, in the configuration bench.py times.

The oracle cannot build all weights of 262,144 - 4,194,304 nodes in test time, so each test
checks a seeded random sample of nodes one by one (stencil rows bit for bit, weights and
derivatives against the FP64 and binary128 oracles), and checks what holds at any size on
every node: the gather-sum of every node against the oracle's own sum of the same weights,
and one RK4 step against the degree-4 Taylor polynomial of the operator it steps.

Workloads (the same recipes as bench.py):
  - 512 x 512 periodic lattice, +-0.3 s jitter (seed 2), Wendland C2, order 8 at h = 2.2 s
    (d/dx, d/dy, nabla^2, nabla^8) and order 6 at h = 1.8 s (d/dx, d/dy, nabla^2, nabla^6);
  - 1000 x 1000 wall-bounded set, spacing varying 4x, per-node order 2-8 (seed 4);
  - 2048 x 2048 periodic lattice, +-0.1 s jitter (seed 5), quadratic ABFs in the dW0/dr-only
    form, order 8 at h = 2.2 s: the RK4 workload.
"""
import os

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


def _sample(n, count, seed):
    return np.unique((S.uniform01(seed, count) * n).astype(np.int64))


def _check_sampled(ns, k, ops, rp, col, w, status, q, rbf="wendland_c2", order=None, abf_form="chain", label=""):
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    orp, ocol = oracle.neighbours(ns.xy, ns.h, ns.periodic, ns.lo, ns.hi, queries=q)
    assert np.array_equal(rp_q, orp) and np.array_equal(col_q, ocol), label
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q, rbf=rbf, order=order, abf_form=abf_form)
    assert np.array_equal(status[q], r64["status"]), label
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label=label)
    return rp_q, col_q, idx, r64, rld


def _check_apply_all_nodes(L, rp, col, w, f):
    """Every node: the GPU gather-sum against the oracle's sum of the same weights, within the
    bound of two summation orders, ~N u sum_j |(f_j - f_i) w_j|."""
    import torch

    out = L.apply(torch.from_numpy(f).to(torch.device("cuda", 0))).cpu().numpy()
    ref = oracle.apply(rp, col, w, f)
    absterm = np.abs(f[col] - np.repeat(f, np.diff(rp)))[:, None] * np.abs(w)
    bound = np.add.reduceat(absterm, rp[:-1], axis=0).T
    assert np.all(np.abs(out - ref) <= 1e-14 * bound + 1e-300)
    return out


def _hard_nodes():
    """The ill-conditioned stencils of this workload, chosen by the oracle alone
    (tests/golden/hard_nodes_lattice512_k8.txt)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hard_nodes_lattice512_k8.txt")
    return np.loadtxt(path, dtype=np.int64, comments="#")


@pytest.fixture(scope="module")
def lattice512_k8():
    """The FP64 GPU build of the 512^2 order-8 workload and its derivatives (the reference the
    mixed builds' outliers are picked against)."""
    k, ops = 8, ("dx", "dy", "lap", "lap4")
    ns = S.jittered_lattice(512, 2.2, k, jitter=0.3, seed=2)
    f = S.fourier_field(n_modes=16, kmax=32, seed=3).value(ns.xy)
    L, rp, col, w, status, _ = G.gpu_run(ns, k, ops, precision="fp64")
    import torch

    d = L.apply(torch.from_numpy(f).to(torch.device("cuda", 0))).cpu().numpy()
    L.close()
    return ns, f, rp, col, w, status, d


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_tc"])
def test_lattice512_order8(lattice512_k8, precision):
    """Sampled nodes of the full-size order-8 workload, against the binary128 oracle: 200 random
    nodes, the 148 ill-conditioned ones the oracle picks (smallest pivot ratios, largest FP64
    errors), and -- for the mixed builds -- every node whose derivatives differ from the FP64
    build's by more than 1e-8 of the operator's largest value over all nodes.  All precisions stay within the
    FP64 floor-aware tolerance; the mixed builds (adaptive refinement on the FP64 residual of the
    moment conditions) must in addition be as accurate as the FP64 oracle on every one of these
    nodes, weights and derivatives (within a factor 2, or 1e-11)."""
    import torch

    ns, f, rp64, col64, w64, st64, d64 = lattice512_k8
    k, ops = 8, ("dx", "dy", "lap", "lap4")
    if precision == "fp64":
        rp, col, w, status, out = rp64, col64, w64, st64, d64
        L = None
    else:
        L, rp, col, w, status, _ = G.gpu_run(ns, k, ops, precision=precision)
        assert np.array_equal(rp, rp64) and np.array_equal(col, col64)
        out = L.apply(torch.from_numpy(f).to(torch.device("cuda", 0))).cpu().numpy()
    # the tail of the difference from the FP64 build: more than 1e-8 of each operator's largest
    # value over all nodes (tens of nodes)
    sc_all = np.abs(d64).max(axis=1, keepdims=True)
    outliers = np.nonzero((np.abs(out - d64) / sc_all).max(axis=0) > 1e-8)[0]
    assert len(outliers) < 1000, len(outliers)
    # each operator's typical scale: its largest value over 200 random nodes (the largest over
    # all nodes belongs to an ill-conditioned stencil whose nabla^8 value is ~1e4 times larger)
    q_rand = _sample(ns.n, 200, seed=101)
    sc_r = np.abs(d64[:, q_rand]).max(axis=1, keepdims=True)
    q = np.unique(np.concatenate([q_rand, _hard_nodes(), outliers]))
    label = f"512^2 k=8 {precision}"
    rp_q, col_q, idx, r64, rld = _check_sampled(ns, k, ops, rp, col, w, status, q, label=label)
    _check_apply_all_nodes_values(rp, col, w, f, out)  # the gather-sum of every node
    d_ld = oracle.apply(rp_q, col_q, rld["w"], f, queries=q, precision=G.REF_PRECISION)
    d_64 = oracle.apply(rp_q, col_q, r64["w"], f, queries=q)
    sc = np.abs(d_ld).max(axis=1)
    e_gpu = np.abs(out[:, q] - d_ld).max(axis=1) / sc
    e_64 = np.abs(d_64 - d_ld).max(axis=1) / sc
    assert np.all(e_gpu <= np.maximum(G.TOL_FLOOR_MAX, G.FLOOR_FACTOR * e_64)), (e_gpu, e_64)
    if precision != "fp64":
        # per node: derivatives (relative to the operator's typical scale) and weights (relative
        # over the stencil) no worse than the FP64 oracle's, beyond a factor 2 at the rounding floor
        ed_gpu = (np.abs(out[:, q] - d_ld) / sc_r).max(axis=0)
        ed_64 = (np.abs(d_64 - d_ld) / sc_r).max(axis=0)
        bad = ed_gpu > np.maximum(G.TOL_FLOOR_MAX, 2.0 * ed_64)
        assert not bad.any(), (q[bad], ed_gpu[bad], ed_64[bad])
        ew_gpu = G.node_rel_err(w[idx], rld["w"], rp_q).max(axis=1)
        ew_64 = G.node_rel_err(r64["w"], rld["w"], rp_q).max(axis=1)
        assert np.all(ew_gpu <= np.maximum(G.TOL_FLOOR_MAX, 2.0 * ew_64)), (q[ew_gpu > np.maximum(G.TOL_FLOOR_MAX, 2.0 * ew_64)])
        info = L.get_build_info()
        assert sum(info["refine_steps"]) == ns.n and info["fp64_rebuilt"] == 0
        L.close()


def _check_apply_all_nodes_values(rp, col, w, f, out):
    """Every node's gather-sum against the oracle's sum of the same weights (two summation
    orders of one sum)."""
    absterm = np.abs(f[col] - np.repeat(f, np.diff(rp)))[:, None] * np.abs(w)
    bound = np.add.reduceat(absterm, rp[:-1], axis=0).T
    assert np.all(np.abs(out - oracle.apply(rp, col, w, f)) <= 1e-14 * bound + 1e-300)


def test_lattice512_order6_and_fp32_apply():
    import torch

    k, ops = 6, ("dx", "dy", "lap", "lap3")
    ns = S.jittered_lattice(512, 1.8, k, jitter=0.3, seed=2)
    L, rp, col, w, status, _ = G.gpu_run(ns, k, ops)
    q = _sample(ns.n, 200, seed=102)
    _check_sampled(ns, k, ops, rp, col, w, status, q, label="512^2 k=6")
    f = S.fourier_field(n_modes=16, kmax=32, seed=3).value(ns.xy)
    full = _check_apply_all_nodes(L, rp, col, w, f)
    # FP32 weights and field through the tuned FP32 kernel: within a few ulp(float) of
    # sum_j (|f_j| + |f_i|) |w_j| of the FP64 result
    L32, _, _, w32, _, _ = G.gpu_run(ns, k, ops, weight_dtype="f32")
    assert np.array_equal(w32, w.astype(np.float32).astype(np.float64))
    f32 = L32.apply(torch.from_numpy(f.astype(np.float32)).to(torch.device("cuda", 0))).cpu().numpy()
    absterm = (np.abs(f[col]) + np.abs(np.repeat(f, np.diff(rp))))[:, None] * np.abs(w)
    bound = np.add.reduceat(absterm, rp[:-1], axis=0).T
    assert np.all(np.abs(f32 - full) <= 64 * 2.0 ** -24 * bound + 2.0 ** -24 * np.abs(full))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_tc"])
def test_walls_1m_variable_order(precision):
    ns = S.variable_wall_nodes(1000, seed=4)
    ops = ("dx", "dy", "lap")
    L, rp, col, w, status, _ = G.gpu_run(ns, 8, ops, order=ns.order, precision=precision)
    q = _sample(ns.n, 200, seed=103)
    # and every wall-band node class: include some nodes on the boundary
    wall = np.nonzero((ns.xy[:, 0] == 0.0) | (ns.xy[:, 1] == 1.0))[0]
    q = np.unique(np.concatenate([q, wall[:: max(1, len(wall) // 40)]]))
    _check_sampled(ns, 8, ops, rp, col, w, status, q, order=ns.order, label=f"walls 1M {precision}")


def test_rk4_lattice2048_order8():
    """The time-stepping workload: sampled weights against the oracle; one RK4 step of the
    graph-replayed stage kernels equals the degree-4 Taylor polynomial of dt A applied to u,
    with A u = sum_d beta_d L^d u evaluated by four labfm_apply calls (any size, FP64); and
    100 steps stay within the spatial and temporal error of the exact solution for FP64 and
    for FP32 fields."""
    import torch

    from paper_1912_06441_gb300 import Labfm

    k, ops = 8, ("dx", "dy", "lap", "lap4")
    ns = S.jittered_lattice(2048, 2.2, k, jitter=0.1, seed=5)
    dev = torch.device("cuda", 0)
    L = Labfm(0)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
    st = torch.full((ns.n,), -1, dtype=torch.int32, device=dev)
    L.build_weights(G.c_matrix(k, ops), uniform_order=k, rbf="quadratic", abf_form="dw0", node_status=st)
    status = st.cpu().numpy()
    assert (status == 0).all()
    rp_d, col_d = L.get_neighbours()
    rp, col = rp_d.cpu().numpy(), col_d.cpu().numpy()
    q = _sample(ns.n, 96, seed=104)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    w_q = L.get_weights()[torch.from_numpy(idx).to(dev)].cpu().numpy()  # only the sampled rows
    orp, ocol = oracle.neighbours(ns.xy, ns.h, True, queries=q)
    assert np.array_equal(rp_q, orp) and np.array_equal(col_q, ocol)
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q, rbf="quadratic", abf_form="dw0")
    G.assert_weights_parity(w_q, r64, rld, rp_q, label="2048^2 rk4 set")
    h = ns.h[0]
    beta = np.array([-1.0, -0.5, 1e-3, -1e-3 * h ** 8])
    dt = 5e-5  # 0.8 x 2.785 / rho with rho ~ 45 / h for this node set
    u0 = S.sincos_field().value(ns.xy)
    b = torch.tensor(beta, device=dev)[:, None]

    def A(v):
        return (b * L.apply(v)).sum(0)

    u = torch.from_numpy(u0).to(dev)
    z1 = A(u)
    z2 = A(z1)
    z3 = A(z2)
    z4 = A(z3)
    taylor = u + dt * z1 + dt ** 2 / 2 * z2 + dt ** 3 / 6 * z3 + dt ** 4 / 24 * z4
    step = u.clone()
    L.step(beta, step, dt, 1)
    scale = float(u.abs().max())
    assert float((step - taylor).abs().max()) < 1e-12 * scale
    # 100 steps: FP64 and FP32 fields against the exact advected, decayed mode
    T = 100 * dt
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    exact = np.exp(-8 * np.pi ** 2 * 1e-3 * T) * np.sin(2 * np.pi * (x - T)) * np.cos(2 * np.pi * (y - 0.5 * T))
    errs = {}
    for dt_name, tdt in (("f64", torch.float64), ("f32", torch.float32)):
        v = torch.from_numpy(u0).to(dev, tdt)
        L.step(beta, v, dt, 100)
        got = v.cpu().numpy().astype(np.float64)
        errs[dt_name] = np.abs(got - exact).max()
    assert errs["f64"] < 1e-7, errs
    assert errs["f32"] < 1e-5, errs


def test_rk4_oracle_leg_2048_subsample_and_independent_256():
    """The time-stepping workload's oracle leg (as bench.py reports it): at the 65,536 nodes of
    the 2048^2 set's 256^2 subsample the GPU's stencil rows equal the oracle's bit for bit and
    its FP64 weights agree with the FP64 oracle's (normwise per node, and derivatives relative to
    the sum of their terms); on an independent 256^2 set with the same parameters, 1000 graph-
    replayed RK4 steps with FP64 fields equal the oracle's 1000 steps to 1e-11 of max|u|, and
    with FP32 fields (FP64 or FP32 weights) to the FP32 rounding floor, 5e-6."""
    import torch

    import bench
    import paper_1912_06441_gb300 as P

    r = bench.rk4_oracle_leg(torch, P, torch.device("cuda", 0), 0)
    sub = r["subsample_2048"]
    assert sub["stencils_bit_exact"] and sub["oracle_status_ok"] == sub["nodes"] == 65536
    assert max(sub["weights_normwise"]["max"]) <= 1e-9, sub["weights_normwise"]
    assert max(sub["deriv_err_over_term_sum"]["max"]) <= 1e-11, sub["deriv_err_over_term_sum"]
    rk = r["independent_256_rk4"]
    assert rk["gpu_f64_fields_f64_weights"]["max_diff_vs_oracle"] <= 1e-11, rk
    for key in ("gpu_f32_fields_f64_weights", "gpu_f32_fields_f32_weights"):
        assert rk[key]["max_diff_vs_oracle"] <= 5e-6, rk
    assert rk["oracle_l2_err_vs_exact"] < 1e-7
