"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Stencils must match bit for bit.  Weights and derivatives are compared per node with the
binary128 oracle, within max(1e-11, 30 x the FP64 oracle's own error) -- the FP64 floor is
~1e-13 at k = 4 but ~1e-8 (worst node) at k = 8, where two correct FP64 computations that
differ only in summation order already disagree (see tests/gpu_common.py).
"""
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

    P.load_library()  # fails loudly if the extension was not built


# ---------------------------------------------------------------------------------- stencils

NBR_CASES = [
    ("lattice64_h1.4_periodic", lambda: S.jittered_lattice(64, 1.4, 4, seed=1)),
    ("lattice61_h2.2_periodic_ragged", lambda: S.jittered_lattice(61, 2.2, 8, seed=2)),
    ("lattice50_h3.0_walls", lambda: S.jittered_lattice(50, 3.0, 4, seed=3, periodic=False)),
    ("lattice8_two_cells_periodic", lambda: S.jittered_lattice(8, 1.8, 4, seed=4)),
    ("lattice6_one_cell_periodic", lambda: S.jittered_lattice(6, 3.0, 4, seed=5)),
    ("variable_spacing_walls", lambda: S.variable_wall_nodes(48, seed=4)),
    # radius tiny against the box: the search caps its grid at 4n + 64 cells (coarse cells of
    # ~100 nodes each)
    ("cluster_capped_grid_walls", lambda: S.lattice_clusters(40, 1.4, [(0.3, 0.3)], 0.04, seed=21)),
]


@pytest.mark.parametrize("name,make", NBR_CASES, ids=[c[0] for c in NBR_CASES])
def test_neighbours_bit_exact(name, make):
    import torch

    from paper_1912_06441_gb300 import Labfm

    ns = make()
    L = Labfm(0)
    dev = torch.device("cuda", 0)
    nnz = L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), ns.periodic,
                             ns.lo, ns.hi)
    rp, col = L.get_neighbours()
    orp, ocol = oracle.neighbours(ns.xy, ns.h, ns.periodic, ns.lo, ns.hi)
    assert nnz == len(ocol)
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert np.array_equal(col.cpu().numpy(), ocol)


def test_neighbours_capped_grid_two_clusters():
    """100,352 nodes in two dense blocks at opposite corners of the unit box (spacing 1e-4,
    h = 1.4e-4): a grid of side 2h would have 12.8 M cells, the search caps it at 4n + 64 and
    its cells hold ~350 nodes each.  Sampled rows (both blocks' edges included) against the
    oracle's brute force, bit for bit; no row reaches across the gap between the blocks."""
    import torch

    from paper_1912_06441_gb300 import Labfm

    ns = S.lattice_clusters(224, 1.4, [(0.05, 0.05), (0.9, 0.9)], 0.0224, seed=22)
    dev = torch.device("cuda", 0)
    L = Labfm(0)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), False, ns.lo, ns.hi)
    rp_d, col_d = L.get_neighbours()
    rp, col = rp_d.cpu().numpy(), col_d.cpu().numpy()
    half = ns.n // 2
    q = np.unique(np.concatenate([(S.uniform01(23, 300) * ns.n).astype(np.int64),
                                  np.arange(0, 224), np.arange(half - 224, half + 224), np.arange(ns.n - 224, ns.n)]))
    rp_q, col_q, _ = G.rows_of(rp, col, q)
    orp, ocol = oracle.neighbours(ns.xy, ns.h, False, ns.lo, ns.hi, queries=q)
    assert np.array_equal(rp_q, orp) and np.array_equal(col_q, ocol)
    # rows never cross between the blocks
    node = np.repeat(np.arange(ns.n), np.diff(rp))
    assert np.array_equal(node < half, col < half)


def test_neighbours_single_node_and_empty_rows():
    import torch

    from paper_1912_06441_gb300 import Labfm

    dev = torch.device("cuda", 0)
    L = Labfm(0)
    assert L.build_neighbours(torch.tensor([[0.5, 0.5]], dtype=torch.float64, device=dev),
                              torch.tensor([0.1], dtype=torch.float64, device=dev), False) == 0
    rp, col = L.get_neighbours()
    assert rp.cpu().tolist() == [0, 0] and col.numel() == 0
    # two far-apart clusters: rows of isolated nodes are empty
    xy = np.array([[0.1, 0.1], [0.11, 0.1], [0.9, 0.9]])
    h = np.full(3, 0.01)
    L.build_neighbours(torch.from_numpy(xy).to(dev), torch.from_numpy(h).to(dev), False)
    rp, col = L.get_neighbours()
    orp, ocol = oracle.neighbours(xy, h, False)
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(col.cpu().numpy(), ocol)


# ---------------------------------------------------------------------------------- weights


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_weights_parity_by_order(k):
    rbf = {1: "wendland_c2", 2: "quadratic", 3: "cone", 4: "wendland_c2", 5: "wendland_c6", 6: "wendland_c2",
           7: "quadratic", 8: "wendland_c2"}[k]
    ns = S.jittered_lattice(37, G.HS[k], k, seed=10 + k)  # 1369 nodes: not a multiple of any block size
    ops = G.OPS[k]
    _, rp, col, w, status, nbad = G.gpu_run(ns, k, ops, rbf=rbf)
    q = np.arange(0, ns.n, 3)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    orp, ocol = oracle.neighbours(ns.xy, ns.h, True, queries=q)
    assert np.array_equal(rp_q, orp) and np.array_equal(col_q, ocol)
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q, rbf=rbf)
    assert np.array_equal(status[q], r64["status"])
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label=f"k={k}")


@pytest.mark.parametrize("rbf", ["wendland_c2", "quadratic", "cone", "wendland_c6", "gaussian"])
def test_weights_parity_by_kernel(rbf):
    k = 4
    ns = S.jittered_lattice(40, 1.6, k, seed=21)
    ops = G.OPS[k]
    _, rp, col, w, status, _ = G.gpu_run(ns, k, ops, rbf=rbf)
    q = np.arange(0, ns.n, 4)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q, rbf=rbf)
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label=rbf)


@pytest.mark.parametrize("k,hs", [(4, 3.0), (8, 2.7)])
def test_weights_parity_multi_chunk_stencils(k, hs):
    """Stencils longer than one shared-memory chunk (64 / 72 neighbours) take the chunked path."""
    ns = S.jittered_lattice(40, hs, k, seed=31)
    ops = G.OPS[k]
    _, rp, col, w, status, _ = G.gpu_run(ns, k, ops)
    assert np.diff(rp).min() > (64 if k < 7 else 72)
    q = np.arange(0, ns.n, 5)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q)
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label=f"chunked k={k}")


@pytest.mark.parametrize("k,hs,rbf", [(2, 1.6, "quadratic"), (4, 2.0, "cone"), (6, 2.0, "wendland_c6"),
                                      (8, 2.2, "quadratic"), (8, 2.8, "wendland_c2")])
def test_weights_parity_dw0_form(k, hs, rbf):
    """LABFM_ABF_DW0_ONLY: every ABF element dW0/dr d^alpha|r| (the form the stability results of
    Sec. 4.2 belong to), FP64 build against the oracle's dw0 form."""
    ns = S.jittered_lattice(36, hs, k, seed=40 + k, jitter=0.2)
    ops = G.OPS[k]
    _, rp, col, w, status, _ = G.gpu_run(ns, k, ops, rbf=rbf, abf_form="dw0")
    q = np.arange(1, ns.n, 3)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q, rbf=rbf, abf_form="dw0")
    assert np.array_equal(status[q], r64["status"])
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label=f"dw0 k={k} {rbf}")
    # the two forms differ (elements 3-9 change) unless the kernel's d2W0/dq2 vanishes identically
    if rbf != "cone":
        _, _, _, w_chain, _, _ = G.gpu_run(ns, k, ops, rbf=rbf)
        assert np.abs(w_chain - w).max() > 1e-6 * np.abs(w).max()


def test_weights_variable_order_and_walls():
    """Per-node order 2..8 on a non-periodic set with varying spacing (one-sided stencils at walls)."""
    ns = S.variable_wall_nodes(40, seed=4)
    ops = ("dx", "dy", "lap")
    kmax = 8
    _, rp, col, w, status, _ = G.gpu_run(ns, kmax, ops, order=ns.order)
    q = np.arange(0, ns.n, 3)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, kmax, ops, q, rp_q, col_q, order=ns.order)
    assert np.array_equal(status[q], r64["status"])
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label="variable order")


def test_weights_random_orders_one_launch():
    """Every order 1..8 mixed at random over a periodic set (h = 2.2 s, enough neighbours for
    order 8): the one-launch build over all orders equals the oracle node by node (statuses and
    weights)."""
    ns = S.jittered_lattice(36, 2.2, 8, seed=61)
    order = (1 + np.floor(S.uniform01(62, ns.n) * 8)).astype(np.int8)
    ops = ("dx", "dy")
    _, rp, col, w, status, _ = G.gpu_run(ns, 8, ops, order=order)
    assert set(np.unique(order)) == set(range(1, 9))
    q = np.arange(1, ns.n, 2)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, 8, ops, q, rp_q, col_q, order=order)
    assert np.array_equal(status[q], r64["status"])
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label="random orders")


def test_fp32_weight_storage():
    k = 6
    ns = S.jittered_lattice(32, G.HS[k], k, seed=41)
    ops = G.OPS[k]
    _, rp, col, w32, _, _ = G.gpu_run(ns, k, ops, weight_dtype="f32")
    _, _, _, w64, _, _ = G.gpu_run(ns, k, ops, weight_dtype="f64")
    assert np.array_equal(w32, w64.astype(np.float32).astype(np.float64))


# ---------------------------------------------------------------------------------- status codes


def test_status_codes_match_oracle():
    """Undersampled (N_i < p), collinear (singular M) and coincident (non-finite M) stencils."""
    xs = np.linspace(0.3, 0.7, 21)
    line = np.stack([xs, np.full_like(xs, 0.5)], 1)  # collinear nodes
    sparse = np.array([[0.1, 0.1], [0.12, 0.1], [0.1, 0.13]])  # 2 neighbours < p
    dup = np.array([[0.8, 0.8], [0.8, 0.8]])  # coincident pair
    rng = S.uniform01(77, 40).reshape(20, 2) * 0.08 + 0.76
    xy = np.concatenate([line, sparse, dup, rng])
    h = np.full(len(xy), 0.06)
    ns = S.NodeSet(xy=xy, h=h, s=h, order=np.full(len(xy), 2, np.int8), periodic=False, lo=(0.0, 0.0),
                   hi=(1.0, 1.0))
    ops = ("dx", "dy", "lap")
    _, rp, col, w, status, nbad = G.gpu_run(ns, 2, ops)
    q = np.arange(ns.n)
    r64 = oracle.build_weights(ns.xy, ns.h, False, rp, col, G.c_matrix(2, ops), k=2, queries=q)
    assert np.array_equal(status, r64["status"])
    assert nbad == int(np.sum(status != 0))
    assert set(status.tolist()) >= {1, 2, 3}
    for t in np.nonzero(status)[0]:
        assert np.all(w[rp[t]:rp[t + 1]] == 0)


# ---------------------------------------------------------------------------------- apply


@pytest.mark.parametrize("k", [4, 6, 8])
def test_apply_parity(k):
    import torch

    ns = S.jittered_lattice(48, G.HS[k], k, seed=50 + k)
    ops = G.OPS[k]
    L, rp, col, w, status, _ = G.gpu_run(ns, k, ops)
    f = S.fourier_field(n_modes=8, kmax=4, seed=3).value(ns.xy)
    dev = torch.device("cuda", 0)
    out = L.apply(torch.from_numpy(f).to(dev)).cpu().numpy()
    # (a) the gather-sum itself: same weights through the oracle's apply.  Two summation
    # orders of sum_j (f_j - f_i) w_j differ by at most ~N u sum_j |(f_j - f_i) w_j|.
    ref_same = oracle.apply(rp, col, w, f)
    absterm = np.abs(f[col] - np.repeat(f, np.diff(rp)))[:, None] * np.abs(w)
    bound = np.add.reduceat(absterm, rp[:-1], axis=0).T  # [n_ops, n]
    assert np.all(np.abs(out - ref_same) <= 1e-14 * bound + 1e-300)
    # (b) end to end against the binary128 oracle, bounded by the FP64 oracle's own error
    q = np.arange(0, ns.n, 4)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q)
    d_ld = oracle.apply(rp_q, col_q, rld["w"], f, queries=q, precision=G.REF_PRECISION)
    d_64 = oracle.apply(rp_q, col_q, r64["w"], f, queries=q)
    sc = np.abs(d_ld).max(axis=1)
    e_gpu = (np.abs(out[:, q] - d_ld).max(axis=1)) / sc
    e_64 = (np.abs(d_64 - d_ld).max(axis=1)) / sc
    assert np.all(e_gpu <= np.maximum(G.TOL_FLOOR_MAX, G.FLOOR_FACTOR * e_64)), (e_gpu, e_64)


def test_apply_op_mask_and_fp32():
    import torch

    k = 4
    ns = S.jittered_lattice(40, G.HS[k], k, seed=61)
    ops = G.OPS[k]
    L, rp, col, w, _, _ = G.gpu_run(ns, k, ops)
    f = S.sincos_field().value(ns.xy)
    dev = torch.device("cuda", 0)
    full = L.apply(torch.from_numpy(f).to(dev)).cpu().numpy()
    part = L.apply(torch.from_numpy(f).to(dev), op_mask=0b1010).cpu().numpy()
    assert np.array_equal(part, full[[1, 3]])
    f32 = L.apply(torch.from_numpy(f.astype(np.float32)).to(dev)).cpu().numpy()
    # float fields: (f_j - f_i) w summed in double then rounded, with f rounded to float on
    # input -> error within a few ulp(float) of sum_j |f_j| |w_j| (the operators cancel large terms)
    absterm = (np.abs(f[col]) + np.abs(np.repeat(f, np.diff(rp))))[:, None] * np.abs(w)
    bound = np.add.reduceat(absterm, rp[:-1], axis=0).T
    assert np.all(np.abs(f32 - full) <= 4 * 2.0 ** -24 * bound + 2.0 ** -24 * np.abs(full))


# ---------------------------------------------------------------------------------- RK4


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rk4_parity(dtype):
    import torch

    k = 4
    # h/dr = 2 (as in Sec. 5.1) keeps every eigenvalue of this operator in the left half-plane
    ns = S.jittered_lattice(32, 2.0, k, seed=71, jitter=0.2)
    ops = ("dx", "dy", "lap")
    L, rp, col, w, _, _ = G.gpu_run(ns, k, ops)
    # diffusion-dominated advection-diffusion with the heat-equation step of Sec. 5.1
    # (dt = 0.05 h^2 / kappa): stable, so rounding differences are not amplified
    beta = np.array([-0.1, -0.05, 1.0])
    dt = 0.05 * ns.h[0] ** 2
    u0 = S.sincos_field().value(ns.xy)
    frozen = np.zeros(ns.n, np.uint8)
    frozen[::7] = 1
    dev = torch.device("cuda", 0)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u = torch.from_numpy(u0).to(dev, tdt)
    fz = torch.from_numpy(frozen).to(dev)
    L.step(beta, u, dt, 10, frozen=fz)
    L.step(beta, u, dt, 10, frozen=fz)  # replays the recorded graph
    got = u.cpu().numpy().astype(np.float64)
    ref = oracle.rk4(rp, col, w, beta, u0, dt, 20, frozen=frozen)
    tol = 1e-12 if dtype == "f64" else 2e-5
    assert np.abs(got - ref).max() < tol * np.abs(ref).max()
    assert np.array_equal(got[::7], u0[::7].astype(np.float32 if dtype == "f32" else np.float64).astype(np.float64))


def test_rk4_parity_order8_hyperviscosity():
    """The time-stepping operator at order 8: advection + diffusion + the -alpha nabla^8
    hyperviscosity of Sec. 4.2 (alpha = 1e-3 h^8), quadratic ABFs in the dw0 form on +-0.2 dr
    noise, where every eigenvalue has a non-positive real part; 30 steps against the oracle."""
    import torch

    k = 8
    ns = S.jittered_lattice(40, 2.2, k, seed=72, jitter=0.2)
    ops = ("dx", "dy", "lap", "lap4")
    L, rp, col, w, status, _ = G.gpu_run(ns, k, ops, rbf="quadratic", abf_form="dw0")
    assert (status == 0).all()
    h = ns.h[0]
    beta = np.array([-1.0, -0.5, 1e-3, -1e-3 * h ** 8])
    # RK4 step inside its stability region: dt = 2 / rho, rho = spectral radius of the operator
    A = np.zeros((ns.n, ns.n))
    node = np.repeat(np.arange(ns.n), np.diff(rp))
    np.add.at(A, (node, col), w @ beta)
    np.add.at(A, (node, node), -(w @ beta))
    lam = np.linalg.eigvals(A)
    assert lam.real.max() < 1e-9 * np.abs(lam).max()  # no growing mode
    dt = 2.0 / np.abs(lam).max()
    u0 = S.sincos_field().value(ns.xy)
    dev = torch.device("cuda", 0)
    u = torch.from_numpy(u0).to(dev)
    L.step(beta, u, dt, 30)
    got = u.cpu().numpy()
    ref = oracle.rk4(rp, col, w, beta, u0, dt, 30)
    assert np.isfinite(ref).all() and np.abs(ref).max() < 1.01
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


# ---------------------------------------------------------------------------------- errors


def test_argument_and_state_errors():
    import torch

    from paper_1912_06441_gb300 import Labfm, LabfmError

    dev = torch.device("cuda", 0)
    L = Labfm(0)
    xy = torch.rand(100, 2, dtype=torch.float64, device=dev)
    h = torch.full((100,), 0.1, dtype=torch.float64, device=dev)
    with pytest.raises(LabfmError) as e:
        L.apply(torch.zeros(100, dtype=torch.float64, device=dev))
    assert e.value.status == 7
    bad_h = h.clone()
    bad_h[3] = -1.0
    with pytest.raises(LabfmError) as e:
        L.build_neighbours(xy, bad_h, True)
    assert e.value.status == 1
    outside = xy.clone()
    outside[5, 0] = 1.5
    with pytest.raises(LabfmError) as e:
        L.build_neighbours(outside, h, False)
    assert e.value.status == 1
    L.build_neighbours(xy, h, True)
    order = torch.full((100,), 9, dtype=torch.int8, device=dev)
    with pytest.raises(LabfmError) as e:
        L.build_weights(G.c_matrix(2, ("dx",)), order=order)
    assert e.value.status == 1
    # rbf values outside LABFM_RBF_* | LABFM_ABF_DW0_ONLY are rejected on the host
    import ctypes as ct

    C = np.zeros((1, 44))
    C[0, 0] = 1.0
    nbad = ct.c_int64()
    for bad_rbf in (5, 0x200, 0x101 | 0x400, -1):
        st = L.lib.labfm_build_weights(L._ctx, None, 2, bad_rbf, 1, C.ctypes.data_as(ct.c_void_p), 0, 0, None,
                                       ct.byref(nbad))
        assert st == 1, bad_rbf
    st = L.lib.labfm_build_weights(L._ctx, None, 2, 0x101, 1, C.ctypes.data_as(ct.c_void_p), 0, 0, None,
                                   ct.byref(nbad))
    assert st in (0, 5)
