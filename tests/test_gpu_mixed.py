"""Parity of the mixed-precision build (double-float assembly and LU on the FP32 pipes, FP64
residual refinement) with the oracle, under the same floor-aware tolerance as the FP64 build."""
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


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7, 8])
def test_mixed_weights_parity_by_order(k):
    ns = S.jittered_lattice(37, G.HS[k], k, seed=10 + k)
    ops = G.OPS[k]
    _, rp, col, w, status, _ = G.gpu_run(ns, k, ops, precision="mixed")
    q = np.arange(0, ns.n, 3)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q)
    assert np.array_equal(status[q], r64["status"])
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label=f"mixed k={k}")


@pytest.mark.parametrize("k,hs,rbf", [(4, 2.0, "quadratic"), (8, 2.2, "quadratic")])
def test_mixed_weights_parity_dw0_form(k, hs, rbf):
    """The dW0/dr-only ABF form (LABFM_ABF_DW0_ONLY) through the mixed-precision build."""
    ns = S.jittered_lattice(36, hs, k, seed=50 + k, jitter=0.2)
    ops = G.OPS[k]
    _, rp, col, w, status, _ = G.gpu_run(ns, k, ops, rbf=rbf, precision="mixed", abf_form="dw0")
    q = np.arange(2, ns.n, 3)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q, rbf=rbf, abf_form="dw0")
    assert np.array_equal(status[q], r64["status"])
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label=f"mixed dw0 k={k}")


def test_mixed_refinement_reaches_the_fp64_floor():
    """At k = 8 the double-float solution alone is far from FP64 (condition numbers ~1e12);
    each refinement step on the reproduction residual brings it down to the FP64 floor."""
    k = 8
    ns = S.jittered_lattice(32, G.HS[k], k, seed=18)
    ops = G.OPS[k]
    q = np.arange(0, ns.n, 3)
    med = []
    for nref in (0, 1, 2):
        _, rp, col, w, status, _ = G.gpu_run(ns, k, ops, precision="mixed", refine=nref)
        rp_q, col_q, idx = G.rows_of(rp, col, q)
        if nref == 0:
            r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q)
            ok = (r64["status"] == 0) & (rld["status"] == 0)
            floor = np.median(G.node_rel_err(r64["w"], rld["w"], rp_q)[ok])
        med.append(np.median(G.node_rel_err(w[idx], rld["w"], rp_q)[ok]))
    assert med[1] < med[0] and med[2] <= med[1] * 1.5, med
    assert med[2] <= max(G.TOL_FLOOR_MEDIAN, G.FLOOR_FACTOR * floor), (med, floor)


def test_mixed_variable_order_and_walls():
    ns = S.variable_wall_nodes(40, seed=4)
    ops = ("dx", "dy", "lap")
    _, rp, col, w, status, _ = G.gpu_run(ns, 8, ops, order=ns.order, precision="mixed")
    q = np.arange(0, ns.n, 3)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, 8, ops, q, rp_q, col_q, order=ns.order)
    assert np.array_equal(status[q], r64["status"])
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label="mixed variable order")


@pytest.mark.parametrize("k,hs", [(4, 3.0), (8, 2.7)])
def test_mixed_multi_chunk_stencils(k, hs):
    ns = S.jittered_lattice(40, hs, k, seed=31)
    ops = G.OPS[k]
    _, rp, col, w, status, _ = G.gpu_run(ns, k, ops, precision="mixed")
    assert np.diff(rp).min() > (64 if k < 7 else 72)
    q = np.arange(0, ns.n, 5)
    rp_q, col_q, idx = G.rows_of(rp, col, q)
    r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q)
    G.assert_weights_parity(w[idx], r64, rld, rp_q, label=f"mixed chunked k={k}")


@pytest.mark.parametrize("k", [2, 5])
def test_mixed_status_codes_match_oracle(k):
    """Undersampled (N_i < p), collinear (singular M) and coincident (non-finite M) stencils.  At
    order 2 the mixed build hands the node set to the FP64 kernel (orders below 5 are built in
    FP64); at order 5 the mixed kernels flag the nodes themselves."""
    xs = np.linspace(0.3, 0.7, 41)
    line = np.stack([xs, np.full_like(xs, 0.5)], 1)  # collinear nodes, 24 neighbours each
    sparse = np.array([[0.1, 0.1], [0.12, 0.1], [0.1, 0.13]])  # 2 neighbours < p
    dup = np.array([[0.8, 0.8], [0.8, 0.8]])  # coincident pair
    rng = S.uniform01(77, 80).reshape(40, 2) * 0.08 + 0.76
    xy = np.concatenate([line, sparse, dup, rng])
    h = np.full(len(xy), 0.06)
    ns = S.NodeSet(xy=xy, h=h, s=h, order=np.full(len(xy), k, np.int8), periodic=False, lo=(0.0, 0.0),
                   hi=(1.0, 1.0))
    ops = ("dx", "dy", "lap")
    _, rp, col, w, status, nbad = G.gpu_run(ns, k, ops, precision="mixed")
    r64 = oracle.build_weights(ns.xy, ns.h, False, rp, col, G.c_matrix(k, ops), k=k, queries=np.arange(ns.n))
    assert np.array_equal(status, r64["status"])
    assert set(status.tolist()) >= {1, 2, 3}
    for t in np.nonzero(status)[0]:
        assert np.all(w[rp[t]:rp[t + 1]] == 0)


def test_mixed_matches_fp64_build_derivatives():
    """Derivatives from the mixed build against the FP64 build on the GPU (order 6): the
    two agree to the FP64 floor."""
    import torch

    k = 6
    ns = S.jittered_lattice(64, G.HS[k], k, seed=2)
    ops = G.OPS[k]
    f = S.fourier_field(16, 8, seed=3).value(ns.xy)
    dev = torch.device("cuda", 0)
    outs = []
    for prec in ("fp64", "mixed"):
        L, rp, col, w, status, _ = G.gpu_run(ns, k, ops, precision=prec)
        outs.append(L.apply(torch.from_numpy(f).to(dev)).cpu().numpy())
    err = np.linalg.norm(outs[1] - outs[0], axis=1) / np.linalg.norm(outs[0], axis=1)
    assert np.all(err < 1e-8), err


@pytest.mark.parametrize("form,tpr", [("registers", 1), ("shared2", 2), ("shared4", 4)])
@pytest.mark.parametrize("tc", [False, True])
def test_every_inversion_form_matches_oracle(form, tpr, tc, monkeypatch):
    """Each form of the mixed builds' Gauss-Jordan inversion (rows in registers; 2 or 4 threads
    per row in shared memory), fixed through LABFM_MIXED_INVERSION, at orders 5 and 8: weights
    against the oracle under the floor-aware tolerance, and the status codes of undersampled,
    collinear and coincident stencils (order 5)."""
    monkeypatch.setenv("LABFM_MIXED_INVERSION", form)
    prec = "mixed_tc" if tc else "mixed"
    for k in (5, 8):
        ns = S.jittered_lattice(30, G.HS[k], k, seed=60 + k)
        ops = G.OPS[k]
        L, rp, col, w, status, _ = G.gpu_run(ns, k, ops, precision=prec)
        assert L.get_build_info()["mixed_inv_threads_per_row"][k] == tpr
        q = np.arange(1, ns.n, 4)
        rp_q, col_q, idx = G.rows_of(rp, col, q)
        r64, rld = G.oracle_refs(ns, k, ops, q, rp_q, col_q)
        assert np.array_equal(status[q], r64["status"])
        G.assert_weights_parity(w[idx], r64, rld, rp_q, label=f"{prec} {form} k={k}")
        L.close()
    xs = np.linspace(0.3, 0.7, 41)
    xy = np.concatenate([np.stack([xs, np.full_like(xs, 0.5)], 1), [[0.1, 0.1], [0.12, 0.1], [0.1, 0.13]],
                         [[0.8, 0.8], [0.8, 0.8]], S.uniform01(77, 80).reshape(40, 2) * 0.08 + 0.76])
    h = np.full(len(xy), 0.06)
    ns = S.NodeSet(xy=xy, h=h, s=h, order=np.full(len(xy), 5, np.int8), periodic=False, lo=(0.0, 0.0),
                   hi=(1.0, 1.0))
    L, rp, col, w, status, _ = G.gpu_run(ns, 5, ("dx", "dy", "lap"), precision=prec)
    r64 = oracle.build_weights(ns.xy, ns.h, False, rp, col, G.c_matrix(5, ("dx", "dy", "lap")), k=5,
                               queries=np.arange(ns.n))
    assert np.array_equal(status, r64["status"]) and set(status.tolist()) >= {1, 2, 3}
    L.close()
