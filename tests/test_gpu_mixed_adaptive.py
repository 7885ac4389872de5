"""The adaptive refinement of the mixed-precision builds and its FP64 fallback.

By default a mixed build refines each node on the FP64 residual of the moment conditions of
Sec. 3.1 until its weights stop changing; a node whose corrections grow instead (its moment
matrix too ill conditioned for the double-float inverse) is built again by the FP64 path.

Node sets: a node whose 66 neighbours lie on three circles about it, the radii perturbed by a
relative delta (labfm_synth.three_ring_stencil: at order 8 its moment matrix is singular on the
exact circles, with a condition number growing as delta^-2), and a very noisy order-8 lattice
below the paper's critical h/dr (h = 2.0 s, jitter +-0.49 s; Sec. 3.2 gives 2.1 for k = 8)."""
import numpy as np
import pytest

import labfm_synth as S
import oracle
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

K = 8
OPS = ("dx", "dy", "lap", "lap4")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1912_06441_gb300 as P

    P.load_library()


def _runs(ns, precisions=("fp64", "mixed", "mixed_tc")):
    out = {}
    for prec in precisions:
        L, rp, col, w, st, nbad = G.gpu_run(ns, K, OPS, precision=prec)
        out[prec] = (rp, col, w, st, L.get_build_info())
        L.close()
    return out


def _same_rows(w, w64, rp):
    return np.array([np.array_equal(w[rp[i]:rp[i + 1]], w64[rp[i]:rp[i + 1]]) for i in range(len(rp) - 1)])


@pytest.mark.parametrize("precision", ["mixed", "mixed_tc"])
def test_diverging_nodes_are_rebuilt_in_fp64(precision):
    """delta = 1e-6 (condition number ~1e18): the refinement of the centre node cannot contract,
    so the FP64 build redoes it -- its weights are then the FP64 build's, bit for bit.  Every
    node the build reports as rebuilt is one whose weights equal the FP64 build's, and the
    statuses agree with the FP64 build."""
    ns = S.three_ring_stencil(1e-6)
    r = _runs(ns, ("fp64", precision))
    rp, col, w64, st64, _ = r["fp64"]
    _, _, w, st, info = r[precision]
    assert np.array_equal(st, st64)
    same = _same_rows(w, w64, rp) & (st == 0)
    assert same[0], "the centre node was not handed to the FP64 build"
    assert info["fp64_rebuilt"] == int(same.sum())
    # every node with a full elimination took refinement steps, the rebuilt ones included
    assert sum(info["refine_steps"]) == int((st == 0).sum())


@pytest.mark.parametrize("precision", ["mixed", "mixed_tc"])
def test_refinement_recovers_where_fp64_loses_accuracy(precision):
    """delta = 1e-5 (condition number ~2e15): the FP64 build's weights of the centre node are off
    by ~1e-3 against the binary128 oracle, the refined mixed weights by < 1e-6."""
    ns = S.three_ring_stencil(1e-5)
    r = _runs(ns, ("fp64", precision))
    rp, col, w64, st64, _ = r["fp64"]
    _, _, w, st, info = r[precision]
    q = np.array([0])
    rq = oracle.build_weights(ns.xy, ns.h, False, rp[:2], col[:rp[1]], G.c_matrix(K, OPS), k=K, queries=q,
                              precision=G.REF_PRECISION, lo=ns.lo, hi=ns.hi)
    e64 = G.node_rel_err(w64[:rp[1]], rq["w"], rp[:2]).max()
    em = G.node_rel_err(w[:rp[1]], rq["w"], rp[:2]).max()
    assert e64 > 1e-5, e64
    assert em < 1e-6 and em < e64 / 100, (em, e64)


@pytest.mark.parametrize("precision", ["mixed", "mixed_tc"])
def test_noisy_lattice_below_critical_spacing(precision):
    """h = 2.0 s, jitter +-0.49 s, 48^2 nodes: every node, weights against the binary128 oracle.
    Nodes the FP64 build redid carry its weights exactly; every other node is at least as
    accurate as the FP64 oracle (to 1e-11), and the refinement took more than one step on some."""
    ns = S.jittered_lattice(48, 2.0, K, jitter=0.49, seed=35)
    r = _runs(ns, ("fp64", precision))
    rp, col, w64, st64, _ = r["fp64"]
    _, _, w, st, info = r[precision]
    assert np.array_equal(st, st64)
    q = np.arange(ns.n)
    r64, rq = G.oracle_refs(ns, K, OPS, q, rp, col)
    ok = (st == 0) & (rq["status"] == 0)
    rebuilt = _same_rows(w, w64, rp) & ok
    assert info["fp64_rebuilt"] == int(rebuilt.sum())
    e = G.node_rel_err(w, rq["w"], rp).max(axis=1)
    e64 = G.node_rel_err(r64["w"], rq["w"], rp).max(axis=1)
    keep = ok & ~rebuilt
    assert np.all(e[keep] <= np.maximum(G.TOL_FLOOR_MAX, 2.0 * e64[keep])), np.max(e[keep] / np.maximum(1e-11, e64[keep]))
    assert sum(info["refine_steps"][2:]) > 0
