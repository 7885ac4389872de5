"""Write hard_nodes_lattice512_k8.txt: the ill-conditioned stencils of the 512 x 512 order-8
derivative workload, chosen by the CPU oracle alone (no GPU result enters the list).

The workload: 512 x 512 periodic jittered lattice (+-0.3 s, seed 2), h = 2.2 s, Wendland C2,
order 8, operators d/dx, d/dy, nabla^2, nabla^8, applied to 16 random Fourier modes (k <= 32,
seed 3).  At order 8 the moment matrices are ill conditioned and the FP64 build loses accuracy
to round-off (Sec. 4.1 ascribes its k = 8 errors to round-off); these are the nodes where it
loses the most.

Recipe: the oracle's stencils of every node (brute force, split over processes); the FP64
oracle's weights of every node with the smallest pivot ratio min |pivot| / max |M| of its
elimination; the binary128 oracle on the 2,000 nodes of smallest pivot ratio; then the union of
the 100 nodes of smallest pivot ratio and the 100 nodes among the 2,000 whose FP64 derivatives
differ most from the binary128 ones (relative to the largest |derivative| of each operator over
all nodes).  Takes a few minutes: run  python tests/golden/make_hard_nodes_lattice512_k8.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "hard_nodes_lattice512_k8.txt")
OPS = ("dx", "dy", "lap", "lap4")


def workload():
    import labfm_synth as S

    ns = S.jittered_lattice(512, 2.2, 8, jitter=0.3, seed=2)
    f = S.fourier_field(n_modes=16, kmax=32, seed=3).value(ns.xy)
    C = np.stack([S.op_c_vector(o, 8) for o in OPS])
    return ns, f, C


def _rows(args):
    import oracle

    n0, n1 = args
    ns, _, _ = workload()
    return oracle.neighbours(ns.xy, ns.h, True, queries=np.arange(n0, n1))


def main():
    import oracle

    ns, f, C = workload()
    nproc = os.cpu_count() or 1
    cuts = np.linspace(0, ns.n, nproc + 1).astype(np.int64)
    with mp.get_context("spawn").Pool(nproc) as pool:
        parts = pool.map(_rows, [(cuts[t], cuts[t + 1]) for t in range(nproc)])
    rp = np.concatenate([[0], np.cumsum(np.concatenate([np.diff(r) for r, _ in parts]))])
    col = np.concatenate([c for _, c in parts])
    r64 = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=8)
    assert (r64["status"] == 0).all()
    d64 = oracle.apply(rp, col, r64["w"], f)
    scale = np.abs(d64).max(axis=1)
    cand = np.sort(np.argsort(r64["piv_ratio"], kind="stable")[:2000])
    lens = rp[cand + 1] - rp[cand]
    sub_rp = np.concatenate([[0], np.cumsum(lens)])
    sub_col = np.concatenate([col[rp[i]:rp[i + 1]] for i in cand])
    rq = oracle.build_weights(ns.xy, ns.h, True, sub_rp, sub_col, C, k=8, queries=cand, precision="q")
    dq = oracle.apply(sub_rp, sub_col, rq["w"], f, queries=cand, precision="q")
    err = (np.abs(d64[:, cand] - dq) / scale[:, None]).max(axis=0)
    worst_piv = np.argsort(r64["piv_ratio"], kind="stable")[:100]
    worst_err = cand[np.argsort(-err, kind="stable")[:100]]
    nodes = np.unique(np.concatenate([worst_piv, worst_err]))
    with open(OUT, "w") as fh:
        fh.write("# Ill-conditioned order-8 stencils of the 512 x 512 jittered lattice (+-0.3 s, seed 2),\n")
        fh.write("# h = 2.2 s, Wendland C2, ops dx dy lap lap4 (Sec. 4.1: FP64 round-off at k = 8), chosen\n")
        fh.write("# by the CPU oracle: the 100 smallest pivot ratios and the 100 largest FP64-vs-binary128\n")
        fh.write("# derivative errors; written by make_hard_nodes_lattice512_k8.py (oracle only).\n")
        fh.write(f"# largest FP64 oracle derivative error among them: {err.max():.3e}\n")
        for i in nodes:
            fh.write(f"{int(i)}\n")
    print(OUT, len(nodes), "nodes; max FP64 error", err.max())


if __name__ == "__main__":
    main()
