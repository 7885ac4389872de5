"""Benchmark of the LABFM hot path on GB300.

One step = the whole path over the 512 x 512 jittered periodic lattice (262,144 nodes,
+-0.3 s jitter, h = 2.2 s, Wendland C2, order k = 8, p = 44): stencil search, FP64 weight
build for d/dx, d/dy, nabla^2 and nabla^8, application of the four operators to a sum of
16 random Fourier modes, and one classical RK4 step of advection-diffusion with nabla^8
hyperviscosity.  The headline value is nodes per second through that step (Mnodes/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl labfm|reference]

``--impl reference`` times the CPU oracle (plain C, FP64) on a bounded sample of the same
workload on the host cores.  Under torchrun each rank runs its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import labfm_synth as S  # noqa: E402

METRIC = "order-8 weight build Mnodes/s; apply GB/s vs HBM; mixed vs FP64 at ≤1e-8 err"
N_SIDE, HS, K, JITTER = 512, 2.2, 8, 0.3
SKIP_LARGE = False  # --skip-large: leave out the heat-equation, Burgers and Poisson runs (thousands
                    # of small launches), the 4.2M-node RK4 and the 1M-node wall workloads
OPS = ("dx", "dy", "lap", "lap4")
def workload_name():
    return (f"2D periodic jittered lattice {N_SIDE}x{N_SIDE} (+-{JITTER}s), h={HS}s, Wendland C2, order {K} "
            f"(p=44), FP64 weights for dx, dy, lap, lap4; apply to 16 Fourier modes (k<=32); 1 RK4 step")
C_ADV = (1.0, 0.5)
NU = 1e-3
HV = 1e-3  # hyperviscosity coefficient alpha = HV * h^8 of the -alpha nabla^8 term


def p_of_k(k):
    return (k * k + 3 * k) // 2


def build_flops_per_node(k, ni, n_ops):
    """Algorithmic FP64 flops of the weight build for one node (p = p(k), N_i neighbours):
    ABF/monomial evaluation (the |r|-derivative polynomials: 2 flops per coefficient),
    assembly 2 p^2 N_i, elimination 2/3 p^3 + 2 p^2 n_ops (both triangular sweeps of the
    right-hand sides), weights 2 p N_i n_ops."""
    p = p_of_k(k)
    coef = sum((n + 1) * (n + 1) for n in range(1, k + 1))
    return 2 * coef * ni + 2 * p * p * ni + (2.0 / 3.0) * p ** 3 + 2 * p * p * n_ops + 2 * p * ni * n_ops


def apply_bytes(n, nnz, n_ops, wbytes=8, fbytes=8):
    """Algorithmic bytes of one application of n_ops operators: per stencil entry one int32
    index and n_ops weights; per node f_i, row pointer and n_ops outputs (the f_j gathers hit
    L2 and count once per node)."""
    return nnz * (4 + n_ops * wbytes) + n * (fbytes + 8 + n_ops * fbytes)


def scan_launches(n):
    items = 2048
    nb = (n + items - 1) // items
    if nb <= 1:
        return 1
    return 2 + scan_launches(nb)


def ncells_of(h, box=1.0):
    """Cells of the stencil-search grid for uniform h on the unit box (same rule as the library)."""
    nc = max(1, int(np.floor(box / (2.0 * h * (1.0 + 1e-9)))))
    return nc * nc


def nbr_launches(n, ncells):
    # check, assign, scan(cells)+total, scatter, count sweep, scan(rows)+total, fill sweep
    return 1 + 1 + scan_launches(ncells) + 1 + 1 + 1 + scan_launches(n) + 1 + 1


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples (the JSON line carries their summary); LABFM_CLOCKS_DIR keeps them
        self.path = os.path.join(os.environ.get("LABFM_CLOCKS_DIR") or tempfile.gettempdir(),
                                 f"labfm_clocks_{os.getpid()}.csv")

    def start(self):
        if not shutil.which("nvidia-smi"):
            return
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                     stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_fp64_peak(torch, dev):
    """FP64 dense peak measured here with cuBLAS DGEMM (4096^3, best of 5), in TFLOP/s."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


def measured_fp32_peak(torch, dev):
    """FP32 FFMA peak measured here with cuBLAS SGEMM (8192^3, TF32 off: the FP32 pipes), TFLOP/s."""
    n = 8192
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        a = torch.randn(n, n, dtype=torch.float32, device=dev)
        b = torch.randn(n, n, dtype=torch.float32, device=dev)
        torch.matmul(a, b)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return 2.0 * n ** 3 / best / 1e12


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback"


def workload(seed_offset=0):
    ns = S.jittered_lattice(N_SIDE, HS, K, jitter=JITTER, seed=2 + 100 * seed_offset)
    field = S.fourier_field(n_modes=16, kmax=32, seed=3 + 100 * seed_offset)
    C = np.stack([S.op_c_vector(o, K) for o in OPS])
    h = ns.h[0]
    beta = np.array([-C_ADV[0], -C_ADV[1], NU, -HV * h ** 8])
    # explicit RK4 step: advective CFL 0.5 on the lattice spacing, bounded by the diffusive limit
    s = 1.0 / N_SIDE
    dt = min(0.5 * s / np.hypot(*C_ADV), 0.1 * s * s / NU)
    return ns, field, C, beta, dt


def cpu_baseline(ns, field, C, sample=1024, seed=9):
    """The oracle as it stands on a bounded sample of the workload: brute-force stencils of
    `sample` nodes over all N, FP64 weights and the four operators, timed on the host cores."""
    import oracle

    threads = os.cpu_count() or 1
    q = np.sort(np.unique((S.uniform01(seed, sample) * ns.n).astype(np.int64)))
    f = field.value(ns.xy)
    oracle.build("f64")
    t0 = time.perf_counter()
    rp, col = oracle.neighbours(ns.xy, ns.h, True, queries=q)
    r = oracle.build_weights(ns.xy, ns.h, True, rp, col, C, k=K, queries=q, nthreads=threads)
    oracle.apply(rp, col, r["w"], f, queries=q, nthreads=threads)
    t = time.perf_counter() - t0
    return {"value": len(q) / t / 1e6, "unit": "Mnodes/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(q)} of {ns.n} nodes: brute-force stencils over all nodes (1 thread), "
                      f"FP64 build + apply of 4 operators ({threads} OpenMP threads)",
            "seconds": t}


# Per-order accuracy workloads: 512^2 jittered lattices (+-0.3 s), h/s above the critical h/dr of
# Sec. 3.2 for each order, Wendland C2, and d/dx, d/dy, nabla^2 and the highest even power of the
# Laplacian the order reproduces (the hyperviscosity operator of Sec. 4.2).
ACC_HS = {2: 1.2, 3: 1.3, 4: 1.4, 5: 1.6, 6: 1.8, 7: 2.0, 8: 2.2}
ACC_SAMPLE = 512


def acc_ops(k):
    m = min(k // 2, 4)
    return ("dx", "dy", "lap") + ((f"lap{m}",) if m >= 2 else ())


def hard_nodes():
    """The ill-conditioned stencils of the order-8 workload that the oracle picks
    (tests/golden/hard_nodes_lattice512_k8.txt)."""
    return np.loadtxt(os.path.join(ROOT, "tests", "golden", "hard_nodes_lattice512_k8.txt"), dtype=np.int64,
                      comments="#")


def _err_stats(d, ref):
    """Per operator, over the sampled nodes: |d - ref| relative to the operator's largest |ref|
    (median, p99, max, fraction of nodes <= 1e-8) and the normalised L2 norm of Sec. 4.1."""
    sc = np.abs(ref).max(axis=1, keepdims=True)
    e = np.abs(d - ref) / sc
    return {"median": np.median(e, axis=1).tolist(), "p99": np.percentile(e, 99, axis=1).tolist(),
            "max": e.max(axis=1).tolist(), "frac_le_1e-8": (e <= 1e-8).mean(axis=1).tolist(),
            "l2": (np.linalg.norm(d - ref, axis=1) / np.linalg.norm(ref, axis=1)).tolist()}


def accuracy_vs_oracle(torch, P, dev, local_rank):
    """The oracle leg's accuracy table: for k = 2..8, the derivatives of every build variant
    (FP64; mixed and mixed_tc with the default adaptive refinement; mixed_tc weights stored in
    FP32 and applied to an FP32 field) at ACC_SAMPLE seeded nodes (plus, at k = 8, the oracle's
    ill-conditioned nodes, reported apart) against the same oracle in IEEE binary128; the FP64
    oracle beside them as the floor of FP64 arithmetic."""
    import oracle

    out = {"reference": "oracle in IEEE binary128 (same algorithm)", "sample_nodes": ACC_SAMPLE,
           "workload": "512^2 jittered lattice (+-0.3 s, seed 2), Wendland C2, h/s = " +
                       ", ".join(f"{ACC_HS[k]} (k={k})" for k in ACC_HS) + "; 16 Fourier modes (k <= 32)",
           "orders": {}}
    f_all = S.fourier_field(n_modes=16, kmax=32, seed=3)
    for k in range(2, 9):
        ops = acc_ops(k)
        ns = S.jittered_lattice(N_SIDE, ACC_HS[k], k, jitter=JITTER, seed=2)
        f = f_all.value(ns.xy)
        C = np.stack([S.op_c_vector(o, k) for o in ops])
        q_rand = np.unique((S.uniform01(900 + k, ACC_SAMPLE) * ns.n).astype(np.int64))
        sets = {"sample": q_rand}
        if k == 8 and N_SIDE == 512:
            sets["ill_conditioned"] = hard_nodes()
        q = np.unique(np.concatenate(list(sets.values())))
        L = P.Labfm(local_rank)
        L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
        rp_d, col_d = L.get_neighbours()
        rp = rp_d.cpu().numpy()
        lens = rp[q + 1] - rp[q]
        rp_q = np.concatenate([[0], np.cumsum(lens)])
        col_q = np.concatenate([col_d[int(rp[i]):int(rp[i + 1])].cpu().numpy() for i in q])
        rq = oracle.build_weights(ns.xy, ns.h, True, rp_q, col_q, C, k=k, queries=q, precision="q")
        r64 = oracle.build_weights(ns.xy, ns.h, True, rp_q, col_q, C, k=k, queries=q)
        d_q = oracle.apply(rp_q, col_q, rq["w"], f, queries=q, precision="q")
        d_64 = oracle.apply(rp_q, col_q, r64["w"], f, queries=q)
        pos = {name: np.searchsorted(q, sel) for name, sel in sets.items()}
        variants = {}
        fd = torch.from_numpy(f).to(dev)
        f32 = torch.from_numpy(f.astype(np.float32)).to(dev)
        for name, prec, wdt in (("fp64", "fp64", "f64"), ("mixed", "mixed", "f64"), ("mixed_tc", "mixed_tc", "f64"),
                                ("mixed_tc_f32_storage", "mixed_tc", "f32")):
            L.build_weights(C, uniform_order=k, precision=prec, weight_dtype=wdt)
            d = L.apply(fd if wdt == "f64" else f32).cpu().numpy().astype(np.float64)[:, q]
            variants[name] = (d, L.get_build_info() if prec != "fp64" else None)
        rec = {"ops": list(ops), "h_over_s": ACC_HS[k]}
        for sname, ps in pos.items():
            blk = {"nodes": int(len(ps)), "fp64_oracle": _err_stats(d_64[:, ps], d_q[:, ps])}
            for name, (d, info) in variants.items():
                blk[name] = _err_stats(d[:, ps], d_q[:, ps])
            rec[sname] = blk
        rec["refine_steps"] = {name: info["refine_steps"] for name, (d, info) in variants.items() if info}
        rec["fp64_rebuilt"] = {name: info["fp64_rebuilt"] for name, (d, info) in variants.items() if info}
        out["orders"][str(k)] = rec
        L.close()
    return out


def kernel_source_hash():
    import hashlib

    hsh = hashlib.sha256()
    for f in ("build_fp64.cu", "abf.cuh"):
        with open(os.path.join(ROOT, "paper_1912_06441_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()


def build_traffic(n):
    """DRAM bytes per launch of the build kernel from the committed ncu capture, scaled by
    node count; None if the kernel source changed since the capture."""
    prof = os.path.join(ROOT, "profiles", "build_fp64_traffic.json")
    try:
        with open(prof) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    if rec.get("source_sha256") != kernel_source_hash():
        return None
    return rec["dram_bytes_per_node"] * n


def _time(torch, fn, reps=3):
    best = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def deriv_errors(d, ref):
    """Per operator: |d - ref| relative to max |ref| (median, 99th percentile, max over nodes)
    and the normalised L2 norm of Sec. 4.1."""
    d = d.astype(np.float64)
    ref = ref.astype(np.float64)
    sc = np.abs(ref).max(axis=1, keepdims=True)
    e = np.abs(d - ref) / sc
    return {"l2": (np.linalg.norm(d - ref, axis=1) / np.linalg.norm(ref, axis=1)).tolist(),
            "median": np.median(e, axis=1).tolist(), "p99": np.percentile(e, 99, axis=1).tolist(),
            "max": e.max(axis=1).tolist(), "frac_nodes_le_1e-8": (e <= 1e-8).mean(axis=1).tolist()}


def mixed_vs_fp64(torch, P, dev, local_rank, nsx, k, ops, field):
    """Mixed-precision and FP64 builds of the same node set: build time, the refinement steps
    the nodes took, and the difference of the mixed derivatives from the FP64 ones (both on the
    GPU), per operator.  The difference is not an error of the mixed build: against the binary128
    oracle the FP64 build is the less accurate of the two (accuracy_vs_oracle)."""
    n = nsx.n
    L = P.Labfm(local_rank)
    L.build_neighbours(torch.from_numpy(nsx.xy).to(dev), torch.from_numpy(nsx.h).to(dev), True)
    C = np.stack([S.op_c_vector(o, k) for o in ops])
    f = torch.from_numpy(field.value(nsx.xy)).to(dev)
    res = {}
    ders = {}
    for prec in ("fp64", "mixed", "mixed_tc"):
        L.build_weights(C, uniform_order=k, precision=prec)
        ms = _time(torch, lambda: L.build_weights(C, uniform_order=k, precision=prec))
        ders[prec] = L.apply(f).cpu().numpy()
        res[prec] = {"ms": ms, "mnodes_per_s": n / (ms * 1e-3) / 1e6}
        info = L.get_build_info()
        if prec == "fp64":
            res[prec]["fp64_group_threads"] = info["fp64_group_threads"]
        else:
            res[prec].update(info)
    res["speedup_mixed_over_fp64"] = res["fp64"]["ms"] / res["mixed"]["ms"]
    res["speedup_mixed_tc_over_fp64"] = res["fp64"]["ms"] / res["mixed_tc"]["ms"]
    # the FP64 build's algorithmic flops per node (the same work for every variant) over each
    # variant's time: FP64-equivalent TFLOP/s, set against the FP64 pipe's measured peak
    ni = L.nnz / n
    flops = build_flops_per_node(k, ni, len(ops)) * n
    for prec in ("fp64", "mixed", "mixed_tc"):
        res[prec]["fp64_equivalent_tflops"] = flops / (res[prec]["ms"] * 1e-3) / 1e12
    res["ops"] = list(ops)
    res["deriv_diff_mixed_vs_fp64"] = deriv_errors(ders["mixed"], ders["fp64"])
    res["deriv_diff_mixed_tc_vs_fp64"] = deriv_errors(ders["mixed_tc"], ders["fp64"])
    res["refinement"] = "adaptive (per node, at most 6 steps; diverging nodes rebuilt in FP64)"
    L.close()
    return res


def extra_measurements(torch, P, dev, local_rank, ns, field, hbm):
    """Outside the timed step: FP64 and mixed-precision builds at order 8 and order 6
    (h = 1.8 s, nabla^6 for the hyperviscosity operator) with the mixed-vs-FP64 derivative
    errors, and the FP32-weight / FP32-field apply."""
    out = {}
    n = ns.n
    out["order8_mixed_vs_fp64"] = mixed_vs_fp64(torch, P, dev, local_rank, ns, K, OPS, field)
    ns6 = S.jittered_lattice(N_SIDE, 1.8, 6, jitter=JITTER, seed=2)
    out["order6_mixed_vs_fp64"] = mixed_vs_fp64(torch, P, dev, local_rank, ns6, 6, ("dx", "dy", "lap", "lap3"),
                                                field)
    L32 = P.Labfm(local_rank)
    xy = torch.from_numpy(ns.xy).to(dev)
    h = torch.from_numpy(ns.h).to(dev)
    L32.build_neighbours(xy, h, True)
    C = np.stack([S.op_c_vector(o, K) for o in OPS])
    L32.build_weights(C, uniform_order=K, weight_dtype="f32")
    f32 = torch.from_numpy(field.value(ns.xy).astype(np.float32)).to(dev)
    o32 = torch.empty((len(OPS), n), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    L32.apply(f32, out=o32)  # tunes the launch shape
    flush.zero_()
    # 20 back-to-back launches: the 325 MB the kernel streams exceed the 129 MB L2, so each
    # launch reads its weights from HBM; the average leaves out the host launch latency
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        L32.apply(f32, out=o32)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    by = apply_bytes(n, L32.nnz, len(OPS), wbytes=4, fbytes=4)
    out["apply_f32"] = {"kernel": "k_apply<4,float,float>", "ms": ms, "achieved_gbs": by / (ms * 1e-3) / 1e9,
                        "frac_of_hbm": by / (ms * 1e-3) / 1e9 / hbm, "algorithmic_bytes": by,
                        "derivatives_per_s": len(OPS) * n / (ms * 1e-3),
                        "timing": f"mean of {reps} back-to-back launches (inputs larger than L2)"}
    L32.close()
    if not SKIP_LARGE:
        out["heat_dirichlet_k4"] = heat_dirichlet(torch, P, dev, local_rank)
        out["burgers_cole_k4"] = burgers_cole(torch, P, dev, local_rank)
        out["poisson_periodic_k4"] = poisson_periodic(torch, P, dev, local_rank)
        out["poisson_neumann_k4"] = poisson_neumann(torch, P, dev, local_rank)
        out["poisson_annulus"] = poisson_annulus(torch, P, dev, local_rank)
        out["rk4_2048"] = rk4_large(torch, P, dev, local_rank)
        out["walls_1m_variable_order"] = walls_variable_order(torch, P, dev, local_rank)
    return out


def heat_dirichlet(torch, P, dev, local_rank, k=4, h_over_H=0.0125, chunk=5000):
    """The heat equation with Dirichlet walls of Sec. 5.1 at the finest resolution of its table:
    161 x 161 nodes (h/dr = 2, interior noise eps/dr = 0.5, wall nodes and the two rows inside
    them on the lattice), quadratic ABFs in the dW0/dr form, order 4, u(x, 0) = sin(pi x) and 0
    on the other walls (frozen), RK4 from zero interior values to t* = 8 pi^2 t = 100 in graph
    replays of `chunk` steps; error of the steady state against the exact one."""
    ns = S.dirichlet_square(int(round(2.0 / h_over_H)) + 1, 2.0, k, 0.5, seed=100 + k)
    L = P.Labfm(local_rank)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), False)
    st = torch.zeros(ns.n, dtype=torch.int32, device=dev)
    nbad = L.build_weights(np.stack([S.op_c_vector("lap", k)]), uniform_order=k, rbf="quadratic",
                           abf_form="dw0", node_status=st)
    # spectral radius of the Laplacian on the internal rows (power iteration, walls held at 0)
    keep = torch.from_numpy(~ns.wall).to(dev, torch.float64)
    v = torch.randn(ns.n, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    rho = 0.0
    for _ in range(100):
        v = v * keep
        v = L.apply(v / v.norm())[0] * keep
        rho = float(v.norm())
    dt = min(0.05 * ns.h[0] ** 2, 0.8 * 2.785 / rho)  # Sec. 5.1's 0.05 h^2, within the RK4 region
    nsteps = int(math.ceil(100.0 / (8.0 * math.pi ** 2) / dt))
    nchunks = (nsteps + chunk - 1) // chunk
    field = S.HeatSteadyField()
    ub = field.boundary(ns.xy, ns.wall)
    u = torch.from_numpy(ub).to(dev)
    fz = torch.from_numpy(ns.wall.astype(np.uint8)).to(dev)
    L.step([1.0], u, dt, chunk, frozen=fz)  # records the graph (tunes the stage shape first)
    u.copy_(torch.from_numpy(ub).to(dev))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(nchunks):
        L.step([1.0], u, dt, chunk, frozen=fz)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    got = u.cpu().numpy()
    ex = field.value(ns.xy)
    steps = nchunks * chunk
    res = {"nodes": ns.n, "nnz": int(L.nnz), "order": k, "h_over_H": h_over_H, "flagged_nodes": int(nbad),
           "spectral_radius_h2": rho * ns.h[0] ** 2, "dt_over_h2": dt / ns.h[0] ** 2, "steps": steps,
           "t_star": 8.0 * math.pi ** 2 * dt * steps, "ms": ms, "steps_per_s": steps / (ms * 1e-3),
           "us_per_step": ms * 1e3 / steps,
           "l2_err_vs_exact_steady": float(np.linalg.norm(got - ex) / np.linalg.norm(ex)),
           "paper_l2_err": 2.9e-10, "walls_unchanged": bool(np.array_equal(got[ns.wall], ub[ns.wall]))}
    L.close()
    return res


def burgers_cole(torch, P, dev, local_rank, k=4, nside=161, Re=100.0, T=1.0, chunk=500):
    """The periodic Burgers' problem of Sec. 5.3: u = sin(2 pi x), v = 0 on a 161 x 161 noisy
    Cartesian set (h/dr = 2, eps/dr = 0.2), quadratic ABFs in the dW0/dr form, order 4,
    Re = 100, RK4 to t = 1 with the time step of Eq. (tstep) in graph replays of `chunk` steps;
    error against Cole's exact solution."""
    ns = S.jittered_lattice(nside, 2.0, k, jitter=0.2 / math.sqrt(2), seed=7)
    L = P.Labfm(local_rank)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
    nbad = L.build_weights(np.stack([S.op_c_vector(o, k) for o in ("dx", "dy", "lap")]), uniform_order=k,
                           rbf="quadratic", abf_form="dw0", node_status=torch.zeros(ns.n, dtype=torch.int32, device=dev))
    h = ns.h[0]
    nsteps = int(math.ceil(T / min(0.2 * h, 0.05 * h * h * Re) / chunk)) * chunk
    dt = T / nsteps
    beta = [0.0, 0.0, 1.0 / Re]
    u0 = torch.from_numpy(np.sin(2 * np.pi * ns.xy[:, 0])).to(dev)
    u, v = u0.clone(), torch.zeros(ns.n, dtype=torch.float64, device=dev)
    L.step_burgers(beta, u, v, dt, chunk)  # records the graph (tunes the stage shape first)
    u.copy_(u0)
    v.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(nsteps // chunk):
        L.step_burgers(beta, u, v, dt, chunk)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    ex = S.ColeBurgersSolution(Re).u(ns.xy[:, 0], T)
    got = u.cpu().numpy()
    res = {"nodes": ns.n, "nnz": int(L.nnz), "order": k, "Re": Re, "T": T, "flagged_nodes": int(nbad),
           "steps": nsteps, "dt": dt, "ms": ms, "steps_per_s": nsteps / (ms * 1e-3), "us_per_step": ms * 1e3 / nsteps,
           "l2_err_vs_cole": float(np.linalg.norm(got - ex) / np.linalg.norm(ex)),
           "max_abs_v": float(v.abs().max())}
    L.close()
    return res


def poisson_periodic(torch, P, dev, local_rank, k=4, nside=512, tol=1e-10):
    """The periodic Poisson problem of Sec. 5.2 at 512 x 512 nodes (h/dr = 2, eps/dr = 0.5,
    quadratic ABFs in the dW0/dr form, order 4): phi = sin 2 pi x sin 2 pi y, node 0 fixed,
    solved by labfm_solve (Jacobi-preconditioned BiCGStab, FP64) from zero to a relative
    residual of 1e-10; error against the exact solution."""
    ns = S.jittered_lattice(nside, 2.0, k, jitter=0.5 / math.sqrt(2), seed=3)
    L = P.Labfm(local_rank)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
    nbad = L.build_weights(np.stack([S.op_c_vector("lap", k)]), uniform_order=k, rbf="quadratic", abf_form="dw0",
                           node_status=torch.zeros(ns.n, dtype=torch.int32, device=dev))
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    ex = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    f = -8 * np.pi ** 2 * ex
    f[0] = ex[0]
    dm = np.zeros(ns.n, np.uint8)
    dm[0] = 1
    fd, dmd = torch.from_numpy(f).to(dev), torch.from_numpy(dm).to(dev)
    phi = torch.zeros(ns.n, dtype=torch.float64, device=dev)
    L.solve(0, fd, phi, dmd, tol=tol, max_iter=100000)  # warm (allocations, first launches)
    phi.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters, resid = L.solve(0, fd, phi, dmd, tol=tol, max_iter=100000)  # synchronises at the end
    ms = (time.perf_counter() - t0) * 1e3
    got = phi.cpu().numpy()
    spmv_bytes = L.nnz * (4 + 8) + ns.n * (8 + 8 + 8 + 8)  # col, w; row_ptr, x_i, out, one dot operand
    res = {"nodes": ns.n, "nnz": int(L.nnz), "order": k, "flagged_nodes": int(nbad), "tol": tol, "iterations": iters,
           "true_rel_residual": resid, "ms": ms, "us_per_iteration": ms * 1e3 / max(iters, 1),
           "l2_err_vs_exact": float(np.linalg.norm(got - ex) / np.linalg.norm(ex)),
           "spmv_bytes": spmv_bytes, "timing": "host wall clock around the call (it synchronises)"}
    L.close()
    return res


def poisson_neumann(torch, P, dev, local_rank, k=4, nside=257, tol=1e-10):
    """Poisson's equation with the Neumann ghost-node rows of Sec. 5.2: the unit square of
    labfm_synth.neumann_square at 257 x 257 lattice nodes plus one ghost per Neumann wall node
    (Dirichlet walls at x = 0, 1; Neumann walls at y = 0, 1; h/dr = 2, interior noise eps/dr = 0.5,
    quadratic ABFs in the dW0/dr form, order 4), phi = sin(2 pi x + 0.3) cos(3 pi y - 0.2) (nonzero
    normal derivative on both Neumann walls), solved by labfm_solve_neumann from zero to a
    relative residual of 1e-10; error against phi at the lattice nodes."""
    q = S.neumann_square(nside, 2.0, k, 0.5, seed=21)
    ns = q.ns
    L = P.Labfm(local_rank)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), False, ns.lo, ns.hi)
    C = np.stack([S.op_c_vector(o, k) for o in ("dx", "dy", "lap")])
    st = torch.zeros(ns.n, dtype=torch.int32, device=dev)
    L.build_weights(C, uniform_order=k, rbf="quadratic", abf_form="dw0", node_status=st)
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    a, b = 2 * np.pi, 3 * np.pi
    ex = np.sin(a * x + 0.3) * np.cos(b * y - 0.2)
    f = np.where(q.dirichlet, ex, -(a * a + b * b) * ex)
    xb, yb = x[q.parent], y[q.parent]
    f[q.ghost] = q.normal[:, 1] * (-b * np.sin(a * xb + 0.3) * np.sin(b * yb - 0.2))  # n = (0, +-1)
    fd = torch.from_numpy(f).to(dev)
    dmd = torch.from_numpy(q.dirichlet.astype(np.uint8)).to(dev)
    nm = (torch.from_numpy(q.ghost).to(dev), torch.from_numpy(q.parent).to(dev), torch.from_numpy(q.normal).to(dev),
          0, 1)
    phi = torch.zeros(ns.n, dtype=torch.float64, device=dev)
    L.solve(2, fd, phi, dmd, tol=tol, max_iter=100000, neumann=nm)  # warm (allocations, first launches)
    phi.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters, resid = L.solve(2, fd, phi, dmd, tol=tol, max_iter=100000, neumann=nm)  # synchronises at the end
    ms = (time.perf_counter() - t0) * 1e3
    got = phi.cpu().numpy()
    keep = np.ones(ns.n, bool)
    keep[q.ghost] = False
    status = st.cpu().numpy()
    res = {"nodes": ns.n, "ghost_rows": int(len(q.ghost)), "nnz": int(L.nnz), "order": k, "tol": tol,
           "flagged_lattice_nodes": int((status[keep] != 0).sum()), "flagged_ghost_nodes": int((status[~keep] != 0).sum()),
           "iterations": iters, "true_rel_residual": resid, "ms": ms, "us_per_iteration": ms * 1e3 / max(iters, 1),
           "l2_err_vs_exact": float(np.linalg.norm(got[keep] - ex[keep]) / np.linalg.norm(ex[keep])),
           "timing": "host wall clock around the call (it synchronises)"}
    L.close()
    return res


ANNULUS_TABLE = {  # Sec. 5.2, Table of the annular problem: relative L2 error at h/H = 2/m, m = 97, 193, 385
    2: (9.1e-3, 2.3e-3, 5.9e-4), 3: (9.5e-3, 2.4e-3, 6.0e-4), 4: (1.4e-4, 6.5e-6, 3.6e-7)}


def poisson_annulus(torch, P, dev, local_rank, levels=(97, 193, 385), tol=2e-12):
    """The annular Poisson problem of Sec. 5.2 on the GPU at the three finest resolutions of its
    table (h/H = 2/97, 2/193, 2/385; up to 110 k nodes), k = 2, 3, 4: nodes by
    labfm_synth.annulus_nodes (the paper's shifting rule, seed 31), quadratic ABFs in the dw0
    form, h = 2 dr; Dirichlet g1 = 0 on the outer circle, Neumann g2 = cos(3 theta) on the inner
    one through ghost rows; labfm_solve_neumann from zero to a relative residual of 2e-12; error
    against r sin(4 pi r) cos(3 theta) beside the printed one."""
    out = {"printed": {str(k): v for k, v in ANNULUS_TABLE.items()}, "levels": list(levels)}
    for k in (2, 3, 4):
        rows = []
        for m in levels:
            q = S.annulus_nodes(m, k, seed=31)
            ns = q.ns
            L = P.Labfm(local_rank)
            L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), False, ns.lo, ns.hi)
            C = np.stack([S.op_c_vector(o, k) for o in ("dx", "dy", "lap")])
            st = torch.zeros(ns.n, dtype=torch.int32, device=dev)
            L.build_weights(C, uniform_order=k, rbf="quadratic", abf_form="dw0", node_status=st)
            x, y = ns.xy[:, 0], ns.xy[:, 1]
            ex = S.annulus_solution(x, y)
            f = np.where(q.dirichlet, 0.0, S.annulus_source(x, y))
            f[q.ghost] = np.cos(3 * np.arctan2(y[q.parent], x[q.parent]))
            nm = (torch.from_numpy(q.ghost).to(dev), torch.from_numpy(q.parent).to(dev),
                  torch.from_numpy(q.normal).to(dev), 0, 1)
            phi = torch.zeros(ns.n, dtype=torch.float64, device=dev)
            keep = np.ones(ns.n, bool)
            keep[q.ghost] = False
            t0 = time.perf_counter()
            try:
                iters, resid = L.solve(2, torch.from_numpy(f).to(dev), phi,
                                       torch.from_numpy(q.dirichlet.astype(np.uint8)).to(dev), tol=tol,
                                       max_iter=100000, neumann=nm)
                ok = True
            except P.LabfmError as e:
                iters, resid, ok = L.last_solve[0], L.last_solve[1], False
            ms = (time.perf_counter() - t0) * 1e3
            got = phi.cpu().numpy()
            rows.append({"m": m, "nodes": ns.n, "ghosts": int(len(q.ghost)), "converged": ok, "iterations": iters,
                         "true_rel_residual": resid, "ms": ms,
                         "flagged_nodes": int((st.cpu().numpy()[keep] != 0).sum()),
                         "l2_err": float(np.linalg.norm(got[keep] - ex[keep]) / np.linalg.norm(ex[keep]))})
            L.close()
        out[str(k)] = rows
    return out


RK4_JITTER = 0.1       # noise of the time-stepping node set: every order-8 stencil well conditioned
RK4_RBF = "quadratic"  # the kernel of the PDE tests of Sec. 5
RK4_ABF = "dw0"        # dW0/dr-only ABFs: the form the stability results of Sec. 4.2 belong to


def spectral_radius(torch, L, beta, iters=80):
    """Largest |lambda| of u -> sum_d beta_d L^d(u) by power iteration through labfm_apply."""
    dev = torch.device("cuda", L.device)
    g = torch.Generator(device=dev).manual_seed(0)
    v = torch.randn(L.n, dtype=torch.float64, device=dev, generator=g)
    v /= v.norm()
    b = torch.tensor(beta, dtype=torch.float64, device=dev)[:, None]
    rho = 0.0
    for _ in range(iters):
        wv = (b * L.apply(v)).sum(0)
        rho = float(wv.norm())
        v = wv / rho
    return rho


def rk4_large(torch, P, dev, local_rank, n_side=2048, nsteps=1000):
    """The time-stepping workload: 2048^2 jittered periodic nodes (+-0.1 s), order 8, quadratic
    ABFs in the dW0/dr-only form, weights built once, then nsteps of RK4 for
    u_t + c.grad u = nu lap u - alpha nabla^8 u (c = (1, 0.5), nu = 1e-3, alpha = 1e-3 h^8)
    replayed from one CUDA graph; FP32 fields with FP64 weights and with FP32 weights; error
    against the exact advected, decayed mode."""
    ns = S.jittered_lattice(n_side, HS, K, jitter=RK4_JITTER, seed=5)
    n = ns.n
    C = np.stack([S.op_c_vector(o, K) for o in OPS])
    h = ns.h[0]
    beta = [-C_ADV[0], -C_ADV[1], NU, -HV * h ** 8]
    res = {"nodes": n, "steps": nsteps, "jitter": RK4_JITTER, "rbf": RK4_RBF, "abf_form": RK4_ABF}
    xy = torch.from_numpy(ns.xy).to(dev)
    hh = torch.from_numpy(ns.h).to(dev)
    u0 = S.sincos_field().value(ns.xy)
    dt = None
    for wdt in ("f64", "f32"):
        L = P.Labfm(local_rank)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        L.build_neighbours(xy, hh, True)
        nbad = L.build_weights(C, uniform_order=K, rbf=RK4_RBF, abf_form=RK4_ABF, weight_dtype=wdt,
                               node_status=torch.zeros(n, dtype=torch.int32, device=dev))
        e1.record()
        e1.synchronize()
        if dt is None:
            # advective CFL 0.5, and 0.8 x the RK4 stability radius on the real axis against the
            # spectral radius of the right-hand side (FP64 weights)
            rho = spectral_radius(torch, L, beta)
            s = 1.0 / n_side
            dt = min(0.5 * s / float(np.hypot(*C_ADV)), 0.8 * 2.785 / rho)
            res["spectral_radius"] = rho
            res["dt"] = dt
        u = torch.from_numpy(u0.astype(np.float32)).to(dev)
        L.step(beta, u, dt, nsteps)  # warm: tunes the stage launch shape and records the graph
        u.copy_(torch.from_numpy(u0.astype(np.float32)).to(dev))
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        L.step(beta, u, dt, nsteps)
        t1.record()
        t1.synchronize()
        ms = t0.elapsed_time(t1)
        T = dt * nsteps
        x, y = ns.xy[:, 0], ns.xy[:, 1]
        exact = np.exp(-8 * np.pi ** 2 * NU * T) * np.sin(2 * np.pi * (x - C_ADV[0] * T)) * \
            np.cos(2 * np.pi * (y - C_ADV[1] * T))
        got = u.cpu().numpy().astype(np.float64)
        if wdt == "f32":
            # the FP32 apply of all four operators on this 4.2M-node set (1.3 GB per launch)
            f = torch.from_numpy(u0.astype(np.float32)).to(dev)
            o = torch.empty((len(OPS), n), dtype=torch.float32, device=dev)
            L.apply(f, out=o)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            for _ in range(10):
                L.apply(f, out=o)
            a1.record()
            a1.synchronize()
            ams = a0.elapsed_time(a1) / 10
            aby = apply_bytes(n, L.nnz, len(OPS), wbytes=4, fbytes=4)
            res["apply_f32"] = {"ms": ams, "achieved_gbs": aby / (ams * 1e-3) / 1e9,
                                "frac_of_hbm": aby / (ams * 1e-3) / 1e9 / hbm_peak()[0],
                                "derivatives_per_s": len(OPS) * n / (ams * 1e-3)}
            del f, o
        wb = 8 if wdt == "f64" else 4
        stage_bytes = L.nnz * (4 + wb) + n * (8 + 4 + 4 * 3)  # col + combined weight; row_ptr, u, src, acc, next
        sub = (np.arange(n) // n_side % 8 == 0) & (np.arange(n) % n_side % 8 == 0)  # the 256^2 subsample
        res[f"weights_{wdt}"] = {
            "build_ms": e0.elapsed_time(e1), "flagged_nodes": int(nbad), "T": T,
            "ms_per_step": ms / nsteps, "steps_per_s": nsteps / (ms * 1e-3),
            "stage_gbs": 4 * stage_bytes / (ms / nsteps * 1e-3) / 1e9,
            "l2_err_vs_exact": float(np.linalg.norm(got - exact) / np.linalg.norm(exact)),
            "l2_err_vs_exact_256_subsample": float(np.linalg.norm(got[sub] - exact[sub]) /
                                                   np.linalg.norm(exact[sub])),
            "max_abs_u": float(np.abs(got).max())}
        del u
        L.close()
        torch.cuda.empty_cache()
    res["nnz"] = int(L.nnz)
    return res


def _host_spectral_radius(A, iters=80):
    """Largest |lambda| of the sparse matrix A by power iteration on the host (seeded start)."""
    v = np.random.default_rng(0).standard_normal(A.shape[0])
    v /= np.linalg.norm(v)
    rho = 0.0
    for _ in range(iters):
        wv = A @ v
        rho = float(np.linalg.norm(wv))
        v = wv / rho
    return rho


def rk4_oracle_leg(torch, P, dev, local_rank, n_side=2048, sub_side=256, nsteps=1000):
    """The time-stepping workload against the oracle.  (1) The 2048^2 set's 256^2 subsample (every
    8th lattice node in x and y): the GPU's stencil rows against the oracle's (bit for bit), and
    the derivatives of u0 through the GPU's FP64 weights against the FP64 oracle's weights at
    those 65,536 nodes.  (2) An independent 256^2 set with the same parameters (seed 6): nsteps
    of RK4 by the oracle (its own stencils, weights and FP64 fields) against the GPU's graph-
    replayed steps with FP32 fields on FP64 weights and on FP32 weights (and FP64 fields on FP64
    weights, the floor), all from the same dt."""
    import oracle

    out = {"reference": "FP64 oracle"}
    C = np.stack([S.op_c_vector(o, K) for o in OPS])
    ns = S.jittered_lattice(n_side, HS, K, jitter=RK4_JITTER, seed=5)
    n = ns.n
    sub = np.nonzero((np.arange(n) // n_side % 8 == 0) & (np.arange(n) % n_side % 8 == 0))[0]
    u0 = S.sincos_field().value(ns.xy)
    L = P.Labfm(local_rank)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
    L.build_weights(C, uniform_order=K, rbf=RK4_RBF, abf_form=RK4_ABF)
    rp_d, col_d = L.get_neighbours()
    rp = rp_d.cpu().numpy()
    lens = rp[sub + 1] - rp[sub]
    rows = torch.from_numpy(np.concatenate([np.arange(rp[i], rp[i + 1]) for i in sub])).to(dev)
    col_sub = col_d[rows].cpu().numpy()
    w_gpu = L.get_weights()[rows].cpu().numpy().astype(np.float64)
    d_gpu = L.apply(torch.from_numpy(u0).to(dev))[:, torch.from_numpy(sub).to(dev)].cpu().numpy()
    L.close()
    del rows, rp_d, col_d
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    orp, ocol = oracle.neighbours_large(ns.xy, ns.h, True, queries=sub)
    r = oracle.build_weights(ns.xy, ns.h, True, orp, ocol, C, k=K, rbf=RK4_RBF, abf_form=RK4_ABF, queries=sub)
    d_or = oracle.apply(orp, ocol, r["w"], u0, queries=sub)
    exact_rows = bool(np.array_equal(np.diff(orp), lens) and np.array_equal(ocol, col_sub))
    res = {"nodes": int(len(sub)), "stencils_bit_exact": exact_rows, "oracle_status_ok": int((r["status"] == 0).sum()),
           "oracle_s": time.perf_counter() - t0}
    if exact_rows:
        # per node and operator: the weights normwise, ||w_gpu - w_oracle|| / ||w_oracle||, and the
        # derivative of u0 relative to the sum of its terms, |d_gpu - d_oracle| / sum_j |(u_j - u_i) w_ji|
        # (the nabla^8 of a smooth mode at h ~ 1e-3 cancels terms ~1e14 times larger than the
        # result, so its error relative to the result itself only measures that cancellation)
        starts = orp[:-1]
        wn = np.sqrt(np.add.reduceat(r["w"] ** 2, starts, axis=0)).T
        wd = np.sqrt(np.add.reduceat((w_gpu - r["w"]) ** 2, starts, axis=0)).T / wn
        terms = np.abs(u0[ocol] - np.repeat(u0[sub], lens))[:, None] * np.abs(r["w"])
        dd = np.abs(d_gpu - d_or) / np.add.reduceat(terms, starts, axis=0).T
        res["weights_normwise"] = {"median": np.median(wd, axis=1).tolist(), "max": wd.max(axis=1).tolist()}
        res["deriv_err_over_term_sum"] = {"median": np.median(dd, axis=1).tolist(), "max": dd.max(axis=1).tolist()}
        res["deriv_err_vs_scale"] = _err_stats(d_gpu, d_or)
    out["subsample_2048"] = res
    # (2) an independent 256^2 set, full RK4 on both sides
    ns = S.jittered_lattice(sub_side, HS, K, jitter=RK4_JITTER, seed=6)
    h = ns.h[0]
    beta = np.array([-C_ADV[0], -C_ADV[1], NU, -HV * h ** 8])
    u0 = S.sincos_field().value(ns.xy)
    t0 = time.perf_counter()
    orp, ocol = oracle.neighbours_large(ns.xy, ns.h, True)
    r = oracle.build_weights(ns.xy, ns.h, True, orp, ocol, C, k=K, rbf=RK4_RBF, abf_form=RK4_ABF)
    rho = _host_spectral_radius(oracle.operator_matrix(orp, ocol, r["w"], beta))
    dt = min(0.5 / sub_side / float(np.hypot(*C_ADV)), 0.8 * 2.785 / rho)
    u_or = oracle.rk4(orp, ocol, r["w"], beta, u0, dt, nsteps)
    oracle_s = time.perf_counter() - t0
    T = dt * nsteps
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    exact = np.exp(-8 * np.pi ** 2 * NU * T) * np.sin(2 * np.pi * (x - C_ADV[0] * T)) * \
        np.cos(2 * np.pi * (y - C_ADV[1] * T))
    rk = {"nodes": ns.n, "seed": 6, "steps": nsteps, "dt": dt, "spectral_radius_oracle": rho, "oracle_s": oracle_s,
          "oracle_l2_err_vs_exact": float(np.linalg.norm(u_or - exact) / np.linalg.norm(exact))}
    sc = float(np.abs(u_or).max())
    for wdt, fdt in (("f64", torch.float64), ("f64", torch.float32), ("f32", torch.float32)):
        L = P.Labfm(local_rank)
        L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
        L.build_weights(C, uniform_order=K, rbf=RK4_RBF, abf_form=RK4_ABF, weight_dtype=wdt)
        u = torch.from_numpy(u0).to(dev, fdt)
        L.step(beta, u, dt, nsteps)
        got = u.cpu().numpy().astype(np.float64)
        L.close()
        key = f"gpu_{'f64' if fdt == torch.float64 else 'f32'}_fields_{wdt}_weights"
        rk[key] = {"max_diff_vs_oracle": float(np.abs(got - u_or).max() / sc),
                   "l2_diff_vs_oracle": float(np.linalg.norm(got - u_or) / np.linalg.norm(u_or)),
                   "l2_err_vs_exact": float(np.linalg.norm(got - exact) / np.linalg.norm(exact))}
    out["independent_256_rk4"] = rk
    return out


def walls_variable_order(torch, P, dev, local_rank, n_side=1000):
    """Non-periodic unit square with walls, spacing varying 4x, per-node order 2..8 (capped at 4
    near walls): the build with nodes bucketed by (order, stencil size), in FP64 (one persistent
    launch over all orders) and in mixed precision (orders 2-4 in that launch, orders 5-8 through
    the mixed kernels), with the group sizes the build autotuner chose."""
    ns = S.variable_wall_nodes(n_side, seed=4)
    n = ns.n
    L = P.Labfm(local_rank)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), False)
    order = torch.from_numpy(ns.order.astype(np.int8)).to(dev)
    C = np.stack([S.op_c_vector(o, 8) for o in ("dx", "dy", "lap")])
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    res = {"nodes": n, "nnz": int(L.nnz), "order_counts": {int(k): int(v) for k, v in
                                                           zip(*np.unique(ns.order, return_counts=True))}}
    for prec in ("fp64", "mixed", "mixed_tc"):
        L.build_weights(C, order=order, precision=prec, node_status=status)
        ms = _time(torch, lambda: L.build_weights(C, order=order, precision=prec, node_status=status), reps=2)
        st = status.cpu().numpy()
        res[prec] = {"ms": ms, "mnodes_per_s": n / (ms * 1e-3) / 1e6,
                     "flagged_nodes": int((st != 0).sum())}
        res[prec].update(L.get_build_info())
    L.close()
    return res


def max_over_ranks(torch, x, world, device):
    """The largest of every rank's x (the slowest replica sets a multi-GPU step time)."""
    if world <= 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replicas_throughput(world, nodes_per_rank, ms_per_step):
    """Whole-job Mnodes/s of `world` replicas, each building nodes_per_rank nodes per step."""
    return world * nodes_per_rank / (ms_per_step * 1e-3) / 1e6


def run_reference(args, rank, world):
    if rank != 0:
        return
    ns, field, C, beta, dt = workload()
    for _ in range(args.warmup):
        cpu_baseline(ns, field, C, sample=256)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(ns, field, C, sample=args.ref_sample))
    v = float(np.mean([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mnodes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean([x["seconds"] for x in vals])) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(), "sample_nodes": args.ref_sample},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "Mnodes/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_labfm(args, rank, world, local_rank):
    import torch

    import paper_1912_06441_gb300 as P

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    P.load_library()
    ns, field, C, beta, dt = workload(seed_offset=rank)
    n = ns.n
    f_host = field.value(ns.xy)
    xy_h = torch.from_numpy(ns.xy).pin_memory()
    h_h = torch.from_numpy(ns.h).pin_memory()
    f_h = torch.from_numpy(f_host).pin_memory()
    u0 = S.sincos_field().value(ns.xy)
    xy = xy_h.to(dev)
    h = h_h.to(dev)
    f = f_h.to(dev)
    u = torch.from_numpy(u0).to(dev)
    out = torch.empty((len(OPS), n), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    L = P.Labfm(local_rank)

    def step(ev=None):
        if ev is not None:
            ev[0].record()
        L.build_neighbours(xy, h, True)
        if ev is not None:
            ev[1].record()
        L.build_weights(C, uniform_order=K)
        if ev is not None:
            ev[2].record()
        L.apply(f, out=out)
        if ev is not None:
            ev[3].record()
        L.step(beta, u, dt, 1)
        if ev is not None:
            ev[4].record()

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record()
    for s in range(args.steps):
        flush.zero_()
        step(evs[s])
    t_end.record()
    barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    phase = np.array([[evs[s][t].elapsed_time(evs[s][t + 1]) for t in range(4)] for s in range(args.steps)])
    total_ms = max_over_ranks(torch, total_ms, world, dev)
    ms_per_step = total_ms / args.steps
    value = replicas_throughput(world, n, ms_per_step)

    # e2e through the public API from pinned host buffers: H2D of xy, h, f; D2H of the
    # derivatives and the stepped field, every step
    out_h = torch.empty((len(OPS), n), dtype=torch.float64).pin_memory()
    u_h = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(e2e_steps):
        xy.copy_(xy_h, non_blocking=True)
        h.copy_(h_h, non_blocking=True)
        f.copy_(f_h, non_blocking=True)
        step()
        out_h.copy_(out, non_blocking=True)
        u_h.copy_(u, non_blocking=True)
    e1.record()
    barrier()
    e2e_ms = max_over_ranks(torch, e0.elapsed_time(e1) / e2e_steps, world, dev)
    h2d = xy_h.numel() * 8 + h_h.numel() * 8 + f_h.numel() * 8
    d2h = out_h.numel() * 8 + u_h.numel() * 8

    if rank != 0:
        return
    nnz = L.nnz
    ni = nnz / n
    build_ms = float(np.mean(phase[:, 1]))
    apply_ms = float(np.mean(phase[:, 2]))
    fp64_peak = measured_fp64_peak(torch, dev)
    bflops = build_flops_per_node(K, ni, len(OPS)) * n
    b_ach = bflops / (build_ms * 1e-3) / 1e12
    abytes = apply_bytes(n, nnz, len(OPS))
    a_ach = abytes / (apply_ms * 1e-3) / 1e9
    hbm, hbm_src = hbm_peak()
    traffic = build_traffic(n)
    line = {
        "metric": METRIC, "value": value, "unit": "Mnodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(), "nodes": n, "nnz": nnz, "order": K, "ops": list(OPS),
                   "l2": "256 MB buffer written between timed steps (inside the timed region)",
                   "parallelism": f"replicas x{world}"},
        "phases_ms": {"neighbours": float(np.mean(phase[:, 0])), "build_fp64": build_ms, "apply": apply_ms,
                      "rk4_step": float(np.mean(phase[:, 3]))},
        "roofline": {"bound": "alu", "kernel": "k_build_fp64<8> (FP64 weight build)", "achieved": b_ach,
                     "peak": fp64_peak, "unit": "TFLOP/s", "frac": b_ach / fp64_peak, "traffic": traffic,
                     "peak_source": "cuBLAS DGEMM 4096^3 measured in this run (FP64 pipe)",
                     "algorithmic_flops_per_node": bflops / n},
        "apply_roofline": {"bound": "hbm", "kernel": "k_apply<4,double,double>", "achieved": a_ach, "peak": hbm,
                           "unit": "GB/s", "frac": a_ach / hbm, "peak_source": hbm_src,
                           "algorithmic_bytes": abytes,
                           "derivatives_per_s": len(OPS) * n / (apply_ms * 1e-3),
                           # on GB300 this FP64 kernel is bound by the FP64 pipe, not by HBM: one
                           # subtraction and n_ops multiply-adds per stencil entry
                           "fp64_pipe": {"achieved_tflops": nnz * (1 + 2 * len(OPS)) / (apply_ms * 1e-3) / 1e12,
                                         "peak_tflops": fp64_peak,
                                         "frac": nnz * (1 + 2 * len(OPS)) / (apply_ms * 1e-3) / 1e12 / fp64_peak},
                           "f32_variant": None},
        "build_mnodes_per_s": n / (build_ms * 1e-3) / 1e6,
        "e2e": {"value": replicas_throughput(world, n, e2e_ms), "unit": "Mnodes/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        # per step: stencil search, one build launch (uniform order), one apply, and the RK4
        # step (operator combination + 4 stage kernels)
        "gpu_launches": args.steps * (nbr_launches(n, ncells_of(HS / N_SIDE)) + 1 + 1 + 1 + 4),
        "clocks": clk,
    }
    line["build_tuning"] = L.get_build_info()["fp64_group_threads"]
    line["extra"] = extra_measurements(torch, P, dev, local_rank, ns, field, hbm)
    fp32_peak = measured_fp32_peak(torch, dev)
    line["extra"]["peaks"] = {"fp64_tflops": fp64_peak, "fp64_source": "cuBLAS DGEMM 4096^3 (FP64 pipe)",
                              "fp32_tflops": fp32_peak, "fp32_source": "cuBLAS SGEMM 8192^3, TF32 off (FFMA pipes)",
                              "hbm_gbs": hbm, "hbm_source": hbm_src}
    for key in ("order8_mixed_vs_fp64", "order6_mixed_vs_fp64"):
        for prec in ("fp64", "mixed", "mixed_tc"):
            r = line["extra"][key][prec]
            r["fp64_equivalent_frac_of_fp64_peak"] = r["fp64_equivalent_tflops"] / fp64_peak
    a32 = line["extra"].get("apply_f32")
    if a32:  # the HBM-bound variant of the apply, beside the FP64-pipe-bound one above
        line["apply_roofline"]["f32_variant"] = {
            "kernel": a32["kernel"], "achieved": a32["achieved_gbs"], "peak": hbm, "unit": "GB/s",
            "frac": a32["frac_of_hbm"], "algorithmic_bytes": a32["algorithmic_bytes"], "timing": a32["timing"],
            "at_4M_nodes_frac": line["extra"].get("rk4_2048", {}).get("apply_f32", {}).get("frac_of_hbm")}
    if not args.no_cpu_baseline:
        # the oracle leg: the CPU baseline, and the accuracy of every build variant against it
        line["cpu_baseline"] = cpu_baseline(ns, field, C, sample=args.cpu_sample)
        line["extra"]["accuracy_vs_oracle"] = accuracy_vs_oracle(torch, P, dev, local_rank)
        if not SKIP_LARGE:
            line["extra"]["rk4_2048"]["oracle"] = rk4_oracle_leg(torch, P, dev, local_rank)
    print(json.dumps(line), flush=True)
    L.close()


PROFILE_CASES = ("apply_f32_512", "apply_f64_512", "stage_df_1024", "stage_f32_1024", "build_fp64_256",
                 "build_mixed_256", "build_mixed_tc_256", "solve_poisson_512")


def profile_case(name):
    """A small, untimed run of one kernel family, for profiler captures (ncu -k ... python bench.py
    --profile NAME): the workloads above at sizes that hold a few GB at most."""
    import torch

    import paper_1912_06441_gb300 as P

    dev = torch.device("cuda", 0)
    L = P.Labfm(0)
    if name == "solve_poisson_512":
        # the periodic Poisson workload of bench.py, 40 BiCGStab iterations (stopped short on purpose)
        ns = S.jittered_lattice(512, 2.0, 4, jitter=0.5 / math.sqrt(2), seed=3)
        L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
        L.build_weights(np.stack([S.op_c_vector("lap", 4)]), uniform_order=4, rbf="quadratic", abf_form="dw0")
        f = torch.from_numpy(-8 * np.pi ** 2 * np.sin(2 * np.pi * ns.xy[:, 0]) * np.sin(2 * np.pi * ns.xy[:, 1])).to(dev)
        dm = torch.zeros(ns.n, dtype=torch.uint8, device=dev)
        dm[0] = 1
        for _ in range(2):
            phi = torch.zeros(ns.n, dtype=torch.float64, device=dev)
            try:
                L.solve(0, f, phi, dm, tol=1e-14, max_iter=40)
            except P.LabfmError:
                pass
    elif name.startswith("apply") or name.startswith("build"):
        n_side = 512 if name.startswith("apply") else 256
        ns = S.jittered_lattice(n_side, HS, K, jitter=JITTER, seed=2)
        C = np.stack([S.op_c_vector(o, K) for o in OPS])
        L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
        wdt = "f32" if name == "apply_f32_512" else "f64"
        prec = {"build_mixed_256": "mixed", "build_mixed_tc_256": "mixed_tc"}.get(name, "fp64")
        for _ in range(1 if name.startswith("apply") else 3):
            L.build_weights(C, uniform_order=K, precision=prec, weight_dtype=wdt)
        if name.startswith("apply"):
            f = torch.from_numpy(field_for_profile(ns)).to(dev, torch.float32 if wdt == "f32" else torch.float64)
            for _ in range(30):
                L.apply(f)
    else:
        ns = S.jittered_lattice(1024, HS, K, jitter=RK4_JITTER, seed=5)
        C = np.stack([S.op_c_vector(o, K) for o in OPS])
        L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), True)
        L.build_weights(C, uniform_order=K, rbf=RK4_RBF, abf_form=RK4_ABF,
                        weight_dtype="f64" if name == "stage_df_1024" else "f32")
        h = ns.h[0]
        u = torch.from_numpy(S.sincos_field().value(ns.xy).astype(np.float32)).to(dev)
        for _ in range(3):
            L.step([-C_ADV[0], -C_ADV[1], NU, -HV * h ** 8], u, 1e-4, 2)
    torch.cuda.synchronize()
    L.close()


def field_for_profile(ns):
    return S.fourier_field(n_modes=16, kmax=32, seed=3).value(ns.xy)


def main():
    global N_SIDE, SKIP_LARGE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="labfm", choices=["labfm", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=1024)
    ap.add_argument("--ref-sample", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-large", action="store_true",
                    help="leave out the heat-equation, Burgers, Poisson, 2048^2 RK4 and 1000^2 wall workloads (profiler captures)")
    ap.add_argument("--n-side", type=int, default=512,
                    help="lattice side (default 512; smaller sizes are for profiler captures only)")
    ap.add_argument("--profile", choices=PROFILE_CASES, default=None,
                    help="run one small untimed case of a kernel family for a profiler capture, then exit")
    args = ap.parse_args()
    if args.profile:
        profile_case(args.profile)
        return
    N_SIDE = args.n_side
    SKIP_LARGE = args.skip_large or args.n_side != 512
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_labfm(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
