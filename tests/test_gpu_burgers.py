"""Burgers' equation (Sec. 5.3) on the CUDA path: labfm_step_burgers against the oracle's RK4 of
the same discrete system (FP64 and FP32, with frozen nodes and a hyperviscosity operator), and
the periodic problem with Cole's exact solution at the resolutions of the oracle's pin."""
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


def _setup(nside, k, ops, eps=0.2, seed=7, weight_dtype="f64"):
    ns = S.jittered_lattice(nside, 2.0, k, jitter=eps / math.sqrt(2), seed=seed)
    L, rp, col, w, status, _ = G.gpu_run(ns, k, ops, rbf="quadratic", abf_form="dw0", weight_dtype=weight_dtype)
    assert (status == 0).all()
    return ns, L, rp, col, w


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_burgers_parity(dtype):
    """k = 4, 32^2 nodes, operators d/dx, d/dy, nabla^2 and nabla^4: 40 steps of Burgers' equation
    with Re = 100 and a biharmonic hyperviscosity -alpha nabla^4 (alpha = 1e-2 h^4, Sec. 4.2), a
    two-dimensional initial field and every fifth node frozen, against the oracle's RK4 on the
    GPU's own weights (FP64: 1e-12 relative; FP32 fields and weights: 2e-5)."""
    import torch

    k, ops, Re = 4, ("dx", "dy", "lap", "lap2"), 100.0
    ns, L, rp, col, w = _setup(32, k, ops, weight_dtype=dtype)
    h = ns.h[0]
    beta = np.array([0.0, 0.0, 1.0 / Re, -1e-2 * h ** 4])
    x, y = ns.xy[:, 0], ns.xy[:, 1]
    u0 = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    v0 = 0.5 * np.cos(2 * np.pi * x) * np.sin(4 * np.pi * y)
    frozen = np.zeros(ns.n, np.uint8)
    frozen[::5] = 1
    dt = min(0.2 * h, 0.05 * h * h * Re)
    dev = torch.device("cuda", 0)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u = torch.from_numpy(u0).to(dev, tdt)
    v = torch.from_numpy(v0).to(dev, tdt)
    fz = torch.from_numpy(frozen).to(dev)
    L.step_burgers(beta, u, v, dt, 20, frozen=fz)
    L.step_burgers(beta, u, v, dt, 20, frozen=fz)  # replays the recorded graph
    gu, gv = u.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    ru, rv = oracle.rk4_burgers(rp, col, w, beta, u0.astype(tdt_np(dtype)), v0.astype(tdt_np(dtype)), dt, 40,
                                frozen=frozen)
    tol = 1e-12 if dtype == "f64" else 2e-5
    scale = max(np.abs(ru).max(), np.abs(rv).max())
    assert np.abs(gu - ru).max() < tol * scale and np.abs(gv - rv).max() < tol * scale
    cast = u0.astype(tdt_np(dtype)).astype(np.float64), v0.astype(tdt_np(dtype)).astype(np.float64)
    assert np.array_equal(gu[::5], cast[0][::5]) and np.array_equal(gv[::5], cast[1][::5])


def tdt_np(dtype):
    return np.float64 if dtype == "f64" else np.float32


def test_burgers_cole_convergence_on_gpu():
    """The periodic problem (u = sin(2 pi x), v = 0, Re = 100, k = 4, h/dr = 2, eps/dr = 0.2) to
    t = 0.4 at h/H = 2/81 and 2/161: the GPU solution equals the oracle's RK4 on the oracle's own
    weights to 1e-9, v stays 0, and the error against Cole's solution falls at the oracle pin's
    rate (3.0 - 4.8)."""
    import torch

    k, Re, T = 4, 100.0, 0.4
    errs = []
    for nside in (81, 161):
        ns, L, rp, col, _ = _setup(nside, k, ("dx", "dy", "lap"))
        h = ns.h[0]
        nsteps = int(math.ceil(T / min(0.2 * h, 0.05 * h * h * Re)))
        dt = T / nsteps
        u0 = np.sin(2 * np.pi * ns.xy[:, 0])
        dev = torch.device("cuda", 0)
        u = torch.from_numpy(u0).to(dev)
        v = torch.zeros(ns.n, dtype=torch.float64, device=dev)
        L.step_burgers([0.0, 0.0, 1.0 / Re], u, v, dt, nsteps)
        gu, gv = u.cpu().numpy(), v.cpu().numpy()
        orp, ocol = oracle.neighbours(ns.xy, ns.h, True)
        ow = oracle.build_weights(ns.xy, ns.h, True, orp, ocol, G.c_matrix(k, ("dx", "dy", "lap")), k=k,
                                  rbf="quadratic", abf_form="dw0")["w"]
        ru, _ = oracle.rk4_burgers(orp, ocol, ow, [0.0, 0.0, 1.0 / Re], u0, np.zeros(ns.n), dt, nsteps)
        assert np.abs(gu - ru).max() < 1e-9 * np.abs(ru).max()
        assert np.abs(gv).max() == 0.0
        ex = S.ColeBurgersSolution(Re).u(ns.xy[:, 0], T)
        errs.append(np.linalg.norm(gu - ex) / np.linalg.norm(ex))
        L.close()
    rate = math.log(errs[0] / errs[1]) / math.log(161 / 81)
    assert 3.0 <= rate <= 4.8, (errs, rate)


def test_burgers_argument_checks():
    import torch

    from paper_1912_06441_gb300 import LabfmError

    ns, L, _, _, _ = _setup(16, 2, ("dy", "dx", "lap"))  # operators 0, 1 not (d/dx, d/dy)
    dev = torch.device("cuda", 0)
    u = torch.zeros(ns.n, dtype=torch.float64, device=dev)
    v = torch.zeros(ns.n, dtype=torch.float64, device=dev)
    with pytest.raises(LabfmError):
        L.step_burgers([0.0, 0.0, 0.01], u, v, 1e-3, 1)
    ns, L, _, _, _ = _setup(16, 2, ("dx", "dy", "lap"))
    with pytest.raises(LabfmError):
        L.step_burgers([0.0, 0.0, 0.01], u, u, 1e-3, 1)  # u and v the same buffer
    L.step_burgers([0.0, 0.0, 0.01], u, v, 1e-3, 0)  # nothing to do


def test_burgers_2d_cole_hopf_on_gpu():
    """Both velocity components active (the two-dimensional Cole-Hopf solution, Re = 10, k = 4,
    t = 0.1): the GPU equals the oracle's RK4 on the oracle's weights to 1e-10 at h/H = 2/41 and
    2/81, and the error against the exact solution falls at rate 3.5 - 4.5 (oracle: 3.97)."""
    import torch

    k, Re, T = 4, 10.0, 0.1
    sol = S.ColeHopf2DSolution(Re=Re)
    errs = []
    for nside in (41, 81):
        ns, L, rp, col, _ = _setup(nside, k, ("dx", "dy", "lap"), seed=8)
        h = ns.h[0]
        nsteps = int(math.ceil(T / min(0.2 * h, 0.05 * h * h * Re)))
        dt = T / nsteps
        u0, v0 = sol.uv(ns.xy, 0.0)
        dev = torch.device("cuda", 0)
        u, v = torch.from_numpy(u0).to(dev), torch.from_numpy(v0).to(dev)
        L.step_burgers([0.0, 0.0, 1.0 / Re], u, v, dt, nsteps)
        gu, gv = u.cpu().numpy(), v.cpu().numpy()
        orp, ocol = oracle.neighbours(ns.xy, ns.h, True)
        ow = oracle.build_weights(ns.xy, ns.h, True, orp, ocol, G.c_matrix(k, ("dx", "dy", "lap")), k=k,
                                  rbf="quadratic", abf_form="dw0")["w"]
        ru, rv = oracle.rk4_burgers(orp, ocol, ow, [0.0, 0.0, 1.0 / Re], u0, v0, dt, nsteps)
        scale = max(np.abs(ru).max(), np.abs(rv).max())
        assert np.abs(gu - ru).max() < 1e-10 * scale and np.abs(gv - rv).max() < 1e-10 * scale
        eu, ev = sol.uv(ns.xy, T)
        errs.append(math.sqrt(np.sum((gu - eu) ** 2 + (gv - ev) ** 2) / np.sum(eu ** 2 + ev ** 2)))
        L.close()
    rate = math.log(errs[0] / errs[1]) / math.log(81 / 41)
    assert 3.5 <= rate <= 4.5, (errs, rate)


@pytest.mark.parametrize("field,weights", [("f32", "f64"), ("f64", "f32")])
def test_burgers_mixed_field_and_weight_types(field, weights):
    """Field and weight types that differ: the sums run in double.  20 steps of the two-
    dimensional problem against the oracle on the same weights and inputs: FP32 fields are rounded
    at every stage (2e-5); with FP32 weights the combined linear weight sum_d beta_d w^d is summed
    in double and kept as a float, one more rounding of ~6e-8 of it (1e-6)."""
    import torch

    k, Re = 4, 10.0
    ns, L, rp, col, w = _setup(32, k, ("dx", "dy", "lap"), weight_dtype=weights, seed=8)
    sol = S.ColeHopf2DSolution(Re=Re)
    u0, v0 = sol.uv(ns.xy, 0.0)
    h = ns.h[0]
    dt = min(0.2 * h, 0.05 * h * h * Re)
    dev = torch.device("cuda", 0)
    tdt = torch.float32 if field == "f32" else torch.float64
    u, v = torch.from_numpy(u0).to(dev, tdt), torch.from_numpy(v0).to(dev, tdt)
    L.step_burgers([0.0, 0.0, 1.0 / Re], u, v, dt, 20)
    gu, gv = u.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if field == "f32" else (lambda a: a)
    ru, rv = oracle.rk4_burgers(rp, col, w, [0.0, 0.0, 1.0 / Re], cast(u0), cast(v0), dt, 20)
    scale = max(np.abs(ru).max(), np.abs(rv).max())
    tol = 2e-5 if field == "f32" else 1e-6
    assert np.abs(gu - ru).max() < tol * scale and np.abs(gv - rv).max() < tol * scale
