"""GB300-native Local Anisotropic Basis Function Method (LABFM) stencil library.

A thin ctypes binding over ``liblabfm.so`` (C ABI in ``include/labfm.h``).  Every step of
the method -- stencil search, ABF/monomial evaluation, moment-matrix assembly, elimination,
weight formation, operator application and RK4 stepping -- runs in the library's CUDA
kernels; this module only checks arguments, passes device pointers and the current torch
stream, and wraps context-owned buffers as torch tensors.  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from .build import LIB as _LIB_PATH, build_library

__all__ = ["Labfm", "LabfmError", "load_library", "RBF", "PREC", "DTYPE", "NODE", "C_FUNCTIONS"]

RBF = {"wendland_c2": 0, "quadratic": 1, "cone": 2, "wendland_c6": 3, "gaussian": 4}
PREC = {"fp64": 0, "mixed": 1, "mixed_tc": 2}
ABF_FORM = {"chain": 0, "dw0": 0x100}  # LABFM_ABF_DW0_ONLY: every ABF element is dW0/dr d^alpha|r|


def precision_code(precision: str, refine: int | None = None) -> int:
    """C ABI precision value: LABFM_PREC_FP64, LABFM_PREC_MIXED[_TC] or LABFM_PREC_MIXED[_TC]_REFINE(refine)."""
    code = PREC[precision]
    if refine is not None:
        if precision not in ("mixed", "mixed_tc") or not 0 <= refine <= 4:
            raise ValueError("refine applies to precision='mixed' or 'mixed_tc', 0..4 steps")
        code |= (refine + 1) << 8
    return code
DTYPE = {"f64": 0, "f32": 1}
NODE = {"ok": 0, "singular": 1, "undersampled": 2, "nonfinite": 3}
STATUS = {0: "LABFM_OK", 1: "LABFM_ERR_ARG", 2: "LABFM_ERR_CUDA", 3: "LABFM_ERR_NOMEM", 4: "LABFM_ERR_CAPACITY",
          5: "LABFM_ERR_SINGULAR", 6: "LABFM_ERR_TIMEOUT", 7: "LABFM_ERR_STATE", 8: "LABFM_ERR_NOT_CONVERGED"}
PMAX = 44
MAX_OPS = 8

# every symbol include/labfm.h declares
C_FUNCTIONS = ["labfm_create", "labfm_destroy", "labfm_last_error", "labfm_set_stream", "labfm_build_neighbours",
               "labfm_get_neighbours", "labfm_build_weights", "labfm_get_weights", "labfm_apply", "labfm_step",
               "labfm_step_burgers", "labfm_solve", "labfm_solve_neumann", "labfm_build_neighbours_noalloc",
               "labfm_get_build_info"]
NOALLOC_MAX_NODES = 262144  # LABFM_NOALLOC_MAX_NODES

_lib = None


class LabfmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str | None = None, build_if_missing: bool = False):
    """Load liblabfm.so (built by ``__graft_entry__.build()`` or ``paper_1912_06441_gb300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        if not build_if_missing:
            raise OSError(f"liblabfm not built ({p}); run `python -m paper_1912_06441_gb300.build`")
        build_library()
    lib = ct.CDLL(p)
    P, I, I64, U32, D = ct.c_void_p, ct.c_int, ct.c_int64, ct.c_uint32, ct.c_double
    lib.labfm_create.argtypes = [ct.POINTER(P), I, P]
    lib.labfm_create.restype = I
    lib.labfm_destroy.argtypes = [P]
    lib.labfm_destroy.restype = None
    lib.labfm_last_error.argtypes = [P]
    lib.labfm_last_error.restype = ct.c_char_p
    lib.labfm_set_stream.argtypes = [P, P]
    lib.labfm_set_stream.restype = I
    lib.labfm_build_neighbours.argtypes = [P, I64, P, P, I, P, P, ct.POINTER(I64)]
    lib.labfm_build_neighbours.restype = I
    lib.labfm_get_neighbours.argtypes = [P, ct.POINTER(P), ct.POINTER(P), ct.POINTER(I64), ct.POINTER(I64)]
    lib.labfm_get_neighbours.restype = I
    lib.labfm_build_weights.argtypes = [P, P, I, I, I, P, I, I, P, ct.POINTER(I64)]
    lib.labfm_build_weights.restype = I
    lib.labfm_get_weights.argtypes = [P, ct.POINTER(P), ct.POINTER(I), ct.POINTER(I)]
    lib.labfm_get_weights.restype = I
    lib.labfm_apply.argtypes = [P, U32, P, I, P]
    lib.labfm_apply.restype = I
    lib.labfm_step.argtypes = [P, P, P, I, D, I64, P]
    lib.labfm_step.restype = I
    lib.labfm_step_burgers.argtypes = [P, P, P, P, I, D, I64, P]
    lib.labfm_step_burgers.restype = I
    lib.labfm_solve.argtypes = [P, I, P, P, P, D, I, ct.POINTER(I), ct.POINTER(D)]
    lib.labfm_solve.restype = I
    lib.labfm_solve_neumann.argtypes = [P, I, P, P, P, I64, P, P, P, I, I, D, I, ct.POINTER(I), ct.POINTER(D)]
    lib.labfm_solve_neumann.restype = I
    lib.labfm_build_neighbours_noalloc.argtypes = [I, P, I64, P, P, I, P, P, P, P, I64, ct.POINTER(I64)]
    lib.labfm_build_neighbours_noalloc.restype = I
    lib.labfm_get_build_info.argtypes = [P, ct.POINTER(_BuildInfo)]
    lib.labfm_get_build_info.restype = I
    if path is None:
        _lib = lib
    return lib


class _BuildInfo(ct.Structure):
    """labfm_build_info"""
    _fields_ = [("refine_steps", ct.c_int64 * 8), ("fp64_rebuilt", ct.c_int64), ("fp64_group_threads", ct.c_int32 * 9),
                ("mixed_inv_threads_per_row", ct.c_int32 * 9)]


class _DevView:
    """__cuda_array_interface__ wrapper so torch can view a context-owned device buffer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


def _torch():
    import torch

    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return DTYPE["f64"]
    if t.dtype == torch.float32:
        return DTYPE["f32"]
    raise TypeError(f"field dtype must be float64 or float32, got {t.dtype}")


class Labfm:
    """One library context on one CUDA device.  Method names follow the C ABI."""

    def __init__(self, device: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("labfm needs a CUDA device; no CPU fallback exists")
        self.lib = load_library()
        self.device = device
        self._ctx = ct.c_void_p()
        with torch.cuda.device(device):
            stream = torch.cuda.current_stream(device).cuda_stream
        st = self.lib.labfm_create(ct.byref(self._ctx), device, ct.c_void_p(stream))
        if st != 0:
            raise LabfmError(st, "labfm_create failed")
        self._stream = stream
        self.n = 0
        self.nnz = 0
        self.n_ops = 0

    # -- helpers -------------------------------------------------------------------------------
    def _check(self, st):
        if st != 0:
            raise LabfmError(st, self.lib.labfm_last_error(self._ctx).decode())

    def _sync_stream(self):
        torch = _torch()
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            self._check(self.lib.labfm_set_stream(self._ctx, ct.c_void_p(s)))
            self._stream = s

    def _dev(self, t, dtype, name, numel=None):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.device.index != self.device:
            raise ValueError(f"{name} must be a torch tensor on cuda:{self.device}")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if numel is not None and self.n > 0 and t.numel() != numel:
            raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
        return ct.c_void_p(t.data_ptr())

    def close(self):
        if self._ctx:
            self.lib.labfm_destroy(self._ctx)
            self._ctx = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI ---------------------------------------------------------------------------------
    def build_neighbours(self, xy, h, periodic: bool, box_lo=(0.0, 0.0), box_hi=(1.0, 1.0)) -> int:
        """Stencils |r_ji| < 2 h_i, j != i (Sec. 2).  xy: cuda float64 [n, 2]; h: cuda float64 [n]."""
        torch = _torch()
        n = int(h.numel())
        pxy = self._dev(xy, torch.float64, "xy", 2 * n)
        ph = self._dev(h, torch.float64, "h", n)
        self._sync_stream()
        lo = (ct.c_double * 2)(*box_lo)
        hi = (ct.c_double * 2)(*box_hi)
        nnz = ct.c_int64()
        self._check(self.lib.labfm_build_neighbours(self._ctx, n, pxy, ph, int(bool(periodic)), lo, hi, ct.byref(nnz)))
        self.n, self.nnz = n, int(nnz.value)
        return self.nnz

    def get_neighbours(self):
        """(row_ptr int64 [n+1], col int32 [nnz]) as torch views of context-owned memory."""
        torch = _torch()
        rp, cl = ct.c_void_p(), ct.c_void_p()
        n, nnz = ct.c_int64(), ct.c_int64()
        self._check(self.lib.labfm_get_neighbours(self._ctx, ct.byref(rp), ct.byref(cl), ct.byref(n), ct.byref(nnz)))
        dev = torch.device("cuda", self.device)
        row_ptr = torch.as_tensor(_DevView(rp.value, (n.value + 1,), "<i8"), device=dev)
        col = torch.as_tensor(_DevView(cl.value or 0, (nnz.value,), "<i4"), device=dev) if nnz.value else \
            torch.zeros(0, dtype=torch.int32, device=dev)
        return row_ptr, col

    def build_weights(self, C, order=None, uniform_order: int = 4, rbf: str = "wendland_c2",
                      precision: str = "fp64", weight_dtype: str = "f64", node_status=None,
                      refine: int | None = None, abf_form: str = "chain") -> int:
        """Weights w_ji^d for the target vectors C (rows, D ordering, Sec. 2); returns #flagged nodes.

        ``abf_form`` "chain" keeps the full chain rule in the ABF elements 1-9 (Appendix A as
        printed), "dw0" truncates every element to dW0/dr d^alpha|r| (LABFM_ABF_DW0_ONLY).

        Raises LabfmError(LABFM_ERR_SINGULAR) only if ``node_status`` is None and a node was
        flagged; with a node_status tensor the flags are returned there and the count here."""
        torch = _torch()
        Cn = np.atleast_2d(np.asarray(C, dtype=np.float64))
        n_ops = Cn.shape[0]
        if n_ops < 1 or n_ops > MAX_OPS or Cn.shape[1] > PMAX:
            raise ValueError("C must be [n_ops <= 8, p <= 44]")
        Cp = np.zeros((n_ops, PMAX))
        Cp[:, : Cn.shape[1]] = Cn
        Cp = np.ascontiguousarray(Cp)
        po = None if order is None else self._dev(order, torch.int8, "order", self.n)
        ps = None if node_status is None else self._dev(node_status, torch.int32, "node_status", self.n)
        self._sync_stream()
        nbad = ct.c_int64()
        st = self.lib.labfm_build_weights(self._ctx, po, int(uniform_order), RBF[rbf] | ABF_FORM[abf_form], n_ops,
                                          Cp.ctypes.data_as(ct.c_void_p), precision_code(precision, refine),
                                          DTYPE[weight_dtype], ps,
                                          ct.byref(nbad))
        if st == 5 and node_status is not None:
            st = 0
        self._check(st)
        self.n_ops = n_ops
        return int(nbad.value)

    def get_build_info(self):
        """Statistics of the last weight build: {"refine_steps": [nodes taking 0..7 refinement
        steps], "fp64_rebuilt": nodes the FP64 build redid (mixed builds; zeros after FP64),
        "fp64_group_threads": {order: threads per node of the FP64 kernel},
        "mixed_inv_threads_per_row": {order: threads per row of the mixed inversion}}."""
        info = _BuildInfo()
        self._check(self.lib.labfm_get_build_info(self._ctx, ct.byref(info)))
        return {"refine_steps": list(info.refine_steps), "fp64_rebuilt": int(info.fp64_rebuilt),
                "fp64_group_threads": {k: int(info.fp64_group_threads[k]) for k in range(1, 9)
                                       if info.fp64_group_threads[k]},
                "mixed_inv_threads_per_row": {k: int(info.mixed_inv_threads_per_row[k]) for k in range(1, 9)
                                              if info.mixed_inv_threads_per_row[k]}}

    def get_weights(self):
        """Context-owned weights as a torch view [nnz, n_ops]."""
        torch = _torch()
        w, dt, no = ct.c_void_p(), ct.c_int(), ct.c_int()
        self._check(self.lib.labfm_get_weights(self._ctx, ct.byref(w), ct.byref(dt), ct.byref(no)))
        typestr = "<f8" if dt.value == 0 else "<f4"
        if self.nnz == 0:
            return torch.zeros((0, no.value), dtype=torch.float64 if dt.value == 0 else torch.float32,
                               device=torch.device("cuda", self.device))
        return torch.as_tensor(_DevView(w.value, (self.nnz, no.value), typestr), device=torch.device("cuda", self.device))

    def apply(self, f, op_mask: int | None = None, out=None):
        """out[s, i] = sum_j (f_j - f_i) w_ji^d for the selected operators (Eq. general_do)."""
        torch = _torch()
        fdt = _dtype_code(f)
        pf = self._dev(f, f.dtype, "f", self.n)
        mask = (1 << self.n_ops) - 1 if op_mask is None else int(op_mask)
        nsel = bin(mask).count("1")
        if out is None:
            out = torch.empty((nsel, self.n), dtype=f.dtype, device=f.device)
        po = self._dev(out, f.dtype, "out", nsel * self.n)
        self._sync_stream()
        self._check(self.lib.labfm_apply(self._ctx, mask, pf, fdt, po))
        return out

    def step(self, beta, u, dt: float, nsteps: int, frozen=None):
        """nsteps of classical RK4 for du/dt = sum_d beta_d L^d(u) (Sec. 5.1); u is updated in place."""
        torch = _torch()
        b = np.zeros(MAX_OPS)
        bb = np.asarray(beta, dtype=np.float64)
        if bb.shape != (self.n_ops,):
            raise ValueError(f"beta must have {self.n_ops} entries")
        b[: self.n_ops] = bb
        fdt = _dtype_code(u)
        pu = self._dev(u, u.dtype, "u", self.n)
        pz = None if frozen is None else self._dev(frozen, torch.uint8, "frozen", self.n)
        self._sync_stream()
        self._check(self.lib.labfm_step(self._ctx, b.ctypes.data_as(ct.c_void_p), pu, fdt, float(dt), int(nsteps), pz))
        return u

    def step_burgers(self, beta, u, v, dt: float, nsteps: int, frozen=None):
        """nsteps of classical RK4 for Burgers' equation (Sec. 5.3):
        du/dt = -(u L^0(u) + v L^1(u)) + sum_{d>=2} beta_d L^d(u), the same for v; operators 0
        and 1 of the weights must be d/dx and d/dy.  u and v are updated in place."""
        torch = _torch()
        b = np.zeros(MAX_OPS)
        bb = np.asarray(beta, dtype=np.float64)
        if bb.shape != (self.n_ops,):
            raise ValueError(f"beta must have {self.n_ops} entries")
        b[: self.n_ops] = bb
        fdt = _dtype_code(u)
        if v.dtype != u.dtype:
            raise TypeError("u and v must have the same dtype")
        pu = self._dev(u, u.dtype, "u", self.n)
        pv = self._dev(v, v.dtype, "v", self.n)
        pz = None if frozen is None else self._dev(frozen, torch.uint8, "frozen", self.n)
        self._sync_stream()
        self._check(self.lib.labfm_step_burgers(self._ctx, b.ctypes.data_as(ct.c_void_p), pu, pv, fdt, float(dt),
                                                int(nsteps), pz))
        return u, v

    def solve(self, op: int, f, phi, dirichlet=None, tol: float = 1e-10, max_iter: int = 10000, neumann=None):
        """Solve A Phi = F (Sec. 5.2, eq. poisson_system) with the rows of operator `op` and
        identity rows where ``dirichlet`` is set, by Jacobi-preconditioned BiCGStab; phi (float64,
        the initial guess) is overwritten.  ``neumann`` = (ghost, parent, normal, op_x, op_y) adds
        the Neumann ghost-node rows (labfm_solve_neumann): cuda int64 [n_ghost] ghost and parent
        node indices, cuda float64 [n_ghost, 2] normals, and the operator indices of d/dx and d/dy.
        Returns (iterations, true relative residual); raises LabfmError(LABFM_ERR_NOT_CONVERGED) if
        the tolerance is not reached."""
        torch = _torch()
        pf = self._dev(f, torch.float64, "f", self.n)
        pp = self._dev(phi, torch.float64, "phi", self.n)
        pd = None if dirichlet is None else self._dev(dirichlet, torch.uint8, "dirichlet", self.n)
        iters, resid = ct.c_int(0), ct.c_double(0.0)
        if neumann is None:
            self._sync_stream()
            st = self.lib.labfm_solve(self._ctx, int(op), pf, pp, pd, float(tol), int(max_iter), ct.byref(iters),
                                      ct.byref(resid))
        else:
            ghost, parent, normal, op_x, op_y = neumann
            ng = ghost.numel()
            pg = self._dev(ghost, torch.int64, "ghost")
            pa = self._dev(parent, torch.int64, "parent")
            pn = self._dev(normal, torch.float64, "normal")
            if parent.numel() != ng or normal.numel() != 2 * ng:
                raise ValueError("ghost, parent and normal must describe the same n_ghost rows")
            self._sync_stream()
            st = self.lib.labfm_solve_neumann(self._ctx, int(op), pf, pp, pd, int(ng), pg, pa, pn, int(op_x),
                                              int(op_y), float(tol), int(max_iter), ct.byref(iters),
                                              ct.byref(resid))
        self.last_solve = (iters.value, resid.value)
        self._check(st)
        return iters.value, resid.value
