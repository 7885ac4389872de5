"""CPU oracle for the LABFM weight build, operator application and RK4 driver.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` use this package.  The library under
``paper_1912_06441_gb300`` never imports it, and it imports nothing from there.

The numerics live in ``labfm_oracle.c`` (plain C, FP64; further builds of the
same source in ``long double`` and in IEEE binary128 measure the FP64 rounding
floor).  This module compiles it with gcc on first use and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "labfm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict = {}

RBF = {"wendland_c2": 0, "quadratic": 1, "cone": 2, "wendland_c6": 3, "gaussian": 4}
# ABF forms (Appendix A): "chain" keeps the second- and third-derivative chain-rule terms of W0 in
# the elements 1-9 (only elements >= 10 are truncated to dW0/dr d^alpha|r|); "dw0" truncates every
# element to dW0/dr d^alpha|r|.
ABF_FORM = {"chain": 0, "dw0": 0x100}
PMAX = 44
ST_OK, ST_SINGULAR, ST_UNDERSAMPLED, ST_NONFINITE = 0, 1, 2, 3


def lib_path(precision: str = "f64") -> str:
    return os.path.join(_BUILD, f"liblabfm_oracle_{precision}.so")


def _real_flags(precision: str):
    """gcc flags of one instantiation: ``f64`` double, ``ld`` long double (80-bit extended on
    x86-64, IEEE binary128 on aarch64), ``q`` _Float128 (IEEE binary128 on both)."""
    if precision == "f64":
        return ["-std=c11", "-DORC_REAL=double"]
    if precision == "ld":
        return ["-std=c11", "-DORC_REAL=long double"]
    if precision == "q":
        return ["-std=gnu11", "-D__STDC_WANT_IEC_60559_TYPES_EXT__", "-DORC_REAL=_Float128", "-DORC_MANT_DIG=113"]
    raise ValueError(precision)


def build(precision: str = "f64", force: bool = False) -> str:
    """Compile the oracle (``f64``, ``ld`` = long double or ``q`` = binary128) into ``oracle/_build``."""
    out = lib_path(precision)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", *_real_flags(precision), "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_P = ct.c_void_p
_I64 = ct.c_int64
_I = ct.c_int
_D = ct.c_double


def _configure(lib):
    lib.orc_neighbours.argtypes = [_I64, _P, _P, _I, _P, _P, _P, _I64, _P, _P, _I64]
    lib.orc_neighbours.restype = _I
    lib.orc_build_weights.argtypes = [_P, _P, _I, _P, _P, _P, _I64, _P, _P, _P, _I, _I, _I, _P,
                                      _P, _P, _P, _P, _I]
    lib.orc_build_weights.restype = _I
    lib.orc_apply.argtypes = [_P, _I64, _P, _P, _P, _I, _P, _P, _I]
    lib.orc_apply.restype = None
    lib.orc_rk4.argtypes = [_I64, _P, _P, _P, _I, _P, _P, _D, _I64, _P, _I]
    lib.orc_rk4.restype = _I
    lib.orc_rk4_burgers.argtypes = [_I64, _P, _P, _P, _I, _P, _P, _P, _D, _I64, _P, _I]
    lib.orc_rk4_burgers.restype = _I
    lib.orc_rbf_derivs.argtypes = [_I, _D, _P]
    lib.orc_rbf_derivs.restype = None
    lib.orc_dr.argtypes = [_D, _D, _I, _P]
    lib.orc_dr.restype = None
    lib.orc_monomials.argtypes = [_D, _D, _I, _P]
    lib.orc_monomials.restype = None
    lib.orc_abfs.argtypes = [_I, _D, _D, _I, _P]
    lib.orc_abfs.restype = None
    lib.orc_p_of_k.argtypes = [_I]
    lib.orc_p_of_k.restype = _I
    lib.orc_real_mant_bits.argtypes = []
    lib.orc_real_mant_bits.restype = _I
    return lib


def _lib(precision: str = "f64"):
    with _LOCK:
        if precision not in _LIBS:
            _LIBS[precision] = _configure(ct.CDLL(build(precision)))
        return _LIBS[precision]


def compile_variant(source_text: str, out_path: str, precision: str = "f64"):
    """Compile an edited copy of the oracle source and load it (used only by the test that
    plants mistakes in the oracle to check that its pins catch them)."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", "-O2", *_real_flags(precision), "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                    "-o", out_path, src, "-lm"], check=True)
    return _configure(ct.CDLL(out_path))


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def p_of_k(k: int) -> int:
    return int(_lib().orc_p_of_k(k))


def mant_bits(precision: str = "f64") -> int:
    return int(_lib(precision).orc_real_mant_bits())


def neighbours(xy, h, periodic, lo=(0.0, 0.0), hi=(1.0, 1.0), queries=None, precision="f64"):
    """Brute-force stencils (Sec. 2).  Returns (row_ptr int64 [nq+1], col int32 [nnz])."""
    lib = _lib(precision)
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    n = xy.shape[0]
    q = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = n if q is None else q.shape[0]
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    rp = np.zeros(nq + 1, dtype=np.int64)
    rc = lib.orc_neighbours(n, _ptr(xy), _ptr(h), int(periodic), _ptr(lo), _ptr(hi), _ptr(q), nq,
                            _ptr(rp), None, 0)
    assert rc == 0
    col = np.zeros(max(int(rp[-1]), 1), dtype=np.int32)
    rc = lib.orc_neighbours(n, _ptr(xy), _ptr(h), int(periodic), _ptr(lo), _ptr(hi), _ptr(q), nq,
                            _ptr(rp), _ptr(col), col.shape[0])
    assert rc == 0
    return rp, col[: int(rp[-1])]


def neighbours_large(xy, h, periodic, lo=(0.0, 0.0), hi=(1.0, 1.0), queries=None):
    """The stencils of ``neighbours`` for node sets too large for its all-pairs search (millions
    of nodes): scipy's kd-tree proposes, per query, every node within a radius 1e-9 larger than
    2 h_i (a superset of the stencil), and the predicate of Sec. 2 then decides in the same
    floating-point operations as the brute force, in IEEE double without fused multiply-add:
    dx = x_j - x_i (+-L once past L/2 in a periodic box), r2 = dx*dx + dy*dy, r2 < (2 h_i)^2,
    j != i.  Returns (row_ptr int64 [nq+1], col int32 [nnz]), rows ascending in j."""
    from scipy.spatial import cKDTree

    xy = np.ascontiguousarray(xy, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    n = xy.shape[0]
    q = np.arange(n, dtype=np.int64) if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    L = hi - lo
    if periodic:
        tree = cKDTree(xy - lo, boxsize=L)
        pts = xy[q] - lo
    else:
        tree = cKDTree(xy)
        pts = xy[q]
    rmax = float(2.0 * h[q].max()) * (1.0 + 1e-9) if len(q) else 0.0
    cand = tree.query_ball_point(pts, r=rmax)
    cnt = np.array([len(c) for c in cand], dtype=np.int64)
    row = np.repeat(np.arange(len(q), dtype=np.int64), cnt)
    j = np.concatenate([np.asarray(c, dtype=np.int64) for c in cand]) if len(q) else np.zeros(0, np.int64)
    i = q[row]
    dx = xy[j, 0] - xy[i, 0]
    dy = xy[j, 1] - xy[i, 1]
    if periodic:
        dx = np.where(dx > 0.5 * L[0], dx - L[0], np.where(dx < -0.5 * L[0], dx + L[0], dx))
        dy = np.where(dy > 0.5 * L[1], dy - L[1], np.where(dy < -0.5 * L[1], dy + L[1], dy))
    R = 2.0 * h[i]
    keep = (dx * dx + dy * dy < R * R) & (j != i)
    row, j = row[keep], j[keep]
    order = np.lexsort((j, row))
    row, j = row[order], j[order]
    rp = np.zeros(len(q) + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(row, minlength=len(q)))
    return rp, j.astype(np.int32)


def build_weights(xy, h, periodic, row_ptr, col, C, k=None, order=None, rbf="wendland_c2",
                  lo=(0.0, 0.0), hi=(1.0, 1.0), queries=None, precision="f64", nthreads=0,
                  want_mhat=False, abf_form="chain"):
    """Weights for every stencil entry (Eqs. disc_form, lsys, w_abf).

    ``C`` is ``[n_ops, p]`` (or ``[n_ops, 44]``) in D ordering, physical units.
    Returns dict with ``w`` ``[nnz, n_ops]``, ``status`` ``[nq]``, ``piv_ratio``
    ``[nq]`` and optionally ``mhat`` ``[nq, p, p]``.
    """
    lib = _lib(precision)
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    C = np.atleast_2d(np.asarray(C, dtype=np.float64))
    n_ops = C.shape[0]
    Cp = np.zeros((n_ops, PMAX))
    Cp[:, : C.shape[1]] = C
    q = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = xy.shape[0] if q is None else q.shape[0]
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    nnz = int(rp[-1])
    w = np.zeros((max(nnz, 1), n_ops))
    st = np.zeros(nq, dtype=np.int32)
    pr = np.zeros(nq)
    od = None if order is None else np.ascontiguousarray(order, dtype=np.int8)
    mh = np.zeros((nq, PMAX, PMAX)) if want_mhat else None
    rc = lib.orc_build_weights(_ptr(xy), _ptr(h), int(periodic), _ptr(np.asarray(lo, np.float64)),
                               _ptr(np.asarray(hi, np.float64)), _ptr(q), nq, _ptr(rp), _ptr(cl),
                               _ptr(od), int(k or 0), RBF[rbf] | ABF_FORM[abf_form], n_ops, _ptr(Cp), _ptr(w), _ptr(st),
                               _ptr(pr), _ptr(mh), int(nthreads))
    assert rc == 0
    out = {"w": w[:nnz], "status": st, "piv_ratio": pr}
    if want_mhat:
        kk = k if k is not None else int(np.max(order))
        p = p_of_k(kk)
        out["mhat"] = mh.reshape(nq, PMAX * PMAX)[:, : p * p].reshape(nq, p, p)
    return out


def apply(row_ptr, col, w, f, queries=None, precision="f64", nthreads=0):
    """out[d, q] = sum_j (f_j - f_i) w_ji^d (Eq. general_do)."""
    lib = _lib(precision)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    n_ops = w.shape[1]
    q = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = rp.shape[0] - 1
    out = np.zeros((n_ops, nq))
    lib.orc_apply(_ptr(q), nq, _ptr(rp), _ptr(cl), _ptr(w), n_ops, _ptr(f), _ptr(out), int(nthreads))
    return out


def rk4(row_ptr, col, w, beta, u0, dt, nsteps, frozen=None, precision="f64", nthreads=0):
    """Classical RK4 for du/dt = sum_d beta_d L^d(u) over all nodes (Sec. 5.1)."""
    lib = _lib(precision)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    u = np.array(u0, dtype=np.float64, copy=True)
    fz = None if frozen is None else np.ascontiguousarray(frozen, dtype=np.uint8)
    rc = lib.orc_rk4(u.shape[0], _ptr(rp), _ptr(cl), _ptr(w), w.shape[1], _ptr(beta), _ptr(u), float(dt),
                     int(nsteps), _ptr(fz), int(nthreads))
    assert rc == 0
    return u


def rk4_burgers(row_ptr, col, w, beta, u0, v0, dt, nsteps, frozen=None, precision="f64", nthreads=0):
    """Classical RK4 for Burgers' equation (Sec. 5.3): du/dt = -(u L^0(u) + v L^1(u)) +
    sum_{d>=2} beta_d L^d(u) and the same for v, operators 0 and 1 being d/dx and d/dy."""
    lib = _lib(precision)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    u = np.array(u0, dtype=np.float64, copy=True)
    v = np.array(v0, dtype=np.float64, copy=True)
    fz = None if frozen is None else np.ascontiguousarray(frozen, dtype=np.uint8)
    rc = lib.orc_rk4_burgers(u.shape[0], _ptr(rp), _ptr(cl), _ptr(w), w.shape[1], _ptr(beta), _ptr(u), _ptr(v),
                             float(dt), int(nsteps), _ptr(fz), int(nthreads))
    assert rc == 0
    return u, v


def operator_matrix(row_ptr, col, w, beta):
    """The sparse matrix A with (A u)_i = sum_d beta_d sum_j (u_j - u_i) w_ji^d (Eq. general_do):
    off-diagonal entries sum_d beta_d w_ji^d, diagonal minus their row sum (scipy CSR)."""
    import scipy.sparse as sp

    rp = np.asarray(row_ptr, dtype=np.int64)
    n = rp.shape[0] - 1
    wb = np.asarray(w, dtype=np.float64) @ np.asarray(beta, dtype=np.float64)
    node = np.repeat(np.arange(n), np.diff(rp))
    A = sp.csr_matrix((wb, (node, np.asarray(col, dtype=np.int64))), shape=(n, n))
    return (A - sp.diags(np.bincount(node, weights=wb, minlength=n))).tocsr()


def steady_state(row_ptr, col, w, beta, u_fixed, frozen):
    """Steady state of du/dt = sum_d beta_d L^d(u) with the frozen (Dirichlet) nodes held at
    ``u_fixed`` (Sec. 5.1: boundary values prescribed, the equation solved at the internal
    nodes only): the internal values solve A_II u_I = -A_IB u_B, by a sparse direct solve."""
    import scipy.sparse.linalg as spl

    A = operator_matrix(row_ptr, col, w, beta)
    fz = np.asarray(frozen).astype(bool)
    I, B = np.nonzero(~fz)[0], np.nonzero(fz)[0]
    u = np.array(u_fixed, dtype=np.float64, copy=True)
    u[I] = spl.spsolve(A[I][:, I].tocsc(), -(A[I][:, B] @ u[B]))
    return u


def solve_operator(row_ptr, col, w, op, f, dirichlet=None, neumann=None):
    """The global system of Sec. 5.2 (eq. poisson_system): A Phi = F with A_ij = w^op_ji (j != i),
    A_ii = -sum_j w^op_ji, and identity rows (Phi_i = f_i) where ``dirichlet`` is set; by a sparse
    direct solve.

    ``neumann`` = (ghost, parent, normal, op_x, op_y): the ghost-node rows of Sec. 5.2 for a
    Neumann boundary.  Row ghost[g] is replaced by the boundary normal derivative operator of its
    parent node b = parent[g], n_x w^(op_x) + n_y w^(op_y) with (n_x, n_y) = normal[g]:
    A_gj = n_x w^x_jb + n_y w^y_jb for every j in the stencil of b, and A_gb = minus the sum of
    those entries; F_g (= f[ghost[g]]) is the prescribed normal derivative there."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    w = np.asarray(w, dtype=np.float64)
    rp = np.asarray(row_ptr, dtype=np.int64)
    beta = np.zeros(w.shape[1])
    beta[op] = 1.0
    A = operator_matrix(row_ptr, col, w, beta).tolil()
    b = np.array(f, dtype=np.float64, copy=True)
    if dirichlet is not None:
        for i in np.nonzero(np.asarray(dirichlet))[0]:
            A.rows[i] = [int(i)]
            A.data[i] = [1.0]
    if neumann is not None:
        ghost, parent, normal, op_x, op_y = neumann
        normal = np.asarray(normal, dtype=np.float64).reshape(-1, 2)
        for g in range(len(ghost)):
            gi, pb = int(ghost[g]), int(parent[g])
            nx, ny = normal[g]
            row = {}
            total = 0.0
            for e in range(rp[pb], rp[pb + 1]):
                c = nx * w[e, op_x] + ny * w[e, op_y]
                j = int(col[e])
                row[j] = row.get(j, 0.0) + c
                total += c
            row[pb] = row.get(pb, 0.0) - total
            js = sorted(row)
            A.rows[gi] = js
            A.data[gi] = [row[j] for j in js]
    return spl.spsolve(sp.csc_matrix(A), b)


def rbf_derivs(rbf, q, precision="f64"):
    d = np.zeros(4)
    _lib(precision).orc_rbf_derivs(RBF[rbf], float(q), _ptr(d))
    return d


def dr(x, y, kmax, precision="f64"):
    """Table t[a, b] = d^(a+b)|r| / dx^a dy^b at (x, y), a + b <= kmax."""
    out = np.zeros((kmax + 1) * (kmax + 1))
    _lib(precision).orc_dr(float(x), float(y), int(kmax), _ptr(out))
    return out.reshape(kmax + 1, kmax + 1)


def monomials(x, y, k, precision="f64"):
    out = np.zeros(p_of_k(k))
    _lib(precision).orc_monomials(float(x), float(y), int(k), _ptr(out))
    return out


def abfs(rbf, x, y, k, precision="f64", abf_form="chain"):
    out = np.zeros(p_of_k(k))
    _lib(precision).orc_abfs(RBF[rbf] | ABF_FORM[abf_form], float(x), float(y), int(k), _ptr(out))
    return out
