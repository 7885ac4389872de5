"""labfm_build_neighbours_noalloc: the stencil search for callers that cannot allocate device
memory (their memory belongs to another allocator, or they must not allocate while running).
It keeps its scratch in a fixed array inside the library instead of allocating, and must give
exactly the stencils of labfm_build_neighbours.

Called through the C ABI (ctypes) with torch-owned outputs, twice in a row on different node
sets so that the second call cannot lean on what the first left in the shared array.  This file
sorts last so that a run stopping at the first failure has run every other test."""
import ctypes as ct

import numpy as np
import pytest

import labfm_synth as S

pytestmark = pytest.mark.gpu


def _reference(ns):
    import torch

    from paper_1912_06441_gb300 import Labfm

    dev = torch.device("cuda", 0)
    L = Labfm(0)
    L.build_neighbours(torch.from_numpy(ns.xy).to(dev), torch.from_numpy(ns.h).to(dev), ns.periodic, ns.lo, ns.hi)
    rp, col = L.get_neighbours()
    out = rp.cpu().numpy().copy(), col.cpu().numpy().copy()
    L.close()
    return out


def _noalloc(lib, ns, capacity):
    import torch

    dev = torch.device("cuda", 0)
    xy = torch.from_numpy(ns.xy).to(dev)
    h = torch.from_numpy(ns.h).to(dev)
    row_ptr = torch.full((ns.n + 1,), -7, dtype=torch.int64, device=dev)
    col = torch.full((max(capacity, 1),), -7, dtype=torch.int32, device=dev)
    lo = (ct.c_double * 2)(*ns.lo)
    hi = (ct.c_double * 2)(*ns.hi)
    nnz = ct.c_int64(-1)
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = lib.labfm_build_neighbours_noalloc(0, ct.c_void_p(stream), ns.n, ct.c_void_p(xy.data_ptr()),
                                            ct.c_void_p(h.data_ptr()), int(ns.periodic), lo, hi,
                                            ct.c_void_p(row_ptr.data_ptr()), ct.c_void_p(col.data_ptr()),
                                            capacity, ct.byref(nnz))
    torch.cuda.synchronize()
    return st, int(nnz.value), row_ptr.cpu().numpy(), col.cpu().numpy()


def test_noalloc_stencils_match_the_allocating_entry_point():
    import torch

    assert torch.cuda.is_available(), "GPU test"
    import paper_1912_06441_gb300 as P

    lib = P.load_library()
    cases = [S.jittered_lattice(96, 2.2, 8, seed=5),                       # periodic, order-8 radius
             S.jittered_lattice(70, 1.4, 4, seed=6, periodic=False)]      # walls, smaller radius
    for ns in cases:  # two calls in a row through the same scratch array
        rp_ref, col_ref = _reference(ns)
        st, nnz, rp, col = _noalloc(lib, ns, capacity=len(col_ref) + 17)
        assert st == 0, st
        assert nnz == len(col_ref)
        assert np.array_equal(rp, rp_ref)
        assert np.array_equal(col[:nnz], col_ref)  # integer output: bit for bit
        assert np.all(col[nnz:] == -7)             # nothing written past the stencils


def test_noalloc_reports_capacity_and_size_limits():
    import paper_1912_06441_gb300 as P

    lib = P.load_library()
    ns = S.jittered_lattice(40, 1.4, 4, seed=8)
    rp_ref, col_ref = _reference(ns)
    st, nnz, rp, col = _noalloc(lib, ns, capacity=10)
    assert st == 4 and nnz == len(col_ref)  # LABFM_ERR_CAPACITY, with the size needed
    assert np.array_equal(rp, rp_ref)
    big = S.jittered_lattice(513, 1.4, 4, seed=9)  # 263,169 nodes > LABFM_NOALLOC_MAX_NODES
    assert big.n > P.NOALLOC_MAX_NODES
    st, _, _, _ = _noalloc(lib, big, capacity=1)
    assert st == 4


def test_noalloc_allocates_nothing_after_its_first_call():
    """The call that exists so that a caller need not allocate must not allocate either: once
    the first call on the device has loaded the library's device code (the fixed array with it),
    a second call leaves the device's free memory unchanged."""
    import torch

    import paper_1912_06441_gb300 as P

    lib = P.load_library()
    ns = S.jittered_lattice(128, 2.2, 8, seed=12)
    rp_ref, col_ref = _reference(ns)
    dev = torch.device("cuda", 0)
    xy = torch.from_numpy(ns.xy).to(dev)
    h = torch.from_numpy(ns.h).to(dev)
    row_ptr = torch.empty(ns.n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(len(col_ref), dtype=torch.int32, device=dev)
    lo = (ct.c_double * 2)(*ns.lo)
    hi = (ct.c_double * 2)(*ns.hi)
    nnz = ct.c_int64(-1)
    stream = torch.cuda.current_stream(dev).cuda_stream

    def call():
        return lib.labfm_build_neighbours_noalloc(0, ct.c_void_p(stream), ns.n, ct.c_void_p(xy.data_ptr()),
                                                  ct.c_void_p(h.data_ptr()), int(ns.periodic), lo, hi,
                                                  ct.c_void_p(row_ptr.data_ptr()), ct.c_void_p(col.data_ptr()),
                                                  len(col_ref), ct.byref(nnz))

    assert call() == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for _ in range(3):
        assert call() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, (free0, free1)
    assert np.array_equal(row_ptr.cpu().numpy(), rp_ref) and np.array_equal(col.cpu().numpy(), col_ref)


def test_noalloc_capped_grid_matches_the_oracle():
    """Node sets whose radius is tiny against the box, so that the cell grid is capped: at
    4n + 64 cells (1,600 nodes in one dense block), and at the fixed array's cell limit (100,352
    nodes in two blocks: the allocating entry point then uses a finer grid than this one).  The
    stencils must be the oracle's, bit for bit (all rows of the small set, sampled rows of the
    large one), and the allocating entry point's on every row."""
    import oracle

    import paper_1912_06441_gb300 as P

    lib = P.load_library()
    small = S.lattice_clusters(40, 1.4, [(0.3, 0.3)], 0.04, seed=21)
    st, nnz, rp, col = _noalloc(lib, small, capacity=200000)
    assert st == 0
    orp, ocol = oracle.neighbours(small.xy, small.h, False, small.lo, small.hi)
    assert np.array_equal(rp, orp) and np.array_equal(col[:nnz], ocol)

    big = S.lattice_clusters(224, 1.4, [(0.05, 0.05), (0.9, 0.9)], 0.0224, seed=22)
    assert 4 * big.n + 64 > P.NOALLOC_MAX_NODES  # the fixed array's limit is the binding cap
    rp_ref, col_ref = _reference(big)
    st, nnz, rp, col = _noalloc(lib, big, capacity=len(col_ref))
    assert st == 0 and nnz == len(col_ref)
    assert np.array_equal(rp, rp_ref) and np.array_equal(col, col_ref)
    q = np.unique(np.concatenate([(S.uniform01(24, 300) * big.n).astype(np.int64), np.arange(0, 224),
                                  np.arange(big.n - 224, big.n)]))
    lens = rp[q + 1] - rp[q]
    sub = np.concatenate([[0], np.cumsum(lens)])
    idx = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in q])
    orp, ocol = oracle.neighbours(big.xy, big.h, False, big.lo, big.hi, queries=q)
    assert np.array_equal(sub, orp) and np.array_equal(col[idx], ocol)
