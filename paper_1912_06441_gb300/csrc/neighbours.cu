// Stencil search (Sec. 2: all j != i with |r_ji| < 2 h_i) on a uniform cell grid.
//
// Cells have side >= 2 h_max, so every neighbour of a node lies in its own cell or one of
// the 8 cells around it (with wrap-around in a periodic box).  Nodes are counting-sorted by
// cell; one thread per node (in cell order, so a warp sweeps the same few cells) counts its
// neighbours, a prefix sum gives the CSR row pointers, a second sweep writes the column
// indices, and each row is sorted ascending.  The distance test is evaluated in IEEE double
// with explicitly rounded operations (no fused multiply-add), so the result does not depend
// on the compiler's contraction choices; a float pre-classification with a proven error bound
// settles every candidate that is not within a thin shell at the radius (on GB300 the double
// test costs FP64-pipe time per candidate), and the shell goes to the double test, so the
// stencils are those of the double test bit for bit.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "labfm_internal.cuh"

namespace labfm {
namespace {

constexpr int NB_THREADS = 256;

struct Grid {
    double lo[2], L[2], halfL[2], inv_cs[2];
    int nc[2];
    int periodic;
    // float pre-filter of the distance test (used where cell_xyf is given): box sides and half
    // sides in float, the bound E on |dx_float - dx| (roundings of the coordinates, the
    // difference and the wrap), and the largest (2h)^2 for which the float wrap cannot differ
    // from the double one on a candidate near the radius
    float Lf[2], halfLf[2];
    float E;
    double r2_wrap_max;
};

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// Validate nodes and find max h.  misc[0] = bits of max h, misc[1] = number of bad nodes.
__global__ void k_check(int64_t n, const double *__restrict__ xy, const double *__restrict__ h, double lo0, double lo1,
                        double hi0, double hi1, unsigned long long *__restrict__ misc)
{
    __shared__ unsigned long long s_max[NB_THREADS / 32];
    __shared__ unsigned int s_bad[NB_THREADS / 32];
    unsigned long long mx = 0;
    unsigned int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x = xy[2 * i], y = xy[2 * i + 1], hv = h[i];
        bool ok = isfinite(x) && isfinite(y) && isfinite(hv) && hv > 0.0 && x >= lo0 && x <= hi0 && y >= lo1 &&
                  y <= hi1;
        if (!ok) bad++;
        else mx = max(mx, dbits(hv));  // positive doubles order like their bit patterns
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_max[w] = mx;
        s_bad[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < NB_THREADS / 32; t++) {
            mx = max(mx, s_max[t]);
            bad += s_bad[t];
        }
        atomicMax(&misc[0], mx);
        if (bad) atomicAdd(&misc[1], (unsigned long long)bad);
    }
}

__device__ __forceinline__ int cell_coord(double x, double lo, double inv_cs, int nc)
{
    double t = __dmul_rn(__dsub_rn(x, lo), inv_cs);
    int c = (int)floor(t);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_assign(int64_t n, const double *__restrict__ xy, Grid g, int32_t *__restrict__ cell_of,
                              int32_t *__restrict__ cell_count)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx = cell_coord(xy[2 * i], g.lo[0], g.inv_cs[0], g.nc[0]);
    int cy = cell_coord(xy[2 * i + 1], g.lo[1], g.inv_cs[1], g.nc[1]);
    int c = cy * g.nc[0] + cx;
    cell_of[i] = c;
    atomicAdd(&cell_count[c], 1);
}

__global__ void k_cell_scatter(int64_t n, const double *__restrict__ xy, const int32_t *__restrict__ cell_of,
                               const int64_t *__restrict__ cell_start, int32_t *__restrict__ cursor,
                               int32_t *__restrict__ cell_nodes, double2 *__restrict__ cell_xy,
                               float2 *__restrict__ cell_xyf)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell_of[i];
    int64_t pos = cell_start[c] + atomicAdd(&cursor[c], 1);
    cell_nodes[pos] = (int32_t)i;
    const double x = xy[2 * i], y = xy[2 * i + 1];
    cell_xy[pos] = make_double2(x, y);
    if (cell_xyf) cell_xyf[pos] = make_float2((float)x, (float)y);
}

// The up-to-3 distinct cell coordinates around c along one axis.
__device__ __forceinline__ int axis_cells(int c, int nc, int periodic, int out[3])
{
    int m = 0;
    for (int d = -1; d <= 1; d++) {
        int v = c + d;
        if (periodic) {
            v = v < 0 ? v + nc : (v >= nc ? v - nc : v);
        } else if (v < 0 || v >= nc) {
            continue;
        }
        bool dup = false;
        for (int t = 0; t < m; t++) dup |= (out[t] == v);
        if (!dup) out[m++] = v;
    }
    return m;
}

// The exact distance test of Sec. 2 in IEEE double, explicitly rounded (no contraction).
__device__ __forceinline__ bool within_exact(double qx, double qy, double xi, double yi, double R2, const Grid &g)
{
    double dx = __dsub_rn(qx, xi);
    double dy = __dsub_rn(qy, yi);
    if (g.periodic) {
        if (dx > g.halfL[0]) dx = __dsub_rn(dx, g.L[0]);
        else if (dx < -g.halfL[0]) dx = __dadd_rn(dx, g.L[0]);
        if (dy > g.halfL[1]) dy = __dsub_rn(dy, g.L[1]);
        else if (dy < -g.halfL[1]) dy = __dadd_rn(dy, g.L[1]);
    }
    double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    return r2 < R2;
}

// One sweep over the candidate cells of node i.  WRITE = false: count; true: write col[].
// With cell_xyf, each candidate is first classified in float: r2f, the squared distance from
// the float coordinates, differs from the double r2 by at most D = 2E(|dx_f| + |dy_f|) + 2E^2 +
// 2^-23 r2f (E bounds the error of dx_f and dy_f); a candidate with r2f below or above
// (2h)^2 by more than 2D + 2^-23 (2h)^2 is decided there, and only the rest (a thin shell at the
// radius) takes the double test.  The result is the double test's, bit for bit; on GB300 the
// double test costs FP64-pipe time per candidate, the float one does not.
template <bool WRITE>
__global__ void k_sweep(int64_t n, const double *__restrict__ xy, const double *__restrict__ h, Grid g,
                        const int32_t *__restrict__ cell_of, const int64_t *__restrict__ cell_start,
                        const int32_t *__restrict__ cell_nodes, const double2 *__restrict__ cell_xy,
                        const float2 *__restrict__ cell_xyf, int32_t *__restrict__ counts,
                        const int64_t *__restrict__ row_ptr, int32_t *__restrict__ col)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int i = cell_nodes[t];
    double xi = xy[2 * (int64_t)i], yi = xy[2 * (int64_t)i + 1];
    double R = 2.0 * h[i];
    double R2 = __dmul_rn(R, R);
    // float classification only where the float wrap cannot flip a candidate near the radius
    const bool filt = cell_xyf != nullptr && (!g.periodic || R2 <= g.r2_wrap_max);
    const float xif = (float)xi, yif = (float)yi, R2f = (float)R2;
    const float E = g.E;
    int c = cell_of[i];
    int cx = c % g.nc[0], cy = c / g.nc[0];
    int xs[3], ys[3];
    int mx = axis_cells(cx, g.nc[0], g.periodic, xs);
    int my = axis_cells(cy, g.nc[1], g.periodic, ys);
    int cnt = 0;
    int64_t base = WRITE ? row_ptr[i] : 0;
    for (int a = 0; a < my; a++) {
        for (int b = 0; b < mx; b++) {
            int cc = ys[a] * g.nc[0] + xs[b];
            int64_t s = cell_start[cc], e = cell_start[cc + 1];
            for (int64_t p = s; p < e; p++) {
                int j = cell_nodes[p];
                if (j == i) continue;
                bool in;
                int decided = 0;  // 1: inside, 2: outside, 0: to the double test
                if (filt) {
                    const float2 qf = cell_xyf[p];
                    float dxf = qf.x - xif, dyf = qf.y - yif;
                    if (g.periodic) {
                        if (dxf > g.halfLf[0]) dxf -= g.Lf[0];
                        else if (dxf < -g.halfLf[0]) dxf += g.Lf[0];
                        if (dyf > g.halfLf[1]) dyf -= g.Lf[1];
                        else if (dyf < -g.halfLf[1]) dyf += g.Lf[1];
                    }
                    const float r2f = fmaf(dxf, dxf, dyf * dyf);
                    const float D = 2.0f * E * (fabsf(dxf) + fabsf(dyf)) + 2.0f * E * E + 1.1920929e-7f * r2f;
                    const float M = 2.0f * D + 1.1920929e-7f * R2f;
                    decided = r2f < R2f - M ? 1 : (r2f > R2f + M ? 2 : 0);
                }
                if (decided) {
                    in = decided == 1;
                } else {
                    const double2 q = cell_xy[p];
                    in = within_exact(q.x, q.y, xi, yi, R2, g);
                }
                if (in) {
                    if (WRITE) col[base + cnt] = j;
                    cnt++;
                }
            }
        }
    }
    if (!WRITE) {
        counts[i] = cnt;
    } else {
        // insertion sort of the row (stencils hold tens of entries)
        int32_t *row = col + base;
        for (int u = 1; u < cnt; u++) {
            int32_t v = row[u];
            int w = u - 1;
            while (w >= 0 && row[w] > v) {
                row[w + 1] = row[w];
                w--;
            }
            row[w + 1] = v;
        }
    }
}

}  // namespace

// The float pre-filter's constants: E = 2^-21 (B + L) bounds |dx_float - dx| (B the largest
// coordinate magnitude of the box, L its larger side: the float roundings of both coordinates,
// of their difference and of the wrap, each at most 2^-24 of a magnitude below 2B + L), and the
// float test is used in a periodic box only for (2h)^2 <= (0.45 L_min)^2, where a candidate whose
// float and double wraps differ (|dx| within E of L/2) lies far outside the radius either way.
static void set_float_filter(Grid &g, const double lo[2], const double hi[2])
{
    double B = 0.0, Lmax = 0.0, Lmin = 1e300;
    for (int d = 0; d < 2; d++) {
        B = std::max(B, std::max(std::fabs(lo[d]), std::fabs(hi[d])));
        Lmax = std::max(Lmax, g.L[d]);
        Lmin = std::min(Lmin, g.L[d]);
        g.Lf[d] = (float)g.L[d];
        g.halfLf[d] = (float)g.halfL[d];
    }
    g.E = (float)std::ldexp(B + Lmax, -21);
    g.r2_wrap_max = (0.45 * Lmin) * (0.45 * Lmin);
}

labfm_status run_neighbours(labfm_ctx *ctx, int64_t n, const double *xy, const double *h, int periodic,
                            const double lo[2], const double hi[2], int64_t *nnz_out)
{
    cudaStream_t s = ctx->stream;
    ctx->n = 0;
    ctx->nnz = 0;
    LABFM_CUDA_TRY(ctx, ctx->misc.reserve(4096));
    unsigned long long *misc = ctx->misc.as<unsigned long long>();
    LABFM_CUDA_TRY(ctx, cudaMemsetAsync(misc, 0, 2 * sizeof(unsigned long long), s));
    int nb = (int)std::min<int64_t>((n + NB_THREADS - 1) / NB_THREADS, (int64_t)ctx->num_sms * 8);
    k_check<<<nb, NB_THREADS, 0, s>>>(n, xy, h, lo[0], lo[1], hi[0], hi[1], misc);
    LABFM_CUDA_TRY(ctx, cudaGetLastError());
    unsigned long long *hs = (unsigned long long *)ctx->host_small;
    LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(hs, misc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hs[1] != 0)
        return fail(ctx, LABFM_ERR_ARG, std::to_string(hs[1]) + " node(s) with non-finite or out-of-box coordinates or h <= 0");
    double hmax;
    memcpy(&hmax, &hs[0], sizeof hmax);

    Grid g{};
    g.periodic = periodic;
    double ncell_d[2];
    for (int d = 0; d < 2; d++) {
        g.lo[d] = lo[d];
        g.L[d] = hi[d] - lo[d];
        g.halfL[d] = 0.5 * g.L[d];
        // side >= 2 h_max with a relative margin far above the rounding of the cell coordinate
        ncell_d[d] = std::floor(g.L[d] / (2.0 * hmax * (1.0 + 1e-9)));
        if (!(ncell_d[d] >= 1.0)) ncell_d[d] = 1.0;
    }
    // keep the grid to about 4 cells per node (coarser cells stay correct, just hold more nodes)
    double cap = 4.0 * (double)n + 64.0;
    if (ncell_d[0] * ncell_d[1] > cap) {
        double f = std::sqrt(ncell_d[0] * ncell_d[1] / cap);
        for (int d = 0; d < 2; d++) ncell_d[d] = std::max(1.0, std::floor(ncell_d[d] / f));
    }
    if (ncell_d[0] * ncell_d[1] > (double)(1 << 28))
        return fail(ctx, LABFM_ERR_CAPACITY, "cell grid exceeds 2^28 cells");
    for (int d = 0; d < 2; d++) {
        g.nc[d] = (int)ncell_d[d];
        g.inv_cs[d] = (double)g.nc[d] / g.L[d];
    }
    set_float_filter(g, lo, hi);
    int64_t ncells = (int64_t)g.nc[0] * g.nc[1];

    LABFM_CUDA_TRY(ctx, ctx->cell_of.reserve(sizeof(int32_t) * n));
    LABFM_CUDA_TRY(ctx, ctx->cell_count.reserve(sizeof(int32_t) * ncells));
    LABFM_CUDA_TRY(ctx, ctx->cell_start.reserve(sizeof(int64_t) * (ncells + 1)));
    LABFM_CUDA_TRY(ctx, ctx->cell_nodes.reserve(sizeof(int32_t) * n + sizeof(double2) * n + sizeof(float2) * n + 64));
    LABFM_CUDA_TRY(ctx, ctx->counts.reserve(sizeof(int32_t) * n));
    LABFM_CUDA_TRY(ctx, ctx->row_ptr.reserve(sizeof(int64_t) * (n + 1)));
    int32_t *cell_of = ctx->cell_of.as<int32_t>();
    int32_t *cell_count = ctx->cell_count.as<int32_t>();
    int64_t *cell_start = ctx->cell_start.as<int64_t>();
    int32_t *cell_nodes = ctx->cell_nodes.as<int32_t>();
    size_t xy_off = ((sizeof(int32_t) * n + 15) / 16) * 16;
    double2 *cell_xy = (double2 *)((char *)ctx->cell_nodes.ptr + xy_off);
    float2 *cell_xyf = (float2 *)(cell_xy + n);
    int32_t *counts = ctx->counts.as<int32_t>();
    int64_t *row_ptr = ctx->row_ptr.as<int64_t>();

    int nbn = (int)((n + NB_THREADS - 1) / NB_THREADS);
    LABFM_CUDA_TRY(ctx, cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * ncells, s));
    k_cell_assign<<<nbn, NB_THREADS, 0, s>>>(n, xy, g, cell_of, cell_count);
    LABFM_CUDA_TRY(ctx, cudaGetLastError());
    LABFM_CUDA_TRY(ctx, exclusive_scan_i32_to_i64(cell_count, cell_start, ncells, ctx->scan_tmp, s));
    LABFM_CUDA_TRY(ctx, cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * ncells, s));
    k_cell_scatter<<<nbn, NB_THREADS, 0, s>>>(n, xy, cell_of, cell_start, cell_count, cell_nodes, cell_xy, cell_xyf);
    LABFM_CUDA_TRY(ctx, cudaGetLastError());
    k_sweep<false><<<nbn, NB_THREADS, 0, s>>>(n, xy, h, g, cell_of, cell_start, cell_nodes, cell_xy, cell_xyf, counts,
                                              nullptr, nullptr);
    LABFM_CUDA_TRY(ctx, cudaGetLastError());
    LABFM_CUDA_TRY(ctx, exclusive_scan_i32_to_i64(counts, row_ptr, n, ctx->scan_tmp, s));
    int64_t *nnz_h = (int64_t *)ctx->host_small;
    LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(nnz_h, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    int64_t nnz = *nnz_h;
    if (nnz >= ((int64_t)1 << 40)) return fail(ctx, LABFM_ERR_CAPACITY, "too many stencil entries");
    LABFM_CUDA_TRY(ctx, ctx->col.reserve(sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
    k_sweep<true><<<nbn, NB_THREADS, 0, s>>>(n, xy, h, g, cell_of, cell_start, cell_nodes, cell_xy, cell_xyf, nullptr,
                                             row_ptr, ctx->col.as<int32_t>());
    LABFM_CUDA_TRY(ctx, cudaGetLastError());
    LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    ctx->n = n;
    ctx->nnz = nnz;
    ctx->periodic = periodic;
    for (int d = 0; d < 2; d++) {
        ctx->lo[d] = lo[d];
        ctx->hi[d] = hi[d];
    }
    LABFM_CUDA_TRY(ctx, ctx->node_xy.reserve(sizeof(double) * 2 * n));
    LABFM_CUDA_TRY(ctx, ctx->node_h.reserve(sizeof(double) * n));
    LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->node_xy.ptr, xy, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s));
    LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->node_h.ptr, h, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    *nnz_out = nnz;
    return LABFM_OK;
}

}  // namespace labfm

// ---------------------------------------------------------------------------------------------
// labfm_build_neighbours_noalloc: the same kernels on a fixed scratch array instead of
// context-owned allocations.
// ---------------------------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int64_t NA_MAXN = LABFM_NOALLOC_MAX_NODES;
constexpr int64_t NA_MAXC = LABFM_NOALLOC_MAX_NODES;  // cells of the search grid
constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t NA_OFF_MISC = 0;
constexpr size_t NA_OFF_CELL_OF = na_align(NA_OFF_MISC + 64);
constexpr size_t NA_OFF_CELL_COUNT = na_align(NA_OFF_CELL_OF + 4 * NA_MAXN);
constexpr size_t NA_OFF_CELL_START = na_align(NA_OFF_CELL_COUNT + 4 * NA_MAXC);
constexpr size_t NA_OFF_CELL_NODES = na_align(NA_OFF_CELL_START + 8 * (NA_MAXC + 1));
constexpr size_t NA_OFF_CELL_XY = na_align(NA_OFF_CELL_NODES + 4 * NA_MAXN);
constexpr size_t NA_OFF_COUNTS = na_align(NA_OFF_CELL_XY + 16 * NA_MAXN);
constexpr size_t NA_OFF_SCAN = na_align(NA_OFF_COUNTS + 4 * NA_MAXN);
constexpr size_t NA_SCAN_ELEMS = 4096;
constexpr size_t NA_BYTES = na_align(NA_OFF_SCAN + 8 * NA_SCAN_ELEMS);  // about 10 MB

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;  // serialises the address lookup (the array itself is not guarded)

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

}  // namespace

// The scratch of labfm_build_neighbours_noalloc (one copy per device that loads the library).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

extern "C" labfm_status labfm_build_neighbours_noalloc(int device, void *stream, int64_t n, const double *xy,
                                                       const double *h, int periodic, const double box_lo[2],
                                                       const double box_hi[2], int64_t *row_ptr, int32_t *col,
                                                       int64_t col_capacity, int64_t *nnz_out)
{
    using namespace labfm;
    if (n < 1 || !xy || !h || !box_lo || !box_hi || !row_ptr || !nnz_out || col_capacity < 0 ||
        (col_capacity > 0 && !col))
        return LABFM_ERR_ARG;
    if (n > NA_MAXN) return LABFM_ERR_CAPACITY;
    for (int d = 0; d < 2; d++)
        if (!std::isfinite(box_lo[d]) || !std::isfinite(box_hi[d]) || !(box_hi[d] > box_lo[d])) return LABFM_ERR_ARG;
    if (device < 0 || device >= NA_MAX_DEVICES) return LABFM_ERR_ARG;
    DeviceGuard guard;
    if (cudaGetDevice(&guard.prev) != cudaSuccess) return LABFM_ERR_CUDA;
    if (guard.prev != device) {
        if (cudaSetDevice(device) != cudaSuccess) return LABFM_ERR_CUDA;
        guard.changed = true;
    }
    // The array's device address, looked up on every call with the device current: in host code
    // g_noalloc_scratch names a host-side stand-in, and an address kept from an earlier call would
    // be stale after the device's primary context was reset (the module is then loaded again).
    // The first call on a device also loads the library's device code there.
    char *base;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LABFM_ERR_CUDA;
        base = static_cast<char *>(p);
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *misc = reinterpret_cast<unsigned long long *>(base + NA_OFF_MISC);
    int32_t *cell_of = reinterpret_cast<int32_t *>(base + NA_OFF_CELL_OF);
    int32_t *cell_count = reinterpret_cast<int32_t *>(base + NA_OFF_CELL_COUNT);
    int64_t *cell_start = reinterpret_cast<int64_t *>(base + NA_OFF_CELL_START);
    int32_t *cell_nodes = reinterpret_cast<int32_t *>(base + NA_OFF_CELL_NODES);
    double2 *cell_xy = reinterpret_cast<double2 *>(base + NA_OFF_CELL_XY);
    int32_t *counts = reinterpret_cast<int32_t *>(base + NA_OFF_COUNTS);
    int64_t *scan_tmp = reinterpret_cast<int64_t *>(base + NA_OFF_SCAN);

#define NA_TRY(expr)                                     \
    do {                                                 \
        if ((expr) != cudaSuccess) return LABFM_ERR_CUDA; \
    } while (0)

    int num_sms = 0;
    NA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    // node check and h_max (the counters start at zero on every call)
    NA_TRY(cudaMemsetAsync(misc, 0, 2 * sizeof(unsigned long long), s));
    int nb = (int)std::min<int64_t>((n + NB_THREADS - 1) / NB_THREADS, (int64_t)num_sms * 8);
    k_check<<<nb, NB_THREADS, 0, s>>>(n, xy, h, box_lo[0], box_lo[1], box_hi[0], box_hi[1], misc);
    NA_TRY(cudaGetLastError());
    unsigned long long hs[2];
    NA_TRY(cudaMemcpyAsync(hs, misc, sizeof hs, cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
    if (hs[1] != 0) return LABFM_ERR_ARG;
    double hmax;
    memcpy(&hmax, &hs[0], sizeof hmax);

    // the same grid rule as labfm_build_neighbours, capped at the scratch's cell count
    Grid g{};
    g.periodic = periodic ? 1 : 0;
    double ncell_d[2];
    for (int d = 0; d < 2; d++) {
        g.lo[d] = box_lo[d];
        g.L[d] = box_hi[d] - box_lo[d];
        g.halfL[d] = 0.5 * g.L[d];
        ncell_d[d] = std::floor(g.L[d] / (2.0 * hmax * (1.0 + 1e-9)));
        if (!(ncell_d[d] >= 1.0)) ncell_d[d] = 1.0;
    }
    double cap = std::min(4.0 * (double)n + 64.0, (double)NA_MAXC);
    if (ncell_d[0] * ncell_d[1] > cap) {
        double f = std::sqrt(ncell_d[0] * ncell_d[1] / cap);
        for (int d = 0; d < 2; d++) ncell_d[d] = std::max(1.0, std::floor(ncell_d[d] / f));
    }
    for (int d = 0; d < 2; d++) {
        g.nc[d] = (int)ncell_d[d];
        g.inv_cs[d] = (double)g.nc[d] / g.L[d];
    }
    const int64_t ncells = (int64_t)g.nc[0] * g.nc[1];
    if (ncells > NA_MAXC) return LABFM_ERR_CAPACITY;

    int nbn = (int)((n + NB_THREADS - 1) / NB_THREADS);
    NA_TRY(cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * ncells, s));
    k_cell_assign<<<nbn, NB_THREADS, 0, s>>>(n, xy, g, cell_of, cell_count);
    NA_TRY(cudaGetLastError());
    NA_TRY(exclusive_scan_i32_to_i64_ws(cell_count, cell_start, ncells, scan_tmp, NA_SCAN_ELEMS, s));
    NA_TRY(cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * ncells, s));
    // (the float pre-filter needs an array the fixed scratch does not hold: the double test alone)
    k_cell_scatter<<<nbn, NB_THREADS, 0, s>>>(n, xy, cell_of, cell_start, cell_count, cell_nodes, cell_xy, nullptr);
    NA_TRY(cudaGetLastError());
    k_sweep<false><<<nbn, NB_THREADS, 0, s>>>(n, xy, h, g, cell_of, cell_start, cell_nodes, cell_xy, nullptr, counts,
                                              nullptr, nullptr);
    NA_TRY(cudaGetLastError());
    NA_TRY(exclusive_scan_i32_to_i64_ws(counts, row_ptr, n, scan_tmp, NA_SCAN_ELEMS, s));
    int64_t nnz = 0;
    NA_TRY(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof nnz, cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
    *nnz_out = nnz;
    if (nnz > col_capacity) return LABFM_ERR_CAPACITY;
    if (nnz > 0) {
        k_sweep<true><<<nbn, NB_THREADS, 0, s>>>(n, xy, h, g, cell_of, cell_start, cell_nodes, cell_xy, nullptr,
                                                 nullptr, row_ptr, col);
        NA_TRY(cudaGetLastError());
    }
    NA_TRY(cudaStreamSynchronize(s));
#undef NA_TRY
    return LABFM_OK;
}
