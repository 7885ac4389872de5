// C ABI of liblabfm: context management, argument checks and dispatch to the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "labfm_internal.cuh"

namespace labfm {

cudaError_t DevBuf::reserve(size_t need)
{
    if (need <= bytes && ptr) return cudaSuccess;
    release();
    size_t want = need < 256 ? 256 : need;
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        return e;
    }
    bytes = want;
    return cudaSuccess;
}

void DevBuf::release()
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

void StepGraph::release()
{
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    u = nullptr;
    v = nullptr;
    frozen = nullptr;
    dtype = -1;
    nsteps = 0;
}

labfm_status fail(labfm_ctx *ctx, labfm_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

labfm_status cuda_fail(labfm_ctx *ctx, cudaError_t e, const char *where)
{
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %d (%s) at %s", (int)e, cudaGetErrorString(e), where);
    return fail(ctx, e == cudaErrorMemoryAllocation ? LABFM_ERR_NOMEM : LABFM_ERR_CUDA, buf);
}

// ---------------------------------------------------------------------------------------------
// Exclusive scan (Blelloch-style in shared memory, recursive over block sums).
// ---------------------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 2 * SCAN_THREADS;

template <class Tin>
__global__ void k_scan_block(const Tin *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                             int64_t *__restrict__ block_sums)
{
    __shared__ int64_t s[SCAN_ITEMS];
    int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS;
    int t = threadIdx.x;
    for (int u = 0; u < 2; u++) {
        int64_t g = base + t + u * SCAN_THREADS;
        s[t + u * SCAN_THREADS] = g < n ? (int64_t)in[g] : 0;
    }
    __syncthreads();
    // up-sweep
    for (int d = 1; d < SCAN_ITEMS; d <<= 1) {
        int idx = (t + 1) * 2 * d - 1;
        if (idx < SCAN_ITEMS) s[idx] += s[idx - d];
        __syncthreads();
    }
    if (t == 0) {
        if (block_sums) block_sums[blockIdx.x] = s[SCAN_ITEMS - 1];
        s[SCAN_ITEMS - 1] = 0;
    }
    __syncthreads();
    // down-sweep
    for (int d = SCAN_ITEMS >> 1; d >= 1; d >>= 1) {
        int idx = (t + 1) * 2 * d - 1;
        if (idx < SCAN_ITEMS) {
            int64_t v = s[idx - d];
            s[idx - d] = s[idx];
            s[idx] += v;
        }
        __syncthreads();
    }
    for (int u = 0; u < 2; u++) {
        int64_t g = base + t + u * SCAN_THREADS;
        if (g < n) out[g] = s[t + u * SCAN_THREADS];
    }
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ block_offsets)
{
    int64_t g = (int64_t)blockIdx.x * SCAN_ITEMS + threadIdx.x;
    int64_t add = block_offsets[blockIdx.x];
    if (g < n) out[g] += add;
    if (g + SCAN_THREADS < n) out[g + SCAN_THREADS] += add;
}

__global__ void k_scan_total(const int64_t *__restrict__ out_excl, const int64_t *__restrict__ last_in_i64,
                             const int32_t *__restrict__ last_in_i32, int64_t n, int64_t *__restrict__ total)
{
    if (n == 0) {
        *total = 0;
        return;
    }
    int64_t last = last_in_i64 ? last_in_i64[n - 1] : (int64_t)last_in_i32[n - 1];
    *total = out_excl[n - 1] + last;
}

template <class Tin>
static cudaError_t scan_rec(const Tin *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s)
{
    int64_t nb = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
    if (nb <= 1) {
        k_scan_block<Tin><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
        return cudaGetLastError();
    }
    int64_t *sums = tmp;
    int64_t *sums_scanned = tmp + nb;
    k_scan_block<Tin><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_rec<int64_t>(sums, sums_scanned, nb, tmp + 2 * nb, s);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, n, sums_scanned);
    return cudaGetLastError();
}

static size_t scan_tmp_elems(int64_t n)
{
    size_t tot = 0;
    while (true) {
        int64_t nb = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
        if (nb <= 1) break;
        tot += 2 * nb;
        n = nb;
    }
    return tot + 16;
}

cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, DevBuf &tmp, cudaStream_t s)
{
    cudaError_t e = tmp.reserve(scan_tmp_elems(n) * sizeof(int64_t));
    if (e != cudaSuccess) return e;
    if (n > 0) {
        e = scan_rec<int64_t>(in, out, n, tmp.as<int64_t>(), s);
        if (e != cudaSuccess) return e;
    }
    k_scan_total<<<1, 1, 0, s>>>(out, in, nullptr, n, out + n);
    return cudaGetLastError();
}

cudaError_t exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, DevBuf &tmp, cudaStream_t s)
{
    cudaError_t e = tmp.reserve(scan_tmp_elems(n) * sizeof(int64_t));
    if (e != cudaSuccess) return e;
    if (n > 0) {
        e = scan_rec<int32_t>(in, out, n, tmp.as<int64_t>(), s);
        if (e != cudaSuccess) return e;
    }
    k_scan_total<<<1, 1, 0, s>>>(out, nullptr, in, n, out + n);
    return cudaGetLastError();
}

size_t scan_workspace_elems(int64_t n) { return scan_tmp_elems(n); }

cudaError_t exclusive_scan_i32_to_i64_ws(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, size_t tmp_elems,
                                         cudaStream_t s)
{
    if (scan_tmp_elems(n) > tmp_elems) return cudaErrorInvalidValue;
    if (n > 0) {
        cudaError_t e = scan_rec<int32_t>(in, out, n, tmp, s);
        if (e != cudaSuccess) return e;
    }
    k_scan_total<<<1, 1, 0, s>>>(out, nullptr, in, n, out + n);
    return cudaGetLastError();
}

}  // namespace labfm

using namespace labfm;

extern "C" {

labfm_status labfm_create(labfm_ctx **out, int device, void *stream)
{
    if (!out) return LABFM_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LABFM_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return LABFM_ERR_CUDA;
    labfm_ctx *ctx = new (std::nothrow) labfm_ctx();
    if (!ctx) return LABFM_ERR_NOMEM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMallocHost(&ctx->host_small, 1024) != cudaSuccess) {  // status words read back by the calls
        delete ctx;
        return LABFM_ERR_NOMEM;
    }
    *out = ctx;
    return LABFM_OK;
}

void labfm_destroy(labfm_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DevBuf *bufs[] = {&ctx->node_xy, &ctx->node_h, &ctx->row_ptr, &ctx->col, &ctx->cell_of, &ctx->cell_count, &ctx->cell_start,
                      &ctx->cell_nodes, &ctx->counts, &ctx->scan_tmp, &ctx->misc, &ctx->w,
                      &ctx->status_tmp, &ctx->wtilde, &ctx->mscratch, &ctx->mrecs, &ctx->mwstore, &ctx->mfallback, &ctx->wcomb, &ctx->rk_acc,
                      &ctx->rk_stage_a, &ctx->rk_stage_b, &ctx->wburg, &ctx->bu_acc, &ctx->bu_stage_a,
                      &ctx->bu_stage_b, &ctx->sol_w, &ctx->sol_vec, &ctx->sol_part, &ctx->sol_gmap, &ctx->sol_wg};
    for (DevBuf *b : bufs) b->release();
    ctx->graph.release();
    ctx->graph_burgers.release();
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->host_small) cudaFreeHost(ctx->host_small);
    delete ctx;
}

const char *labfm_last_error(const labfm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

labfm_status labfm_set_stream(labfm_ctx *ctx, void *stream)
{
    if (!ctx) return LABFM_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    ctx->graph.release();
    ctx->graph_burgers.release();
    return LABFM_OK;
}

labfm_status labfm_build_neighbours(labfm_ctx *ctx, int64_t n, const double *xy, const double *h, int periodic,
                                    const double box_lo[2], const double box_hi[2], int64_t *nnz_out)
{
    if (!ctx) return LABFM_ERR_ARG;
    ctx->err.clear();
    if (n < 1 || n >= ((int64_t)1 << 31)) return fail(ctx, LABFM_ERR_ARG, "n must be in [1, 2^31)");
    if (!xy || !h || !box_lo || !box_hi || !nnz_out) return fail(ctx, LABFM_ERR_ARG, "null pointer argument");
    for (int d = 0; d < 2; d++)
        if (!std::isfinite(box_lo[d]) || !std::isfinite(box_hi[d]) || !(box_hi[d] > box_lo[d]))
            return fail(ctx, LABFM_ERR_ARG, "box must be finite with box_hi > box_lo");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, LABFM_ERR_CUDA, "cudaSetDevice failed");
    ctx->have_weights = false;
    ctx->wcomb_valid = false;
    return run_neighbours(ctx, n, xy, h, periodic ? 1 : 0, box_lo, box_hi, nnz_out);
}

labfm_status labfm_get_neighbours(labfm_ctx *ctx, const int64_t **row_ptr, const int32_t **col, int64_t *n,
                                  int64_t *nnz)
{
    if (!ctx) return LABFM_ERR_ARG;
    if (ctx->n == 0) return fail(ctx, LABFM_ERR_STATE, "no stencils built");
    if (row_ptr) *row_ptr = ctx->row_ptr.as<int64_t>();
    if (col) *col = ctx->col.as<int32_t>();
    if (n) *n = ctx->n;
    if (nnz) *nnz = ctx->nnz;
    return LABFM_OK;
}

labfm_status labfm_build_weights(labfm_ctx *ctx, const int8_t *order, int uniform_order, int rbf, int n_ops,
                                 const double *C, int precision, int weight_dtype, int32_t *node_status,
                                 int64_t *n_bad_out)
{
    if (!ctx) return LABFM_ERR_ARG;
    ctx->err.clear();
    if (ctx->n == 0) return fail(ctx, LABFM_ERR_STATE, "labfm_build_neighbours must come first");
    if (!order && (uniform_order < 1 || uniform_order > LABFM_MAX_ORDER))
        return fail(ctx, LABFM_ERR_ARG, "uniform_order must be in 1..8");
    {
        int base = rbf & LABFM_RBF_MASK, form = rbf & ~LABFM_RBF_MASK;
        if (base < LABFM_RBF_WENDLAND_C2 || base > LABFM_RBF_GAUSSIAN || (form & ~LABFM_ABF_DW0_ONLY))
            return fail(ctx, LABFM_ERR_ARG, "unknown rbf");
    }
    if (n_ops < 1 || n_ops > LABFM_MAX_OPS) return fail(ctx, LABFM_ERR_ARG, "n_ops must be in 1..8");
    if (!C) return fail(ctx, LABFM_ERR_ARG, "C is null");
    for (int t = 0; t < n_ops * LABFM_PMAX; t++)
        if (!std::isfinite(C[t])) return fail(ctx, LABFM_ERR_ARG, "C has a non-finite entry");
    {
        int base = precision & 0xff, forced = (precision >> 8) & 0xf, rest = precision >> 12;
        bool ok = rest == 0 && (base == LABFM_PREC_FP64
                                    ? forced == 0
                                    : ((base == LABFM_PREC_MIXED || base == LABFM_PREC_MIXED_TC) && forced <= 5));
        if (!ok) return fail(ctx, LABFM_ERR_ARG, "unknown precision");
    }
    if (weight_dtype != LABFM_F64 && weight_dtype != LABFM_F32) return fail(ctx, LABFM_ERR_ARG, "bad weight_dtype");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, LABFM_ERR_CUDA, "cudaSetDevice failed");
    ctx->have_weights = false;
    ctx->wcomb_valid = false;
    ctx->wburg_valid = false;
    labfm_status st =
        run_build(ctx, order, uniform_order, rbf, n_ops, C, precision, weight_dtype, node_status, n_bad_out);
    if (st == LABFM_OK || st == LABFM_ERR_SINGULAR) {
        ctx->have_weights = true;
        ctx->n_ops = n_ops;
        ctx->wdtype = weight_dtype;
        // operators 0 and 1 are d/dx and d/dy when their targets are the unit vectors of the
        // first two elements of D (Sec. 2): what labfm_step_burgers needs
        bool g = n_ops >= 2;
        for (int e = 0; e < LABFM_PMAX && g; e++)
            g = C[e] == (e == 0 ? 1.0 : 0.0) && C[LABFM_PMAX + e] == (e == 1 ? 1.0 : 0.0);
        ctx->grad01 = g;
    }
    return st;
}

labfm_status labfm_get_build_info(labfm_ctx *ctx, labfm_build_info *info)
{
    if (!ctx || !info) return LABFM_ERR_ARG;
    if (!ctx->have_weights) return fail(ctx, LABFM_ERR_STATE, "no weights built");
    for (int t = 0; t < 8; t++) info->refine_steps[t] = ctx->info_ref_hist[t];
    info->fp64_rebuilt = ctx->info_fp64_rebuilt;
    for (int k = 0; k <= LABFM_MAX_ORDER; k++) {
        info->fp64_group_threads[k] = ctx->info_group[k];
        info->mixed_inv_threads_per_row[k] = ctx->info_inv_tpr[k];
    }
    return LABFM_OK;
}

labfm_status labfm_get_weights(labfm_ctx *ctx, const void **w, int *dtype, int *n_ops)
{
    if (!ctx) return LABFM_ERR_ARG;
    if (!ctx->have_weights) return fail(ctx, LABFM_ERR_STATE, "no weights built");
    if (w) *w = ctx->w.ptr;
    if (dtype) *dtype = ctx->wdtype;
    if (n_ops) *n_ops = ctx->n_ops;
    return LABFM_OK;
}

labfm_status labfm_apply(labfm_ctx *ctx, uint32_t op_mask, const void *f, int field_dtype, void *out)
{
    if (!ctx) return LABFM_ERR_ARG;
    ctx->err.clear();
    if (!ctx->have_weights) return fail(ctx, LABFM_ERR_STATE, "labfm_build_weights must come first");
    if (!f || !out) return fail(ctx, LABFM_ERR_ARG, "null field or output");
    if (field_dtype != LABFM_F64 && field_dtype != LABFM_F32) return fail(ctx, LABFM_ERR_ARG, "bad field_dtype");
    if (op_mask == 0 || (op_mask >> ctx->n_ops) != 0) return fail(ctx, LABFM_ERR_ARG, "op_mask selects no or unknown operators");
    cudaError_t e = launch_apply(ctx, op_mask, f, field_dtype, out);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "labfm_apply launch");
    return LABFM_OK;
}

labfm_status labfm_step(labfm_ctx *ctx, const double *beta, void *u, int field_dtype, double dt, int64_t nsteps,
                        const uint8_t *frozen)
{
    if (!ctx) return LABFM_ERR_ARG;
    ctx->err.clear();
    if (!ctx->have_weights) return fail(ctx, LABFM_ERR_STATE, "labfm_build_weights must come first");
    if (!beta || !u) return fail(ctx, LABFM_ERR_ARG, "null beta or u");
    if (field_dtype != LABFM_F64 && field_dtype != LABFM_F32) return fail(ctx, LABFM_ERR_ARG, "bad field_dtype");
    if (!std::isfinite(dt) || nsteps < 0) return fail(ctx, LABFM_ERR_ARG, "dt must be finite and nsteps >= 0");
    for (int d = 0; d < ctx->n_ops; d++)
        if (!std::isfinite(beta[d])) return fail(ctx, LABFM_ERR_ARG, "beta has a non-finite entry");
    if (nsteps == 0) return LABFM_OK;
    return run_step(ctx, beta, u, field_dtype, dt, nsteps, frozen);
}

labfm_status labfm_solve(labfm_ctx *ctx, int op, const double *f, double *phi, const uint8_t *dirichlet, double tol,
                         int max_iter, int *iters_out, double *resid_out)
{
    if (!ctx) return LABFM_ERR_ARG;
    ctx->err.clear();
    if (!ctx->have_weights) return fail(ctx, LABFM_ERR_STATE, "labfm_build_weights must come first");
    if (op < 0 || op >= ctx->n_ops) return fail(ctx, LABFM_ERR_ARG, "op must index a built operator");
    if (!f || !phi) return fail(ctx, LABFM_ERR_ARG, "null f or phi");
    if ((const void *)f == (const void *)phi) return fail(ctx, LABFM_ERR_ARG, "f and phi must be distinct buffers");
    if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 1) return fail(ctx, LABFM_ERR_ARG, "need tol > 0 and max_iter >= 1");
    return run_solve(ctx, op, f, phi, dirichlet, SolveNeumann{}, tol, max_iter, iters_out, resid_out);
}

labfm_status labfm_solve_neumann(labfm_ctx *ctx, int op, const double *f, double *phi, const uint8_t *dirichlet,
                                 int64_t n_ghost, const int64_t *ghost, const int64_t *parent, const double *normal,
                                 int op_x, int op_y, double tol, int max_iter, int *iters_out, double *resid_out)
{
    if (!ctx) return LABFM_ERR_ARG;
    ctx->err.clear();
    if (!ctx->have_weights) return fail(ctx, LABFM_ERR_STATE, "labfm_build_weights must come first");
    if (op < 0 || op >= ctx->n_ops) return fail(ctx, LABFM_ERR_ARG, "op must index a built operator");
    if (!f || !phi) return fail(ctx, LABFM_ERR_ARG, "null f or phi");
    if ((const void *)f == (const void *)phi) return fail(ctx, LABFM_ERR_ARG, "f and phi must be distinct buffers");
    if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 1) return fail(ctx, LABFM_ERR_ARG, "need tol > 0 and max_iter >= 1");
    if (n_ghost < 0 || n_ghost > ctx->n) return fail(ctx, LABFM_ERR_ARG, "need 0 <= n_ghost <= n");
    SolveNeumann nm;
    if (n_ghost > 0) {
        if (!ghost || !parent || !normal) return fail(ctx, LABFM_ERR_ARG, "null ghost, parent or normal");
        if (op_x < 0 || op_x >= ctx->n_ops || op_y < 0 || op_y >= ctx->n_ops)
            return fail(ctx, LABFM_ERR_ARG, "op_x and op_y must index built operators");
        nm.n_ghost = n_ghost;
        nm.ghost = ghost;
        nm.parent = parent;
        nm.normal = normal;
        nm.op_x = op_x;
        nm.op_y = op_y;
    }
    return run_solve(ctx, op, f, phi, dirichlet, nm, tol, max_iter, iters_out, resid_out);
}

labfm_status labfm_step_burgers(labfm_ctx *ctx, const double *beta, void *u, void *v, int field_dtype, double dt,
                                int64_t nsteps, const uint8_t *frozen)
{
    if (!ctx) return LABFM_ERR_ARG;
    ctx->err.clear();
    if (!ctx->have_weights) return fail(ctx, LABFM_ERR_STATE, "labfm_build_weights must come first");
    if (!ctx->grad01) return fail(ctx, LABFM_ERR_ARG, "operators 0 and 1 of the weights must be d/dx and d/dy");
    if (!beta || !u || !v) return fail(ctx, LABFM_ERR_ARG, "null beta, u or v");
    if (u == v) return fail(ctx, LABFM_ERR_ARG, "u and v must be distinct buffers");
    if (field_dtype != LABFM_F64 && field_dtype != LABFM_F32) return fail(ctx, LABFM_ERR_ARG, "bad field_dtype");
    if (!std::isfinite(dt) || nsteps < 0) return fail(ctx, LABFM_ERR_ARG, "dt must be finite and nsteps >= 0");
    for (int d = 2; d < ctx->n_ops; d++)
        if (!std::isfinite(beta[d])) return fail(ctx, LABFM_ERR_ARG, "beta has a non-finite entry");
    if (nsteps == 0) return LABFM_OK;
    return run_step_burgers(ctx, beta, u, v, field_dtype, dt, nsteps, frozen);
}

}  // extern "C"
