// Implicit solves with the global operator matrix of Sec. 5.2 (eq. poisson_system):
//   A_ij = w^d_ji (j != i),  A_ii = -sum_j w^d_ji,   so (A x)_i = A_ii x_i + sum_j w^d_ji x_j = L^d_i(x),
// with Dirichlet rows (A_bb = 1, A_bj = 0, F_b = g_b) where the caller's mask is set, and Neumann
// ghost rows (A_gj = n_x w^x_jb + n_y w^y_jb over the stencil of the ghost's parent b, A_gb = minus
// their sum, F_g = the normal derivative at b).  The matrix is never formed: its product is a
// stencil sum over the context's CSR stencils.
//
// Solver: stabilised bi-conjugate gradients (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992)
// with a Jacobi preconditioner M = diag(A), the preconditioned form with y = M^-1 p, z = M^-1 s:
//   rho = (r^, r); beta = (rho / rho_old)(alpha / omega); p = r + beta (p - omega v); y = M^-1 p
//   v = A y; alpha = rho / (r^, v); s = r - alpha v; z = M^-1 s; t = A z
//   omega = (t, s) / (t, t); x += alpha y + omega z; r = s - omega t
// Every scalar stays in device memory: each reducing launch writes per-block partial dot
// products and its last block (an atomic ticket) sums them in a fixed order and forms the
// scalars, so an iteration is five launches with no host round trip (16 iterations recorded once
// per call into a CUDA graph and replayed).  A device flag ends the iteration
// (converged, breakdown, iteration limit); later launches see it and return at once, so the host
// reads the flag once per chunk.
#include <algorithm>
#include <cmath>
#include <vector>

#include "labfm_internal.cuh"

namespace labfm {
namespace {

constexpr int SOLVE_THREADS = 256;
constexpr int SOLVE_G = 4;      // lanes per node in the setup
constexpr int SOLVE_G_MAX = 16; // the product's lanes per node are tuned in {4, 8, 16} x entries in flight {2, 4, 8}
constexpr int SOLVE_VEC_MAX_BLOCKS = 1024;

// device-resident solver state
struct SolveState {
    double rho, rho_old, alpha, omega, beta;
    double bnorm2, rnorm2, snorm2;
    double tol2;       // (tol ||b||)^2
    int done;          // 0 running, 1 converged, 2 breakdown, 3 iteration limit
    int skip;          // ||s|| already within the tolerance: omega = 0, x += alpha y, r = s
    int iters;
    int max_iter;
    unsigned int ticket;  // blocks of the current launch that have written their partial sums
};

// Two sums over the block at once, of values held by the threads whose index is a multiple of
// STRIDE (the others' are ignored), in a fixed order (deterministic); the results are valid in
// warp 0.  The values go through shared memory and warp 0 alone adds them: on GB300 every FP64
// add is scarce, and a shuffle tree in every warp would cost each warp five adds per sum, about
// as many FP64 instructions as a product's stencil entries.  sh: 2 x SOLVE_THREADS / STRIDE.
template <int STRIDE>
__device__ __forceinline__ void block_sum2(double a, double b, double *sh, double &sa, double &sb)
{
    constexpr int NV = SOLVE_THREADS / STRIDE;
    __syncthreads();  // sh is free (an earlier sum may still be reading it)
    if (threadIdx.x % STRIDE == 0) {
        sh[threadIdx.x / STRIDE] = a;
        sh[NV + threadIdx.x / STRIDE] = b;
    }
    __syncthreads();
    sa = sb = 0.0;
    if (threadIdx.x < 32) {
        for (int k = threadIdx.x; k < NV; k += 32) {
            sa += sh[k];
            sb += sh[NV + k];
        }
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
        }
    }
}

// The scalars of the step that follows a reduction (thread 0 of the reducing block):
//   step 0 (after the setup):       rnorm2, bnorm2, rho = rnorm2, alpha = omega = rho_old = 1, beta = 0
//   step 2 (after v = A y):         alpha = rho / (rhat, v)
//   step 4 (after t = A z):         skip = (s, s) <= tol2; omega = (t, s) / (t, t)
//   step 5 (after the x, r update): rho_old = rho, rho = (rhat, r), rnorm2, iters++, convergence,
//                                   beta of the next iteration
// s0..s2: the sums of the three partial slots; s3: the sum of part2 (the (s, s) of phase 2).
__device__ void form_scalars(int step, double s0, double s1, double s2, double s3, SolveState *st)
{
    switch (step) {
    case 0:
        st->rnorm2 = s0;
        st->bnorm2 = s1;
        st->tol2 *= s1 > 0.0 ? s1 : 1.0;
        st->rho = s0;
        st->rho_old = st->alpha = st->omega = 1.0;
        st->beta = 0.0;
        st->iters = 0;
        st->done = (s0 <= st->tol2) ? 1 : 0;
        break;
    case 2:
        st->alpha = st->rho / s0;
        if (s0 == 0.0 || !isfinite(st->alpha)) st->done = 2;
        break;
    case 4:
        st->snorm2 = s3;
        st->skip = s3 <= st->tol2 ? 1 : 0;
        st->omega = st->skip ? 0.0 : (s2 > 0.0 ? s0 / s2 : 0.0);
        if (!isfinite(st->omega)) st->done = 2;
        break;
    default:
        st->rho_old = st->rho;
        st->rho = s0;
        st->rnorm2 = s1;
        st->iters += 1;
        if (s1 <= st->tol2) st->done = 1;
        else if (st->rho == 0.0 || st->omega == 0.0 || !isfinite(s1)) st->done = 2;
        else if (st->iters >= st->max_iter) st->done = 3;
        else {
            st->beta = (st->rho / st->rho_old) * (st->alpha / st->omega);
            if (!isfinite(st->beta)) st->done = 2;
        }
        break;
    }
}

// Called by every block after thread 0 has written the block's partials: the last block to
// arrive sums all partials in a fixed order (deterministic) and forms the scalars of `step`.
// The partials are read through L2 (__ldcg) after the other blocks' fence-then-ticket.
__device__ void last_block_scalars(int nblk, int step, const double *part, int nblk2, const double *part2,
                                   SolveState *st, double *sh)
{
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st->ticket, 1u) == (unsigned)(nblk - 1);
    }
    __syncthreads();
    if (!s_last) return;  // uniform per block
    __threadfence();
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int k = threadIdx.x; k < nblk; k += SOLVE_THREADS) {
        a += __ldcg(part + 3 * k);
        b += __ldcg(part + 3 * k + 1);
        c += __ldcg(part + 3 * k + 2);
    }
    if (part2)
        for (int k = threadIdx.x; k < nblk2; k += SOLVE_THREADS) d += __ldcg(part2 + 3 * k);
    double s0, s1, s2, s3;
    block_sum2<1>(a, b, sh, s0, s1);
    block_sum2<1>(c, d, sh, s2, s3);
    if (threadIdx.x == 0) {
        form_scalars(step, s0, s1, s2, s3, st);
        st->ticket = 0u;  // the next reduction starts from zero (it is a later launch)
    }
}

// weights of operator d as one contiguous FP64 stream, the Jacobi scaling 1 / A_ii, and the
// Dirichlet values into the initial guess: their residuals, search directions and updates are
// then exactly zero, so those entries keep f_i exactly.  SOLVE_G lanes per node.
template <class WT>
__global__ void __launch_bounds__(SOLVE_THREADS) k_solve_setup(int64_t n, const int64_t *__restrict__ row_ptr,
                                                              const WT *__restrict__ w, int n_ops, int op,
                                                              double *__restrict__ wd, double *__restrict__ dinv,
                                                              double *__restrict__ adiag,
                                                              const uint8_t *__restrict__ dirichlet,
                                                              const double *__restrict__ f, double *__restrict__ x)
{
    const int lane = threadIdx.x & (SOLVE_G - 1);
    const int64_t i = ((int64_t)blockIdx.x * SOLVE_THREADS + threadIdx.x) / SOLVE_G;
    double sum = 0.0;
    if (i < n)
        for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += SOLVE_G) {
            const double v = (double)w[e * n_ops + op];
            wd[e] = v;
            sum += v;
        }
    for (int o = SOLVE_G >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (i >= n || lane != 0) return;
    const bool fixed = dirichlet && dirichlet[i];
    if (fixed) x[i] = f[i];
    const double a = -sum;  // A_ii
    adiag[i] = a;
    dinv[i] = fixed ? 1.0 : (a != 0.0 && isfinite(1.0 / a) ? 1.0 / a : 1.0);
}

// Neumann ghost rows (Sec. 5.2): gmap[ghost[g]] = g (gmap starts at -1), with the checks the host
// reads back in flag: bit 0 an index out of range or a ghost that is its own parent, bit 1 a
// ghost listed twice, bit 2 a ghost row also marked Dirichlet, bit 3 a non-finite normal.
__global__ void k_ghost_map(int64_t n, int64_t n_ghost, const int64_t *__restrict__ ghost,
                            const int64_t *__restrict__ parent, const double *__restrict__ normal,
                            const uint8_t *__restrict__ dirichlet, int32_t *__restrict__ gmap,
                            unsigned int *__restrict__ flag)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_ghost) return;
    const int64_t gi = ghost[g], b = parent[g];
    if (!isfinite(normal[2 * g]) || !isfinite(normal[2 * g + 1])) atomicOr(flag, 8u);
    if (gi < 0 || gi >= n || b < 0 || b >= n || gi == b) {
        atomicOr(flag, 1u);
        return;
    }
    if (dirichlet && dirichlet[gi]) atomicOr(flag, 4u);
    if (atomicCAS(&gmap[gi], -1, (int)g) != -1) atomicOr(flag, 2u);
}

// goff[g] = sum over g' < g of the stencil size of parent[g'] (where ghost g's weights start in
// the ghost weight stream), goff[n_ghost] the total; one block, each thread a contiguous run of
// ghosts, then a scan of the per-thread sums in shared memory.  A parent out of range counts 0
// (k_ghost_map has flagged it and the solve stops before any use).
constexpr int GHOST_SCAN_THREADS = 1024;
__global__ void __launch_bounds__(GHOST_SCAN_THREADS) k_ghost_offsets(int64_t n, int64_t n_ghost,
                                                                      const int64_t *__restrict__ parent,
                                                                      const int64_t *__restrict__ row_ptr,
                                                                      int64_t *__restrict__ goff)
{
    __shared__ int64_t sh[GHOST_SCAN_THREADS];
    const int64_t per = (n_ghost + GHOST_SCAN_THREADS - 1) / GHOST_SCAN_THREADS;
    const int64_t g0 = (int64_t)threadIdx.x * per, g1 = g0 + per < n_ghost ? g0 + per : n_ghost;
    auto size_of = [&](int64_t g) -> int64_t {
        const int64_t b = parent[g];
        return (b >= 0 && b < n) ? row_ptr[b + 1] - row_ptr[b] : 0;
    };
    int64_t run = 0;
    for (int64_t g = g0; g < g1; g++) run += size_of(g);
    sh[threadIdx.x] = run;
    __syncthreads();
    for (int o = 1; o < GHOST_SCAN_THREADS; o <<= 1) {  // inclusive scan (Hillis-Steele)
        const int64_t add = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += add;
        __syncthreads();
    }
    int64_t at = sh[threadIdx.x] - run;  // exclusive prefix of this thread's run
    for (int64_t g = g0; g < g1; g++) {
        goff[g] = at;
        at += size_of(g);
    }
    if (threadIdx.x == GHOST_SCAN_THREADS - 1) goff[n_ghost] = sh[threadIdx.x];
}

// The ghost rows' weights and diagonals: row ghost[g] is n_x L^(op_x) + n_y L^(op_y) at the
// parent b (Sec. 5.2): entry e of b's stencil gets c_e = n_x w^(op_x)_e + n_y w^(op_y)_e
// (into wdg from goff[g]), the column of b gets -sum_e c_e (adiag), and the Jacobi scaling uses
// the row's true diagonal, the c_e of the ghost itself within b's stencil (1 if it is absent or
// zero).  SOLVE_G lanes per ghost; runs after k_solve_setup, whose values for these rows it
// replaces.
template <class WT>
__global__ void __launch_bounds__(SOLVE_THREADS) k_solve_setup_ghost(
    int64_t n_ghost, const int64_t *__restrict__ ghost, const int64_t *__restrict__ parent,
    const double *__restrict__ normal, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    const WT *__restrict__ w, int n_ops, int op_x, int op_y, const int64_t *__restrict__ goff,
    double *__restrict__ wdg, double *__restrict__ adiag, double *__restrict__ dinv)
{
    const int lane = threadIdx.x & (SOLVE_G - 1);
    const int64_t g = ((int64_t)blockIdx.x * SOLVE_THREADS + threadIdx.x) / SOLVE_G;
    double sum = 0.0, diag = 0.0;
    int64_t gi = 0;
    if (g < n_ghost) {
        gi = ghost[g];
        const int64_t b = parent[g];
        const double nx = normal[2 * g], ny = normal[2 * g + 1];
        const int64_t rs = row_ptr[b], re = row_ptr[b + 1], o = goff[g] - rs;
        for (int64_t e = rs + lane; e < re; e += SOLVE_G) {
            const double v = nx * (double)w[e * n_ops + op_x] + ny * (double)w[e * n_ops + op_y];
            wdg[o + e] = v;
            sum += v;
            if (col[e] == gi) diag += v;
        }
    }
    for (int o = SOLVE_G >> 1; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        diag += __shfl_xor_sync(0xffffffffu, diag, o);
    }
    if (g >= n_ghost || lane != 0) return;
    adiag[gi] = -sum;
    dinv[gi] = (diag != 0.0 && isfinite(1.0 / diag)) ? 1.0 / diag : 1.0;
}

// The ghost rows as the product kernel reads them (all null when there are none)
struct GhostRows {
    const int32_t *gmap = nullptr;   // [n]: ghost ordinal of row i, or -1
    const int64_t *parent = nullptr; // [n_ghost]
    const int64_t *goff = nullptr;   // [n_ghost + 1]
    const double *wdg = nullptr;     // ghost weight stream
};

// out = A x with the matrix in its global form (Sec. 5.2): out_i = A_ii x_i + sum_j w_ji x_j, one
// FP64 multiply-add per stencil entry (Dirichlet rows: out_i = x_i; a Neumann ghost row: the
// stencil of its parent b with the ghost weights, and the diagonal term on x_b); G lanes per node
// with UNR entries in flight per lane; fused partial dot products (a1 . out), (out . out) into
// part[3 block + 0, 2]
template <int G, int UNR>
__global__ void __launch_bounds__(SOLVE_THREADS) k_solve_spmv(int64_t n, const int64_t *__restrict__ row_ptr,
                                                             const int32_t *__restrict__ col,
                                                             const double *__restrict__ wd,
                                                             const double *__restrict__ adiag,
                                                             const uint8_t *__restrict__ dirichlet,
                                                             const double *__restrict__ x, double *__restrict__ out,
                                                             const double *__restrict__ a1, double *__restrict__ part,
                                                             int step, int nblk2, const double *__restrict__ part2,
                                                             SolveState *__restrict__ st, GhostRows gr)
{
    if (st && st->done) return;
    __shared__ double sh[2 * SOLVE_THREADS];
    const int lane = threadIdx.x & (G - 1);
    const int64_t i = ((int64_t)blockIdx.x * SOLVE_THREADS + threadIdx.x) / G;
    const bool live = i < n;
    int64_t rs = 0, re = 0, woff = 0;
    const double *wrow = wd;
    double xi = 0.0;  // x at the row's diagonal column (i, or a ghost row's parent)
    if (live) {
        int64_t src = i;
        int gidx = -1;
        if (gr.gmap) gidx = gr.gmap[i];
        if (gidx >= 0) src = gr.parent[gidx];
        rs = row_ptr[src];
        re = row_ptr[src + 1];
        xi = x[src];
        if (gidx >= 0) {
            wrow = gr.wdg;
            woff = gr.goff[gidx] - rs;
        }
    }
    double acc = 0.0;
    for (int64_t base = rs; base < re; base += G * UNR) {
        int cj[UNR];
        double wv[UNR];
#pragma unroll
        for (int q = 0; q < UNR; q++) {
            const int64_t e = base + q * G + lane;
            cj[q] = e < re ? __ldcs(col + e) : -1;
            wv[q] = e < re ? __ldcs(wrow + (e + woff)) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < UNR; q++)
            if (cj[q] >= 0) acc = fma(x[cj[q]], wv[q], acc);
    }
    for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    double d1 = 0.0, d3 = 0.0;
    if (live && lane == 0) {
        const double yi = (dirichlet && dirichlet[i]) ? xi : fma(adiag[i], xi, acc);
        out[i] = yi;
        if (a1) d1 = a1[i] * yi;
        d3 = yi * yi;
    }
    if (!part) return;
    double s1, s3;
    block_sum2<G>(d1, d3, sh, s1, s3);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s1;
        part[3 * blockIdx.x + 1] = 0.0;
        part[3 * blockIdx.x + 2] = s3;
    }
    if (step >= 0) last_block_scalars(gridDim.x, step, part, nblk2, part2, st, sh);
}

// the element-wise updates of one iteration, by phase
//   0: r = b - r (r holds A x on entry), rhat = r, p = v = 0; partials (r, r), (b, b)
//   1: p = r + beta (p - omega v); y = dinv p
//   2: s = r - alpha v; z = dinv s; partial (s, s) into part2
//   3: x += alpha y + omega z; r = s - omega t; partials (rhat, r), (r, r)
__global__ void __launch_bounds__(SOLVE_THREADS) k_solve_vec(int64_t n, int phase, const double *__restrict__ b,
                                                            double *__restrict__ x, double *__restrict__ r,
                                                            double *__restrict__ rhat, double *__restrict__ p,
                                                            double *__restrict__ v, double *__restrict__ y,
                                                            double *__restrict__ s, double *__restrict__ z,
                                                            const double *__restrict__ t,
                                                            const double *__restrict__ dinv,
                                                            double *__restrict__ part, SolveState *__restrict__ st)
{
    if (phase != 0 && st->done) return;
    __shared__ double sh[2 * SOLVE_THREADS];
    const double alpha = st ? st->alpha : 0.0, omega = st ? st->omega : 0.0, beta = st ? st->beta : 0.0;
    double d1 = 0.0, d2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        switch (phase) {
        case 0: {
            const double ri = b[i] - r[i];
            r[i] = ri;
            rhat[i] = ri;
            p[i] = 0.0;
            v[i] = 0.0;
            d1 = fma(ri, ri, d1);
            d2 = fma(b[i], b[i], d2);
            break;
        }
        case 1: {
            const double pi = fma(beta, fma(-omega, v[i], p[i]), r[i]);
            p[i] = pi;
            y[i] = dinv[i] * pi;
            break;
        }
        case 2: {
            const double si = fma(-alpha, v[i], r[i]);
            s[i] = si;
            z[i] = dinv[i] * si;
            d1 = fma(si, si, d1);
            break;
        }
        default: {
            x[i] = fma(omega, z[i], fma(alpha, y[i], x[i]));
            const double ri = fma(-omega, t[i], s[i]);
            r[i] = ri;
            d1 = fma(rhat[i], ri, d1);
            d2 = fma(ri, ri, d2);
            break;
        }
        }
    }
    if (phase == 1) return;
    double s1, s2;
    block_sum2<1>(d1, d2, sh, s1, s2);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s1;
        part[3 * blockIdx.x + 1] = s2;
        part[3 * blockIdx.x + 2] = 0.0;
    }
    // phase 0 forms the starting scalars, phase 3 those of the next iteration; the (s, s) of
    // phase 2 is read with omega after t = A z
    if (st && (phase == 0 || phase == 3)) last_block_scalars(gridDim.x, phase == 0 ? 0 : 5, part, 0, nullptr, st, sh);
}

template <int G, int UNR>
cudaError_t launch_spmv_t(int64_t n, const int64_t *rp, const int32_t *cl, const double *wd, const double *adiag,
                          const uint8_t *dirichlet, const double *x, double *out, const double *a1, double *part,
                          int step, int nblk2, const double *part2, SolveState *st, const GhostRows &gr,
                          cudaStream_t q)
{
    const unsigned blocks = (unsigned)((n * G + SOLVE_THREADS - 1) / SOLVE_THREADS);
    k_solve_spmv<G, UNR><<<blocks, SOLVE_THREADS, 0, q>>>(n, rp, cl, wd, adiag, dirichlet, x, out, a1, part, step,
                                                          nblk2, part2, st, gr);
    return cudaGetLastError();
}

cudaError_t launch_spmv(int G, int UNR, int64_t n, const int64_t *rp, const int32_t *cl, const double *wd,
                        const double *adiag, const uint8_t *dirichlet, const double *x, double *out, const double *a1,
                        double *part, int step, int nblk2, const double *part2, SolveState *st, const GhostRows &gr,
                        cudaStream_t q)
{
#define LABFM_SPMV_CASE(g, u)                                                                                   \
    if (G == g && UNR == u) return launch_spmv_t<g, u>(n, rp, cl, wd, adiag, dirichlet, x, out, a1, part, step, \
                                                       nblk2, part2, st, gr, q);
    LABFM_SPMV_CASE(4, 2) LABFM_SPMV_CASE(4, 4) LABFM_SPMV_CASE(4, 8)
    LABFM_SPMV_CASE(8, 2) LABFM_SPMV_CASE(8, 4) LABFM_SPMV_CASE(8, 8)
    LABFM_SPMV_CASE(16, 2) LABFM_SPMV_CASE(16, 4) LABFM_SPMV_CASE(16, 8)
#undef LABFM_SPMV_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

labfm_status run_solve(labfm_ctx *ctx, int op, const double *f, double *phi, const uint8_t *dirichlet,
                       const SolveNeumann &nm, double tol, int max_iter, int *iters_out, double *resid_out)
{
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n, nnz = ctx->nnz;
    const int nblk_setup = (int)((n * SOLVE_G + SOLVE_THREADS - 1) / SOLVE_THREADS);
    const int nblk_vec = (int)std::min<int64_t>((n + SOLVE_THREADS - 1) / SOLVE_THREADS, SOLVE_VEC_MAX_BLOCKS);
    const size_t npart = 3 * (size_t)std::max<int64_t>((n * SOLVE_G_MAX + SOLVE_THREADS - 1) / SOLVE_THREADS, nblk_vec);
    LABFM_CUDA_TRY(ctx, ctx->sol_w.reserve(sizeof(double) * (nnz > 0 ? nnz : 1)));
    LABFM_CUDA_TRY(ctx, ctx->sol_vec.reserve(sizeof(double) * 10 * n));
    LABFM_CUDA_TRY(ctx, ctx->sol_part.reserve(sizeof(double) * (npart + 3 * (size_t)nblk_vec) + sizeof(SolveState)));
    double *V = ctx->sol_vec.as<double>();
    double *dinv = V, *r = V + n, *rhat = V + 2 * n, *p = V + 3 * n, *v = V + 4 * n, *y = V + 5 * n, *sv = V + 6 * n,
           *z = V + 7 * n, *t = V + 8 * n, *adiag = V + 9 * n;
    double *part = ctx->sol_part.as<double>();
    double *part2 = part + npart;  // (s, s) of phase 2, read with omega
    SolveState *st = reinterpret_cast<SolveState *>(part2 + 3 * (size_t)nblk_vec);
    const int64_t *rp = ctx->row_ptr.as<int64_t>();
    const int32_t *cl = ctx->col.as<int32_t>();
    const double *wd = ctx->sol_w.as<double>();
    if (ctx->wdtype == LABFM_F64)
        k_solve_setup<double><<<nblk_setup, SOLVE_THREADS, 0, s>>>(n, rp, ctx->w.as<double>(), ctx->n_ops, op,
                                                               ctx->sol_w.as<double>(), dinv, adiag, dirichlet, f, phi);
    else
        k_solve_setup<float><<<nblk_setup, SOLVE_THREADS, 0, s>>>(n, rp, ctx->w.as<float>(), ctx->n_ops, op,
                                                              ctx->sol_w.as<double>(), dinv, adiag, dirichlet, f, phi);
    LABFM_CUDA_TRY(ctx, cudaGetLastError());
    // Neumann ghost rows: map, checks and weight offsets, read back with one synchronisation;
    // then their weights and diagonals replace what the setup wrote for those rows
    GhostRows gr;
    if (nm.n_ghost > 0) {
        const int64_t ng = nm.n_ghost;
        const size_t map_bytes = ((sizeof(int32_t) * (size_t)n + 15) / 16) * 16;
        LABFM_CUDA_TRY(ctx, ctx->sol_gmap.reserve(map_bytes + sizeof(int64_t) * (size_t)(ng + 1) + 16));
        int32_t *gmap = ctx->sol_gmap.as<int32_t>();
        int64_t *goff = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(gmap) + map_bytes);
        unsigned int *gflag = reinterpret_cast<unsigned int *>(goff + ng + 1);
        LABFM_CUDA_TRY(ctx, cudaMemsetAsync(gmap, 0xff, sizeof(int32_t) * (size_t)n, s));  // -1
        LABFM_CUDA_TRY(ctx, cudaMemsetAsync(gflag, 0, sizeof(unsigned int), s));
        k_ghost_map<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(n, ng, nm.ghost, nm.parent, nm.normal, dirichlet,
                                                                 gmap, gflag);
        k_ghost_offsets<<<1, GHOST_SCAN_THREADS, 0, s>>>(n, ng, nm.parent, rp, goff);
        LABFM_CUDA_TRY(ctx, cudaGetLastError());
        unsigned long long *hs = (unsigned long long *)ctx->host_small;
        LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(&hs[0], goff + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(&hs[1], gflag, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        const unsigned flag = (unsigned)(hs[1] & 0xffffffffull);
        if (flag & 1u) return fail(ctx, LABFM_ERR_ARG, "a ghost or parent index is out of range, or a ghost is its own parent");
        if (flag & 2u) return fail(ctx, LABFM_ERR_ARG, "a ghost row is listed twice");
        if (flag & 4u) return fail(ctx, LABFM_ERR_ARG, "a ghost row is also a Dirichlet row");
        if (flag & 8u) return fail(ctx, LABFM_ERR_ARG, "a ghost normal is not finite");
        const int64_t total = (int64_t)hs[0];
        LABFM_CUDA_TRY(ctx, ctx->sol_wg.reserve(sizeof(double) * (size_t)(total > 0 ? total : 1)));
        double *wdg = ctx->sol_wg.as<double>();
        const unsigned gblk = (unsigned)((ng * SOLVE_G + SOLVE_THREADS - 1) / SOLVE_THREADS);
        if (ctx->wdtype == LABFM_F64)
            k_solve_setup_ghost<double><<<gblk, SOLVE_THREADS, 0, s>>>(ng, nm.ghost, nm.parent, nm.normal, rp, cl,
                                                                     ctx->w.as<double>(), ctx->n_ops, nm.op_x,
                                                                     nm.op_y, goff, wdg, adiag, dinv);
        else
            k_solve_setup_ghost<float><<<gblk, SOLVE_THREADS, 0, s>>>(ng, nm.ghost, nm.parent, nm.normal, rp, cl,
                                                                    ctx->w.as<float>(), ctx->n_ops, nm.op_x,
                                                                    nm.op_y, goff, wdg, adiag, dinv);
        LABFM_CUDA_TRY(ctx, cudaGetLastError());
        gr.gmap = gmap;
        gr.parent = nm.parent;
        gr.goff = goff;
        gr.wdg = wdg;
    }
    SolveState init{};
    init.tol2 = tol * tol;
    init.max_iter = max_iter;
    LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(st, &init, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    // the product's launch shape: tuned once per problem class on this context (not while the
    // caller's stream is being captured, nor below 4096 nodes), kept in the context's table
    int G = 4, UNR = 4;
    {
        const int64_t deg = n > 0 ? (nnz + n / 2) / n : 0;
        int64_t lg = 0;
        while (lg < 62 && ((int64_t)1 << (lg + 1)) <= n) lg++;
        const uint64_t key = ((uint64_t)(deg > 0xffff ? 0xffff : deg) << 40) | ((uint64_t)lg << 32) | (4ull << 24);
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            G = (int)(it->second >> 8);
            UNR = (int)(it->second & 0xff);
        } else {
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            LABFM_CUDA_TRY(ctx, cudaStreamIsCapturing(s, &cap));
            if (cap == cudaStreamCaptureStatusNone && n >= 4096) {
                cudaEvent_t e0, e1;
                LABFM_CUDA_TRY(ctx, cudaEventCreate(&e0));
                LABFM_CUDA_TRY(ctx, cudaEventCreate(&e1));
                float best = 1e30f;
                const int gs[3] = {4, 8, 16}, us[3] = {2, 4, 8};
                cudaError_t te = cudaSuccess;
                for (int gi = 0; gi < 3 && te == cudaSuccess; gi++)
                    for (int ui = 0; ui < 3 && te == cudaSuccess; ui++) {
                        for (int rep = 0; rep < 2 && te == cudaSuccess; rep++) {  // warm-up, then timed
                            if (rep) cudaEventRecord(e0, s);
                            te = launch_spmv(gs[gi], us[ui], n, rp, cl, wd, adiag, dirichlet, f, t, nullptr, part, -1,
                                             0, nullptr, nullptr, gr, s);
                            if (rep) cudaEventRecord(e1, s);
                        }
                        float ms = 0.0f;
                        if (te == cudaSuccess) te = cudaEventSynchronize(e1);
                        if (te == cudaSuccess) te = cudaEventElapsedTime(&ms, e0, e1);
                        if (te == cudaSuccess && ms < best) {
                            best = ms;
                            G = gs[gi];
                            UNR = us[ui];
                        }
                    }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (te != cudaSuccess) return cuda_fail(ctx, te, "solver launch-shape tuning");
                ctx->tuned[key] = ((uint32_t)G << 8) | (uint32_t)UNR;
            }
        }
    }
    // step: the scalars the last block forms (-1: none, and no gating on the state)
    auto spmv = [&](cudaStream_t q, const double *x, double *out, const double *a1, int step) {
        launch_spmv(G, UNR, n, rp, cl, wd, adiag, dirichlet, x, out, a1, part, step, step == 4 ? nblk_vec : 0,
                    step == 4 ? part2 : nullptr, step >= 0 ? st : nullptr, gr, q);
    };
    auto vec = [&](cudaStream_t q, int phase) {
        k_solve_vec<<<nblk_vec, SOLVE_THREADS, 0, q>>>(n, phase, f, phi, r, rhat, p, v, y, sv, z, t, dinv,
                                                       phase == 2 ? part2 : part, st);
    };
    // r = b - A x, r^ = r
    spmv(s, phi, r, nullptr, -1);
    vec(s, 0);                                // + the starting scalars
    LABFM_CUDA_TRY(ctx, cudaGetLastError());
    // one chunk of iterations, recorded once per call into a CUDA graph and replayed
    constexpr int CHUNK = 16;
    auto enqueue_chunk = [&](cudaStream_t q) {
        for (int it = 0; it < CHUNK; it++) {
            vec(q, 1);                        // p, y
            spmv(q, y, v, rhat, 2);           // v = A y, (rhat, v) -> alpha
            vec(q, 2);                        // s, z, (s, s)
            spmv(q, z, t, sv, 4);             // t = A z, (s, t), (t, t) -> omega
            vec(q, 3);                        // x, r, (rhat, r), (r, r) -> rho, beta, convergence
        }
    };
    if (!ctx->capture_stream)
        LABFM_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    LABFM_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_chunk(ctx->capture_stream);
    {
        cudaError_t e = cudaGetLastError();
        cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "BiCGStab chunk capture");
    }
    // Chunks of iterations until the device flag ends them; then the true residual.  BiCGStab
    // restarts from the current iterate (r = F - A Phi, r^ = r), at most MAX_RESTARTS times
    // within max_iter in total, in two cases: the recurrence residual, which drifts from the
    // true one in finite precision, says converged while the true residual is above tol; or the
    // iteration broke down (rho = (r^, r), (r^, v) or omega vanished or was not finite) with a
    // finite iterate.  The second is the usual remedy for a breakdown: the shadow residual r^
    // has become orthogonal to the Krylov space, and a fresh r^ = r starts a new one.  (No
    // launch after the one that flagged the breakdown updates Phi, except when the residual
    // norm itself was not finite, which the finite-residual condition excludes.)
    constexpr int MAX_RESTARTS = 8;
    SolveState h{};
    int total = 0, restarts = 0;
    double resid = 0.0;
    std::vector<double> hp(3 * (size_t)nblk_vec);
    cudaError_t le = cudaSuccess;
    while (true) {
        for (int it = 0; it < max_iter - total && le == cudaSuccess; it += CHUNK) {
            le = cudaGraphLaunch(exec, s);  // the iteration limit stops the last chunk early (done = 3)
            if (le == cudaSuccess) le = cudaMemcpyAsync(&h, st, sizeof(SolveState), cudaMemcpyDeviceToHost, s);
            if (le == cudaSuccess) le = cudaStreamSynchronize(s);
            if (h.done) break;
        }
        if (le != cudaSuccess) break;
        total += h.iters;
        // the true residual ||b - A x|| / ||b||: t = A x, then phase 0 on scratch copies
        spmv(s, phi, t, nullptr, -1);
        k_solve_vec<<<nblk_vec, SOLVE_THREADS, 0, s>>>(n, 0, f, nullptr, t, sv, z, y, nullptr, nullptr, nullptr,
                                                       nullptr, nullptr, part, nullptr);
        le = cudaGetLastError();
        if (le == cudaSuccess)
            le = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s);
        if (le == cudaSuccess) le = cudaStreamSynchronize(s);
        if (le != cudaSuccess) break;
        double rr = 0.0, bb = 0.0;
        for (int k = 0; k < nblk_vec; k++) {
            rr += hp[3 * k];
            bb += hp[3 * k + 1];
        }
        resid = std::sqrt(rr) / (bb > 0.0 ? std::sqrt(bb) : 1.0);
        const bool drifted = h.done == 1 && resid > tol, broke_down = h.done == 2;
        if ((drifted || broke_down) && std::isfinite(resid) && restarts < MAX_RESTARTS && total < max_iter) {
            restarts++;
            init.max_iter = max_iter - total;
            le = cudaMemcpyAsync(st, &init, sizeof(SolveState), cudaMemcpyHostToDevice, s);
            if (le != cudaSuccess) break;
            spmv(s, phi, r, nullptr, -1);
            vec(s, 0);
            le = cudaGetLastError();
            if (le != cudaSuccess) break;
            continue;
        }
        break;
    }
    cudaGraphExecDestroy(exec);
    if (le != cudaSuccess) return cuda_fail(ctx, le, "BiCGStab iterations");
    if (iters_out) *iters_out = total;
    if (resid_out) *resid_out = resid;
    if (h.done == 1 && std::isfinite(resid) && resid <= tol) return LABFM_OK;
    return fail(ctx, LABFM_ERR_NOT_CONVERGED,
                h.done == 2   ? "BiCGStab breakdown (rho, alpha or omega vanished or was not finite)"
                : h.done == 1 ? "the true residual stayed above tol after the restarts"
                              : "BiCGStab did not reach the tolerance within max_iter iterations");
}

}  // namespace labfm
