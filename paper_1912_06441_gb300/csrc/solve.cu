// Implicit solves with the global operator matrix of Sec. 5.2 (eq. poisson_system):
//   A_ij = w^d_ji (j != i),  A_ii = -sum_j w^d_ji,   so (A x)_i = sum_j (x_j - x_i) w^d_ji = L^d_i(x),
// with Dirichlet rows (A_bb = 1, A_bj = 0, F_b = g_b) where the caller's mask is set.  The matrix
// is never formed: its product is a stencil sum over the context's CSR stencils.
//
// Solver: stabilised bi-conjugate gradients (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992)
// with a Jacobi preconditioner M = diag(A), the preconditioned form with y = M^-1 p, z = M^-1 s:
//   rho = (r^, r); beta = (rho / rho_old)(alpha / omega); p = r + beta (p - omega v); y = M^-1 p
//   v = A y; alpha = rho / (r^, v); s = r - alpha v; z = M^-1 s; t = A z
//   omega = (t, s) / (t, t); x += alpha y + omega z; r = s - omega t
// Every scalar stays in device memory: per-block partial dot products, then a one-block kernel
// that forms the scalars, so an iteration is eight launches with no host round trip.  A device
// flag ends the iteration (converged, breakdown); later launches see it and return at once, so
// the host enqueues iterations in chunks and reads the flag once per chunk.
#include <algorithm>
#include <cmath>
#include <vector>

#include "labfm_internal.cuh"

namespace labfm {
namespace {

constexpr int SOLVE_THREADS = 256;
constexpr int SOLVE_MAX_BLOCKS = 1024;  // partial sums per reduction

// device-resident solver state
struct SolveState {
    double rho, rho_old, alpha, omega, beta;
    double bnorm2, rnorm2, snorm2;
    double tol2;       // (tol ||b||)^2
    int done;          // 0 running, 1 converged, 2 breakdown, 3 iteration limit
    int skip;          // ||s|| already within the tolerance: omega = 0, x += alpha y, r = s
    int iters;
    int max_iter;
};

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < SOLVE_THREADS / 32; w++) s += sh[w];  // fixed order: deterministic
    return s;
}

// weights of operator d as one contiguous FP64 stream, the Jacobi scaling 1 / A_ii, and the
// Dirichlet values into the initial guess: their residuals, search directions and updates are
// then exactly zero, so those entries keep f_i exactly
template <class WT>
__global__ void k_solve_setup(int64_t n, const int64_t *__restrict__ row_ptr, const WT *__restrict__ w, int n_ops,
                              int op, double *__restrict__ wd, double *__restrict__ dinv,
                              const uint8_t *__restrict__ dirichlet, const double *__restrict__ f,
                              double *__restrict__ x)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (dirichlet && dirichlet[i]) x[i] = f[i];
        double s = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            const double v = (double)w[e * n_ops + op];
            wd[e] = v;
            s += v;
        }
        const double a = -s;  // A_ii
        dinv[i] = (dirichlet && dirichlet[i]) ? 1.0 : (a != 0.0 && isfinite(1.0 / a) ? 1.0 / a : 1.0);
    }
}

// out = A x (Dirichlet rows: out_i = x_i), one warp per node; optional fused partial dot products
// (a1 . out) and (a2 . out), (out . out) into part[block][0..2]
__global__ void __launch_bounds__(SOLVE_THREADS) k_solve_spmv(int64_t n, const int64_t *__restrict__ row_ptr,
                                                             const int32_t *__restrict__ col,
                                                             const double *__restrict__ wd,
                                                             const uint8_t *__restrict__ dirichlet,
                                                             const double *__restrict__ x, double *__restrict__ out,
                                                             const double *__restrict__ a1,
                                                             const double *__restrict__ a2, double *__restrict__ part,
                                                             const SolveState *__restrict__ st)
{
    if (st && st->done) return;
    __shared__ double sh[SOLVE_THREADS / 32];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (SOLVE_THREADS / 32);
    double d1 = 0.0, d2 = 0.0, d3 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * (SOLVE_THREADS / 32) + (threadIdx.x >> 5); i < n; i += warps) {
        const double xi = x[i];
        double acc = 0.0;
        for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) acc = fma(x[col[e]] - xi, wd[e], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double yi = (dirichlet && dirichlet[i]) ? xi : acc;
        if (lane == 0) {
            out[i] = yi;
            if (a1) d1 = fma(a1[i], yi, d1);
            if (a2) d2 = fma(a2[i], yi, d2);
            d3 = fma(yi, yi, d3);
        }
    }
    if (!part) return;
    const double s1 = block_sum(d1, sh);
    const double s2 = block_sum(d2, sh);
    const double s3 = block_sum(d3, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s1;
        part[3 * blockIdx.x + 1] = s2;
        part[3 * blockIdx.x + 2] = s3;
    }
}

// the element-wise updates of one iteration, by phase
//   0: r = b - r (r holds A x on entry), rhat = r, p = v = 0; partials (r, r), (b, b)
//   1: p = r + beta (p - omega v); y = dinv p
//   2: s = r - alpha v; z = dinv s; partial (s, s)
//   3: x += alpha y + omega z; r = s - omega t; partials (rhat, r), (r, r)
__global__ void __launch_bounds__(SOLVE_THREADS) k_solve_vec(int64_t n, int phase, const double *__restrict__ b,
                                                            double *__restrict__ x, double *__restrict__ r,
                                                            double *__restrict__ rhat, double *__restrict__ p,
                                                            double *__restrict__ v, double *__restrict__ y,
                                                            double *__restrict__ s, double *__restrict__ z,
                                                            const double *__restrict__ t,
                                                            const double *__restrict__ dinv,
                                                            double *__restrict__ part, const SolveState *__restrict__ st)
{
    if (phase != 0 && st->done) return;
    __shared__ double sh[SOLVE_THREADS / 32];
    const double alpha = st->alpha, omega = st->omega, beta = st->beta;
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
    const double s1 = block_sum(d1, sh);
    const double s2 = block_sum(d2, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s1;
        part[3 * blockIdx.x + 1] = s2;
        part[3 * blockIdx.x + 2] = 0.0;
    }
}

// one block: sum the partials in a fixed order and form the scalars of the step that follows
//   step 0 (after setup):      rnorm2, bnorm2, rho = rnorm2, alpha = omega = rho_old = 1
//   step 1 (before phase 1):   beta = (rho / rho_old)(alpha / omega)
//   step 2 (after v = A y):    alpha = rho / (rhat, v)
//   step 3 (after phase 2):    snorm2
//   step 4 (after t = A z):    omega = (t, s) / (t, t)
//   step 5 (after phase 3):    rho_old = rho, rho = (rhat, r), rnorm2, iters++, convergence
__global__ void k_solve_scalars(int nblk, int step, const double *__restrict__ part, SolveState *__restrict__ st)
{
    if (step != 0 && st->done) return;
    __shared__ double sh[3][SOLVE_THREADS];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < nblk; k += SOLVE_THREADS) {
        a += part[3 * k];
        b += part[3 * k + 1];
        c += part[3 * k + 2];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int h = SOLVE_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int q = 0; q < 3; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double s0 = sh[0][0], s1 = sh[1][0];
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
    case 1:
        st->beta = (st->rho / st->rho_old) * (st->alpha / st->omega);
        if (!isfinite(st->beta)) st->done = 2;
        break;
    case 2:
        st->alpha = st->rho / s0;
        if (s0 == 0.0 || !isfinite(st->alpha)) st->done = 2;
        break;
    case 3:
        st->snorm2 = s0;
        st->skip = s0 <= st->tol2 ? 1 : 0;
        break;
    case 4: {
        // the partials of t = A z hold (s . t) in slot 0 and (t . t) in slot 2
        const double ts = s0, tt = sh[2][0];
        st->omega = st->skip ? 0.0 : (tt > 0.0 ? ts / tt : 0.0);
        if (!isfinite(st->omega)) st->done = 2;
        break;
    }
    default:
        st->rho_old = st->rho;
        st->rho = s0;
        st->rnorm2 = s1;
        st->iters += 1;
        if (s1 <= st->tol2) st->done = 1;
        else if (st->rho == 0.0 || st->omega == 0.0 || !isfinite(s1)) st->done = 2;
        else if (st->iters >= st->max_iter) st->done = 3;
        break;
    }
}

}  // namespace

labfm_status run_solve(labfm_ctx *ctx, int op, const double *f, double *phi, const uint8_t *dirichlet, double tol,
                       int max_iter, int *iters_out, double *resid_out)
{
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n, nnz = ctx->nnz;
    LABFM_CUDA_TRY(ctx, ctx->sol_w.reserve(sizeof(double) * (nnz > 0 ? nnz : 1)));
    LABFM_CUDA_TRY(ctx, ctx->sol_vec.reserve(sizeof(double) * 9 * n));
    LABFM_CUDA_TRY(ctx, ctx->sol_part.reserve(sizeof(double) * 3 * SOLVE_MAX_BLOCKS + sizeof(SolveState)));
    double *V = ctx->sol_vec.as<double>();
    double *dinv = V, *r = V + n, *rhat = V + 2 * n, *p = V + 3 * n, *v = V + 4 * n, *y = V + 5 * n, *sv = V + 6 * n,
           *z = V + 7 * n, *t = V + 8 * n;
    double *part = ctx->sol_part.as<double>();
    SolveState *st = reinterpret_cast<SolveState *>(part + 3 * SOLVE_MAX_BLOCKS);
    const int nblk_vec = (int)std::min<int64_t>((n + SOLVE_THREADS - 1) / SOLVE_THREADS, SOLVE_MAX_BLOCKS);
    const int nblk_mv = (int)std::min<int64_t>((n + SOLVE_THREADS / 32 - 1) / (SOLVE_THREADS / 32), SOLVE_MAX_BLOCKS);
    {
        const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16);
        if (ctx->wdtype == LABFM_F64)
            k_solve_setup<double><<<blocks, 256, 0, s>>>(n, ctx->row_ptr.as<int64_t>(), ctx->w.as<double>(),
                                                         ctx->n_ops, op, ctx->sol_w.as<double>(), dinv, dirichlet, f,
                                                         phi);
        else
            k_solve_setup<float><<<blocks, 256, 0, s>>>(n, ctx->row_ptr.as<int64_t>(), ctx->w.as<float>(), ctx->n_ops,
                                                        op, ctx->sol_w.as<double>(), dinv, dirichlet, f, phi);
        LABFM_CUDA_TRY(ctx, cudaGetLastError());
    }
    SolveState init{};
    init.tol2 = tol * tol;
    init.skip = 0;
    init.max_iter = max_iter;
    LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(st, &init, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    const int64_t *rp = ctx->row_ptr.as<int64_t>();
    const int32_t *cl = ctx->col.as<int32_t>();
    const double *wd = ctx->sol_w.as<double>();
    auto spmv = [&](const double *x, double *out, const double *a1, const double *a2, const SolveState *gate) {
        k_solve_spmv<<<nblk_mv, SOLVE_THREADS, 0, s>>>(n, rp, cl, wd, dirichlet, x, out, a1, a2, part, gate);
    };
    auto vec = [&](int phase) {
        k_solve_vec<<<nblk_vec, SOLVE_THREADS, 0, s>>>(n, phase, f, phi, r, rhat, p, v, y, sv, z, t, dinv, part, st);
    };
    auto scalars = [&](int nblk, int step) { k_solve_scalars<<<1, SOLVE_THREADS, 0, s>>>(nblk, step, part, st); };
    // r = b - A x, r^ = r
    spmv(phi, r, nullptr, nullptr, nullptr);
    vec(0);
    scalars(nblk_vec, 0);
    LABFM_CUDA_TRY(ctx, cudaGetLastError());
    SolveState h{};
    const int chunk = 16;
    for (int it = 0; it < max_iter; it += chunk) {
        for (int q = 0; q < chunk && it + q < max_iter; q++) {
            scalars(nblk_vec, 1);      // beta (the partials of the previous step are not read)
            vec(1);                    // p, y
            spmv(y, v, rhat, nullptr, st);
            scalars(nblk_mv, 2);       // alpha
            vec(2);                    // s, z
            scalars(nblk_vec, 3);      // ||s||
            spmv(z, t, sv, nullptr, st);
            scalars(nblk_mv, 4);       // omega from (s . t) and (t . t)
            vec(3);                    // x, r
            scalars(nblk_vec, 5);      // rho, ||r||, convergence
        }
        LABFM_CUDA_TRY(ctx, cudaGetLastError());
        LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(&h, st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (h.done) break;
    }
    // the true residual ||b - A x|| / ||b||
    spmv(phi, t, nullptr, nullptr, nullptr);
    LABFM_CUDA_TRY(ctx, cudaGetLastError());
    {
        // reuse phase 0 on scratch copies: r = b - A x into sv, partial (r, r) and (b, b)
        k_solve_vec<<<nblk_vec, SOLVE_THREADS, 0, s>>>(n, 0, f, nullptr, t, sv, z, y, nullptr, nullptr, nullptr,
                                                       nullptr, nullptr, part, st);
        LABFM_CUDA_TRY(ctx, cudaGetLastError());
    }
    std::vector<double> hp(3 * (size_t)nblk_vec);
    LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s));
    LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    double rr = 0.0, bb = 0.0;
    for (int k = 0; k < nblk_vec; k++) {
        rr += hp[3 * k];
        bb += hp[3 * k + 1];
    }
    const double resid = std::sqrt(rr) / (bb > 0.0 ? std::sqrt(bb) : 1.0);
    if (iters_out) *iters_out = h.iters;
    if (resid_out) *resid_out = resid;
    if (h.done == 1 && std::isfinite(resid)) return LABFM_OK;
    return fail(ctx, LABFM_ERR_NOT_CONVERGED,
                h.done == 2 ? "BiCGStab breakdown (rho, alpha or omega vanished or was not finite)"
                            : "BiCGStab did not reach the tolerance within max_iter iterations");
}

}  // namespace labfm
