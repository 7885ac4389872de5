// FP64 weight build (Sec. 3.1-3.2): per node, monomials X and ABFs W of every neighbour,
// M = sum_j X_j (outer) W_j (Eq. disc_form), Gaussian elimination with partial pivoting of
// M Psi = C^d for all operators at once (Eq. lsys), and w_j^d = W_j . Psi^d (Eq. w_abf).
//
// One CTA per node (persistent over a node list).  Neighbour data are staged in shared
// memory in chunks of NB neighbours: Xs[j][m], Ws[j][n] (row stride LDX, a multiple of 4 so
// that a thread's 4 consecutive W values are one 32-byte load).  The p x p assembly is tiled
// 2 x 4 per thread in registers across chunks.  The augmented matrix [M | Chat] (Chat_alpha =
// C_alpha h^-|alpha|) is then eliminated in shared memory, one column per step, in the space of
// the X staging (X is not read again), which keeps a CTA within a quarter of the SM's shared
// memory: four CTAs per SM.
#include <algorithm>
#include <cmath>
#include <vector>

#include "abf.cuh"

namespace labfm {
namespace {

constexpr int BUILD_THREADS = 256;

template <int K> struct Cfg {
    static constexpr int P = p_of_k(K);
    static constexpr int LDX = (P + 3) / 4 * 4;
    static constexpr int NB = K >= 7 ? 72 : 64;
    static constexpr int TM = 2, TN = 4;
    static constexpr int RG = (P + TM - 1) / TM, CG = (P + TN - 1) / TN;
    static_assert(RG * CG <= BUILD_THREADS, "assembly tile grid exceeds the CTA");
    static constexpr int LDA = P + MAX_OPS + 1;  // augmented row stride (odd: fewer bank conflicts)
    // the augmented matrix reuses the X staging (X is not read after the assembly)
    static_assert((size_t)P * LDA <= (size_t)NB * LDX, "augmented matrix fits the X staging");
    static constexpr size_t smem_bytes = sizeof(double) * ((size_t)2 * NB * LDX);
};

struct BuildArgs {
    int64_t n_list;           // nodes in this launch
    const int32_t *list;      // node ids, or null: node = list index
    const double *xy;         // [2n]
    const double *h;          // [n]
    const int64_t *row_ptr;
    const int32_t *col;
    int periodic;
    double L[2], halfL[2];
    int rbf;
    int n_ops;
    void *w;  // [nnz][n_ops]
    int wdtype;
    int32_t *node_status;     // may be null
    unsigned long long *n_bad;
    double C[MAX_OPS * PMAX];  // target vectors, row d = C^d (physical units)
};

// Shared memory of one CTA beyond the X/W staging: the scalars and small arrays of the node being
// built, carved from the dynamic allocation (so that a kernel holding several orders allocates
// them once, not once per order).
struct NodeShared {
    double psi[PMAX * MAX_OPS];  // Psi^d, kept while X and W are staged again
    double invpiv[PMAX];         // 1 / pivot of each column, reused by the back substitution
    double hpow[KMAX + 1];       // h^-n
    double inv;
    int piv;
    int flag;  // bit 0: zero/non-finite pivot, bit 1: non-finite weight, bit 2: non-finite M
};

template <int K> constexpr size_t node_smem_bytes() { return Cfg<K>::smem_bytes + sizeof(NodeShared); }
constexpr size_t max_node_smem_bytes()
{
    return std::max({node_smem_bytes<1>(), node_smem_bytes<2>(), node_smem_bytes<3>(), node_smem_bytes<4>(),
                     node_smem_bytes<5>(), node_smem_bytes<6>(), node_smem_bytes<7>(), node_smem_bytes<8>()});
}

// The whole build of node i at order K by the CTA: stage X and W, assemble M, eliminate
// [M | Chat], weights.  Ends synchronised (the shared memory is reused by the next node).
template <int K>
__device__ __forceinline__ void build_node(const BuildArgs &A, int64_t i, double *smem)
{
    using C = Cfg<K>;
    constexpr int P = C::P, LDX = C::LDX, NB = C::NB, LDA = C::LDA, TM = C::TM, TN = C::TN;
    double *Xs = smem;                 // [NB][LDX]
    double *Ws = Xs + NB * LDX;        // [NB][LDX]
    double *Am = Xs;                   // [P][LDA]  augmented [M | Chat], over the X staging
    NodeShared &sh = *reinterpret_cast<NodeShared *>(Ws + NB * LDX);
    double *s_psi = sh.psi, *s_invpiv = sh.invpiv, *s_hpow = sh.hpow;
    int &s_piv = sh.piv, &s_flag = sh.flag;
    double &s_inv = sh.inv;

    const int tid = threadIdx.x;
    const int n_ops = A.n_ops;
    const int W_ = P + n_ops;  // used columns of the augmented matrix
    const int rg = tid / C::CG, cg = tid % C::CG;
    const bool tile_active = tid < C::RG * C::CG;

    {
        const int64_t rs = A.row_ptr[i], re = A.row_ptr[i + 1];
        const int ni = (int)(re - rs);
        if (ni < P) {
            for (int64_t t = tid; t < (int64_t)ni * n_ops; t += BUILD_THREADS) {
                if (A.wdtype == LABFM_F64) ((double *)A.w)[rs * n_ops + t] = 0.0;
                else ((float *)A.w)[rs * n_ops + t] = 0.0f;
            }
            if (tid == 0) {
                if (A.node_status) A.node_status[i] = LABFM_NODE_UNDERSAMPLED;
                atomicAdd(A.n_bad, 1ull);
            }
            return;
        }
        const double xi = A.xy[2 * i], yi = A.xy[2 * i + 1], hi = A.h[i];
        const double ihi = 1.0 / hi;
        if (tid == 0) {
            double s = 1.0;
            for (int t = 0; t <= K; t++) {
                s_hpow[t] = s;
                s *= ihi;
            }
        }

        double acc[TM][TN];
#pragma unroll
        for (int a = 0; a < TM; a++)
#pragma unroll
            for (int b = 0; b < TN; b++) acc[a][b] = 0.0;

        const int nchunks = (ni + NB - 1) / NB;
        for (int ch = 0; ch < nchunks; ch++) {
            const int j0 = ch * NB;
            const int nj = min(NB, ni - j0);
            for (int t = tid; t < nj; t += BUILD_THREADS) {
                int j = A.col[rs + j0 + t];
                double dx = A.xy[2 * (int64_t)j] - xi, dy = A.xy[2 * (int64_t)j + 1] - yi;
                if (A.periodic) {
                    if (dx > A.halfL[0]) dx -= A.L[0];
                    else if (dx < -A.halfL[0]) dx += A.L[0];
                    if (dy > A.halfL[1]) dy -= A.L[1];
                    else if (dy < -A.halfL[1]) dy += A.L[1];
                }
                double *X = Xs + t * LDX, *W = Ws + t * LDX;
                eval_xw<K>(dx * ihi, dy * ihi, A.rbf, X, W);
#pragma unroll
                for (int e = P; e < LDX; e++) X[e] = W[e] = 0.0;
            }
            __syncthreads();
            if (tile_active) {
                for (int j = 0; j < nj; j++) {
                    const double *X = Xs + j * LDX + rg * TM;
                    const double *W = Ws + j * LDX + cg * TN;
                    double xv[TM], wv[TN];
#pragma unroll
                    for (int a = 0; a < TM; a++) xv[a] = X[a];
                    double2 w01 = *reinterpret_cast<const double2 *>(W);
                    double2 w23 = *reinterpret_cast<const double2 *>(W + 2);
                    wv[0] = w01.x;
                    wv[1] = w01.y;
                    wv[2] = w23.x;
                    wv[3] = w23.y;
#pragma unroll
                    for (int a = 0; a < TM; a++)
#pragma unroll
                        for (int b = 0; b < TN; b++) acc[a][b] = fma(xv[a], wv[b], acc[a][b]);
                }
            }
            if (ch + 1 < nchunks) __syncthreads();
        }
        // M into the augmented matrix, scaled targets into its right-hand columns
        if (tid == 0) s_flag = 0;
        __syncthreads();
        if (tile_active) {
            bool finite = true;
#pragma unroll
            for (int a = 0; a < TM; a++)
#pragma unroll
                for (int b = 0; b < TN; b++) {
                    int m = rg * TM + a, c = cg * TN + b;
                    if (m < P && c < P) {
                        Am[m * LDA + c] = acc[a][b];
                        finite &= isfinite(acc[a][b]);
                    }
                }
            // a non-finite entry of M (a neighbour on top of node i: singular ABFs)
            if (!finite) atomicOr(&s_flag, 4);
        }
        for (int t = tid; t < P * n_ops; t += BUILD_THREADS) {
            int m = t / n_ops, d = t % n_ops;
            Am[m * LDA + P + d] = A.C[d * PMAX + m] * s_hpow[elem_degree(m)];
        }
        __syncthreads();
        const bool bad_m = (s_flag & 4) != 0;

        // Gaussian elimination with partial pivoting (first largest |pivot| wins)
        for (int c = 0; c < P && !bad_m; c++) {
            if (tid < 32) {
                double best = -1.0;
                int br = c;
                for (int r = c + tid; r < P; r += 32) {
                    double v = fabs(Am[r * LDA + c]);
                    if (v > best) {
                        best = v;
                        br = r;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    double ob = __shfl_xor_sync(0xffffffffu, best, o);
                    int orr = __shfl_xor_sync(0xffffffffu, br, o);
                    if (ob > best || (ob == best && orr < br)) {
                        best = ob;
                        br = orr;
                    }
                }
                if (tid == 0) {
                    s_piv = br;
                    double pv = Am[br * LDA + c];
                    if (!(best > 0.0) || !isfinite(best)) {
                        s_flag |= 1;
                        s_inv = 0.0;
                    } else {
                        s_inv = 1.0 / pv;
                    }
                    s_invpiv[c] = s_inv;
                }
            }
            __syncthreads();
            const int pr = s_piv;
            if (pr != c) {
                for (int t = c + tid; t < W_; t += BUILD_THREADS) {
                    double a = Am[c * LDA + t];
                    Am[c * LDA + t] = Am[pr * LDA + t];
                    Am[pr * LDA + t] = a;
                }
                __syncthreads();
            }
            const double inv = s_inv;
            for (int r = c + 1 + tid; r < P; r += BUILD_THREADS) Am[r * LDA + c] *= inv;
            __syncthreads();
            const int nr = P - c - 1, nc = W_ - c - 1;
            for (int t = tid; t < nr * nc; t += BUILD_THREADS) {
                int r = c + 1 + t / nc, q = c + 1 + t % nc;
                Am[r * LDA + q] = fma(-Am[r * LDA + c], Am[c * LDA + q], Am[r * LDA + q]);
            }
            __syncthreads();
        }
        // back substitution on the n_ops right-hand sides
        for (int c = P - 1; c >= 0 && !bad_m; c--) {
            if (tid < n_ops) Am[c * LDA + P + tid] *= s_invpiv[c];
            __syncthreads();
            for (int t = tid; t < c * n_ops; t += BUILD_THREADS) {
                int r = t / n_ops, d = t % n_ops;
                Am[r * LDA + P + d] = fma(-Am[r * LDA + c], Am[c * LDA + P + d], Am[r * LDA + P + d]);
            }
            __syncthreads();
        }
        const bool singular = (s_flag & 5) != 0;  // no weights from a failed elimination
        for (int t = tid; t < P * n_ops; t += BUILD_THREADS) {
            const int m = t / n_ops, d = t - m * n_ops;
            s_psi[m * MAX_OPS + d] = Am[m * LDA + P + d];
        }
        __syncthreads();

        // weights w_j^d = W_j . Psi^d
        for (int ch = 0; ch < nchunks; ch++) {
            const int j0 = ch * NB;
            const int nj = min(NB, ni - j0);
            if (nchunks > 1) {  // the staged W of earlier chunks were overwritten: recompute
                __syncthreads();
                for (int t = tid; t < nj; t += BUILD_THREADS) {
                    int j = A.col[rs + j0 + t];
                    double dx = A.xy[2 * (int64_t)j] - xi, dy = A.xy[2 * (int64_t)j + 1] - yi;
                    if (A.periodic) {
                        if (dx > A.halfL[0]) dx -= A.L[0];
                        else if (dx < -A.halfL[0]) dx += A.L[0];
                        if (dy > A.halfL[1]) dy -= A.L[1];
                        else if (dy < -A.halfL[1]) dy += A.L[1];
                    }
                    eval_xw<K>(dx * ihi, dy * ihi, A.rbf, Xs + t * LDX, Ws + t * LDX);
                }
                __syncthreads();
            }
            for (int t = tid; t < nj * n_ops; t += BUILD_THREADS) {
                int j = t / n_ops, d = t % n_ops;
                double s = 0.0;
                if (!singular) {
                    const double *W = Ws + j * LDX;
#pragma unroll 4
                    for (int m = 0; m < P; m++) s = fma(W[m], s_psi[m * MAX_OPS + d], s);
                    if (!isfinite(s)) {
                        atomicOr(&s_flag, 2);
                        s = 0.0;
                    }
                }
                int64_t idx = (rs + j0 + j) * n_ops + d;
                if (A.wdtype == LABFM_F64) ((double *)A.w)[idx] = s;
                else ((float *)A.w)[idx] = (float)s;
            }
        }
        __syncthreads();
        const int flag = s_flag;
        if (flag & 2) {  // a weight was not finite: the whole node is zeroed
            for (int64_t t = tid; t < (int64_t)ni * n_ops; t += BUILD_THREADS) {
                if (A.wdtype == LABFM_F64) ((double *)A.w)[rs * n_ops + t] = 0.0;
                else ((float *)A.w)[rs * n_ops + t] = 0.0f;
            }
        }
        if (tid == 0) {
            int st = (flag & 4)   ? LABFM_NODE_NONFINITE
                     : (flag & 1) ? LABFM_NODE_SINGULAR
                     : (flag & 2) ? LABFM_NODE_NONFINITE
                                  : LABFM_NODE_OK;
            if (A.node_status) A.node_status[i] = st;
            if (st != LABFM_NODE_OK) atomicAdd(A.n_bad, 1ull);
        }
        __syncthreads();  // shared state is reused by the next node
    }
}

// One order for all listed nodes (persistent over the list).
template <int K>
__global__ void __launch_bounds__(BUILD_THREADS, 4) k_build_fp64(BuildArgs A)
{
    extern __shared__ __align__(16) double smem[];
    for (int64_t li = blockIdx.x; li < A.n_list; li += gridDim.x)
        build_node<K>(A, A.list ? (int64_t)A.list[li] : li, smem);
}

// Every order in one persistent launch (per-node order, Sec. 4.1 walls and variable resolution):
// the list holds the nodes by ascending order, and CTAs take them from the end, so that the
// costliest nodes go first and the cheap ones fill the tail.
__global__ void __launch_bounds__(BUILD_THREADS, 4) k_build_fp64_orders(BuildArgs A, const int8_t *__restrict__ order)
{
    extern __shared__ __align__(16) double smem[];
    for (int64_t li = blockIdx.x; li < A.n_list; li += gridDim.x) {
        const int64_t i = A.list[A.n_list - 1 - li];
        switch (order[i]) {
        case 1: build_node<1>(A, i, smem); break;
        case 2: build_node<2>(A, i, smem); break;
        case 3: build_node<3>(A, i, smem); break;
        case 4: build_node<4>(A, i, smem); break;
        case 5: build_node<5>(A, i, smem); break;
        case 6: build_node<6>(A, i, smem); break;
        case 7: build_node<7>(A, i, smem); break;
        default: build_node<8>(A, i, smem); break;
        }
    }
}

template <int K>
static cudaError_t launch_k(const BuildArgs &a, int num_sms, cudaStream_t s)
{
    using C = Cfg<K>;
    constexpr size_t smem = node_smem_bytes<K>();
    cudaError_t e = cudaFuncSetAttribute(k_build_fp64<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_fp64<K>, BUILD_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = std::min<int64_t>(a.n_list, (int64_t)num_sms * per_sm);
    if (grid < 1) return cudaSuccess;
    k_build_fp64<K><<<(unsigned)grid, BUILD_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_all_orders(const BuildArgs &a, const int8_t *order, int num_sms, cudaStream_t s)
{
    constexpr size_t smem = max_node_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_build_fp64_orders, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_fp64_orders, BUILD_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = std::min<int64_t>(a.n_list, (int64_t)num_sms * per_sm);
    if (grid < 1) return cudaSuccess;
    k_build_fp64_orders<<<(unsigned)grid, BUILD_THREADS, smem, s>>>(a, order);
    return cudaGetLastError();
}

static cudaError_t launch_order(int k, const BuildArgs &a, int num_sms, cudaStream_t s)
{
    switch (k) {
    case 1: return launch_k<1>(a, num_sms, s);
    case 2: return launch_k<2>(a, num_sms, s);
    case 3: return launch_k<3>(a, num_sms, s);
    case 4: return launch_k<4>(a, num_sms, s);
    case 5: return launch_k<5>(a, num_sms, s);
    case 6: return launch_k<6>(a, num_sms, s);
    case 7: return launch_k<7>(a, num_sms, s);
    default: return launch_k<8>(a, num_sms, s);
    }
}

// Bucket nodes by order: counts per order, then a stable list of node ids per order.
__global__ void k_order_count(int64_t n, const int8_t *__restrict__ order, unsigned long long *__restrict__ cnt,
                              unsigned long long *__restrict__ bad)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = order[i];
    if (k < 1 || k > KMAX) {
        atomicAdd(bad, 1ull);
        return;
    }
    atomicAdd(&cnt[k], 1ull);
}

__global__ void k_order_scatter(int64_t n, const int8_t *__restrict__ order, const unsigned long long *__restrict__ base,
                                unsigned long long *__restrict__ cursor, int32_t *__restrict__ list)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = order[i];
    if (k < 1 || k > KMAX) return;
    unsigned long long pos = base[k] + atomicAdd(&cursor[k], 1ull);
    list[pos] = (int32_t)i;
}

}  // namespace

// Refinement steps of a mixed build: LABFM_PREC_MIXED[_TC]_REFINE(n) fixes n; otherwise each
// node refines until it converges (at most NREF_ADAPTIVE steps; one for most nodes).
constexpr int NREF_ADAPTIVE = 6;
static int precision_nref(int precision, bool &adaptive)
{
    int forced = (precision >> 8) & 0xf;  // LABFM_PREC_MIXED_REFINE(n) stores n + 1 here
    adaptive = forced == 0;
    return forced ? forced - 1 : NREF_ADAPTIVE;
}

labfm_status run_build(labfm_ctx *ctx, const int8_t *order, int uniform_order, int rbf, int n_ops, const double *Cin,
                       int precision, int weight_dtype, int32_t *node_status, int64_t *n_bad_out)
{
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n;
    const int base_prec = precision & 0xff;
    const bool mixed = base_prec == LABFM_PREC_MIXED || base_prec == LABFM_PREC_MIXED_TC;
    size_t wbytes = (size_t)ctx->nnz * n_ops * (weight_dtype == LABFM_F64 ? 8 : 4);
    LABFM_CUDA_TRY(ctx, ctx->w.reserve(wbytes > 0 ? wbytes : 8));
    if (mixed) LABFM_CUDA_TRY(ctx, ctx->wtilde.reserve((size_t)ctx->nnz * n_ops * 8 + 8));
    LABFM_CUDA_TRY(ctx, ctx->misc.reserve(4096));
    unsigned long long *dmisc = ctx->misc.as<unsigned long long>();
    // misc layout: [0] bad nodes, [1] bad orders, [2..10] order counts, [11..19] bases, [20..28] cursors,
    // [30] tensor-core waits that gave up, [31] nodes handed to the FP64 build, [32..39] nodes by
    // refinement steps
    constexpr int NMISC = 40;
    LABFM_CUDA_TRY(ctx, cudaMemsetAsync(dmisc, 0, NMISC * sizeof(unsigned long long), s));
    for (int t = 0; t < 8; t++) ctx->info_ref_hist[t] = 0;
    ctx->info_fp64_rebuilt = 0;

    BuildArgs a{};
    a.xy = ctx->node_xy.as<double>();
    a.h = ctx->node_h.as<double>();
    a.row_ptr = ctx->row_ptr.as<int64_t>();
    a.col = ctx->col.as<int32_t>();
    a.periodic = ctx->periodic;
    for (int d = 0; d < 2; d++) {
        a.L[d] = ctx->hi[d] - ctx->lo[d];
        a.halfL[d] = 0.5 * a.L[d];
    }
    a.rbf = rbf;
    a.n_ops = n_ops;
    a.w = ctx->w.ptr;
    a.wdtype = weight_dtype;
    a.node_status = node_status;
    a.n_bad = dmisc;
    for (int t = 0; t < n_ops * PMAX; t++) a.C[t] = Cin[t];

    MixedArgsPublic m{};
    if (mixed) {
        m.xy = a.xy;
        m.h = a.h;
        m.row_ptr = a.row_ptr;
        m.col = a.col;
        m.periodic = a.periodic;
        for (int d = 0; d < 2; d++) {
            m.L[d] = a.L[d];
            m.halfL[d] = a.halfL[d];
        }
        m.rbf = rbf;
        m.n_ops = n_ops;
        m.w = a.w;
        m.wdtype = weight_dtype;
        m.wt = ctx->wtilde.as<double>();
        m.node_status = node_status;
        m.n_bad = dmisc;
        m.num_sms = ctx->num_sms;
        m.tc = base_prec == LABFM_PREC_MIXED_TC;
        m.tc_timeout = dmisc + 30;
        m.fb_count = dmisc + 31;
        m.ref_hist = dmisc + 32;
        LABFM_CUDA_TRY(ctx, ctx->mfallback.reserve(sizeof(int32_t) * (n > 0 ? n : 1)));
        m.fb_list = ctx->mfallback.as<int32_t>();
        for (int t = 0; t < n_ops * PMAX; t++) m.C[t] = Cin[t];
        for (int d = 0; d < n_ops; d++) {
            int l = 0;
            for (int e = 0; e < PMAX; e++)
                if (Cin[d * PMAX + e] != 0.0) l = std::max(l, (int)elem_degree(e));
            m.lmax[d] = l;
        }
    }
    auto launch = [&](int k, const int32_t *list, int64_t n_list) -> cudaError_t {
        if (!mixed) {
            a.list = list;
            a.n_list = n_list;
            return launch_order(k, a, ctx->num_sms, s);
        }
        m.list = list;
        m.n_list = n_list;
        bool adaptive = false;
        m.nref = precision_nref(precision, adaptive);
        m.adaptive = adaptive ? 1 : 0;
        // per-node matrices of one batch: at most 2^18 nodes (4.2 GB at k = 8)
        m.batch_nodes = std::max<int64_t>(1, std::min<int64_t>(n_list, (int64_t)1 << 18));
        cudaError_t e = ctx->mscratch.reserve(mixed_scratch_bytes_per_node(k) * (size_t)m.batch_nodes + 256);
        if (e != cudaSuccess) return e;
        m.scratch = ctx->mscratch.ptr;
        e = ctx->mrecs.reserve(mixed_record_bytes() * (size_t)ctx->nnz + 256);
        if (e != cudaSuccess) return e;
        m.recs = ctx->mrecs.ptr;
        // W of every entry, kept from the assembly for the weights kernel (8 bytes per element);
        // above 24 GB the weights kernel evaluates W again instead
        const size_t wbytes_k = (size_t)8 * p_of_k(k) * (size_t)ctx->nnz;
        m.wstore = nullptr;
        if (wbytes_k <= ((size_t)24 << 30) && ctx->mwstore.reserve(wbytes_k + 256) == cudaSuccess)
            m.wstore = ctx->mwstore.ptr;
        else
            cudaGetLastError();  // a failed reservation only disables the store
        return launch_build_mixed(k, m, s);
    };

    unsigned long long *hs = (unsigned long long *)ctx->host_small;
    if (!order) {
        LABFM_CUDA_TRY(ctx, launch(uniform_order, nullptr, n));
    } else {
        int nb = (int)((n + 255) / 256);
        k_order_count<<<nb, 256, 0, s>>>(n, order, dmisc + 2, dmisc + 1);
        LABFM_CUDA_TRY(ctx, cudaGetLastError());
        LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(hs, dmisc, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (hs[1] != 0) return fail(ctx, LABFM_ERR_ARG, "order[] has entries outside 1..8");
        unsigned long long cnt[KMAX + 1], base[KMAX + 1];
        unsigned long long acc = 0;
        for (int k = 0; k <= KMAX; k++) {
            cnt[k] = hs[2 + k];
            base[k] = acc;
            acc += cnt[k];
        }
        LABFM_CUDA_TRY(ctx, ctx->status_tmp.reserve(sizeof(int32_t) * (n > 0 ? n : 1)));
        int32_t *list = ctx->status_tmp.as<int32_t>();
        for (int k = 0; k <= KMAX; k++) hs[k] = base[k];
        LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(dmisc + 11, hs, sizeof(base), cudaMemcpyHostToDevice, s));
        k_order_scatter<<<nb, 256, 0, s>>>(n, order, dmisc + 11, dmisc + 20, list);
        LABFM_CUDA_TRY(ctx, cudaGetLastError());
        if (!mixed) {
            // every order in one persistent launch over the whole (ascending-order) list
            a.list = list;
            a.n_list = (int64_t)acc;
            LABFM_CUDA_TRY(ctx, launch_all_orders(a, order, ctx->num_sms, s));
        } else {
            for (int k = KMAX; k >= 1; k--) {
                if (!cnt[k]) continue;
                LABFM_CUDA_TRY(ctx, launch(k, list + base[k], (int64_t)cnt[k]));
            }
        }
    }
    LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(hs, dmisc, NMISC * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hs[30]) return fail(ctx, LABFM_ERR_TIMEOUT, "a tensor-core completion wait gave up");
    if (mixed && hs[31]) {
        // nodes whose refinement diverged (the double-float inverse too inaccurate for the
        // iteration to contract): the FP64 build writes their weights and statuses
        const int64_t nfb = (int64_t)hs[31];
        ctx->info_fp64_rebuilt = nfb;
        a.list = ctx->mfallback.as<int32_t>();
        a.n_list = nfb;
        if (!order) LABFM_CUDA_TRY(ctx, launch_order(uniform_order, a, ctx->num_sms, s));
        else LABFM_CUDA_TRY(ctx, launch_all_orders(a, order, ctx->num_sms, s));
        LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(hs, dmisc, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    if (mixed)
        for (int t = 0; t < 8; t++) ctx->info_ref_hist[t] = (int64_t)hs[32 + t];
    int64_t nbad = (int64_t)hs[0];
    if (n_bad_out) *n_bad_out = nbad;
    if (nbad) return fail(ctx, LABFM_ERR_SINGULAR, std::to_string(nbad) + " node(s) flagged");
    return LABFM_OK;
}

}  // namespace labfm
