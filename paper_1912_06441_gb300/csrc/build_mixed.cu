// Mixed-precision weight build.  Same method as build_fp64.cu (Eqs. disc_form, lsys, w_abf),
// with the arithmetic placed where GB300 has throughput: its FP32 pipes issue ~64x the FP64
// rate, so the bulk runs in double-float (pairs of FP32, ~48 bits; df64.cuh) and FP64 is kept
// for the polynomial-reproduction residual.  Three kernels per batch of nodes, handing off
// through global scratch:
//   A  k_mixed_assemble (CTA per node): X and W of every neighbour in double-float, then
//      M = sum_j X_j (outer) W_j in double-float register tiles  -> M (global).
//   B  k_mixed_invert (two threads per row, the matrix in shared memory): Gauss-Jordan
//      inversion of M with partial pivoting (interchanges undone on the columns) -> M^-1.
//   C  k_mixed_weights (CTA per node): Psi~ = M^-1 C~, w~ = W . Psi~, then refinement steps on
//      the residual of the moment conditions of Sec. 3.1
//          r = C~ - sum_j X_j w~_j   (FP64)        w~ <- w~ + W . (M^-1 r)
//      and the physical weights w = h^-l_d w~.  A fixed number of steps when the caller forces
//      one; by default each node refines until its weights stop changing (adaptive: see
//      refine_decision), and a node whose corrections grow instead is handed to the FP64 build.
// Targets are scaled per operator d by h^(l_d - |alpha|), l_d = highest degree with a non-zero
// entry of C^d, so that Psi~ stays within float range; w = h^-l_d w~ is the same similarity
// transform as the FP64 build (exact in exact arithmetic).
#include <cmath>

#include <cuda_bf16.h>

#include "abf.cuh"
#include "df64.cuh"

namespace labfm {
namespace {

constexpr int MIX_THREADS = 256;
static_assert(MIX_THREADS / 32 >= MAX_OPS, "a warp per operator in the weights kernel's sums");
constexpr int PARTS = 3;            // threads per neighbour in the X/W evaluation
constexpr int NREC = 8;             // per-neighbour record: q, 1/q, u, v, W0', W0'', W0'''

template <int K> struct MCfg {
    static constexpr int P = p_of_k(K);
    static constexpr int TM = 2, TN = 4;
    static constexpr int RG = (P + TM - 1) / TM, CG = (P + TN - 1) / TN;
    // row stride (df) of the per-neighbour arrays: odd, so that the 8-byte accesses of consecutive
    // neighbours (threads) fall on distinct bank pairs, and wide enough for the tile's columns
    static constexpr int LDX = (CG * TN > P ? CG * TN : P) | 1;
    static constexpr int NB = K >= 7 ? 72 : 64;
    static_assert(NB * PARTS <= MIX_THREADS, "one evaluation pass per chunk");
    static_assert(RG * CG <= MIX_THREADS, "assembly tile grid exceeds the CTA");
    static_assert(CG * TN <= LDX, "the tile's interleaved columns stay within a staged row");
    // kernel A: Xf, Wf (df) + neighbour records
    static constexpr size_t smemA = 8 * ((size_t)2 * NB * LDX + (size_t)NB * NREC);
    // kernel C: Xd (double), Wf (df), records, Psi/rhs (df), the chunk's w~ (double) and its
    // last corrections (float); M^-1 is read from global memory (through L1), which keeps three
    // CTAs per SM
    static constexpr size_t smemC = 8 * ((size_t)2 * NB * LDX + (size_t)NB * NREC + (size_t)2 * P * MAX_OPS +
                                         (size_t)NB * MAX_OPS) + 4 * (size_t)NB * MAX_OPS;
};

struct DfTables {
    df invfact2[KMAX + 1][KMAX + 1];  // 1 / (a! b!) as a double-float
    float rpoly[PMAX][KMAX + 1];      // the |r|-derivative polynomials (integers, exact in float)
};

constexpr DfTables make_df_tables()
{
    DfTables T{};
    const RPolyTable R = make_rpoly_table();
    for (int e = 0; e < PMAX; e++)
        for (int t = 0; t <= KMAX; t++) T.rpoly[e][t] = static_cast<float>(R.c[e][t]);
    double f[KMAX + 1] = {1, 1, 2, 6, 24, 120, 720, 5040, 40320};
    for (int a = 0; a <= KMAX; a++)
        for (int b = 0; b <= KMAX; b++) {
            double x = 1.0 / (f[a] * f[b]);
            float h = static_cast<float>(x);
            float l = static_cast<float>(x - static_cast<double>(h));
            T.invfact2[a][b] = df{h, l};
        }
    return T;
}

__constant__ DfTables c_dft = make_df_tables();

struct Rec;

struct MixedArgs {
    int64_t n_list;       // nodes in this batch
    const int32_t *list;  // node ids, or null: node = list index + list_base
    int64_t list_base;
    const double *xy;
    const double *h;
    const int64_t *row_ptr;
    const int32_t *col;
    int periodic;
    double L[2], halfL[2];
    int rbf;
    int n_ops;
    int nref;           // refinement steps: exactly this many, or at most this many when adaptive
    int adaptive;       // 1: per-node stopping rule (refine_decision)
    int32_t *fb_list;   // nodes whose refinement diverged, for the FP64 build (adaptive only)
    unsigned long long *fb_count;
    unsigned long long *ref_hist;  // [NREF_MAX + 1] nodes by number of refinement steps taken
    void *w;            // [nnz][n_ops] output
    int wdtype;
    double *wt;         // [nnz][n_ops] scratch: unscaled weights w~ in double
    df *Mg;             // [n_list][mstride] scratch: M (row-major), then M^-1 (column-major)
    int64_t mstride;    // elements per node in Mg (p^2)
    int *flag;          // [n_list] scratch: per-node failure bits
    Rec *recs;          // [nnz] per-entry preamble (k_mixed_records)
    df *wstore;         // [nnz][wstride] W of every entry in double-float, written by the assembly
                        // and read by the weights kernel; null: the weights kernel evaluates W again
    int64_t wstride;    // elements per entry in wstore (p)
    unsigned long long *tc_timeout;  // tensor-core assembly: waits that gave up
    int32_t *node_status;
    unsigned long long *n_bad;
    int lmax[MAX_OPS];
    double C[MAX_OPS * PMAX];
};

__device__ __forceinline__ int64_t node_of(const MixedArgs &A, int64_t li)
{
    return A.list ? (int64_t)A.list[li] : A.list_base + li;
}

// Degrees handled by evaluation part `part` of NP (each part carries a similar (n+1)^2 workload):
// NP = 3: part 0: 8, 3, 1   part 1: 7, 4, 2   part 2: 6, 5
// NP = 4: part 0: 8, 1      part 1: 7, 2      part 2: 6, 3      part 3: 5, 4
template <int NP>
__device__ __forceinline__ bool part_has_degree(int part, int n)
{
    static_assert(NP == 3 || NP == 4, "three or four parts");
    if (NP == 3) {
        switch (part) {
        case 0: return n == 8 || n == 3 || n == 1;
        case 1: return n == 7 || n == 4 || n == 2;
        default: return n == 6 || n == 5;
        }
    }
    switch (part) {
    case 0: return n == 8 || n == 1;
    case 1: return n == 7 || n == 2;
    case 2: return n == 6 || n == 3;
    default: return n == 5 || n == 4;
    }
}

// X (when Xf != null) and W in double-float for the degrees of `part` of one neighbour, from
// its record (polar form q, (u, v) as in abf.cuh's eval_xw).
template <int K, int NP>
__device__ __forceinline__ void eval_xw_part(const df *__restrict__ rec, int part, df *__restrict__ Xf,
                                             df *__restrict__ Wf)
{
    const df q = rec[0], iq = rec[1], u = rec[2], v = rec[3], d1 = rec[4], d2 = rec[5], d3 = rec[6];
    df up[K + 1], vp[K + 1];
    up[0] = vp[0] = df{1.0f, 0.0f};
#pragma unroll
    for (int t = 1; t <= K; t++) {
        up[t] = df_mul(up[t - 1], u);
        vp[t] = df_mul(vp[t - 1], v);
    }
    df qn = df{1.0f, 0.0f}, iqn = df{1.0f, 0.0f};
#pragma unroll
    for (int n = 1; n <= K; n++) {
        if (n > 1) {
            qn = df_mul(qn, q);
            iqn = df_mul(iqn, iq);
        } else {
            qn = q;
        }
        if (!part_has_degree<NP>(part, n)) continue;
        // d^alpha|r| = P_alpha(u, v) q^(1-n): with gn = W0'(q) / q^(n-1) the dW0/dr term is P gn
        const df gn = df_mul(d1, iqn);
        df mono[K + 1];
#pragma unroll
        for (int t = 0; t <= n; t++) mono[t] = df_mul(up[t], vp[n - t]);
        // second derivatives of |r| for the chain rule of the degree-3 elements
        df rxx = df{0.0f, 0.0f}, rxy = rxx, ryy = rxx;
        if (n == 3) {
            rxx = df_mul(vp[2], iq);
            rxy = df_neg(df_mul(df_mul(u, v), iq));
            ryy = df_mul(up[2], iq);
        }
#pragma unroll
        for (int a = n; a >= 0; a--) {
            const int b = n - a;
            const int e = p_of_k(n - 1) + b;
            if (Xf) Xf[e] = df_mul(df_mul(qn, mono[a]), c_dft.invfact2[a][b]);
            // P_alpha(u, v) = sum_t c_t u^t v^(n-t) with integer c_t (exact floats): each product
            // c m is split exactly (TwoProduct), the high parts summed with TwoSum and the low
            // parts and sum errors collected in one float, renormalised once at the end
            float sh = 0.0f, sl = 0.0f;
#pragma unroll
            for (int t = a & 1; t <= n; t += 2) {  // P_alpha has only the terms of a's parity
                const float c = c_dft.rpoly[e][t];
                if (c != 0.0f) {
                    const float ph = __fmul_rn(c, mono[t].hi);
                    float pl = __fmaf_rn(c, mono[t].hi, -ph);
                    pl = __fmaf_rn(c, mono[t].lo, pl);
                    float s2, err;
                    two_sum(sh, ph, s2, err);
                    sh = s2;
                    sl = __fadd_rn(sl, __fadd_rn(err, pl));
                }
            }
            df s;
            two_sum(sh, sl, s.hi, s.lo);  // |sl| may exceed |sh| when P_alpha nearly vanishes
            df wv = df_mul(s, gn);
            // chain rule for |alpha| <= 3 (all radial derivatives), W0' only for |alpha| >= 4 (Appendix A)
            if (n == 2) {
                wv = df_fma(d2, a == 2 ? up[2] : (a == 1 ? df_mul(u, v) : vp[2]), wv);
            } else if (n == 3) {
                if (a == 3) wv = df_fma(d3, up[3], df_fma(d2, df_mul(df{3.0f, 0.0f}, df_mul(u, rxx)), wv));
                if (a == 2)
                    wv = df_fma(d3, df_mul(up[2], v),
                                df_fma(d2, df_add(df_mul(v, rxx), df_mul(df{2.0f, 0.0f}, df_mul(u, rxy))), wv));
                if (a == 1)
                    wv = df_fma(d3, df_mul(u, vp[2]),
                                df_fma(d2, df_add(df_mul(u, ryy), df_mul(df{2.0f, 0.0f}, df_mul(v, rxy))), wv));
                if (a == 0) wv = df_fma(d3, vp[3], df_fma(d2, df_mul(df{3.0f, 0.0f}, df_mul(v, ryy)), wv));
            }
            Wf[e] = wv;
        }
    }
}

// FP64 preamble of one stencil entry, converted once to double-float (kernel k_mixed_records):
// the scaled offset (x, y) in double, and q, 1/q, u, v and the first three radial derivatives
// of W0 in double-float.
struct Rec {
    double x, y;
    df v[7];
};
static_assert(sizeof(Rec) == 72, "record layout");

// One warp per node: every stencil entry's preamble (the only FP64 work of the X/W evaluation).
__global__ void __launch_bounds__(256) k_mixed_records(MixedArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    Rec *recs = A.recs;
    for (int64_t li = wg; li < A.n_list; li += nw) {
        const int64_t i = A.list ? (int64_t)A.list[li] : A.list_base + li;
        const int64_t rs = A.row_ptr[i], re = A.row_ptr[i + 1];
        const double xi = A.xy[2 * i], yi = A.xy[2 * i + 1];
        const double ihi = 1.0 / A.h[i];
        for (int64_t e = rs + lane; e < re; e += 32) {
            const int j = A.col[e];
            double dx = A.xy[2 * (int64_t)j] - xi, dy = A.xy[2 * (int64_t)j + 1] - yi;
            if (A.periodic) {
                if (dx > A.halfL[0]) dx -= A.L[0];
                else if (dx < -A.halfL[0]) dx += A.L[0];
                if (dy > A.halfL[1]) dy -= A.L[1];
                else if (dy < -A.halfL[1]) dy += A.L[1];
            }
            const double x = dx * ihi, y = dy * ihi;
            const double qd = sqrt(x * x + y * y);
            const double iqd = 1.0 / qd;
            double d1, d2, d3;
            rbf_derivs(A.rbf, qd, d1, d2, d3);
            Rec r;
            r.x = x;
            r.y = y;
            r.v[0] = df_from_double(qd);
            r.v[1] = df_from_double(iqd);
            r.v[2] = df_from_double(x * iqd);
            r.v[3] = df_from_double(y * iqd);
            r.v[4] = df_from_double(d1);
            r.v[5] = df_from_double(d2);
            r.v[6] = df_from_double(d3);
            recs[e] = r;
        }
    }
}

// Stage neighbours j0 .. j0+nj-1 of node i from their records: X in FP64 (when Xd != null, one
// thread per neighbour), then X (when Xf != null) and W in double-float (PARTS threads per
// neighbour, a warp on one part).  Ends synchronised.
template <int K>
__device__ __forceinline__ void stage_chunk(const MixedArgs &A, int64_t rs, int j0, int nj, double *Xd, df *Xf,
                                            df *Wf, df *Nrec)
{
    using C = MCfg<K>;
    constexpr int P = C::P, LDX = C::LDX;
    static_assert(LDX - P >= 0, "padding");
    // records -> shared memory (coalesced: an entry's 72 bytes as nine 8-byte words)
    const double *src = reinterpret_cast<const double *>(A.recs + rs + j0);
    for (int t = threadIdx.x; t < nj * 9; t += MIX_THREADS) {
        const int jj = t / 9, w = t - jj * 9;
        if (w >= 2) reinterpret_cast<double *>(Nrec + jj * NREC)[w - 2] = src[t];
    }
    __syncthreads();
    if (Xd) {
        for (int t = threadIdx.x; t < nj; t += MIX_THREADS) {
            const double x = src[t * 9], y = src[t * 9 + 1];
            // x^a / a! and y^b / b!: one FP64 multiply per element of X
            double xs[K + 1], ys[K + 1], xp = 1.0, yp = 1.0;
            xs[0] = ys[0] = 1.0;
#pragma unroll
            for (int q = 1; q <= K; q++) {
                xp *= x;
                yp *= y;
                xs[q] = xp * c_invfact2.v[q][0];
                ys[q] = yp * c_invfact2.v[q][0];
            }
            double *X = Xd + t * LDX;
#pragma unroll
            for (int e = 0; e < P; e++) {
                const int a = elem_a(e), b = elem_degree(e) - a;
                X[e] = xs[a] * ys[b];
            }
#pragma unroll
            for (int e = P; e < LDX; e++) X[e] = 0.0;
        }
    }
    if (A.wstore && !Xf) {
        // W as the assembly stored it (coalesced: consecutive threads, consecutive elements)
        const df *ws = A.wstore + (rs + j0) * A.wstride;
        for (int t = threadIdx.x; t < nj * P; t += MIX_THREADS) {
            const int jj = t / P, e = t - jj * P;
            Wf[jj * LDX + e] = ws[jj * A.wstride + e];
        }
    } else {
        for (int t = threadIdx.x; t < nj * PARTS; t += MIX_THREADS) {
            const int part = t / nj, jj = t - part * nj;
            eval_xw_part<K, PARTS>(Nrec + jj * NREC, part, Xf ? Xf + jj * LDX : nullptr, Wf + jj * LDX);
        }
    }
    // the padding columns the tiles read
    if constexpr (LDX > P) {
        for (int t = threadIdx.x; t < nj * (LDX - P); t += MIX_THREADS) {
            const int jj = t / (LDX - P), e = P + t % (LDX - P);
            if (Xf) Xf[jj * LDX + e] = df{0.0f, 0.0f};
            Wf[jj * LDX + e] = df{0.0f, 0.0f};
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void mark_undersampled(const MixedArgs &A, int64_t li, int64_t i, int64_t rs, int ni)
{
    const int n_ops = A.n_ops;
    for (int64_t t = threadIdx.x; t < (int64_t)ni * n_ops; t += blockDim.x) {
        if (A.wdtype == LABFM_F64) ((double *)A.w)[rs * n_ops + t] = 0.0;
        else ((float *)A.w)[rs * n_ops + t] = 0.0f;
    }
    if (threadIdx.x == 0) A.flag[li] = 8;
}

// ------------------------------------------------------------------------------------------
// A: X, W and M in double-float
// ------------------------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void assemble_node(const MixedArgs &A, int64_t li, double *smem_d, int &s_bad)
{
    using C = MCfg<K>;
    constexpr int P = C::P, LDX = C::LDX, NB = C::NB, TM = C::TM, TN = C::TN;
    df *Xf = reinterpret_cast<df *>(smem_d);  // [NB][LDX]
    df *Wf = Xf + NB * LDX;                   // [NB][LDX]
    df *Nrec = Wf + NB * LDX;                 // [NB][NREC]
    const int tid = threadIdx.x;
    const int rg = tid / C::CG, cg = tid % C::CG;
    const bool tile_active = tid < C::RG * C::CG;

    const int64_t i = node_of(A, li);
    const int64_t rs = A.row_ptr[i], re = A.row_ptr[i + 1];
    const int ni = (int)(re - rs);
    if (ni < P) {
        mark_undersampled(A, li, i, rs, ni);
        return;
    }
    df acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; a++)
#pragma unroll
        for (int b = 0; b < TN; b++) acc[a][b] = df{0.0f, 0.0f};
    for (int j0 = 0; j0 < ni; j0 += NB) {
        const int nj = min(NB, ni - j0);
        stage_chunk<K>(A, rs, j0, nj, nullptr, Xf, Wf, Nrec);
        if (A.wstore) {
            df *ws = A.wstore + (rs + j0) * A.wstride;
            for (int t = tid; t < nj * P; t += MIX_THREADS) {
                const int jj = t / P, e = t - jj * P;
                ws[jj * A.wstride + e] = Wf[jj * LDX + e];
            }
        }
        if (tile_active) {
            for (int j = 0; j < nj; j++) {
                const df *X = Xf + j * LDX + rg * TM;
                // columns cg, cg + CG, ...: a warp's loads of one column slot are consecutive
                // 8-byte values (distinct banks), where four consecutive columns per thread (two
                // 16-byte loads) put threads 4 apart on the same banks
                const df *W = Wf + j * LDX + cg;
                df xv[TM], wv[TN];
#pragma unroll
                for (int a = 0; a < TM; a++) xv[a] = X[a];
#pragma unroll
                for (int b = 0; b < TN; b++) wv[b] = W[b * C::CG];
#pragma unroll
                for (int a = 0; a < TM; a++)
#pragma unroll
                    for (int b = 0; b < TN; b++) acc[a][b] = df_fma(xv[a], wv[b], acc[a][b]);
            }
        }
        __syncthreads();
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (tile_active) {
        df *Mg = A.Mg + li * A.mstride;
        bool finite = true;
#pragma unroll
        for (int a = 0; a < TM; a++)
#pragma unroll
            for (int b = 0; b < TN; b++) {
                int m = rg * TM + a, c = cg + b * C::CG;
                if (m < P && c < P) {
                    Mg[m * P + c] = acc[a][b];
                    finite &= df_isfinite(acc[a][b]);
                }
            }
        if (!finite) s_bad = 4;  // a neighbour on top of node i: singular ABFs
    }
    __syncthreads();
    if (tid == 0) A.flag[li] = s_bad;
}

template <int K>
__global__ void __launch_bounds__(MIX_THREADS, 3) k_mixed_assemble(MixedArgs A)
{
    extern __shared__ __align__(16) double smem_d[];
    __shared__ int s_bad;
    for (int64_t li = blockIdx.x; li < A.n_list; li += gridDim.x) assemble_node<K>(A, li, smem_d, s_bad);
}

// ------------------------------------------------------------------------------------------
// A': M on the tensor cores (tcgen05), exact in BF16 slices.
//
// Every X_alpha(j) and W_beta(j) of a chunk of <= 64 neighbours is scaled by a power of two
// common to its row over the chunk, 2^-e, e = the exponent of the row's largest magnitude, and
// cut into NSL = 7 BF16 slices of 8 bits:
//     v 2^-e = sum_{s=1..7} c_s 2^-8s,   c_1 in [-256, 256], c_s in [-128, 128] (s > 1),
// integers, so exact in BF16 (8 significant bits), with |remainder| <= 2^-57 (relative to the
// row's largest value; a value far below it keeps fewer bits, hence seven slices rather than
// six: order-8 rows span up to ~2^20 across a stencil).  For each level t = a + b (2..8) the
// products of slices a of X and b of W over the chunk are summed on the tensor cores into one
// FP32 accumulator per level:
//     D_t[alpha][beta] = sum_{a + b = t} sum_j cX_a[alpha](j) cW_b[beta](j),
// every partial sum an integer of magnitude <= 64 (2 * 256 * 128 + 5 * 128 * 128) < 2^24, so
// the FP32 accumulation is exact.  Then M[alpha][beta] = 2^(eX + eW) sum_t D_t 2^-8t in
// double-float (levels >= 9 lie below 2^-56 of the leading one and are not formed).
//
// Operands sit in shared memory in the K-major core-matrix layout without swizzle (8 rows x 16
// bytes per core matrix; K-adjacent core matrices 128 B apart, 8-row groups 1 KB apart for a
// 64-deep chunk).  A = X slice (rows alpha, M = 128: rows >= p are don't-care), B = W slice
// (rows beta, N = p rounded up to 16), K = neighbours.  Accumulators D_t live in tensor memory
// (lane = alpha, column = (t - t0) N + beta); the CTA holds 256 columns, two CTAs per SM.
// ------------------------------------------------------------------------------------------
constexpr int TC_THREADS = 256;
constexpr int NSL = 7;          // slices per operand
constexpr int TC_KC = 64;       // neighbours per chunk (the K of one pass)
constexpr int TC_PARTS = 4;     // threads per neighbour in the X/W evaluation: one pass of the CTA
static_assert(TC_KC * TC_PARTS == TC_THREADS, "every thread evaluates one (neighbour, part)");
constexpr int TC_ROWB = TC_KC / 8 * 128;  // bytes per 8-row group of an operand slice
constexpr int TC_TMEM_COLS = 256;

template <int K> struct TcCfg {
    static constexpr int P = p_of_k(K);
    static constexpr int PN = (P + 15) / 16 * 16;        // N of one level (columns)
    static constexpr int RA = (P + 7) / 8 * 8;           // rows stored per X slice
    static constexpr int SA = RA / 8 * TC_ROWB;          // bytes per X slice
    static constexpr int SB = PN / 8 * TC_ROWB;          // bytes per W slice
    static constexpr int A_BYTES = (NSL - 1) * SA + 16 * TC_ROWB;  // the last slice's 128-row window
    static constexpr int B_BYTES = NSL * SB;
    // levels per tensor-memory round: the columns fit the allocation, and the exact int64
    // combination of a round's levels (each < 2^24, 8 bits apart) stays below 2^63
    static constexpr int LPR = TC_TMEM_COLS / PN < 5 ? TC_TMEM_COLS / PN : 5;
    // row stride (df) of the staging arrays: odd, so that the 8-byte accesses of consecutive
    // neighbours (threads) fall on distinct bank pairs
    static constexpr int LDS = P % 2 ? P : P + 1;
    // row stride (df) of M in shared memory: odd, so that the epilogue's lanes (consecutive rows,
    // one column) fall on distinct bank pairs
    static constexpr int LDSM = P % 2 ? P : P + 1;
    static constexpr size_t smem = (size_t)A_BYTES + B_BYTES + 8 * (size_t)P * LDSM + 16;
    static_assert((size_t)TC_KC * LDS * 8 <= (size_t)A_BYTES && (size_t)TC_KC * LDS * 8 <= (size_t)B_BYTES,
                  "staging fits the operand regions");
    static_assert(P <= 64, "rows alpha in the first two lane quadrants");
};

__device__ __forceinline__ uint32_t tc_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle, LBO = 128 B (K direction), SBO = 1 KB
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(TC_ROWB >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t tc_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, int accumulate)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

// Bounded wait for the completion of phase `parity` of the mbarrier (polls; false: gave up).
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, int polls = 1 << 20)
{
    for (int it = 0; it < polls; it++) {
        uint32_t done;
        asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity));
        if (done) return true;
    }
    return false;
}

// 2^e as a float for |e| <= 126 (clamped: values beyond lie outside the double-float range)
__device__ __forceinline__ float tc_pow2(int e)
{
    e = max(-126, min(127, e));
    return __int_as_float((e + 127) << 23);
}

// exponent e with |v| < 2^e for every v of magnitude <= m (m = max |hi| of a row), 0 for m = 0
__device__ __forceinline__ int tc_row_exp(float m) { return m > 0.0f ? ilogbf(m) + 1 : 0; }

// byte offset of element (row r, k) in a K-major core-matrix slice
__device__ __forceinline__ int tc_off(int r, int k) { return (r >> 3) * TC_ROWB + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// Shared state of the tensor-core assembly, kept by the kernel across the nodes of a CTA.
struct TcShared {
    uint32_t max[2 * PMAX];  // per-row max |hi| of X (0..P-1) and W (P..2P-1) over the chunk
    int e[2 * PMAX];         // the rows' scaling exponents
    int bad, abort;
    uint32_t pending;        // the mbarrier phase whose MMAs a timed-out wait left behind
};

// M of list entry li on the tensor cores (the CTA's tensor memory `tmem`, mbarrier `mbar` with
// its current `phase`).  Returns with ts.abort set if a completion wait gave up.
template <int K>
__device__ __forceinline__ void tc_node(const MixedArgs &A, int64_t li, unsigned char *smem_tc, TcShared &ts,
                                        uint32_t tmem, uint32_t mbar, uint32_t &phase)
{
    using C = TcCfg<K>;
    constexpr int P = C::P, PN = C::PN, LDS = C::LDS;
    unsigned char *sA = smem_tc;                      // X slices (and the X staging)
    unsigned char *sB = smem_tc + C::A_BYTES;         // W slices (and the W staging)
    df *sM = reinterpret_cast<df *>(sB + C::B_BYTES);  // M of the node, accumulated over chunks
    df *Xst = reinterpret_cast<df *>(sA);
    df *Wst = reinterpret_cast<df *>(sB);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // epilogue role: warps 0, 1, 4, 5 read lane quadrants 0 and 1 (alpha = lane + 32 q);
    // warps w and w + 4 take the two halves of the beta columns
    const int q = warp & 3, half = warp >> 2;
    const int alpha = 32 * q + lane;
    const bool epi = q < 2;
    const int64_t i = node_of(A, li);
    const int64_t rs = A.row_ptr[i], re = A.row_ptr[i + 1];
    const int ni = (int)(re - rs);
    if (ni < P) {
        mark_undersampled(A, li, i, rs, ni);
        return;
    }
    if (tid == 0) ts.bad = 0;
    for (int j0 = 0; j0 < ni; j0 += TC_KC) {
        const int nj = min(TC_KC, ni - j0);
        const int ksteps = (nj + 15) / 16;
        // 1. X and W of the chunk in double-float (TC_PARTS threads per neighbour)
        if (tid < 2 * P) ts.max[tid] = 0u;
        for (int t = tid; t < TC_KC * TC_PARTS; t += TC_THREADS) {
            const int part = t / TC_KC, jj = t - part * TC_KC;
            if (jj < nj)
                eval_xw_part<K, TC_PARTS>(A.recs[rs + j0 + jj].v, part, Xst + jj * LDS, Wst + jj * LDS);
        }
        __syncthreads();
        if (A.wstore) {  // W for the weights kernel (the staging is read-only until the next barrier)
            df *ws = A.wstore + (rs + j0) * A.wstride;
            for (int t = tid; t < nj * P; t += TC_THREADS) {
                const int jj = t / P, e = t - jj * P;
                ws[jj * A.wstride + e] = Wst[jj * LDS + e];
            }
        }
        // 2. octets (row r of one operand, 8 consecutive neighbours) to registers, and the
        //    row maxima of |hi| (as ordered bit patterns: non-negative floats compare as integers)
        constexpr int NOCT = 2 * P * (TC_KC / 8);
        constexpr int PER = (NOCT + TC_THREADS - 1) / TC_THREADS;
        df val[PER][8];
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int o = tid + u * TC_THREADS;
            const int opnd = o / (P * (TC_KC / 8)), rem = o - opnd * (P * (TC_KC / 8));
            const int r = rem % P, oct = rem / P;
            uint32_t m = 0u;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const int jj = 8 * oct + c;
                val[u][c] = (o < NOCT && jj < nj) ? (opnd == 0 ? Xst : Wst)[jj * LDS + r] : df{0.0f, 0.0f};
                m = max(m, __float_as_uint(fabsf(val[u][c].hi)));  // NaN and inf sort above finite
            }
            if (o < NOCT && m) atomicMax(&ts.max[opnd * P + r], m);
        }
        __syncthreads();
        // 3. slices -> BF16 operands, one 16-byte core-matrix row (8 neighbours) per store;
        //    K positions nj .. 16 ksteps - 1 are zero
        if (tid < 2 * P) {
            const uint32_t mb = ts.max[tid];
            ts.e[tid] = tc_row_exp(mb >= 0x7f800000u ? 0.0f : __uint_as_float(mb));
        }
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int o = tid + u * TC_THREADS;
            const int opnd = o / (P * (TC_KC / 8)), rem = o - opnd * (P * (TC_KC / 8));
            const int r = rem % P, oct = rem / P;
            if (o >= NOCT || 8 * oct >= 16 * ksteps) continue;
            const uint32_t mb = ts.max[opnd * P + r];
            if (mb >= 0x7f800000u) ts.bad = 4;  // a neighbour on top of node i: singular ABFs
            const float sc = tc_pow2(-tc_row_exp(mb >= 0x7f800000u ? 0.0f : __uint_as_float(mb)));
            float rh[8], rl[8];
#pragma unroll
            for (int c = 0; c < 8; c++) {
                rh[c] = val[u][c].hi * sc;
                rl[c] = val[u][c].lo * sc;
            }
            unsigned char *base = (opnd == 0 ? sA : sB) + tc_off(r, 8 * oct);
            const int sstride = opnd == 0 ? C::SA : C::SB;
#pragma unroll
            for (int sl = 1; sl <= NSL; sl++) {
                const float up = tc_pow2(8 * sl), dn = tc_pow2(-8 * sl);
                uint32_t packed[4];
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    const float c0 = rintf(rh[c] * up), c1 = rintf(rh[c + 1] * up);  // integers, |c| <= 256
                    two_sum(__fsub_rn(rh[c], c0 * dn), rl[c], rh[c], rl[c]);          // exact remainders
                    two_sum(__fsub_rn(rh[c + 1], c1 * dn), rl[c + 1], rh[c + 1], rl[c + 1]);
                    __nv_bfloat162 pr = __floats2bfloat162_rn(c0, c1);
                    packed[c / 2] = *reinterpret_cast<uint32_t *>(&pr);
                }
                *reinterpret_cast<uint4 *>(base + (sl - 1) * sstride) =
                    make_uint4(packed[0], packed[1], packed[2], packed[3]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // 4. per round of levels: issue, wait, read out
        for (int t0 = 2; t0 <= NSL + 1 && !ts.abort; t0 += C::LPR) {
            const int t1 = min(NSL + 1, t0 + C::LPR - 1);
            asm volatile("tcgen05.fence::after_thread_sync;");  // the last read-out is complete
            if (tid == 0) {
                uint64_t ad[NSL], bd[NSL];
                const uint32_t a0 = tc_smem_u32(sA), b0 = tc_smem_u32(sB);
#pragma unroll
                for (int sl = 0; sl < NSL; sl++) {
                    ad[sl] = tc_desc(a0 + sl * C::SA);
                    bd[sl] = tc_desc(b0 + sl * C::SB);
                }
                // one MMA per (X slice a, K step): B = the W slices b_lo .. b_hi that pair with a
                // inside the round (adjacent rows), D shifted so that column block b lands in
                // level a + b's accumulator.  a = 1 covers every level of the round, so its
                // first K step initialises all of them.
                for (int a = 1; a <= NSL && a < t1; a++) {
                    const int b_lo = max(1, t0 - a), b_hi = min(NSL, t1 - a);
                    if (b_lo > b_hi) continue;
                    const uint32_t idesc = tc_idesc((b_hi - b_lo + 1) * PN);
                    const uint32_t dcol = (uint32_t)((a + b_lo - t0) * PN);
                    for (int ks = 0; ks < ksteps; ks++)  // +256 B per K step = +16 in the address field
                        tc_mma(tmem + dcol, ad[a - 1] + (uint64_t)(16 * ks), bd[b_lo - 1] + (uint64_t)(16 * ks),
                               idesc, (a == 1 && ks == 0) ? 0 : 1);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    mbar));
            }
            const bool ok = tc_wait(mbar, phase);
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!ok) {
                if (tid == 0) {
                    ts.abort = 1;
                    ts.pending = phase ^ 1u;
                    atomicAdd(A.tc_timeout, 1ull);
                }
            } else if (epi) {
                // thread (alpha, half): M[alpha][beta] for its half of the beta columns,
                // accumulated over the rounds and chunks in shared memory.  The levels of a
                // round are exact integers < 2^24: S = sum_t D_t 2^(8 (t1 - t)) is exact in
                // int64 (< 2^57), and M += 2^(eX + eW - 8 t1) S.
                const bool own = alpha < P;
                constexpr int HB = PN / 2;  // columns per half
                df *Mrow = sM + (own ? alpha : 0) * C::LDSM;
                const int ex = ts.e[own ? alpha : 0] - 8 * t1;
                for (int g = 0; g < HB; g += 8) {
                    // all levels of this round for 8 columns: issue the loads, then one wait
                    uint32_t v[C::LPR][8];
#pragma unroll
                    for (int l = 0; l < C::LPR; l++) {
                        if (t0 + l <= t1) {
                            asm volatile(
                                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                : "=r"(v[l][0]), "=r"(v[l][1]), "=r"(v[l][2]), "=r"(v[l][3]), "=r"(v[l][4]),
                                  "=r"(v[l][5]), "=r"(v[l][6]), "=r"(v[l][7])
                                : "r"(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(l * PN + half * HB + g)));
                        }
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (own) {
#pragma unroll
                        for (int c = 0; c < 8; c++) {
                            const int beta = half * HB + g + c;
                            if (beta >= P) continue;
                            long long S = 0;
#pragma unroll
                            for (int l = 0; l < C::LPR; l++)
                                if (t0 + l <= t1) S = S * 256 + (long long)__float2int_rn(__uint_as_float(v[l][c]));
                            // S = H 2^32 + L1 2^16 + L0, |H| < 2^25, L1, L0 < 2^16: three exact floats
                            const int H = (int)(S >> 32);
                            const uint32_t L = (uint32_t)S;
                            float sh, sl;
                            two_sum((float)H * 4294967296.0f, (float)(L >> 16) * 65536.0f, sh, sl);
                            sl = __fadd_rn(sl, (float)(L & 0xffffu));
                            fast_two_sum(sh, sl, sh, sl);
                            const float sc = tc_pow2(ex + ts.e[P + beta]);
                            const df add = df{sh * sc, sl * sc};
                            Mrow[beta] = (j0 == 0 && t0 == 2) ? add : df_add(Mrow[beta], add);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
        if (ts.abort) break;
    }
    if (ts.abort) return;
    // M of the node -> global
    df *Mg = A.Mg + li * A.mstride;
    bool finite = true;
    for (int u = tid; u < P * P; u += TC_THREADS) {
        const int r = u / P;
        const df v = sM[r * C::LDSM + (u - r * P)];
        finite &= df_isfinite(v);
        Mg[u] = v;
    }
    if (!finite) ts.bad = 4;
    __syncthreads();
    if (tid == 0) A.flag[li] = ts.bad;
    __syncthreads();
}

// CTA set-up of the tensor-core assembly: the mbarrier and 256 tensor-memory columns.
__device__ __forceinline__ void tc_setup(uint64_t &s_mbar, uint32_t &s_tmem, TcShared &ts)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(&s_mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        ts.abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

// CTA tear-down.  After a wait that gave up, the MMAs of that commit may still be writing tensor
// memory: wait for them once more (bounded, 4x longer) before the memory is released.  The call
// reports LABFM_ERR_TIMEOUT either way and its weights are undefined.  (Not exercised on the GPU:
// making a wait run out would leave tensor-core work in flight on a shared GPU.)
__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t mbar, const TcShared &ts)
{
    if (ts.abort) tc_wait(mbar, ts.pending, 1 << 22);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

template <int K>
__global__ void __launch_bounds__(TC_THREADS, 2) k_mixed_assemble_tc(MixedArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ TcShared ts;
    tc_setup(s_mbar, s_tmem, ts);
    const uint32_t tmem = s_tmem, mbar = tc_smem_u32(&s_mbar);
    uint32_t phase = 0;
    for (int64_t li = blockIdx.x; li < A.n_list; li += gridDim.x) {
        tc_node<K>(A, li, smem_tc, ts, tmem, mbar, phase);
        if (ts.abort) break;
    }
    tc_teardown(tmem, mbar, ts);
}

// ------------------------------------------------------------------------------------------
// B: Gauss-Jordan inversion with partial pivoting, in double-float.  Two forms, the build
// autotuner choosing per order: each row in the registers of one thread (k_mixed_invert_rr,
// below), or one CTA per node with TPR (2 or 4) threads per row of the working matrix in shared
// memory:
// thread t updates the columns q = h, h + TPR, h + 2 TPR, ... of row t / TPR (h = t % TPR), so
// that TPR P lanes do work and each thread's update is 1/TPR of a row.  Zero columns pad P to a
// multiple WC of TPR.  The row stride LDM (in 8-byte words) is TPR times an odd number, so the
// 16 lanes of a half-warp (16 / TPR rows, TPR column classes) touch 16 distinct bank pairs.  Per
// pivot column c:
//   1. argmax of |M[r][c]| over r >= c (lanes h = 0; warp shuffles, then the warps through
//      shared memory; the lowest row wins a tie);
//   2. rows c and argmax exchanged (threads over columns), the pivot row and the pivot column
//      (after the exchange) published in shared memory;
//   3. f = M[r][c] / p, M[r][q] -= f M[c][q] on the thread's columns (q != c), M[r][c] = -f;
//      row c: M[c][q] /= p, M[c][c] = 1 / p.
// The row interchanges are undone on the columns when the result is written out.
// ------------------------------------------------------------------------------------------
template <int P, int TPR> struct InvCfg {
    static_assert(TPR == 2 || TPR == 4, "two or four threads per row");
    static constexpr int PART = (P + TPR - 1) / TPR;                         // columns per thread
    static constexpr int WC = TPR * PART;                                     // working columns
    static constexpr int LDM = (WC / TPR) % 2 ? WC : WC + TPR;                // TPR x odd
    static constexpr int NT = (TPR * P + 31) / 32 * 32;                       // threads, whole warps
    static constexpr int NW = NT / 32;
    static_assert(NT >= WC && NT >= TPR * P, "a thread per column and TPR per row");
    static_assert((LDM / TPR) % 2 == 1 && LDM % TPR == 0 && LDM >= WC, "row stride");
};

// Shared memory of the inversion of one p x p matrix with TPR threads per row.
template <int P, int TPR> struct InvShared {
    df m[P * InvCfg<P, TPR>::LDM];
    df prow[InvCfg<P, TPR>::WC];
    df pcol[P];
    float best[InvCfg<P, TPR>::NW];
    int br[InvCfg<P, TPR>::NW];
    int src[P];
    signed char piv[P];
};

// M^-1 of list entry li at order K by a CTA of InvCfg<p, TPR>::NT threads.
template <int K, int TPR>
__device__ __forceinline__ void invert_node(const MixedArgs &A, int64_t li, InvShared<p_of_k(K), TPR> &sh)
{
    constexpr int P = p_of_k(K);
    using I = InvCfg<P, TPR>;
    constexpr int PART = I::PART, WC = I::WC, LDM = I::LDM, NT = I::NT, NW = I::NW;
    df *s_m = sh.m, *s_prow = sh.prow, *s_pcol = sh.pcol;
    float *s_best = sh.best;
    int *s_br = sh.br, *s_src = sh.src;
    signed char *s_piv = sh.piv;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int r = t / TPR, hf = t % TPR;
    const bool own = r < P;

    if (A.flag[li] != 0) return;  // uniform per CTA
    const df *Mg = A.Mg + li * A.mstride;
    for (int u = t; u < P * P; u += NT) {
        const int rr = u / P;
        s_m[rr * LDM + (u - rr * P)] = Mg[u];
    }
    if (WC > P)
        for (int u = t; u < P * (WC - P); u += NT) s_m[(u / (WC - P)) * LDM + P + u % (WC - P)] = df{0.0f, 0.0f};
    __syncthreads();
    bool zero = false;
    for (int c = 0; c < P; c++) {
        float best = (own && hf == 0 && r >= c) ? fabsf(s_m[r * LDM + c].hi) : -1.0f;
        int br = own ? r : P;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int orr = __shfl_xor_sync(0xffffffffu, br, o);
            if (ob > best || (ob == best && orr < br)) {
                best = ob;
                br = orr;
            }
        }
        if (lane == 0) {
            s_best[warp] = best;
            s_br[warp] = br;
        }
        __syncthreads();
        best = s_best[0];
        br = s_br[0];
#pragma unroll
        for (int w = 1; w < NW; w++)
            if (s_best[w] > best) {  // later warps hold higher rows: strict keeps the lowest
                best = s_best[w];
                br = s_br[w];
            }
        if (!(best > 0.0f) || !isfinite(best)) {
            zero = true;
            break;
        }
        // best > 0 comes from a lane h = 0 of a row r >= c, so c <= br < P
        if (t == 0) s_piv[c] = (signed char)br;
        if (t < WC) {  // column t: exchange rows c and br, publish the pivot row
            const df a = s_m[c * LDM + t], b = s_m[br * LDM + t];
            s_prow[t] = b;
            if (br != c) {
                s_m[c * LDM + t] = b;
                s_m[br * LDM + t] = a;
            }
            // row t's entry of the pivot column after the exchange (rows c and br from the
            // values this thread just read when t == c; other rows are not being written)
            if (t == c) {
                s_pcol[c] = b;
                if (br != c) s_pcol[br] = a;
            } else if (t < P && t != br) {
                s_pcol[t] = s_m[t * LDM + c];
            }
        }
        __syncthreads();
        const df inv = df_recip(s_prow[c]);
        if (own) {
            df *row = s_m + r * LDM + hf;  // this thread's columns: row[TPR q]
            const bool mine = (c % TPR) == hf;
            if (r == c) {
#pragma unroll
                for (int q = 0; q < PART; q++) row[TPR * q] = df_mul(row[TPR * q], inv);
                if (mine) row[c - hf] = inv;
            } else {
                const df f = df_mul(s_pcol[r], inv);
                const df *pr = s_prow + hf;
#pragma unroll
                for (int q = 0; q < PART; q++) row[TPR * q] = df_fms(f, pr[TPR * q], row[TPR * q]);
                if (mine) row[c - hf] = df_neg(f);
            }
        }
        __syncthreads();
    }
    if (zero) {
        if (t == 0) A.flag[li] = 1;
        __syncthreads();
        return;
    }
    // column order of the result: undo the interchanges, last first
    if (t == 0) {
        for (int q = 0; q < P; q++) s_src[q] = q;
        for (int c = P - 1; c >= 0; c--) {
            const int pr = s_piv[c];
            const int a = s_src[c];
            s_src[c] = s_src[pr];
            s_src[pr] = a;
        }
    }
    __syncthreads();
    df *Mo = A.Mg + li * A.mstride;
    for (int u = t; u < P * P; u += NT) {  // column-major: element (rr, q) at q * P + rr
        const int q = u / P, rr = u - q * P;
        Mo[u] = s_m[rr * LDM + s_src[q]];
    }
    __syncthreads();
}

template <int K, int TPR>
__global__ void __launch_bounds__(InvCfg<p_of_k(K), TPR>::NT) k_mixed_invert(MixedArgs A)
{
    __shared__ InvShared<p_of_k(K), TPR> sh;
    for (int64_t li = blockIdx.x; li < A.n_list; li += gridDim.x) invert_node<K, TPR>(A, li, sh);
}

// The same Gauss-Jordan inversion with each row of M held in the registers of one thread (one
// "thread per row"), NPC nodes per CTA.  Rows are not exchanged: the pivot of column c is the
// largest |M[r][c]| (then the lowest r) over the rows not yet used as pivots, found with a
// shared-memory atomicMax on (|hi| bits, ~r); every row then holds its columns c .. p-1 in
// a[0 .. p-1-c] and the finished columns of the inverse behind them: the update
//     a[k-1] = a[k] - f prow[k]  (k = 1 .. p-1),   a[p-1] = -f,   f = M[r][c] / pivot
// (the pivot row: a[k-1] = a[k] / pivot, a[p-1] = 1 / pivot) shifts the row by one column, so
// that every register index is fixed at compile time and the pivot column is always a[0].  With
// E the product of the row operations, E M = Pi (the permutation of the pivot rows) and
// M^-1 = Pi^T E: after p steps a[c] of row r is E[r][p_c], p_c the pivot row of column c, and
// it is row s_r of the inverse (s_r the column row r was pivot of) at column p_c.  Against the
// shared-memory version: one shared load (the broadcast pivot row) per multiply-add instead of
// two loads and a store, and two barriers per column instead of three.
// Nodes per CTA: 2, 5, 7, 8 for p = 44, 35, 27, 20 (88 of 96, 175 of 192, 189 of 192, 160 of 160
// lanes busy).  CTAs per SM from a register budget of 2p + 40 per thread (the row's 2p floats and
// the rest): at p = 44, 128 registers, five CTAs per SM, a few spilled values; a budget without
// spills (151 registers, four CTAs per SM) measured 1 % slower.
template <int P> struct RrCfg {
    static constexpr int NPC = P > 40 ? 2 : (P > 30 ? 5 : (P > 24 ? 7 : 8));
    static constexpr int NT = (NPC * P + 31) / 32 * 32;
    static constexpr int MINB = 65536 / (NT * (2 * P + 40)) > 0 ? 65536 / (NT * (2 * P + 40)) : 1;
};

template <int P, int NPC> struct RrShared {
    unsigned long long key[NPC][2];  // pivot candidates of columns of even / odd index
    df prow[NPC][P];                 // the pivot row (a[1 ..] before the update)
    df inv[NPC];                     // 1 / pivot
    unsigned char pivrow[NPC][P];    // p_c
};

template <int K>
__global__ void __launch_bounds__(RrCfg<p_of_k(K)>::NT, RrCfg<p_of_k(K)>::MINB) k_mixed_invert_rr(MixedArgs A)
{
    constexpr int P = p_of_k(K), NPC = RrCfg<P>::NPC;
    __shared__ RrShared<P, NPC> sh;
    const int t = threadIdx.x;
    const int nl = t / P, r = t - nl * P;
    const bool slot = nl < NPC;
    for (int64_t g = blockIdx.x; g * NPC < A.n_list; g += gridDim.x) {
        const int64_t li = g * NPC + nl;
        bool active = slot && li < A.n_list;
        if (active) active = A.flag[li] == 0;
        df a[P];
        if (active) {
            const df *row = A.Mg + li * A.mstride + r * P;
#pragma unroll
            for (int k = 0; k < P; k++) a[k] = row[k];
        } else {
#pragma unroll
            for (int k = 0; k < P; k++) a[k] = df{0.0f, 0.0f};
        }
        if (t < NPC) sh.key[t][0] = 0ull;
        __syncthreads();
        bool used = false, dead = false;
        int mystep = 0;
        for (int c = 0; c < P; c++) {
            const int b = c & 1;
            if (active && !used) {
                const unsigned long long key = ((unsigned long long)__float_as_uint(fabsf(a[0].hi)) << 32) |
                                               (unsigned long long)(0xffffffffu - (unsigned)r);
                atomicMax(&sh.key[nl][b], key);
            }
            if (t < NPC) sh.key[t][b ^ 1] = 0ull;
            __syncthreads();
            const unsigned long long key = slot ? sh.key[nl][b] : 0ull;
            const unsigned mag = (unsigned)(key >> 32);
            const int pr = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
            // |pivot| zero, infinite or NaN (NaN bit patterns sort above every finite value)
            if (!(mag > 0u && mag < 0x7f800000u)) dead = true;
            const bool go = active && !dead;
            if (go && r == pr) {
#pragma unroll
                for (int k = 1; k < P; k++) sh.prow[nl][k] = a[k];
                sh.inv[nl] = df_recip(a[0]);
                sh.pivrow[nl][c] = (unsigned char)r;
                used = true;
                mystep = c;
            }
            __syncthreads();
            if (go) {
                // one update for every row (no divergent branch for the pivot row): the pivot
                // row clears its registers and takes f = -1/pivot, so that its a[k-1] =
                // 0 - f prow[k] = prow[k] / pivot and a[p-1] = -f = 1/pivot
                const df inv = sh.inv[nl];
                df f = df_mul(a[0], inv);
                if (r == pr) {
                    f = df_neg(inv);
#pragma unroll
                    for (int k = 1; k < P; k++) a[k] = df{0.0f, 0.0f};
                }
                const df *pw = sh.prow[nl];
#pragma unroll
                for (int k = 1; k < P; k++) a[k - 1] = df_fms(f, pw[k], a[k]);
                a[P - 1] = df_neg(f);
            }
        }
        if (active) {
            if (dead) {
                if (r == 0) A.flag[li] = 1;
            } else {
                df *out = A.Mg + li * A.mstride + mystep;  // column-major, as the shared form
#pragma unroll
                for (int c = 0; c < P; c++) out[sh.pivrow[nl][c] * P] = a[c];
            }
        }
        __syncthreads();  // sh.pivrow and the keys are rewritten by the next group
    }
}

// ------------------------------------------------------------------------------------------
// C: Psi~ = M^-1 C~, w~ = W . Psi~, FP64 residual refinement, physical weights
//
// Adaptive refinement.  Step t changes the weights by dw_t (t = 0: the first solve, dw_0 = w_0);
// eta_t = max_d ||dw_t,d|| / ||w_t,d|| over the node's stencil (eta_0 = 1).  Refinement with an
// approximate inverse contracts the error by a factor rho per step, and the correction dw_t is
// close to the error before it, so rho ~ eta_t / eta_(t-1) and the error left after step t is
// about eta_t^2 / eta_(t-1).  The node stops after step t >= 1 when
//   - that estimate is below 2^-44 (~6e-14: within a few hundred ulps of double precision), or
//   - eta_t > eta_(t-1) / 2: the corrections no longer shrink, because they are at the rounding
//     level of the FP64 residual (the floor of the method on this stencil), or because the
//     inverse is too inaccurate for the iteration to contract (cond(M) u_df >~ 1); in the latter
//     case, recognised by eta_t > 1e-3, the node is rebuilt in FP64 (fb_list), or
//   - t = NREF_MAX.
// Most nodes stop after one step, with no residual evaluated after it.
// ------------------------------------------------------------------------------------------
constexpr int NREF_MAX = 6;
constexpr float REF_EPS = 5.6843419e-14f;  // 2^-44
constexpr float REF_DIVERGED = 1e-3f;

// Thread 0: the decision after step `it` from the per-operator sums of dw^2 and w^2 in shared
// memory.  Returns 1 to continue, 0 to stop, 2 to stop and rebuild the node in FP64.
__device__ __forceinline__ int refine_decision(int it, int nmax, int n_ops, const float *dw2, const float *w2,
                                               float eta_prev, float &eta)
{
    eta = 0.0f;
    for (int d = 0; d < n_ops; d++)
        if (w2[d] > 0.0f) eta = fmaxf(eta, sqrtf(dw2[d] / w2[d]));
    if (it == 0) {
        eta = 1.0f;
        return nmax > 0 ? 1 : 0;
    }
    if (!(eta <= 1e30f)) return 2;  // not finite
    if (eta > 0.5f * eta_prev) return eta > REF_DIVERGED ? 2 : 0;
    if (eta * eta <= REF_EPS * eta_prev) return 0;
    return it < nmax ? 1 : 0;
}

// Per-node shared state of the weights kernel.
struct WShared {
    double hneg[KMAX + 1], hpos[KMAX + 1];
    double res[PMAX * MAX_OPS];
    float dw2[MAX_OPS], w2[MAX_OPS];  // per operator: sum of dw^2 and of w^2 over the stencil
    float eta;
    int flag, go;
};

// Weights of list entry li at order K (dynamic shared memory of MCfg<K>::smemC bytes).
template <int K>
__device__ __forceinline__ void weights_node(const MixedArgs &A, int64_t li, double *smem_d, WShared &ws)
{
    using C = MCfg<K>;
    constexpr int P = C::P, LDX = C::LDX, NB = C::NB;
    double *Xd = smem_d;                                     // [NB][LDX]
    df *Wf = reinterpret_cast<df *>(Xd + NB * LDX);          // [NB][LDX]
    df *Nrec = Wf + NB * LDX;                                // [NB][NREC]
    df *Rhs = Nrec + NB * NREC;                              // [P][MAX_OPS] right-hand sides
    df *Psi = Rhs + P * MAX_OPS;                             // [P][MAX_OPS]
    double *Wt = reinterpret_cast<double *>(Psi + P * MAX_OPS);  // [NB][MAX_OPS] w~ of the chunk
    float *Vt = reinterpret_cast<float *>(Wt + NB * MAX_OPS);    // [NB][MAX_OPS] the last correction of w~
    double *s_hneg = ws.hneg, *s_hpos = ws.hpos, *s_res = ws.res;
    float *s_dw2 = ws.dw2, *s_w2 = ws.w2;
    float &s_eta = ws.eta;
    int &s_flag = ws.flag, &s_go = ws.go;
    const int tid = threadIdx.x;
    const int n_ops = A.n_ops;

    const int64_t i = node_of(A, li);
    const int64_t rs = A.row_ptr[i], re = A.row_ptr[i + 1];
    const int ni = (int)(re - rs);
    const int fl = A.flag[li];
    if (fl & 8) {  // undersampled: weights already zeroed by kernel A
        if (tid == 0) {
            if (A.node_status) A.node_status[i] = LABFM_NODE_UNDERSAMPLED;
            atomicAdd(A.n_bad, 1ull);
        }
        return;
    }
    if (fl != 0) {
        for (int64_t t = tid; t < (int64_t)ni * n_ops; t += MIX_THREADS) {
            if (A.wdtype == LABFM_F64) ((double *)A.w)[rs * n_ops + t] = 0.0;
            else ((float *)A.w)[rs * n_ops + t] = 0.0f;
        }
        if (tid == 0) {
            if (A.node_status) A.node_status[i] = (fl & 4) ? LABFM_NODE_NONFINITE : LABFM_NODE_SINGULAR;
            atomicAdd(A.n_bad, 1ull);
        }
        return;
    }
    const double hi = A.h[i];
    const double ihi = 1.0 / hi;
    if (tid == 0) {
        double s = 1.0, t = 1.0;
        for (int q = 0; q <= KMAX; q++) {
            s_hneg[q] = s;
            s_hpos[q] = t;
            s *= ihi;
            t *= hi;
        }
        s_flag = 0;
    }
    const df *__restrict__ Mi = A.Mg + li * A.mstride;  // M^-1 of the node (global)
    __syncthreads();
    // scaled targets C~_alpha = C_alpha h^(l_d - |alpha|)
    for (int t = tid; t < P * n_ops; t += MIX_THREADS) {
        int m = t / n_ops, d = t % n_ops;
        int deg = elem_degree(m), l = A.lmax[d];
        double sc = l >= deg ? s_hpos[l - deg] : s_hneg[deg - l];
        s_res[m * MAX_OPS + d] = A.C[d * PMAX + m] * sc;
        Rhs[m * MAX_OPS + d] = df_from_double(s_res[m * MAX_OPS + d]);
    }
    const int nchunks = (ni + NB - 1) / NB;
    if (nchunks == 1) stage_chunk<K>(A, rs, 0, ni, Xd, nullptr, Wf, Nrec);
    else __syncthreads();

    float eta_prev = 1.0f;
    int go = 1;
    int it = 0;
    for (;; it++) {
        // Psi (or its correction) = M^-1 Rhs, thread per (m, d)
        for (int t = tid; t < P * n_ops; t += MIX_THREADS) {
            int m = t / n_ops, d = t % n_ops;
            df s0 = df{0.0f, 0.0f}, s1 = s0;
            const df *col = Mi + m;  // M^-1 is column-major: a warp's rows m are adjacent
            int q = 0;
            for (; q + 1 < P; q += 2) {
                s0 = df_fma(col[q * P], Rhs[q * MAX_OPS + d], s0);
                s1 = df_fma(col[(q + 1) * P], Rhs[(q + 1) * MAX_OPS + d], s1);
            }
            if (q < P) s0 = df_fma(col[q * P], Rhs[q * MAX_OPS + d], s0);
            Psi[m * MAX_OPS + d] = df_add(s0, s1);
        }
        // w~ (+)= W . Psi over the chunks; the residual r = C~ - sum_j X_j w~_j accumulates
        for (int t = tid; t < P * n_ops; t += MIX_THREADS) {
            int m = t / n_ops, d = t % n_ops;
            int deg = elem_degree(m), l = A.lmax[d];
            double sc = l >= deg ? s_hpos[l - deg] : s_hneg[deg - l];
            s_res[m * MAX_OPS + d] = A.C[d * PMAX + m] * sc;
        }
        if (tid < MAX_OPS) {
            s_dw2[tid] = 0.0f;
            if (it == 0) s_w2[tid] = 0.0f;
        }
        __syncthreads();
        for (int ch = 0; ch < nchunks; ch++) {
            const int j0 = ch * NB, nj = min(NB, ni - j0);
            if (nchunks > 1) stage_chunk<K>(A, rs, j0, nj, Xd, nullptr, Wf, Nrec);
            for (int t = tid; t < nj * n_ops; t += MIX_THREADS) {
                int j = t / n_ops, d = t % n_ops;
                df s0 = df{0.0f, 0.0f}, s1 = s0;
                const df *W = Wf + j * LDX;
                int m = 0;
                for (; m + 1 < P; m += 2) {
                    s0 = df_fma(W[m], Psi[m * MAX_OPS + d], s0);
                    s1 = df_fma(W[m + 1], Psi[(m + 1) * MAX_OPS + d], s1);
                }
                if (m < P) s0 = df_fma(W[m], Psi[m * MAX_OPS + d], s0);
                const df sv = df_add(s0, s1);
                const double v = df_to_double(sv);
                const int64_t idx = (rs + j0 + j) * n_ops + d;
                const double wv = it == 0 ? v : A.wt[idx] + v;
                A.wt[idx] = wv;
                Wt[j * MAX_OPS + d] = wv;
                Vt[j * MAX_OPS + d] = sv.hi;  // the change in float (no FP64 conversion)
            }
            __syncthreads();
            if (A.adaptive) {
                // per operator (warp d): the chunk's sum of dw^2 in float; the sum of w^2 is that of
                // the first pass (w = dw_0), kept for the later ones, where w changes by a relative
                // eta << 1 (its effect on eta_t is of the order of eta_t itself)
                const int wp = tid >> 5, ln = tid & 31;
                if (wp < n_ops) {
                    float a2 = 0.0f;
                    for (int j = ln; j < nj; j += 32) {
                        const float vf = Vt[j * MAX_OPS + wp];
                        a2 = fmaf(vf, vf, a2);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, o);
                    if (ln == 0) {
                        s_dw2[wp] += a2;
                        if (it == 0) s_w2[wp] += a2;
                    }
                }
                __syncthreads();
            }
            // the residual of this pass is needed only if another step follows; with one
            // chunk the adaptive decision is known here, before the residual is formed
            bool res;
            if (!A.adaptive) {
                res = it < A.nref;
            } else if (nchunks == 1) {
                if (tid == 0) {
                    float eta;
                    s_go = refine_decision(it, A.nref, n_ops, s_dw2, s_w2, eta_prev, eta);
                    s_eta = eta;
                }
                __syncthreads();
                res = s_go == 1;
            } else {
                res = it < A.nref;
            }
            if (res) {
                for (int t = tid; t < P * n_ops; t += MIX_THREADS) {
                    int m = t / n_ops, d = t % n_ops;
                    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                    int j = 0;
                    for (; j + 3 < nj; j += 4) {
                        s0 = fma(Xd[j * LDX + m], Wt[j * MAX_OPS + d], s0);
                        s1 = fma(Xd[(j + 1) * LDX + m], Wt[(j + 1) * MAX_OPS + d], s1);
                        s2 = fma(Xd[(j + 2) * LDX + m], Wt[(j + 2) * MAX_OPS + d], s2);
                        s3 = fma(Xd[(j + 3) * LDX + m], Wt[(j + 3) * MAX_OPS + d], s3);
                    }
                    for (; j < nj; j++) s0 = fma(Xd[j * LDX + m], Wt[j * MAX_OPS + d], s0);
                    s_res[m * MAX_OPS + d] -= (s0 + s1) + (s2 + s3);
                }
            }
            __syncthreads();
        }
        if (A.adaptive) {
            if (nchunks > 1) {
                if (tid == 0) {
                    float eta;
                    s_go = refine_decision(it, A.nref, n_ops, s_dw2, s_w2, eta_prev, eta);
                    s_eta = eta;
                }
                __syncthreads();
            }
            go = s_go;
            eta_prev = s_eta;
            if (go != 1) break;
        } else if (it == A.nref) {
            break;
        }
        for (int t = tid; t < P * n_ops; t += MIX_THREADS) {
            int m = t / n_ops, d = t % n_ops;
            Rhs[m * MAX_OPS + d] = df_from_double(s_res[m * MAX_OPS + d]);
        }
        __syncthreads();
    }
    if (tid == 0 && A.ref_hist) atomicAdd(&A.ref_hist[min(it, NREF_MAX)], 1ull);
    if (go == 2) {
        // the corrections grew: the FP64 build redoes this node (weights and status)
        if (tid == 0) A.fb_list[atomicAdd(A.fb_count, 1ull)] = (int32_t)i;
        __syncthreads();
        return;
    }

    // physical weights w = h^-l_d w~
    for (int64_t t = tid; t < (int64_t)ni * n_ops; t += MIX_THREADS) {
        int d = (int)(t % n_ops);
        double v = A.wt[rs * n_ops + t] * s_hneg[A.lmax[d]];
        if (!isfinite(v)) {
            atomicOr(&s_flag, 2);
            v = 0.0;
        }
        if (A.wdtype == LABFM_F64) ((double *)A.w)[rs * n_ops + t] = v;
        else ((float *)A.w)[rs * n_ops + t] = (float)v;
    }
    __syncthreads();
    if (s_flag & 2) {
        for (int64_t t = tid; t < (int64_t)ni * n_ops; t += MIX_THREADS) {
            if (A.wdtype == LABFM_F64) ((double *)A.w)[rs * n_ops + t] = 0.0;
            else ((float *)A.w)[rs * n_ops + t] = 0.0f;
        }
    }
    if (tid == 0) {
        const int st = (s_flag & 2) ? LABFM_NODE_NONFINITE : LABFM_NODE_OK;
        if (A.node_status) A.node_status[i] = st;
        if (st != LABFM_NODE_OK) atomicAdd(A.n_bad, 1ull);
    }
    __syncthreads();
}

template <int K>
__global__ void __launch_bounds__(MIX_THREADS, 3) k_mixed_weights(MixedArgs A)
{
    extern __shared__ __align__(16) double smem_d[];
    __shared__ WShared ws;
    for (int64_t li = blockIdx.x; li < A.n_list; li += gridDim.x) weights_node<K>(A, li, smem_d, ws);
}

template <class KernelT>
cudaError_t launch_persistent(KernelT kern, const MixedArgs &a, int threads, size_t smem, int64_t units, int num_sms,
                              cudaStream_t s, int max_per_sm = 1 << 30)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm > max_per_sm) per_sm = max_per_sm;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = std::min<int64_t>(units, (int64_t)num_sms * per_sm);
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_records(const MixedArgs &a, int num_sms, cudaStream_t s)
{
    const int64_t blocks = std::min<int64_t>((a.n_list + 7) / 8, (int64_t)num_sms * 16);
    if (blocks > 0) k_mixed_records<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// two CTAs per SM, each holding TC_TMEM_COLS of the 512 tensor-memory columns for its whole run:
// the shared-memory request (>= 80 KB, <= 113 KB) keeps a third CTA off the SM
template <class KernelT>
cudaError_t launch_tc(KernelT kern, const MixedArgs &a, size_t smem_needed, int num_sms, cudaStream_t s)
{
    const size_t smem = std::max<size_t>(smem_needed, 80 * 1024);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(a.n_list, 2 * (int64_t)num_sms);
    if (grid > 0) kern<<<(unsigned)grid, TC_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_mixed_k(const MixedArgs &a, int num_sms, bool tc, int inv_tpr, cudaStream_t s)
{
    using C = MCfg<K>;
    cudaError_t e = launch_records(a, num_sms, s);
    if (e != cudaSuccess) return e;
    if (tc) e = launch_tc(k_mixed_assemble_tc<K>, a, TcCfg<K>::smem, num_sms, s);
    else e = launch_persistent(k_mixed_assemble<K>, a, MIX_THREADS, C::smemA, a.n_list, num_sms, s);
    if (e != cudaSuccess) return e;
    if (inv_tpr == 1)
        e = launch_persistent(k_mixed_invert_rr<K>, a, RrCfg<C::P>::NT, 0, (a.n_list + RrCfg<C::P>::NPC - 1) / RrCfg<C::P>::NPC,
                              num_sms, s);
    else if (inv_tpr == 4) e = launch_persistent(k_mixed_invert<K, 4>, a, InvCfg<C::P, 4>::NT, 0, a.n_list, num_sms, s);
    else e = launch_persistent(k_mixed_invert<K, 2>, a, InvCfg<C::P, 2>::NT, 0, a.n_list, num_sms, s);
    if (e != cudaSuccess) return e;
    return launch_persistent(k_mixed_weights<K>, a, MIX_THREADS, C::smemC, a.n_list, num_sms, s);
}

MixedArgs make_args(const MixedArgsPublic &p)
{
    MixedArgs a{};
    a.xy = p.xy;
    a.h = p.h;
    a.row_ptr = p.row_ptr;
    a.col = p.col;
    a.periodic = p.periodic;
    for (int d = 0; d < 2; d++) {
        a.L[d] = p.L[d];
        a.halfL[d] = p.halfL[d];
    }
    a.rbf = p.rbf;
    a.n_ops = p.n_ops;
    a.nref = p.nref;
    a.adaptive = p.adaptive;
    a.fb_list = p.fb_list;
    a.fb_count = p.fb_count;
    a.ref_hist = p.ref_hist;
    a.w = p.w;
    a.wdtype = p.wdtype;
    a.wt = p.wt;
    a.node_status = p.node_status;
    a.n_bad = p.n_bad;
    a.recs = reinterpret_cast<Rec *>(p.recs);
    a.tc_timeout = p.tc_timeout;
    a.wstore = reinterpret_cast<df *>(p.wstore);
    for (int d = 0; d < MAX_OPS; d++) a.lmax[d] = p.lmax[d];
    for (int t = 0; t < MAX_OPS * PMAX; t++) a.C[t] = p.C[t];
    return a;
}

}  // namespace

size_t mixed_record_bytes() { return sizeof(Rec); }

size_t mixed_scratch_bytes_per_node(int k)
{
    const int p = p_of_k(k);
    return sizeof(df) * (size_t)p * p + sizeof(int);
}

cudaError_t launch_build_mixed(int k, const MixedArgsPublic &p, cudaStream_t s)
{
    if (k < MIXED_MIN_ORDER || k > KMAX) return cudaErrorInvalidValue;
    MixedArgs a = make_args(p);
    const int pk = p_of_k(k);
    a.mstride = (int64_t)pk * pk;
    a.wstride = pk;
    // scratch holds batch_nodes matrices; the node list is processed batch by batch
    const int64_t batch = p.batch_nodes;
    for (int64_t b0 = 0; b0 < p.n_list; b0 += batch) {
        a.n_list = std::min<int64_t>(batch, p.n_list - b0);
        a.list = p.list ? p.list + b0 : nullptr;
        a.list_base = p.list ? 0 : b0;
        a.Mg = reinterpret_cast<df *>(p.scratch);
        a.flag = reinterpret_cast<int *>(reinterpret_cast<char *>(p.scratch) + sizeof(df) * (size_t)a.mstride * batch);
        cudaError_t e;
        switch (k) {
        case 5: e = launch_mixed_k<5>(a, p.num_sms, p.tc != 0, p.inv_tpr, s); break;
        case 6: e = launch_mixed_k<6>(a, p.num_sms, p.tc != 0, p.inv_tpr, s); break;
        case 7: e = launch_mixed_k<7>(a, p.num_sms, p.tc != 0, p.inv_tpr, s); break;
        default: e = launch_mixed_k<8>(a, p.num_sms, p.tc != 0, p.inv_tpr, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace labfm
