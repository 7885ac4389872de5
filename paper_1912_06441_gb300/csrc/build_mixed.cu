// Mixed-precision weight build.  Same method as build_fp64.cu (Eqs. disc_form, lsys, w_abf),
// with the arithmetic placed where GB300 has throughput:
//   - X and W of each neighbour are evaluated in FP64 (X stays in FP64 for the residual);
//   - M = sum_j X_j (outer) W_j and the partial-pivoting LU of M run in double-float
//     (pairs of FP32 on the FP32 pipes, ~48 bits), giving Psi~ and w~ = W . Psi~;
//   - then `nref` steps of iterative refinement on the polynomial-reproduction residual
//         r = C~ - sum_j X_j w~_j        (computed in FP64; Sec. 2.1: the moments of w must
//                                         equal the targets C)
//         w~ <- w~ + W . (LU^-1 r)       (correction solve in double-float).
// The targets are scaled per operator d by h^(l_d - |alpha|), l_d = highest degree with a
// non-zero entry of C^d, so that Psi~ stays within float range; the stored weight is
// w = h^-l_d w~, the same similarity transform as the FP64 build (exact in exact arithmetic).
#include <cmath>

#include "abf.cuh"
#include "df64.cuh"

namespace labfm {
namespace {

constexpr int MIX_THREADS = 256;

template <int K> struct MCfg {
    static constexpr int P = p_of_k(K);
    static constexpr int LDX = (P + 3) / 4 * 4;
    static constexpr int NB = K >= 7 ? 72 : 64;
    static constexpr int TM = 2, TN = 4;
    static constexpr int RG = (P + TM - 1) / TM, CG = (P + TN - 1) / TN;
    static_assert(RG * CG <= MIX_THREADS, "assembly tile grid exceeds the CTA");
    static constexpr int LDA = P + MAX_OPS + 1;
    // Xd (double) + Xf (df) + Wf (df, first written as double) + Af (df) + residual (double)
    static constexpr size_t smem_bytes = 8 * ((size_t)3 * NB * LDX + (size_t)P * LDA + (size_t)P * MAX_OPS);
};

struct MixedArgs {
    int64_t n_list;
    const int32_t *list;
    const double *xy;
    const double *h;
    const int64_t *row_ptr;
    const int32_t *col;
    int periodic;
    double L[2], halfL[2];
    int rbf;
    int n_ops;
    int nref;
    void *w;        // [nnz][n_ops] output
    int wdtype;
    double *wt;     // [nnz][n_ops] scratch: unscaled weights w~ in double
    int32_t *node_status;
    unsigned long long *n_bad;
    int lmax[MAX_OPS];  // l_d
    double C[MAX_OPS * PMAX];
};

template <int K>
__device__ __forceinline__ void stage_chunk(const MixedArgs &A, int64_t rs, int j0, int nj, double xi, double yi,
                                            double ihi, double *Xd, df *Xf, df *Wf)
{
    using C = MCfg<K>;
    constexpr int P = C::P, LDX = C::LDX;
    for (int t = threadIdx.x; t < nj; t += MIX_THREADS) {
        int j = A.col[rs + j0 + t];
        double dx = A.xy[2 * (int64_t)j] - xi, dy = A.xy[2 * (int64_t)j + 1] - yi;
        if (A.periodic) {
            if (dx > A.halfL[0]) dx -= A.L[0];
            else if (dx < -A.halfL[0]) dx += A.L[0];
            if (dy > A.halfL[1]) dy -= A.L[1];
            else if (dy < -A.halfL[1]) dy += A.L[1];
        }
        double *X = Xd + t * LDX;
        double *Wd = reinterpret_cast<double *>(Wf + t * LDX);
        eval_xw<K>(dx * ihi, dy * ihi, A.rbf, X, Wd);
#pragma unroll 4
        for (int e = 0; e < LDX; e++) {
            double xv = e < P ? X[e] : 0.0;
            double wv = e < P ? Wd[e] : 0.0;
            if (e >= P) X[e] = 0.0;
            Xf[t * LDX + e] = df_from_double(xv);
            Wf[t * LDX + e] = df_from_double(wv);  // in place: same 8 bytes
        }
    }
}

template <int K>
__global__ void __launch_bounds__(MIX_THREADS, 2) k_build_mixed(MixedArgs A)
{
    using C = MCfg<K>;
    constexpr int P = C::P, LDX = C::LDX, NB = C::NB, LDA = C::LDA, TM = C::TM, TN = C::TN;
    extern __shared__ __align__(16) double smem_d[];
    double *Xd = smem_d;                                          // [NB][LDX]
    df *Xf = reinterpret_cast<df *>(Xd + NB * LDX);               // [NB][LDX]
    df *Wf = Xf + NB * LDX;                                       // [NB][LDX]
    df *Af = Wf + NB * LDX;                                       // [P][LDA]
    double *Rd = reinterpret_cast<double *>(Af + P * LDA);        // [P][MAX_OPS] residual
    __shared__ int s_pivrow[P];
    __shared__ df s_invp[P];
    __shared__ double s_hneg[KMAX + 1], s_hpos[KMAX + 1];
    __shared__ int s_flag;

    const int tid = threadIdx.x;
    const int n_ops = A.n_ops;
    const int W_ = P + n_ops;
    const int rg = tid / C::CG, cg = tid % C::CG;
    const bool tile_active = tid < C::RG * C::CG;

    for (int64_t li = blockIdx.x; li < A.n_list; li += gridDim.x) {
        const int64_t i = A.list ? (int64_t)A.list[li] : li;
        const int64_t rs = A.row_ptr[i], re = A.row_ptr[i + 1];
        const int ni = (int)(re - rs);
        if (ni < P) {
            for (int64_t t = tid; t < (int64_t)ni * n_ops; t += MIX_THREADS) {
                if (A.wdtype == LABFM_F64) ((double *)A.w)[rs * n_ops + t] = 0.0;
                else ((float *)A.w)[rs * n_ops + t] = 0.0f;
            }
            if (tid == 0) {
                if (A.node_status) A.node_status[i] = LABFM_NODE_UNDERSAMPLED;
                atomicAdd(A.n_bad, 1ull);
            }
            continue;
        }
        const double xi = A.xy[2 * i], yi = A.xy[2 * i + 1], hi = A.h[i];
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

        // ---- assembly of M in double-float, 2 x 4 register tiles ----
        df acc[TM][TN];
#pragma unroll
        for (int a = 0; a < TM; a++)
#pragma unroll
            for (int b = 0; b < TN; b++) acc[a][b] = df{0.0f, 0.0f};
        const int nchunks = (ni + NB - 1) / NB;
        for (int ch = 0; ch < nchunks; ch++) {
            const int j0 = ch * NB, nj = min(NB, ni - j0);
            stage_chunk<K>(A, rs, j0, nj, xi, yi, ihi, Xd, Xf, Wf);
            __syncthreads();
            if (tile_active) {
                for (int j = 0; j < nj; j++) {
                    const df *X = Xf + j * LDX + rg * TM;
                    const df *W = Wf + j * LDX + cg * TN;
                    df xv[TM], wv[TN];
#pragma unroll
                    for (int a = 0; a < TM; a++) xv[a] = X[a];
                    float4 w01 = *reinterpret_cast<const float4 *>(W);
                    float4 w23 = *reinterpret_cast<const float4 *>(W + 2);
                    wv[0] = df{w01.x, w01.y};
                    wv[1] = df{w01.z, w01.w};
                    wv[2] = df{w23.x, w23.y};
                    wv[3] = df{w23.z, w23.w};
#pragma unroll
                    for (int a = 0; a < TM; a++)
#pragma unroll
                        for (int b = 0; b < TN; b++) acc[a][b] = df_fma(xv[a], wv[b], acc[a][b]);
                }
            }
            __syncthreads();
        }
        if (tile_active) {
            bool finite = true;
#pragma unroll
            for (int a = 0; a < TM; a++)
#pragma unroll
                for (int b = 0; b < TN; b++) {
                    int m = rg * TM + a, c = cg * TN + b;
                    if (m < P && c < P) {
                        Af[m * LDA + c] = acc[a][b];
                        finite &= df_isfinite(acc[a][b]);
                    }
                }
            if (!finite) atomicOr(&s_flag, 4);
        }
        // scaled targets C~_alpha = C_alpha h^(l_d - |alpha|)
        for (int t = tid; t < P * n_ops; t += MIX_THREADS) {
            int m = t / n_ops, d = t % n_ops;
            int deg = elem_degree(m);
            int l = A.lmax[d];
            double sc = l >= deg ? s_hpos[l - deg] : s_hneg[deg - l];
            Af[m * LDA + P + d] = df_from_double(A.C[d * PMAX + m] * sc);
        }
        __syncthreads();
        const bool bad_m = (s_flag & 4) != 0;

        // ---- LU with partial pivoting (whole-row swaps, so the factors can be reused) ----
        for (int c = 0; c < P && !bad_m; c++) {
            if (tid < 32) {
                float best = -1.0f;
                int br = c;
                for (int r = c + tid; r < P; r += 32) {
                    float v = df_abs_hi(Af[r * LDA + c]);
                    if (v > best) {
                        best = v;
                        br = r;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    float ob = __shfl_xor_sync(0xffffffffu, best, o);
                    int orr = __shfl_xor_sync(0xffffffffu, br, o);
                    if (ob > best || (ob == best && orr < br)) {
                        best = ob;
                        br = orr;
                    }
                }
                if (tid == 0) {
                    s_pivrow[c] = br;
                    df pv = Af[br * LDA + c];
                    if (!(best > 0.0f) || !isfinite(best)) {
                        s_flag |= 1;
                        s_invp[c] = df{0.0f, 0.0f};
                    } else {
                        s_invp[c] = df_recip(pv);
                    }
                }
            }
            __syncthreads();
            const int pr = s_pivrow[c];
            if (pr != c) {
                for (int t = tid; t < W_; t += MIX_THREADS) {
                    df a = Af[c * LDA + t];
                    Af[c * LDA + t] = Af[pr * LDA + t];
                    Af[pr * LDA + t] = a;
                }
                __syncthreads();
            }
            const df inv = s_invp[c];
            for (int r = c + 1 + tid; r < P; r += MIX_THREADS) Af[r * LDA + c] = df_mul(Af[r * LDA + c], inv);
            __syncthreads();
            const int nr = P - c - 1, nc = W_ - c - 1;
            for (int t = tid; t < nr * nc; t += MIX_THREADS) {
                int r = c + 1 + t / nc, q = c + 1 + t % nc;
                Af[r * LDA + q] = df_fms(Af[r * LDA + c], Af[c * LDA + q], Af[r * LDA + q]);
            }
            __syncthreads();
        }
        // back substitution: Psi~ in columns P..P+n_ops
        for (int c = P - 1; c >= 0 && !bad_m; c--) {
            if (tid < n_ops) Af[c * LDA + P + tid] = df_mul(Af[c * LDA + P + tid], s_invp[c]);
            __syncthreads();
            for (int t = tid; t < c * n_ops; t += MIX_THREADS) {
                int r = t / n_ops, d = t % n_ops;
                Af[r * LDA + P + d] = df_fms(Af[r * LDA + c], Af[c * LDA + P + d], Af[r * LDA + P + d]);
            }
            __syncthreads();
        }
        const bool failed = (s_flag & 5) != 0;

        // ---- w~ = W . Psi~ (double-float), then refinement steps ----
        for (int it = 0; it <= A.nref && !failed; it++) {
            // (it == 0: Psi~ in the RHS columns;  it > 0: correction dPsi in the RHS columns)
            for (int ch = 0; ch < nchunks; ch++) {
                const int j0 = ch * NB, nj = min(NB, ni - j0);
                if (nchunks > 1) {
                    stage_chunk<K>(A, rs, j0, nj, xi, yi, ihi, Xd, Xf, Wf);
                    __syncthreads();
                }
                for (int t = tid; t < nj * n_ops; t += MIX_THREADS) {
                    int j = t / n_ops, d = t % n_ops;
                    df s = df{0.0f, 0.0f};
                    const df *W = Wf + j * LDX;
#pragma unroll 4
                    for (int m = 0; m < P; m++) s = df_fma(W[m], Af[m * LDA + P + d], s);
                    int64_t idx = (rs + j0 + j) * n_ops + d;
                    double v = df_to_double(s);
                    A.wt[idx] = it == 0 ? v : A.wt[idx] + v;
                }
                __syncthreads();
            }
            if (it == A.nref) break;
            // residual r = C~ - sum_j X_j w~_j in FP64 (thread per (alpha, d))
            for (int t = tid; t < P * n_ops; t += MIX_THREADS) {
                int m = t / n_ops, d = t % n_ops;
                int deg = elem_degree(m);
                int l = A.lmax[d];
                double sc = l >= deg ? s_hpos[l - deg] : s_hneg[deg - l];
                Rd[m * MAX_OPS + d] = A.C[d * PMAX + m] * sc;
            }
            for (int ch = 0; ch < nchunks; ch++) {
                const int j0 = ch * NB, nj = min(NB, ni - j0);
                if (nchunks > 1) {
                    __syncthreads();
                    stage_chunk<K>(A, rs, j0, nj, xi, yi, ihi, Xd, Xf, Wf);
                }
                __syncthreads();
                for (int t = tid; t < P * n_ops; t += MIX_THREADS) {
                    int m = t / n_ops, d = t % n_ops;
                    double s = Rd[m * MAX_OPS + d];
                    for (int j = 0; j < nj; j++) s = fma(-Xd[j * LDX + m], A.wt[(rs + j0 + j) * n_ops + d], s);
                    Rd[m * MAX_OPS + d] = s;
                }
            }
            __syncthreads();
            // correction solve with the stored factors: row swaps, unit-lower L, then U
            for (int t = tid; t < P * n_ops; t += MIX_THREADS) {
                int m = t / n_ops, d = t % n_ops;
                Af[m * LDA + P + d] = df_from_double(Rd[m * MAX_OPS + d]);
            }
            __syncthreads();
            if (tid < n_ops) {
                for (int c = 0; c < P; c++) {
                    int pr = s_pivrow[c];
                    if (pr != c) {
                        df a = Af[c * LDA + P + tid];
                        Af[c * LDA + P + tid] = Af[pr * LDA + P + tid];
                        Af[pr * LDA + P + tid] = a;
                    }
                }
            }
            __syncthreads();
            for (int c = 0; c < P - 1; c++) {
                for (int t = tid; t < (P - c - 1) * n_ops; t += MIX_THREADS) {
                    int r = c + 1 + t / n_ops, d = t % n_ops;
                    Af[r * LDA + P + d] = df_fms(Af[r * LDA + c], Af[c * LDA + P + d], Af[r * LDA + P + d]);
                }
                __syncthreads();
            }
            for (int c = P - 1; c >= 0; c--) {
                if (tid < n_ops) Af[c * LDA + P + tid] = df_mul(Af[c * LDA + P + tid], s_invp[c]);
                __syncthreads();
                for (int t = tid; t < c * n_ops; t += MIX_THREADS) {
                    int r = t / n_ops, d = t % n_ops;
                    Af[r * LDA + P + d] = df_fms(Af[r * LDA + c], Af[c * LDA + P + d], Af[r * LDA + P + d]);
                }
                __syncthreads();
            }
        }

        // ---- physical weights w = h^-l_d w~ ----
        for (int64_t t = tid; t < (int64_t)ni * n_ops; t += MIX_THREADS) {
            int d = (int)(t % n_ops);
            double v = failed ? 0.0 : A.wt[rs * n_ops + t] * s_hneg[A.lmax[d]];
            if (!isfinite(v)) {
                atomicOr(&s_flag, 2);
                v = 0.0;
            }
            if (A.wdtype == LABFM_F64) ((double *)A.w)[rs * n_ops + t] = v;
            else ((float *)A.w)[rs * n_ops + t] = (float)v;
        }
        __syncthreads();
        const int flag = s_flag;
        if ((flag & 2) && !failed) {
            for (int64_t t = tid; t < (int64_t)ni * n_ops; t += MIX_THREADS) {
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
        __syncthreads();
    }
}

template <int K>
cudaError_t launch_mixed_k(const MixedArgs &a, int num_sms, cudaStream_t s)
{
    using C = MCfg<K>;
    cudaError_t e = cudaFuncSetAttribute(k_build_mixed<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::smem_bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_mixed<K>, MIX_THREADS, C::smem_bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = std::min<int64_t>(a.n_list, (int64_t)num_sms * per_sm);
    if (grid < 1) return cudaSuccess;
    k_build_mixed<K><<<(unsigned)grid, MIX_THREADS, C::smem_bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_build_mixed(int k, const MixedArgsPublic &p, cudaStream_t s)
{
    MixedArgs a{};
    a.n_list = p.n_list;
    a.list = p.list;
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
    a.w = p.w;
    a.wdtype = p.wdtype;
    a.wt = p.wt;
    a.node_status = p.node_status;
    a.n_bad = p.n_bad;
    for (int d = 0; d < MAX_OPS; d++) a.lmax[d] = p.lmax[d];
    for (int t = 0; t < MAX_OPS * PMAX; t++) a.C[t] = p.C[t];
    switch (k) {
    case 1: return launch_mixed_k<1>(a, p.num_sms, s);
    case 2: return launch_mixed_k<2>(a, p.num_sms, s);
    case 3: return launch_mixed_k<3>(a, p.num_sms, s);
    case 4: return launch_mixed_k<4>(a, p.num_sms, s);
    case 5: return launch_mixed_k<5>(a, p.num_sms, s);
    case 6: return launch_mixed_k<6>(a, p.num_sms, s);
    case 7: return launch_mixed_k<7>(a, p.num_sms, s);
    default: return launch_mixed_k<8>(a, p.num_sms, s);
    }
}

}  // namespace labfm
