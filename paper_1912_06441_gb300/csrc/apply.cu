// Operator application (Eq. general_do) and the RK4 driver (Sec. 5.1).
//
// Both are streaming gather-sums over the CSR stencils: per stencil entry e of node i, read
// col[e] and the weights w[e][*] once (HBM), gather f[col[e]] (stays in L2: the field is
// small next to the weight stream and nodes are numbered in spatial order), and accumulate
// (f_j - f_i) w.  A group of G lanes shares one node: the lanes read consecutive entries, so
// every weight and index load of a warp is a contiguous, fully used segment; UNR entries per
// lane are in flight before the first use.  The partial sums of a group are combined with
// shuffles: by a reduce-scatter over the operators in the apply (each lane ends with one
// operator's sum), by a butterfly tree in the RK4 and Burgers stages.
//
// (G, UNR) is chosen per context by a small autotuner: the first apply (or RK4 run) for a
// given operator count, data types and problem class times every shape once on the real
// stencils and keeps the fastest.
#include <cmath>
#include <type_traits>

#include "df64.cuh"
#include "labfm_internal.cuh"

namespace labfm {
namespace {

constexpr int APPLY_THREADS = 256;

// Weights of entry e (NOPS of them) into wv[], converted to the accumulation type.
template <int NOPS, class WT, class AT>
__device__ __forceinline__ void load_w(const WT *__restrict__ w, int64_t e, AT *wv)
{
    const WT *p = w + e * NOPS;
    if constexpr (NOPS == 4 && sizeof(WT) == 8) {
        double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
        double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
        wv[0] = (AT)a.x; wv[1] = (AT)a.y; wv[2] = (AT)b.x; wv[3] = (AT)b.y;
    } else if constexpr (NOPS == 4 && sizeof(WT) == 4) {
        float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
        wv[0] = (AT)a.x; wv[1] = (AT)a.y; wv[2] = (AT)a.z; wv[3] = (AT)a.w;
    } else if constexpr (NOPS == 2 && sizeof(WT) == 8) {
        double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
        wv[0] = (AT)a.x; wv[1] = (AT)a.y;
    } else {
#pragma unroll
        for (int d = 0; d < NOPS; d++) wv[d] = (AT)__ldcs(p + d);
    }
}

template <class FT, class WT>
using acc_t = typename std::conditional<std::is_same<FT, float>::value && std::is_same<WT, float>::value, float,
                                        double>::type;

// out[sel(d)][i] = sum_j (f_j - f_i) w_ji^d for the operators in mask.
template <int NOPS, class FT, class WT, int UNR>
__global__ void __launch_bounds__(APPLY_THREADS) k_apply(int64_t n, const int64_t *__restrict__ row_ptr,
                                                         const int32_t *__restrict__ col, const WT *__restrict__ w,
                                                         const FT *__restrict__ f, FT *__restrict__ out, uint32_t mask,
                                                         int lg_g)
{
    using AT = acc_t<FT, WT>;
    const int G = 1 << lg_g;  // lanes per node, a power of two
    const int lane = threadIdx.x & (G - 1);
    const int64_t i = ((int64_t)blockIdx.x * APPLY_THREADS + threadIdx.x) >> lg_g;
    const bool live = i < n;
    int64_t rs = 0, re = 0;
    AT fi = 0;
    if (live) {
        rs = row_ptr[i];
        re = row_ptr[i + 1];
        fi = (AT)__ldg(f + i);
    }
    AT acc[NOPS];
#pragma unroll
    for (int d = 0; d < NOPS; d++) acc[d] = 0;
    for (int64_t base = rs; base < re; base += (int64_t)G * UNR) {
        int cj[UNR];
        AT wv[UNR][NOPS];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            int64_t e = base + (int64_t)u * G + lane;
            if (e < re) {
                cj[u] = __ldcs(col + e);
                load_w<NOPS>(w, e, wv[u]);
            } else {
                cj[u] = -1;
#pragma unroll
                for (int d = 0; d < NOPS; d++) wv[u][d] = 0;
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            if (cj[u] >= 0) {
                AT df = (AT)__ldg(f + cj[u]) - fi;
#pragma unroll
                for (int d = 0; d < NOPS; d++) acc[d] = fma(df, wv[u][d], acc[d]);
            }
        }
    }
    // Reduce-scatter over the node's G lanes (G >= NP, NOPS padded to the power of two NP): at
    // offsets G/2, G/4, ... each lane keeps one half of its operators and adds the partner's
    // half, until it holds one operator's partial, d = lane / (G / NP); the remaining offsets
    // add that one value.  NP - 1 + log2(G / NP) adds per lane instead of NOPS log2(G) (FP64
    // adds are scarce), in a fixed order.
    constexpr int NP = NOPS <= 1 ? 1 : NOPS <= 2 ? 2 : NOPS <= 4 ? 4 : 8;
    AT v[NP];
#pragma unroll
    for (int d = 0; d < NP; d++) v[d] = d < NOPS ? acc[d] : (AT)0;
    int o = G >> 1;
#pragma unroll
    for (int m = NP; m > 1; m >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < m / 2; j++) {
            const AT send = upper ? v[j] : v[j + m / 2];
            const AT keep = upper ? v[j + m / 2] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    for (; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    const int per = G / NP;  // lanes holding the same operator's sum
    const int d = lane / per;
    if (live && (lane & (per - 1)) == 0 && d < NOPS && ((mask >> d) & 1u)) {
        const int row = __popc(mask & ((1u << d) - 1u));
        out[(int64_t)row * n + i] = (FT)v[0];
    }
}

// Storage of the combined RK4 weight wc_ji = sum_d beta_d w_ji^d (a context-owned buffer):
//   CW_F64  double                    FP64 weights, FP64 fields: accumulated in double (the
//                                     stencil indices are read from the CSR)
//   CW_F32  int2 (j, w)               FP32 weights: each entry's stencil index and weight as one
//                                     8-byte word, accumulated in the field type
//   CW_DF   int2 (j, hi), float lo    FP64 weights, FP32 fields: the double rounded to a
//                                     double-float pair once, here, so that the stage
//                                     accumulates on the FP32 pipes (about 48 bits, far below the
//                                     FP32 field rounding) instead of converting and multiplying
//                                     in FP64 for every stencil entry; the low parts follow the
//                                     nnz index/high-part words
// Packing the index with the weight gives one wide load per entry for the same bytes.
enum { CW_F64 = 0, CW_F32 = 1, CW_DF = 2 };

int cw_format(int fdt, int wdt) { return wdt == LABFM_F32 ? CW_F32 : (fdt == LABFM_F32 ? CW_DF : CW_F64); }
size_t cw_bytes(int fmt) { return fmt == CW_DF ? 12 : 8; }

template <class WT>
__global__ void k_combine(int64_t nnz, int n_ops, const WT *__restrict__ w, const int32_t *__restrict__ col,
                          void *__restrict__ wc, int fmt, double b0, double b1, double b2, double b3, double b4,
                          double b5, double b6, double b7)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const double b[8] = {b0, b1, b2, b3, b4, b5, b6, b7};
    double s = 0.0;
    for (int d = 0; d < n_ops; d++) s = fma(b[d], (double)w[e * n_ops + d], s);
    if (fmt == CW_F64) {
        ((double *)wc)[e] = s;
    } else if (fmt == CW_F32) {
        ((int2 *)wc)[e] = make_int2(col[e], __float_as_int((float)s));
    } else {
        df v = df_from_double(s);
        ((int2 *)wc)[e] = make_int2(col[e], __float_as_int(v.hi));
        ((float *)((int2 *)wc + nnz))[e] = v.lo;
    }
}

// One RK4 stage.  F_i = sum_j (src_j - src_i) wc_ji (0 on frozen nodes), then
//   stage 0: acc = u + dt/6 F,  nxt = u + dt/2 F
//   stage 1: acc += dt/3 F,     nxt = u + dt/2 F
//   stage 2: acc += dt/3 F,     nxt = u + dt F
//   stage 3: u = acc + dt/6 F
// The per-node update runs in the field type.
template <class FT, int CW, int UNR>
__global__ void __launch_bounds__(APPLY_THREADS) k_rk4_stage(int64_t n, const int64_t *__restrict__ row_ptr,
                                                             const int32_t *__restrict__ col,
                                                             const void *__restrict__ wc_raw,
                                                             const float *__restrict__ wc_lo,
                                                             const FT *__restrict__ src, FT *__restrict__ u,
                                                             FT *__restrict__ acc_buf, FT *__restrict__ nxt,
                                                             const uint8_t *__restrict__ frozen, int stage, FT dt,
                                                             int lg_g)
{
    // AT: type of the stencil sum (double-float for CW_DF); the per-node update runs in FT
    using AT = typename std::conditional<std::is_same<FT, float>::value && CW != CW_F64, float, double>::type;
    using WT = typename std::conditional<CW == CW_F64, double, float2>::type;  // (weight, low part)
    const double *__restrict__ wcd = (const double *)wc_raw;
    const int2 *__restrict__ wcp = (const int2 *)wc_raw;
    const int G = 1 << lg_g;  // lanes per node, a power of two
    const int lane = threadIdx.x & (G - 1);
    const int64_t i = ((int64_t)blockIdx.x * APPLY_THREADS + threadIdx.x) >> lg_g;
    const bool live = i < n;
    int64_t rs = 0, re = 0;
    FT si = 0;
    if (live) {
        rs = row_ptr[i];
        re = row_ptr[i + 1];
        si = src[i];
    }
    AT acc = 0;
    df accd{0.0f, 0.0f};
    // FP32 weights: the stencil stream is software-pipelined (the next batch of UNR entries per
    // lane is loaded before the gathers of the current one, so its latency overlaps them: +8 % at
    // 2048^2); with double-float weights the second batch's registers cost more than the overlap
    // gains (-11 %), so those load each batch just before its gathers
    constexpr bool PIPE = CW == CW_F32;
    int cn[UNR];
    WT wn[UNR];
    auto load_batch = [&](int64_t base) {
#pragma unroll
        for (int q = 0; q < UNR; q++) {
            const int64_t e = base + (int64_t)q * G + lane;
            if (e < re) {
                if constexpr (CW == CW_F64) {
                    cn[q] = __ldcs(col + e);
                    wn[q] = __ldcs(wcd + e);
                } else {
                    const int2 pr = __ldcs(wcp + e);  // stencil index and (high part of the) weight
                    cn[q] = pr.x;
                    wn[q] = make_float2(__int_as_float(pr.y), CW == CW_DF ? __ldcs(wc_lo + e) : 0.0f);
                }
            } else {
                cn[q] = -1;
            }
        }
    };
    if (PIPE && rs < re) load_batch(rs);
    for (int64_t base = rs; base < re; base += (int64_t)G * UNR) {
        if (!PIPE) load_batch(base);
        int cj[UNR];
        WT wv[UNR];
#pragma unroll
        for (int q = 0; q < UNR; q++) {
            cj[q] = cn[q];
            wv[q] = wn[q];
        }
        if (PIPE && base + (int64_t)G * UNR < re) load_batch(base + (int64_t)G * UNR);
#pragma unroll
        for (int q = 0; q < UNR; q++) {
            if (cj[q] >= 0) {
                if constexpr (CW == CW_DF) {
                    float dh, dl;  // src_j - src_i exactly, as a double-float
                    two_sum((float)src[cj[q]], -(float)si, dh, dl);
                    accd = df_fma(df{dh, dl}, df{wv[q].x, wv[q].y}, accd);
                } else if constexpr (CW == CW_F32) {
                    acc = fma((AT)src[cj[q]] - (AT)si, (AT)wv[q].x, acc);
                } else {
                    acc = fma((AT)src[cj[q]] - (AT)si, (AT)wv[q], acc);
                }
            }
        }
    }
    if constexpr (CW == CW_DF) {
        for (int o = G >> 1; o > 0; o >>= 1) {
            df other{__shfl_xor_sync(0xffffffffu, accd.hi, o), __shfl_xor_sync(0xffffffffu, accd.lo, o)};
            accd = df_add(accd, other);
        }
        acc = accd.hi + accd.lo;  // CW_DF comes with FP32 fields
    } else {
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    }
    if (!live || lane != 0) return;
    const FT F = (frozen && frozen[i]) ? (FT)0 : (FT)acc;
    const FT ui = u[i];
    switch (stage) {
    case 0:
        acc_buf[i] = ui + dt * (FT)(1.0 / 6.0) * F;
        nxt[i] = ui + dt * (FT)0.5 * F;
        break;
    case 1:
        acc_buf[i] = acc_buf[i] + dt * (FT)(1.0 / 3.0) * F;
        nxt[i] = ui + dt * (FT)0.5 * F;
        break;
    case 2:
        acc_buf[i] = acc_buf[i] + dt * (FT)(1.0 / 3.0) * F;
        nxt[i] = ui + dt * F;
        break;
    default:
        u[i] = acc_buf[i] + dt * (FT)(1.0 / 6.0) * F;
        break;
    }
}

// ---------------------------------------------------------------------------------------------
// Launch shapes and the autotuner
// ---------------------------------------------------------------------------------------------
struct Shape {
    int G, UNR;
};

// default shape: enough lanes that UNR entries per lane cover an average stencil
Shape default_shape(const labfm_ctx *ctx, int min_g)
{
    double avg = ctx->n > 0 ? (double)ctx->nnz / (double)ctx->n : 0.0;
    int G = 4;
    while (G < 32 && G * 4 < avg) G *= 2;
    if (G < min_g) G = min_g;
    return Shape{G, 4};
}

unsigned blocks_for(int64_t n, int G) { return (unsigned)((n * G + APPLY_THREADS - 1) / APPLY_THREADS); }
int log2_of(int G)
{
    int l = 0;
    while ((1 << l) < G) l++;
    return l;
}

template <int NOPS, class FT, class WT>
cudaError_t launch_apply_shape(labfm_ctx *ctx, Shape sh, uint32_t mask, const void *f, void *out, cudaStream_t s)
{
    const unsigned blocks = blocks_for(ctx->n, sh.G);
    auto args = [&](auto kern) {
        kern<<<blocks, APPLY_THREADS, 0, s>>>(ctx->n, ctx->row_ptr.as<int64_t>(), ctx->col.as<int32_t>(),
                                              (const WT *)ctx->w.ptr, (const FT *)f, (FT *)out, mask, log2_of(sh.G));
    };
    switch (sh.UNR) {
    case 2: args(k_apply<NOPS, FT, WT, 2>); break;
    case 8: args(k_apply<NOPS, FT, WT, 8>); break;
    default: args(k_apply<NOPS, FT, WT, 4>); break;
    }
    return cudaGetLastError();
}

template <class FT, int CW>
cudaError_t launch_stage_shape(labfm_ctx *ctx, Shape sh, const FT *src, FT *u, FT *acc, FT *nxt, const uint8_t *frozen,
                               int stage, double dt, cudaStream_t s)
{
    const unsigned blocks = blocks_for(ctx->n, sh.G);
    const void *wc = ctx->wcomb.ptr;
    const float *wc_lo = CW == CW_DF ? reinterpret_cast<const float *>(ctx->wcomb.as<int2>() + ctx->nnz) : nullptr;
    auto args = [&](auto kern) {
        kern<<<blocks, APPLY_THREADS, 0, s>>>(ctx->n, ctx->row_ptr.as<int64_t>(), ctx->col.as<int32_t>(), wc, wc_lo,
                                              src, u, acc, nxt, frozen, stage, (FT)dt, log2_of(sh.G));
    };
    switch (sh.UNR) {
    case 2: args(k_rk4_stage<FT, CW, 2>); break;
    case 8: args(k_rk4_stage<FT, CW, 8>); break;
    default: args(k_rk4_stage<FT, CW, 4>); break;
    }
    return cudaGetLastError();
}

// Time every shape with `run` (which enqueues one launch on ctx->stream) and keep the fastest.
template <class RunFn>
cudaError_t autotune(labfm_ctx *ctx, uint64_t key, int min_g, RunFn run, Shape &best)
{
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
        best = Shape{(int)(it->second >> 8), (int)(it->second & 0xff)};
        return cudaSuccess;
    }
    best = default_shape(ctx, min_g);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(ctx->stream, &cap);
    if (ce != cudaSuccess) return ce;
    if (cap != cudaStreamCaptureStatusNone) return cudaSuccess;  // caller is recording a graph: no timing
    if (ctx->n < 4096) {  // too small to time meaningfully
        ctx->tuned[key] = ((uint32_t)best.G << 8) | (uint32_t)best.UNR;
        return cudaSuccess;
    }
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    float best_ms = 1e30f;
    const int gs[4] = {4, 8, 16, 32}, us[3] = {2, 4, 8};
    for (int gi = 0; gi < 4 && e == cudaSuccess; gi++) {
        for (int ui = 0; ui < 3 && e == cudaSuccess; ui++) {
            Shape sh{gs[gi], us[ui]};
            if (sh.G < min_g) continue;
            e = run(sh);  // warm-up
            if (e != cudaSuccess) break;
            cudaEventRecord(e0, ctx->stream);
            e = run(sh);
            cudaEventRecord(e1, ctx->stream);
            if (e != cudaSuccess) break;
            e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best = sh;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) ctx->tuned[key] = ((uint32_t)best.G << 8) | (uint32_t)best.UNR;
    return e;
}

// Shapes are tuned per kind of launch, data types and problem class: floor(log2 n) and the mean
// stencil size rounded to an integer, so that rebuilding stencils of the same kind (a moving node
// set, a bench repetition) reuses the choice instead of timing again.
uint64_t tune_key(const labfm_ctx *ctx, int kind, int nops, int fdt, int wdt)
{
    uint64_t lg = 0;
    while (lg < 62 && ((int64_t)1 << (lg + 1)) <= ctx->n) lg++;
    uint64_t deg = ctx->n > 0 ? (uint64_t)((double)ctx->nnz / (double)ctx->n + 0.5) : 0;
    if (deg > 0xffff) deg = 0xffff;
    return (deg << 40) | (lg << 32) | ((uint64_t)kind << 24) | ((uint64_t)nops << 16) | ((uint64_t)fdt << 8) |
           (uint64_t)wdt;
}

template <int NOPS, class FT, class WT>
cudaError_t launch_apply_t(labfm_ctx *ctx, uint32_t mask, const void *f, int fdt, void *out)
{
    const int min_g = NOPS <= 4 ? 4 : 8;  // the reduce-scatter needs G >= NOPS rounded up to 2^k
    Shape sh;
    cudaError_t e = autotune(
        ctx, tune_key(ctx, 1, NOPS, fdt, ctx->wdtype), min_g,
        [&](Shape s) { return launch_apply_shape<NOPS, FT, WT>(ctx, s, mask, f, out, ctx->stream); }, sh);
    if (e != cudaSuccess) return e;
    return launch_apply_shape<NOPS, FT, WT>(ctx, sh, mask, f, out, ctx->stream);
}

template <int NOPS>
cudaError_t launch_apply_n(labfm_ctx *ctx, uint32_t mask, const void *f, int fdt, void *out)
{
    if (ctx->wdtype == LABFM_F64)
        return fdt == LABFM_F64 ? launch_apply_t<NOPS, double, double>(ctx, mask, f, fdt, out)
                                : launch_apply_t<NOPS, float, double>(ctx, mask, f, fdt, out);
    return fdt == LABFM_F64 ? launch_apply_t<NOPS, double, float>(ctx, mask, f, fdt, out)
                            : launch_apply_t<NOPS, float, float>(ctx, mask, f, fdt, out);
}

template <class FT, int CW>
cudaError_t enqueue_steps(labfm_ctx *ctx, void *u, int fdt, double dt, int64_t nsteps, const uint8_t *frozen,
                          cudaStream_t s)
{
    FT *uu = (FT *)u, *acc = ctx->rk_acc.as<FT>(), *sa = ctx->rk_stage_a.as<FT>(), *sb = ctx->rk_stage_b.as<FT>();
    // tune on stage 0, which reads u and writes only the work buffers
    Shape sh;
    cudaError_t e = autotune(
        ctx, tune_key(ctx, 2, 1, fdt, ctx->wdtype), 1,
        [&](Shape sp) { return launch_stage_shape<FT, CW>(ctx, sp, uu, uu, acc, sa, frozen, 0, dt, ctx->stream); },
        sh);
    if (e != cudaSuccess) return e;
    for (int64_t st = 0; st < nsteps; st++) {
        if ((e = launch_stage_shape<FT, CW>(ctx, sh, uu, uu, acc, sa, frozen, 0, dt, s)) != cudaSuccess) return e;
        if ((e = launch_stage_shape<FT, CW>(ctx, sh, sa, uu, acc, sb, frozen, 1, dt, s)) != cudaSuccess) return e;
        if ((e = launch_stage_shape<FT, CW>(ctx, sh, sb, uu, acc, sa, frozen, 2, dt, s)) != cudaSuccess) return e;
        if ((e = launch_stage_shape<FT, CW>(ctx, sh, sa, uu, acc, (FT *)nullptr, frozen, 3, dt, s)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_steps_dt(labfm_ctx *ctx, int fdt, void *u, double dt, int64_t nsteps, const uint8_t *frozen,
                             cudaStream_t s)
{
    switch (cw_format(fdt, ctx->wdtype)) {
    case CW_F64: return enqueue_steps<double, CW_F64>(ctx, u, fdt, dt, nsteps, frozen, s);
    case CW_DF: return enqueue_steps<float, CW_DF>(ctx, u, fdt, dt, nsteps, frozen, s);
    default:
        return fdt == LABFM_F64 ? enqueue_steps<double, CW_F32>(ctx, u, fdt, dt, nsteps, frozen, s)
                                : enqueue_steps<float, CW_F32>(ctx, u, fdt, dt, nsteps, frozen, s);
    }
}

}  // namespace

cudaError_t launch_apply(labfm_ctx *ctx, uint32_t mask, const void *f, int fdt, void *out)
{
    switch (ctx->n_ops) {
    case 1: return launch_apply_n<1>(ctx, mask, f, fdt, out);
    case 2: return launch_apply_n<2>(ctx, mask, f, fdt, out);
    case 3: return launch_apply_n<3>(ctx, mask, f, fdt, out);
    case 4: return launch_apply_n<4>(ctx, mask, f, fdt, out);
    case 5: return launch_apply_n<5>(ctx, mask, f, fdt, out);
    case 6: return launch_apply_n<6>(ctx, mask, f, fdt, out);
    case 7: return launch_apply_n<7>(ctx, mask, f, fdt, out);
    default: return launch_apply_n<8>(ctx, mask, f, fdt, out);
    }
}

labfm_status run_step(labfm_ctx *ctx, const double *beta, void *u, int fdt, double dt, int64_t nsteps,
                      const uint8_t *frozen)
{
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n, nnz = ctx->nnz;
    size_t fsz = fdt == LABFM_F64 ? 8 : 4;
    const int fmt = cw_format(fdt, ctx->wdtype);
    // combined weight, cached while beta, the weights and the storage format are unchanged
    bool same_beta = ctx->wcomb_valid && ctx->wcomb_dtype == fmt;
    for (int d = 0; d < ctx->n_ops && same_beta; d++) same_beta = (ctx->beta_cached[d] == beta[d]);
    if (!same_beta) {
        LABFM_CUDA_TRY(ctx, ctx->wcomb.reserve(cw_bytes(fmt) * (nnz > 0 ? nnz : 1)));
        double b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int d = 0; d < ctx->n_ops; d++) b[d] = beta[d];
        unsigned blocks = (unsigned)((nnz + 255) / 256);
        if (nnz > 0) {
            if (ctx->wdtype == LABFM_F64)
                k_combine<double><<<blocks, 256, 0, s>>>(nnz, ctx->n_ops, ctx->w.as<double>(), ctx->col.as<int32_t>(),
                                                         ctx->wcomb.ptr, fmt,
                                                         b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7]);
            else
                k_combine<float><<<blocks, 256, 0, s>>>(nnz, ctx->n_ops, ctx->w.as<float>(), ctx->col.as<int32_t>(),
                                                        ctx->wcomb.ptr, fmt,
                                                        b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7]);
            LABFM_CUDA_TRY(ctx, cudaGetLastError());
        }
        for (int d = 0; d < ctx->n_ops; d++) ctx->beta_cached[d] = beta[d];
        ctx->wcomb_valid = true;
        ctx->wcomb_dtype = fmt;
    }
    LABFM_CUDA_TRY(ctx, ctx->rk_acc.reserve(fsz * n));
    LABFM_CUDA_TRY(ctx, ctx->rk_stage_a.reserve(fsz * n));
    LABFM_CUDA_TRY(ctx, ctx->rk_stage_b.reserve(fsz * n));

    StepGraph &g = ctx->graph;
    const bool same = g.exec && g.u == u && g.frozen == frozen && g.dtype == fdt && g.dt == dt &&
                      g.nsteps == nsteps && g.n == n && g.nnz == nnz && g.wdtype == ctx->wdtype &&
                      g.row_ptr == ctx->row_ptr.ptr && g.col == ctx->col.ptr && g.wc == ctx->wcomb.ptr &&
                      g.acc == ctx->rk_acc.ptr && g.sa == ctx->rk_stage_a.ptr && g.sb == ctx->rk_stage_b.ptr;
    if (!same) {
        g.release();
        if (!ctx->capture_stream) {
            LABFM_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        }
        // the capture stream must see the combined weights (enqueued on the context stream)
        LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        cudaGraph_t graph = nullptr;
        // shapes are tuned (on the context stream) before the capture begins
        {
            cudaError_t te = enqueue_steps_dt(ctx, fdt, u, dt, 0, frozen, s);
            if (te != cudaSuccess) return cuda_fail(ctx, te, "RK4 stage tuning");
            // the capture stream must not start before the tuning launches end
            LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        }
        LABFM_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_steps_dt(ctx, fdt, u, dt, nsteps, frozen, ctx->capture_stream);
        cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(ctx, e, "RK4 stage capture");
        }
        LABFM_CUDA_TRY(ctx, e2);
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return cuda_fail(ctx, e, "cudaGraphInstantiate");
        }
        g.u = u;
        g.frozen = frozen;
        g.dtype = fdt;
        g.dt = dt;
        g.nsteps = nsteps;
        g.n = n;
        g.nnz = nnz;
        g.wdtype = ctx->wdtype;
        g.row_ptr = ctx->row_ptr.ptr;
        g.col = ctx->col.ptr;
        g.wc = ctx->wcomb.ptr;
        g.acc = ctx->rk_acc.ptr;
        g.sa = ctx->rk_stage_a.ptr;
        g.sb = ctx->rk_stage_b.ptr;
    }
    LABFM_CUDA_TRY(ctx, cudaGraphLaunch(g.exec, s));
    return LABFM_OK;
}

}  // namespace labfm

// ---------------------------------------------------------------------------------------------
// Burgers' equation (Sec. 5.3, eq. burgers): du/dt = -(u d/dx + v d/dy) u + sum_{d>=2} beta_d L^d u,
// and the same for v, by the classical RK4 scheme.  The advection coefficients depend on the
// field, so d/dx and d/dy stay separate sums; the linear operators combine into one weight.
// ---------------------------------------------------------------------------------------------
namespace labfm {
namespace {

// per entry: (w^0, w^1, sum_{d>=2} beta_d w^d), the last summed in double
template <class WT>
__global__ void k_burg_combine(int64_t nnz, int n_ops, const WT *__restrict__ w, WT *__restrict__ wb, double b2,
                               double b3, double b4, double b5, double b6, double b7)
{
    const double bb[6] = {b2, b3, b4, b5, b6, b7};
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const WT *we = w + e * n_ops;
        double s = 0.0;
        for (int d = 2; d < n_ops; d++) s += bb[d - 2] * (double)we[d];
        wb[3 * e] = we[0];
        wb[3 * e + 1] = we[1];
        wb[3 * e + 2] = (WT)s;
    }
}

// One RK4 stage for the pair (u, v).  With the stage's source fields (su, sv):
//   A_x(s)_i = sum_j (s_j - s_i) w^0,  A_y(s)_i = sum_j (s_j - s_i) w^1,  B(s)_i = sum_j (s_j - s_i) wl
//   F_u = -(su_i A_x(su) + sv_i A_y(su)) + B(su),   F_v = -(su_i A_x(sv) + sv_i A_y(sv)) + B(sv)
// (0 on frozen nodes), then the stage updates of k_rk4_stage for both fields; acc and nxt hold
// u in [0, n) and v in [n, 2n).  Sums in double unless fields and weights are both float.
template <class FT, class WT, int UNR>
__global__ void __launch_bounds__(APPLY_THREADS) k_burgers_stage(int64_t n, const int64_t *__restrict__ row_ptr,
                                                                 const int32_t *__restrict__ col,
                                                                 const WT *__restrict__ wb, const FT *__restrict__ su,
                                                                 const FT *__restrict__ sv, FT *__restrict__ u,
                                                                 FT *__restrict__ v, FT *__restrict__ acc,
                                                                 FT *__restrict__ nxt,
                                                                 const uint8_t *__restrict__ frozen, int stage, FT dt,
                                                                 int lg_g)
{
    using AT = typename std::conditional<std::is_same<FT, float>::value && std::is_same<WT, float>::value, float,
                                         double>::type;
    const int G = 1 << lg_g;
    const int lane = threadIdx.x & (G - 1);
    const int64_t i = ((int64_t)blockIdx.x * APPLY_THREADS + threadIdx.x) >> lg_g;
    const bool live = i < n;
    int64_t rs = 0, re = 0;
    AT ui = 0, vi = 0;
    if (live) {
        rs = row_ptr[i];
        re = row_ptr[i + 1];
        ui = (AT)su[i];
        vi = (AT)sv[i];
    }
    AT s[6] = {0, 0, 0, 0, 0, 0};  // A_x(u), A_y(u), B(u), A_x(v), A_y(v), B(v)
    for (int64_t base = rs; base < re; base += (int64_t)G * UNR) {
        int cj[UNR];
        AT w0[UNR], w1[UNR], wl[UNR];
#pragma unroll
        for (int q = 0; q < UNR; q++) {
            const int64_t e = base + (int64_t)q * G + lane;
            if (e < re) {
                cj[q] = __ldcs(col + e);
                w0[q] = (AT)__ldcs(wb + 3 * e);
                w1[q] = (AT)__ldcs(wb + 3 * e + 1);
                wl[q] = (AT)__ldcs(wb + 3 * e + 2);
            } else {
                cj[q] = -1;
            }
        }
#pragma unroll
        for (int q = 0; q < UNR; q++) {
            if (cj[q] >= 0) {
                const AT du = (AT)su[cj[q]] - ui, dv = (AT)sv[cj[q]] - vi;
                s[0] = fma(du, w0[q], s[0]);
                s[1] = fma(du, w1[q], s[1]);
                s[2] = fma(du, wl[q], s[2]);
                s[3] = fma(dv, w0[q], s[3]);
                s[4] = fma(dv, w1[q], s[4]);
                s[5] = fma(dv, wl[q], s[5]);
            }
        }
    }
    for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int t = 0; t < 6; t++) s[t] += __shfl_xor_sync(0xffffffffu, s[t], o);
    if (!live || lane != 0) return;
    const bool fz = frozen && frozen[i];
    const FT Fu = fz ? (FT)0 : (FT)(-(ui * s[0] + vi * s[1]) + s[2]);
    const FT Fv = fz ? (FT)0 : (FT)(-(ui * s[3] + vi * s[4]) + s[5]);
    const FT u0 = u[i], v0 = v[i];
    switch (stage) {
    case 0:
        acc[i] = u0 + dt * (FT)(1.0 / 6.0) * Fu;
        acc[n + i] = v0 + dt * (FT)(1.0 / 6.0) * Fv;
        nxt[i] = u0 + dt * (FT)0.5 * Fu;
        nxt[n + i] = v0 + dt * (FT)0.5 * Fv;
        break;
    case 1:
        acc[i] = acc[i] + dt * (FT)(1.0 / 3.0) * Fu;
        acc[n + i] = acc[n + i] + dt * (FT)(1.0 / 3.0) * Fv;
        nxt[i] = u0 + dt * (FT)0.5 * Fu;
        nxt[n + i] = v0 + dt * (FT)0.5 * Fv;
        break;
    case 2:
        acc[i] = acc[i] + dt * (FT)(1.0 / 3.0) * Fu;
        acc[n + i] = acc[n + i] + dt * (FT)(1.0 / 3.0) * Fv;
        nxt[i] = u0 + dt * Fu;
        nxt[n + i] = v0 + dt * Fv;
        break;
    default:
        u[i] = acc[i] + dt * (FT)(1.0 / 6.0) * Fu;
        v[i] = acc[n + i] + dt * (FT)(1.0 / 6.0) * Fv;
        break;
    }
}

template <class FT, class WT>
cudaError_t launch_burg_stage_shape(labfm_ctx *ctx, Shape sh, const FT *su, const FT *sv, FT *u, FT *v, FT *acc,
                                    FT *nxt, const uint8_t *frozen, int stage, double dt, cudaStream_t s)
{
    const unsigned blocks = blocks_for(ctx->n, sh.G);
    auto args = [&](auto kern) {
        kern<<<blocks, APPLY_THREADS, 0, s>>>(ctx->n, ctx->row_ptr.as<int64_t>(), ctx->col.as<int32_t>(),
                                              ctx->wburg.as<WT>(), su, sv, u, v, acc, nxt, frozen, stage, (FT)dt,
                                              log2_of(sh.G));
    };
    switch (sh.UNR) {
    case 2: args(k_burgers_stage<FT, WT, 2>); break;
    case 8: args(k_burgers_stage<FT, WT, 8>); break;
    default: args(k_burgers_stage<FT, WT, 4>); break;
    }
    return cudaGetLastError();
}

template <class FT, class WT>
cudaError_t enqueue_burgers(labfm_ctx *ctx, void *u_, void *v_, int fdt, double dt, int64_t nsteps,
                            const uint8_t *frozen, cudaStream_t s)
{
    const int64_t n = ctx->n;
    FT *u = (FT *)u_, *v = (FT *)v_;
    FT *acc = ctx->bu_acc.as<FT>(), *sa = ctx->bu_stage_a.as<FT>(), *sb = ctx->bu_stage_b.as<FT>();
    // tune on stage 0, which reads u and v and writes only the work buffers
    Shape sh;
    cudaError_t e = autotune(
        ctx, tune_key(ctx, 3, 2, fdt, ctx->wdtype), 1,
        [&](Shape sp) {
            return launch_burg_stage_shape<FT, WT>(ctx, sp, u, v, u, v, acc, sa, frozen, 0, dt, ctx->stream);
        },
        sh);
    if (e != cudaSuccess) return e;
    for (int64_t st = 0; st < nsteps; st++) {
        if ((e = launch_burg_stage_shape<FT, WT>(ctx, sh, u, v, u, v, acc, sa, frozen, 0, dt, s)) != cudaSuccess)
            return e;
        if ((e = launch_burg_stage_shape<FT, WT>(ctx, sh, sa, sa + n, u, v, acc, sb, frozen, 1, dt, s)) !=
            cudaSuccess)
            return e;
        if ((e = launch_burg_stage_shape<FT, WT>(ctx, sh, sb, sb + n, u, v, acc, sa, frozen, 2, dt, s)) !=
            cudaSuccess)
            return e;
        if ((e = launch_burg_stage_shape<FT, WT>(ctx, sh, sa, sa + n, u, v, acc, (FT *)nullptr, frozen, 3, dt, s)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_burgers_dt(labfm_ctx *ctx, int fdt, void *u, void *v, double dt, int64_t nsteps,
                               const uint8_t *frozen, cudaStream_t s)
{
    if (fdt == LABFM_F64)
        return ctx->wdtype == LABFM_F64 ? enqueue_burgers<double, double>(ctx, u, v, fdt, dt, nsteps, frozen, s)
                                        : enqueue_burgers<double, float>(ctx, u, v, fdt, dt, nsteps, frozen, s);
    return ctx->wdtype == LABFM_F64 ? enqueue_burgers<float, double>(ctx, u, v, fdt, dt, nsteps, frozen, s)
                                    : enqueue_burgers<float, float>(ctx, u, v, fdt, dt, nsteps, frozen, s);
}

}  // namespace

labfm_status run_step_burgers(labfm_ctx *ctx, const double *beta, void *u, void *v, int fdt, double dt,
                              int64_t nsteps, const uint8_t *frozen)
{
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n, nnz = ctx->nnz;
    const size_t fsz = fdt == LABFM_F64 ? 8 : 4, wsz = ctx->wdtype == LABFM_F64 ? 8 : 4;
    bool same_beta = ctx->wburg_valid;
    for (int d = 2; d < ctx->n_ops && same_beta; d++) same_beta = (ctx->beta_burg[d] == beta[d]);
    if (!same_beta) {
        LABFM_CUDA_TRY(ctx, ctx->wburg.reserve(3 * wsz * (nnz > 0 ? nnz : 1)));
        double b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int d = 2; d < ctx->n_ops; d++) b[d] = beta[d];
        if (nnz > 0) {
            const unsigned blocks = (unsigned)std::min<int64_t>((nnz + 255) / 256, (int64_t)ctx->num_sms * 32);
            if (ctx->wdtype == LABFM_F64)
                k_burg_combine<double><<<blocks, 256, 0, s>>>(nnz, ctx->n_ops, ctx->w.as<double>(),
                                                               ctx->wburg.as<double>(), b[2], b[3], b[4], b[5], b[6],
                                                               b[7]);
            else
                k_burg_combine<float><<<blocks, 256, 0, s>>>(nnz, ctx->n_ops, ctx->w.as<float>(),
                                                              ctx->wburg.as<float>(), b[2], b[3], b[4], b[5], b[6],
                                                              b[7]);
            LABFM_CUDA_TRY(ctx, cudaGetLastError());
        }
        for (int d = 2; d < ctx->n_ops; d++) ctx->beta_burg[d] = beta[d];
        ctx->wburg_valid = true;
    }
    LABFM_CUDA_TRY(ctx, ctx->bu_acc.reserve(2 * fsz * n));
    LABFM_CUDA_TRY(ctx, ctx->bu_stage_a.reserve(2 * fsz * n));
    LABFM_CUDA_TRY(ctx, ctx->bu_stage_b.reserve(2 * fsz * n));

    StepGraph &g = ctx->graph_burgers;
    const bool same = g.exec && g.u == u && g.v == v && g.frozen == frozen && g.dtype == fdt && g.dt == dt &&
                      g.nsteps == nsteps && g.n == n && g.nnz == nnz && g.wdtype == ctx->wdtype &&
                      g.row_ptr == ctx->row_ptr.ptr && g.col == ctx->col.ptr && g.wc == ctx->wburg.ptr &&
                      g.acc == ctx->bu_acc.ptr && g.sa == ctx->bu_stage_a.ptr && g.sb == ctx->bu_stage_b.ptr;
    if (!same) {
        g.release();
        if (!ctx->capture_stream) {
            LABFM_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        }
        LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // the combined weights, before the capture stream reads them
        {
            cudaError_t te = enqueue_burgers_dt(ctx, fdt, u, v, dt, 0, frozen, s);  // tuning only
            if (te != cudaSuccess) return cuda_fail(ctx, te, "Burgers stage tuning");
            LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        }
        cudaGraph_t graph = nullptr;
        LABFM_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_burgers_dt(ctx, fdt, u, v, dt, nsteps, frozen, ctx->capture_stream);
        cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(ctx, e, "Burgers stage capture");
        }
        LABFM_CUDA_TRY(ctx, e2);
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return cuda_fail(ctx, e, "cudaGraphInstantiate");
        }
        g.u = u;
        g.v = v;
        g.frozen = frozen;
        g.dtype = fdt;
        g.dt = dt;
        g.nsteps = nsteps;
        g.n = n;
        g.nnz = nnz;
        g.wdtype = ctx->wdtype;
        g.row_ptr = ctx->row_ptr.ptr;
        g.col = ctx->col.ptr;
        g.wc = ctx->wburg.ptr;
        g.acc = ctx->bu_acc.ptr;
        g.sa = ctx->bu_stage_a.ptr;
        g.sb = ctx->bu_stage_b.ptr;
    }
    LABFM_CUDA_TRY(ctx, cudaGraphLaunch(g.exec, s));
    return LABFM_OK;
}

}  // namespace labfm
