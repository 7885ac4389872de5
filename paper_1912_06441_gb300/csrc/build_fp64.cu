// FP64 weight build (Sec. 3.1-3.2): per node, monomials X and ABFs W of every neighbour,
// M = sum_j X_j (outer) W_j (Eq. disc_form), Gaussian elimination with partial pivoting of
// M Psi = C^d for all operators at once (Eq. lsys), and w_j^d = W_j . Psi^d (Eq. w_abf).
//
// A group of G threads per node (persistent over a node list): the whole CTA (G = 256) from order 6
// or 7 up, and two or four nodes per CTA below (G = 128 or 64, each group on its own named
// barrier), where the p x p system is small and a whole CTA would spend its time in barrier
// latency with most threads idle.  G per order is chosen by timing (build autotuner).
// Neighbour data are staged in shared memory in chunks of NB neighbours: Xs[j][m], Ws[j][n]
// (odd row stride LDX, so that the rows of consecutive neighbours start on distinct banks).  The
// p x p assembly is tiled 2 x 4 per thread in registers across chunks (two consecutive rows, four
// columns CG apart).  The augmented
// matrix [M | Chat] (Chat_alpha = C_alpha h^-|alpha|) is then eliminated in shared memory, one
// column per step, in the space of the X staging (X is not read again), which keeps a CTA within
// a quarter of the SM's shared memory: four CTAs per SM.
//
// Per-node orders (walls and variable resolution, Sec. 4.1) run in one persistent launch over
// work items: nodes bucketed by (order, stencil size), taken largest first, an item being one
// node of a CTA-wide order or 256 / G nodes of a grouped one.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "abf.cuh"

namespace labfm {
namespace {

constexpr int BUILD_THREADS = 256;

// Shared memory of one CTA beyond the X/W staging: the scalars and small arrays of the node being
// built, carved from the dynamic allocation (so that a kernel holding several orders allocates
// them once, not once per order).
struct NodeShared {
    double psi[PMAX * MAX_OPS];  // Psi^d, kept while X and W are staged again
    double invpiv[PMAX];         // 1 / pivot of each column, reused by the back substitution
    double hpow[KMAX + 1];       // h^-n
    double inv;
    int flag;
    unsigned char perm[2][PMAX];  // the elimination's rows by position (two lists, alternating)  // bit 0: zero/non-finite pivot, bit 1: non-finite weight, bit 2: non-finite M
};

// The CTA's dynamic shared memory: that of one order-8 node (72-neighbour chunks), so that four
// CTAs fit an SM; a CTA of NG = 256 / G groups gives each group a 1/NG share.
constexpr size_t SMEM_CTA = (sizeof(double) * ((size_t)2 * 72 * 45) + sizeof(NodeShared) + 15) / 16 * 16;

// Register tile (rows x columns of M per thread) of the assembly for p = P, staged row stride LDX
// and G threads: the shape of at most 8 accumulators that needs the fewest FP64 warp instructions
// per neighbour, (warps holding a tile) x (tile size).  A warp's FP64 instruction takes the pipe's
// time for all 32 lanes, masked or not, so a shape that leaves lanes of the last warp idle, or
// pads rows or columns, costs what it wastes (2 x 4 at order 7 needs 6 warps x 8 = 48 where
// 1 x 5 needs 8 x 5 = 40).  Ties keep the earlier, larger shape.
struct TileShape {
    int m, n;
};
constexpr TileShape pick_tile(int P, int LDX, int G)
{
    constexpr TileShape cands[] = {{2, 4}, {4, 2}, {1, 7}, {2, 3}, {3, 2}, {1, 6}, {1, 5},
                                   {1, 4}, {2, 2}, {1, 3}, {1, 2}, {1, 1}};
    TileShape best{0, 0};
    long best_cost = 0;
    for (const TileShape t : cands) {
        const int rg = (P + t.m - 1) / t.m, cg = (P + t.n - 1) / t.n;
        if (rg * cg > G || cg * t.n > LDX || rg * t.m > LDX) continue;
        const long cost = (long)((rg * cg + 31) / 32) * t.m * t.n;
        if (best.m == 0 || cost < best_cost) {
            best = t;
            best_cost = cost;
        }
    }
    return best;
}

template <int K, int G> struct Cfg {
    static constexpr int P = p_of_k(K);
    static constexpr int LDX = (P + 3) / 4 * 4 + 1;  // odd: rows of consecutive neighbours on distinct banks
    static constexpr int NG = BUILD_THREADS / G;  // nodes per CTA
    static_assert(G % 32 == 0 && BUILD_THREADS % G == 0, "groups of whole warps");
    // neighbours per staged chunk: what the group's share of the CTA's shared memory holds, <= 72
    static constexpr size_t GROUP_SMEM = (SMEM_CTA / NG) / 16 * 16;
    static constexpr int NB_FIT = (int)((GROUP_SMEM - sizeof(NodeShared)) / (sizeof(double) * 2 * LDX));
    static constexpr int NB = NB_FIT < 72 ? NB_FIT : 72;
    static constexpr TileShape TILE = pick_tile(P, LDX, G);
    static_assert(TILE.m > 0, "no register tile of at most 8 accumulators fits the group");
    static constexpr int TM = TILE.m, TN = TILE.n;
    static constexpr int RG = (P + TM - 1) / TM, CG = (P + TN - 1) / TN;
    static_assert(RG * CG <= G, "assembly tile grid exceeds the group");
    // The last, partly filled warp of tiles takes its tiles' elements one per lane and slot where
    // that needs fewer FP64 instructions per neighbour than a tile (order 8: 18 tiles = 144
    // elements in 5 slots instead of 8 accumulators; order 7: 105 elements in 4 instead of 5).
    static constexpr int NTILE = RG * CG;
    static constexpr int TAIL_WARP = NTILE / 32;
    static constexpr int TAIL_ELEMS = (NTILE % 32) * TM * TN;
    static constexpr int SLOTS = (TAIL_ELEMS + 31) / 32;
    static constexpr bool SPLIT = NTILE % 32 != 0 && SLOTS < TM * TN;
    static_assert(CG * TN <= LDX, "the tile's interleaved columns stay within a staged row");
    static constexpr int LDA = P + MAX_OPS + 1;  // augmented row stride (odd: fewer bank conflicts)
    // the augmented matrix reuses the X staging (X is not read after the assembly)
    static_assert((size_t)P * LDA <= (size_t)NB * LDX, "augmented matrix fits the X staging");
    static constexpr size_t smem_bytes = sizeof(double) * ((size_t)2 * NB * LDX);
    static_assert(smem_bytes + sizeof(NodeShared) <= GROUP_SMEM, "group staging fits its share");
};

// group sizes a given order may run with (the assembly tile grid must fit the group)
__host__ __device__ constexpr bool group_ok(int K, int G)
{
    return G == 256 || (G == 128 && K <= 6) || (G == 64 && K <= 5);
}

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

// Finiteness from the exponent bits (integer instructions: on GB300 an FP64 compare occupies the
// scarce FP64 pipe as long as a multiply-add)
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// 1 / a by Newton-Raphson iteration (r <- r + r (1 - a r), which squares the relative error of
// r at each step) from the single-precision reciprocal of a's leading 23 mantissa bits, formed
// with integer operations and the FP32 unit: two steps take the start's ~2^-22 to the rounding
// of the last step (within an ulp of 1/a) in four FP64 multiply-adds.  Used for the pivots, where
// one lane's division would hold the warp's share of the FP64 pipe for longer.  Subnormal a and
// |a| >= 2^1022 (a reciprocal at or below the normal range) take the division.
__device__ __forceinline__ double recip_newton(double a)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const int ef = (int)((b >> 52) & 0x7ff);  // biased exponent of a
    if (ef < 1 || ef > 2044) return 1.0 / a;
    const float mf = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff));  // 1.f of a, in [1, 2)
    const unsigned int rb = __float_as_uint(__frcp_rn(mf));                    // in (0.5, 1]
    // r0 = (1 / mf) 2^-(ef - 1023) with a's sign, assembled as a double
    const unsigned long long er = (unsigned long long)((int)((rb >> 23) & 0xff) - 127 - ef + 2046);
    double r = __longlong_as_double((long long)((b & 0x8000000000000000ull) | (er << 52) |
                                                ((unsigned long long)(rb & 0x7fffff) << 29)));
    double e = fma(-a, r, 1.0);
    r = fma(r, e, r);
    e = fma(-a, r, 1.0);
    return fma(r, e, r);
}

// Named barrier of group g of G threads: 1..2 for G = 128, 3..6 for G = 64 (an id is never used
// with two thread counts); the CTA-wide group uses the CTA barrier.
template <int G> __device__ __forceinline__ int group_bar(int g) { return (G == 128 ? 1 : 3) + g; }

// Barrier of one group: the CTA barrier for a CTA-wide group, named barrier `bar` of G threads
// otherwise.
template <int G> __device__ __forceinline__ void gsync(int bar)
{
    if constexpr (G == BUILD_THREADS) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(G) : "memory");
    }
}

// The whole build of node i at order K by a group of G threads (group-local thread index `tid`,
// barrier `bar`): stage X and W, assemble M, eliminate [M | Chat], weights.  Ends synchronised
// (the group's shared memory is reused by its next node).
template <int K, int G>
__device__ __forceinline__ void build_node(const BuildArgs &A, int64_t i, double *smem, int tid, int bar)
{
    using C = Cfg<K, G>;
    constexpr int P = C::P, LDX = C::LDX, NB = C::NB, LDA = C::LDA, TM = C::TM, TN = C::TN;
    double *Xs = smem;                 // [NB][LDX]
    double *Ws = Xs + NB * LDX;        // [NB][LDX]
    double *Am = Xs;                   // [P][LDA]  augmented [M | Chat], over the X staging
    NodeShared &sh = *reinterpret_cast<NodeShared *>(Ws + NB * LDX);
    double *s_psi = sh.psi, *s_invpiv = sh.invpiv, *s_hpow = sh.hpow;
    int &s_flag = sh.flag;
    double &s_inv = sh.inv;

    const int n_ops = A.n_ops;
    const int W_ = P + n_ops;  // used columns of the augmented matrix
    const int rg = tid / C::CG, cg = tid % C::CG;
    const bool tail = C::SPLIT && (tid >> 5) == C::TAIL_WARP;
    const bool tile_active = tid < C::RG * C::CG && !tail;
    // element of slot s of a tail-warp lane: row m and column c of M (element lane + 32 s of the
    // tail warp's tiles, in tile order); a slot past the last element reads the zero padding
    // column LDX - 1 of X and W and is not written
    auto tail_elem = [&](int s, int &m, int &c) {
        const int e = (tid & 31) + 32 * s;
        if (e >= C::TAIL_ELEMS) {
            m = c = LDX - 1;
            return;
        }
        const int tile = C::TAIL_WARP * 32 + e / (TM * TN), w = e % (TM * TN);
        m = (tile / C::CG) * TM + w / TN;
        c = tile % C::CG + (w % TN) * C::CG;
    };

    {
        const int64_t rs = A.row_ptr[i], re = A.row_ptr[i + 1];
        const int ni = (int)(re - rs);
        if (ni < P) {
            for (int64_t t = tid; t < (int64_t)ni * n_ops; t += G) {
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
        const double ihi = recip_newton(hi);
        if (tid == 0) {
            double s = 1.0;
            for (int t = 0; t <= K; t++) {
                s_hpow[t] = s;
                s *= ihi;
            }
        }

        // X and W of the chunk's neighbours into shared memory (thread per neighbour)
        auto stage = [&](int j0, int nj) {
            for (int t = tid; t < nj; t += G) {
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
        };
        double acc[TM][TN];
        auto accumulate = [&](int nj) {
            for (int j = 0; j < nj; j++) {
                const double *X = Xs + j * LDX + rg * TM;
                // columns cg, cg + CG, cg + 2 CG, ...: a warp's loads of one column slot are
                // consecutive doubles (distinct banks), where TN consecutive columns per thread would
                // put threads 4 apart on the same banks
                const double *W = Ws + j * LDX + cg;
                double xv[TM], wv[TN];
#pragma unroll
                for (int a = 0; a < TM; a++) xv[a] = X[a];
#pragma unroll
                for (int b = 0; b < TN; b++) wv[b] = W[b * C::CG];
#pragma unroll
                for (int a = 0; a < TM; a++)
#pragma unroll
                    for (int b = 0; b < TN; b++) acc[a][b] = fma(xv[a], wv[b], acc[a][b]);
            }
        };
        auto accumulate_tail = [&](int nj) {
            int xo[C::SLOTS > 0 ? C::SLOTS : 1], wo[C::SLOTS > 0 ? C::SLOTS : 1];
#pragma unroll
            for (int q = 0; q < C::SLOTS; q++) tail_elem(q, xo[q], wo[q]);
            for (int j = 0; j < nj; j++) {
                const double *X = Xs + j * LDX, *W = Ws + j * LDX;
#pragma unroll
                for (int q = 0; q < C::SLOTS; q++) acc[q / TN][q % TN] = fma(X[xo[q]], W[wo[q]], acc[q / TN][q % TN]);
            }
        };
        // the first chunk apart, so that its ABF evaluation runs before the accumulators exist
        // (most nodes have one chunk; with them live the evaluation spills to local memory)
        const int nchunks = (ni + NB - 1) / NB;
        const int nj0 = min(NB, ni);
        stage(0, nj0);
        gsync<G>(bar);
#pragma unroll
        for (int a = 0; a < TM; a++)
#pragma unroll
            for (int b = 0; b < TN; b++) acc[a][b] = 0.0;
        if (tile_active) accumulate(nj0);
        else if (tail) accumulate_tail(nj0);
        for (int ch = 1; ch < nchunks; ch++) {
            const int j0 = ch * NB;
            const int nj = min(NB, ni - j0);
            gsync<G>(bar);
            stage(j0, nj);
            gsync<G>(bar);
            if (tile_active) accumulate(nj);
            else if (tail) accumulate_tail(nj);
        }
        // M into the augmented matrix, scaled targets into its right-hand columns
        if (tid == 0) s_flag = 0;
        gsync<G>(bar);
        {
            bool finite = true;
            if (tile_active) {
#pragma unroll
                for (int a = 0; a < TM; a++)
#pragma unroll
                    for (int b = 0; b < TN; b++) {
                        int m = rg * TM + a, c = cg + b * C::CG;
                        if (m < P && c < P) {
                            Am[m * LDA + c] = acc[a][b];
                            finite &= finite_bits(acc[a][b]);
                        }
                    }
            } else if (tail) {
#pragma unroll
                for (int q = 0; q < C::SLOTS; q++) {
                    int m, c;
                    tail_elem(q, m, c);
                    if (m < P && c < P) {
                        Am[m * LDA + c] = acc[q / TN][q % TN];
                        finite &= finite_bits(acc[q / TN][q % TN]);
                    }
                }
            }
            // a non-finite entry of M (a neighbour on top of node i: singular ABFs)
            if (!finite) atomicOr(&s_flag, 4);
        }
        for (int t = tid; t < P * n_ops; t += G) {
            int m = t / n_ops, d = t % n_ops;
            Am[m * LDA + P + d] = A.C[d * PMAX + m] * s_hpow[elem_degree(m)];
        }
        gsync<G>(bar);
        const bool bad_m = (s_flag & 4) != 0;

        // Gaussian elimination with partial pivoting (first largest |pivot| wins), the rows left in
        // place: a list of the rows by position (double-buffered, so that the update reads one list
        // while the next is written) stands for the exchanges.  The pivot search compares |entry|
        // as bit patterns (non-negative doubles order like their bits; a zero column gives 0, inf
        // and NaN sort above every finite value and are flagged): integer compares, where FP64
        // compares would take the FP64 pipe's time (7 % of the kernel at order 8, measured).
        // Look-ahead: in the step of column c the group's first warp updates column c + 1, finds
        // its pivot and scales it while the other warps update columns c + 2 on, so that a column
        // costs one group barrier.
        unsigned char *permA = sh.perm[0], *permB = sh.perm[1];
        // pivot of column c by the first warp: `pin` lists the rows by position, `pout` receives
        // the list with positions c and the pivot's exchanged; the column below the pivot is scaled
        auto pivot = [&](int c, const unsigned char *pin, unsigned char *pout) {
            unsigned long long best = 0ull;
            int bk = P;
            for (int k = c + tid; k < P; k += 32) {
                const unsigned long long v = (unsigned long long)__double_as_longlong(Am[pin[k] * LDA + c]) & 0x7fffffffffffffffull;
                if (v > best || (v == best && k < bk)) {
                    best = v;
                    bk = k;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
                if (ob > best || (ob == best && ok < bk)) {
                    best = ob;
                    bk = ok;
                }
            }
            if (bk >= P) bk = c;  // the same on every lane after the butterfly
            if (tid == 0) {
                if (best == 0ull || best >= 0x7ff0000000000000ull) {
                    s_flag |= 1;
                    s_inv = 0.0;
                } else {
                    s_inv = recip_newton(Am[pin[bk] * LDA + c]);
                }
                s_invpiv[c] = s_inv;
            }
            for (int k = tid; k < P; k += 32) pout[k] = pin[k == c ? bk : (k == bk ? c : k)];
            __syncwarp();
            const double inv = s_inv;
            for (int k = c + 1 + tid; k < P; k += 32) Am[pout[k] * LDA + c] *= inv;
        };
        if (!bad_m) {
            if (tid < 32) {
                for (int k = tid; k < P; k += 32) permB[k] = (unsigned char)k;
                __syncwarp();
                pivot(0, permB, permA);
            }
            gsync<G>(bar);
        }
        for (int c = 0; c + 1 < P && !bad_m; c++) {
            const unsigned char *cur = (c & 1) ? permB : permA;  // column c's pivot at position c
            unsigned char *nxt = (c & 1) ? permA : permB;
            const int pr = cur[c];
            const int nr = P - c - 1;
            if (tid < 32) {
                for (int k = c + 1 + tid; k < P; k += 32) {
                    const int r = cur[k];
                    Am[r * LDA + c + 1] = fma(-Am[r * LDA + c], Am[pr * LDA + c + 1], Am[r * LDA + c + 1]);
                }
                __syncwarp();
                pivot(c + 1, cur, nxt);
            } else {
                const int nc = W_ - c - 2;  // columns c + 2 .. W_ - 1
                for (int t = tid - 32; t < nr * nc; t += G - 32) {
                    const int k = c + 1 + t / nc, q = c + 2 + t % nc;
                    const int r = cur[k];
                    Am[r * LDA + q] = fma(-Am[r * LDA + c], Am[pr * LDA + q], Am[r * LDA + q]);
                }
            }
            gsync<G>(bar);
        }
        // back substitution on the n_ops right-hand sides, rows by final position: the column-c
        // step updates positions k < c with x_c; position c - 1 takes its last update there and is
        // scaled to x_(c-1) at once (the same product as scaling it at the start of the next step),
        // by the first n_ops threads apart from the others' updates: a multiply inside the shared
        // loop would take FP64 pipe time in every warp of the loop, masked or not
        const unsigned char *fp = ((P - 1) & 1) ? permB : permA;
        if (!bad_m) {
            if (tid < n_ops) Am[fp[P - 1] * LDA + P + tid] *= s_invpiv[P - 1];
            gsync<G>(bar);
        }
        for (int c = P - 1; c > 0 && !bad_m; c--) {
            const int rc = fp[c];
            if (tid < n_ops) {
                const int r = fp[c - 1];
                Am[r * LDA + P + tid] = fma(-Am[r * LDA + c], Am[rc * LDA + P + tid], Am[r * LDA + P + tid]) * s_invpiv[c - 1];
            }
            for (int t = tid; t < (c - 1) * n_ops; t += G) {
                const int k = t / n_ops, d = t % n_ops;
                const int r = fp[k];
                Am[r * LDA + P + d] = fma(-Am[r * LDA + c], Am[rc * LDA + P + d], Am[r * LDA + P + d]);
            }
            gsync<G>(bar);
        }
        const bool singular = (s_flag & 5) != 0;  // no weights from a failed elimination
        for (int t = tid; t < P * n_ops; t += G) {
            const int m = t / n_ops, d = t - m * n_ops;
            double v = 0.0;  // a non-finite M gives no weights, and no position list is formed
            if (!bad_m) v = Am[fp[m] * LDA + P + d];
            s_psi[m * MAX_OPS + d] = v;
        }
        gsync<G>(bar);

        // weights w_j^d = W_j . Psi^d
        for (int ch = 0; ch < nchunks; ch++) {
            const int j0 = ch * NB;
            const int nj = min(NB, ni - j0);
            if (nchunks > 1) {  // the staged W of earlier chunks were overwritten: recompute
                gsync<G>(bar);
                for (int t = tid; t < nj; t += G) {
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
                gsync<G>(bar);
            }
            for (int t = tid; t < nj * n_ops; t += G) {
                int j = t / n_ops, d = t % n_ops;
                double s = 0.0;
                if (!singular) {
                    const double *W = Ws + j * LDX;
#pragma unroll 4
                    for (int m = 0; m < P; m++) s = fma(W[m], s_psi[m * MAX_OPS + d], s);
                    if (!finite_bits(s)) {
                        atomicOr(&s_flag, 2);
                        s = 0.0;
                    }
                }
                int64_t idx = (rs + j0 + j) * n_ops + d;
                if (A.wdtype == LABFM_F64) ((double *)A.w)[idx] = s;
                else ((float *)A.w)[idx] = (float)s;
            }
        }
        gsync<G>(bar);
        const int flag = s_flag;
        if (flag & 2) {  // a weight was not finite: the whole node is zeroed
            for (int64_t t = tid; t < (int64_t)ni * n_ops; t += G) {
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
        gsync<G>(bar);  // shared state is reused by the next node
    }
}

// One order for all listed nodes (persistent over the list; 256 / G nodes per CTA at a time).
template <int K, int G>
__global__ void __launch_bounds__(BUILD_THREADS, 4) k_build_fp64(BuildArgs A)
{
    using C = Cfg<K, G>;
    extern __shared__ __align__(16) double smem[];
    const int g = threadIdx.x / G;
    double *gs = smem + g * (C::GROUP_SMEM / sizeof(double));
    for (int64_t li = (int64_t)blockIdx.x * C::NG + g; li < A.n_list; li += (int64_t)gridDim.x * C::NG)
        build_node<K, G>(A, A.list ? (int64_t)A.list[li] : li, gs, threadIdx.x % G, group_bar<G>(g));
}

// Work items of the one-launch build over per-node orders: orders from KMAX down; order k has
// n_items[k] items starting at item0[k], item t covering the list entries base[k] + (t -
// item0[k]) NG_k ... of that order, NG_k = 256 / group[k] (the last item may be short).
struct OrderItems {
    int group[KMAX + 1];
    int64_t base[KMAX + 1], cnt[KMAX + 1], item0[KMAX + 1], n_items[KMAX + 1];
    int64_t total;
};

template <int K, int G>
__device__ __forceinline__ void run_item(const BuildArgs &A, const OrderItems &I, int64_t t, double *smem)
{
    if constexpr (group_ok(K, G)) {
        using C = Cfg<K, G>;
        const int g = threadIdx.x / G;
        const int64_t e = (t - I.item0[K]) * C::NG + g;  // entry within order K
        if (e < I.cnt[K])
            build_node<K, G>(A, (int64_t)A.list[I.base[K] + e], smem + g * (C::GROUP_SMEM / sizeof(double)),
                             threadIdx.x % G, group_bar<G>(g));
    }
}

template <int K>
__device__ __forceinline__ void run_item_k(const BuildArgs &A, const OrderItems &I, int64_t t, double *smem)
{
    switch (I.group[K]) {
    case 64: run_item<K, 64>(A, I, t, smem); break;
    case 128: run_item<K, 128>(A, I, t, smem); break;
    default: run_item<K, 256>(A, I, t, smem); break;
    }
}

// Every order in one persistent launch: CTAs take the items in order (the costliest first, the
// list being bucketed by descending (order, stencil size)), so that the cheap ones fill the tail.
// The groups of a CTA run their items independently; where the group size changes from one item
// to the next, the whole CTA meets first, so that no group starts on shared memory (or a named
// barrier) that a group of the previous size still uses.  The item sequence, hence that barrier,
// is the same for every thread of the CTA.
__global__ void __launch_bounds__(BUILD_THREADS, 4) k_build_fp64_items(BuildArgs A, OrderItems I)
{
    extern __shared__ __align__(16) double smem[];
    int prev_group = 0;
    for (int64_t t = blockIdx.x; t < I.total; t += gridDim.x) {
        int k = KMAX;
        while (k > 1 && t >= I.item0[k] + I.n_items[k]) k--;
        if (I.group[k] != prev_group) {
            if (prev_group != 0) __syncthreads();
            prev_group = I.group[k];
        }
        switch (k) {
        case 1: run_item_k<1>(A, I, t, smem); break;
        case 2: run_item_k<2>(A, I, t, smem); break;
        case 3: run_item_k<3>(A, I, t, smem); break;
        case 4: run_item_k<4>(A, I, t, smem); break;
        case 5: run_item_k<5>(A, I, t, smem); break;
        case 6: run_item_k<6>(A, I, t, smem); break;
        case 7: run_item_k<7>(A, I, t, smem); break;
        default: run_item_k<8>(A, I, t, smem); break;
        }
    }
}

// Listed nodes of any orders, one per CTA (the few nodes a mixed build hands back to FP64).
__global__ void __launch_bounds__(BUILD_THREADS, 4) k_build_fp64_any(BuildArgs A, const int8_t *__restrict__ order,
                                                                    int uniform_order)
{
    extern __shared__ __align__(16) double smem[];
    for (int64_t li = blockIdx.x; li < A.n_list; li += gridDim.x) {
        const int64_t i = A.list[li];
        switch (order ? order[i] : uniform_order) {
        case 1: build_node<1, 256>(A, i, smem, threadIdx.x, 0); break;
        case 2: build_node<2, 256>(A, i, smem, threadIdx.x, 0); break;
        case 3: build_node<3, 256>(A, i, smem, threadIdx.x, 0); break;
        case 4: build_node<4, 256>(A, i, smem, threadIdx.x, 0); break;
        case 5: build_node<5, 256>(A, i, smem, threadIdx.x, 0); break;
        case 6: build_node<6, 256>(A, i, smem, threadIdx.x, 0); break;
        case 7: build_node<7, 256>(A, i, smem, threadIdx.x, 0); break;
        default: build_node<8, 256>(A, i, smem, threadIdx.x, 0); break;
        }
    }
}

template <class KernelT, class... Args>
static cudaError_t launch_persistent_build(KernelT kern, int64_t units, int num_sms, cudaStream_t s, Args... args)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CTA);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BUILD_THREADS, SMEM_CTA);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(units, (int64_t)num_sms * per_sm);
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, BUILD_THREADS, SMEM_CTA, s>>>(args...);
    return cudaGetLastError();
}

template <int K>
static cudaError_t launch_k(const BuildArgs &a, int G, int num_sms, cudaStream_t s)
{
    if (G == 64 && group_ok(K, 64))
        return launch_persistent_build(k_build_fp64<K, group_ok(K, 64) ? 64 : 256>, (a.n_list + 3) / 4, num_sms, s, a);
    if (G == 128 && group_ok(K, 128))
        return launch_persistent_build(k_build_fp64<K, group_ok(K, 128) ? 128 : 256>, (a.n_list + 1) / 2, num_sms, s,
                                       a);
    return launch_persistent_build(k_build_fp64<K, 256>, a.n_list, num_sms, s, a);
}

static cudaError_t launch_order(int k, int G, const BuildArgs &a, int num_sms, cudaStream_t s)
{
    switch (k) {
    case 1: return launch_k<1>(a, G, num_sms, s);
    case 2: return launch_k<2>(a, G, num_sms, s);
    case 3: return launch_k<3>(a, G, num_sms, s);
    case 4: return launch_k<4>(a, G, num_sms, s);
    case 5: return launch_k<5>(a, G, num_sms, s);
    case 6: return launch_k<6>(a, G, num_sms, s);
    case 7: return launch_k<7>(a, G, num_sms, s);
    default: return launch_k<8>(a, G, num_sms, s);
    }
}

// Bucketing by (order, stencil size), both descending: key = (KMAX - k) 256 + 255 - min(N_i, 255).
constexpr int NBUCKET = (KMAX + 1) * 256;
__device__ __forceinline__ int bucket_key(int k, int64_t deg) { return (KMAX - k) * 256 + 255 - (int)min(deg, (int64_t)255); }

__global__ void k_bucket_count(int64_t n, const int8_t *__restrict__ order, const int64_t *__restrict__ row_ptr,
                               unsigned int *__restrict__ hist, unsigned long long *__restrict__ bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = order[i];
    if (k < 1 || k > KMAX) {
        atomicAdd(bad, 1ull);
        return;
    }
    atomicAdd(&hist[bucket_key(k, row_ptr[i + 1] - row_ptr[i])], 1u);
}

// cursor[b] starts at the first list position of bucket b
__global__ void k_bucket_scatter(int64_t n, const int8_t *__restrict__ order, const int64_t *__restrict__ row_ptr,
                                 unsigned int *__restrict__ cursor, int32_t *__restrict__ list)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = order[i];
    if (k < 1 || k > KMAX) return;
    list[atomicAdd(&cursor[bucket_key(k, row_ptr[i + 1] - row_ptr[i])], 1u)] = (int32_t)i;
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

// LABFM_MIXED_INVERSION = registers | shared2 | shared4 fixes the form of the mixed builds'
// inversion (rows in registers; 2 or 4 threads per row in shared memory) instead of the build
// autotuner's choice (diagnostics and tests); unset or any other value: the autotuner decides.
static int mixed_inversion_override()
{
    const char *v = std::getenv("LABFM_MIXED_INVERSION");
    if (!v) return 0;
    if (std::strcmp(v, "registers") == 0) return 1;
    if (std::strcmp(v, "shared2") == 0) return 2;
    if (std::strcmp(v, "shared4") == 0) return 4;
    return 0;
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
    // misc layout: [0] bad nodes, [1] bad orders, [30] tensor-core waits that gave up, [31] nodes
    // handed to the FP64 build, [32..39] nodes by refinement steps; from byte 1024 the bucket
    // histogram, from byte 1024 + 4 NBUCKET the bucket cursors
    constexpr int NMISC = 40;
    LABFM_CUDA_TRY(ctx, ctx->misc.reserve(1024 + 8 * (size_t)NBUCKET));
    unsigned long long *dmisc = ctx->misc.as<unsigned long long>();
    unsigned int *d_hist = reinterpret_cast<unsigned int *>(ctx->misc.as<char>() + 1024);
    unsigned int *d_cursor = d_hist + NBUCKET;
    LABFM_CUDA_TRY(ctx, cudaMemsetAsync(dmisc, 0, NMISC * sizeof(unsigned long long), s));
    for (int t = 0; t < 8; t++) ctx->info_ref_hist[t] = 0;
    for (int t = 0; t <= KMAX; t++) ctx->info_group[t] = ctx->info_inv_tpr[t] = 0;
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
    // Orders that the FP64 kernel builds: all of them for LABFM_PREC_FP64; for the mixed builds the
    // orders below MIXED_MIN_ORDER, whose p x p systems (p <= 14) are small and well conditioned:
    // there the cost is latency, which the grouped FP64 kernel hides better than the four-kernel
    // mixed pipeline, and FP64 arithmetic is accurate to the floor.
    auto fp64_route = [&](int k) { return !mixed || k < MIXED_MIN_ORDER; };

    // Group size of the FP64 kernel per order: timed once per (order, mean stencil size, n_ops)
    // on up to 16,384 of the order's real nodes (the autotuner of the build), kept in the
    // context's table.  Not while the caller's stream is being captured, nor below 4,096 nodes.
    auto group_for = [&](int k, const int32_t *list, int64_t cnt, double deg, int &G) -> cudaError_t {
        G = k <= 5 ? 64 : 256;
        const uint64_t dkey = (uint64_t)std::min(deg + 0.5, 65535.0);
        const uint64_t key = (dkey << 40) | ((uint64_t)k << 32) | (5ull << 24) | ((uint64_t)n_ops << 16);
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            G = (int)it->second;
            return cudaSuccess;
        }
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(s, &cap);
        if (e != cudaSuccess) return e;
        if (cap != cudaStreamCaptureStatusNone) return cudaSuccess;
        const int n_ok = (int)group_ok(k, 64) + (int)group_ok(k, 128) + (int)group_ok(k, 256);
        if (n_ok == 1) G = 256;  // one candidate: nothing to time
        if (cnt >= 4096 && n_ok > 1) {
            const int cand[3] = {64, 128, 256};
            float best = 1e30f;
            cudaEvent_t e0, e1;
            if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
            if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
                cudaEventDestroy(e0);
                return e;
            }
            BuildArgs t = a;
            t.list = list;
            t.n_list = std::min<int64_t>(cnt, 16384);
            for (int c = 0; c < 3 && e == cudaSuccess; c++) {
                if (!group_ok(k, cand[c])) continue;
                e = launch_order(k, cand[c], t, ctx->num_sms, s);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                if (e == cudaSuccess) e = launch_order(k, cand[c], t, ctx->num_sms, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e == cudaSuccess && ms < best) {
                    best = ms;
                    G = cand[c];
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (e != cudaSuccess) return e;
        }
        ctx->tuned[key] = (uint32_t)G;
        return cudaSuccess;
    };
    // the mixed kernels over the listed nodes, all at order k
    auto launch_mixed_raw = [&](int k, const int32_t *list, int64_t n_list, int tpr) -> cudaError_t {
        m.list = list;
        m.n_list = n_list;
        m.inv_tpr = tpr;
        bool adaptive = false;
        m.nref = precision_nref(precision, adaptive);
        m.adaptive = adaptive ? 1 : 0;
        // per-node matrices of one batch: at most 2^20 nodes (16 GB at k = 8)
        m.batch_nodes = std::max<int64_t>(1, std::min<int64_t>(n_list, (int64_t)1 << 20));
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
    // Threads per row of the mixed inversion (2 or 4), timed once per (order, mean stencil size,
    // n_ops, precision) on the whole mixed pipeline over up to 16,384 of the order's nodes (the
    // timing runs' counters are cleared afterwards; their weights are overwritten by the build).
    auto launch_mixed = [&](int k, const int32_t *list, int64_t cnt, double deg) -> cudaError_t {
        // untimed (small or captured builds): rows in registers, the form that won every timing
        int tpr = 1;
        const int forced = mixed_inversion_override();
        if (forced) {
            ctx->info_inv_tpr[k] = forced;
            return launch_mixed_raw(k, list, cnt, forced);
        }
        const uint64_t dkey = (uint64_t)std::min(deg + 0.5, 65535.0);
        const uint64_t key = (dkey << 40) | ((uint64_t)k << 32) | (6ull << 24) | ((uint64_t)n_ops << 16) |
                             ((uint64_t)base_prec << 8);
        auto it = ctx->tuned.find(key);
        cudaError_t e = cudaSuccess;
        if (it != ctx->tuned.end()) {
            tpr = (int)it->second;
        } else {
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            e = cudaStreamIsCapturing(s, &cap);
            if (e != cudaSuccess) return e;
            if (cap == cudaStreamCaptureStatusNone && cnt >= 4096) {
                cudaEvent_t e0, e1;
                if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
                if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
                    cudaEventDestroy(e0);
                    return e;
                }
                const int64_t nt = std::min<int64_t>(cnt, 16384);
                float best = 1e30f;
                const int cands[3] = {1, 2, 4};  // threads per row: 1 = rows in registers
                for (int ci = 0; ci < 3 && e == cudaSuccess; ci++) {
                    const int cand = cands[ci];
                    e = launch_mixed_raw(k, list, nt, cand);  // warm-up
                    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                    if (e == cudaSuccess) e = launch_mixed_raw(k, list, nt, cand);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e == cudaSuccess && ms < best) {
                        best = ms;
                        tpr = cand;
                    }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (e != cudaSuccess) return e;
                // the timing runs' flags, rebuild lists and step counts
                e = cudaMemsetAsync(dmisc, 0, sizeof(unsigned long long), s);
                if (e == cudaSuccess) e = cudaMemsetAsync(dmisc + 30, 0, 10 * sizeof(unsigned long long), s);
                if (e != cudaSuccess) return e;
            }
            ctx->tuned[key] = (uint32_t)tpr;
        }
        ctx->info_inv_tpr[k] = tpr;
        return launch_mixed_raw(k, list, cnt, tpr);
    };

    unsigned long long *hs = (unsigned long long *)ctx->host_small;
    if (!order) {
        const int k = uniform_order;
        if (fp64_route(k)) {
            int G = 256;
            LABFM_CUDA_TRY(ctx, group_for(k, nullptr, n, n > 0 ? (double)ctx->nnz / (double)n : 0.0, G));
            ctx->info_group[k] = G;
            LABFM_CUDA_TRY(ctx, cudaMemsetAsync(dmisc, 0, sizeof(unsigned long long), s));  // the timing runs' flags
            a.list = nullptr;
            a.n_list = n;
            LABFM_CUDA_TRY(ctx, launch_order(k, G, a, ctx->num_sms, s));
        } else {
            LABFM_CUDA_TRY(ctx, launch_mixed(k, nullptr, n, n > 0 ? (double)ctx->nnz / (double)n : 0.0));
        }
    } else {
        // bucket the nodes by (order, stencil size), both descending
        LABFM_CUDA_TRY(ctx, cudaMemsetAsync(d_hist, 0, sizeof(unsigned int) * NBUCKET, s));
        const int nb = (int)((n + 255) / 256);
        k_bucket_count<<<nb, 256, 0, s>>>(n, order, a.row_ptr, d_hist, dmisc + 1);
        LABFM_CUDA_TRY(ctx, cudaGetLastError());
        std::vector<unsigned int> hist(NBUCKET);
        LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(hs, dmisc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(hist.data(), d_hist, sizeof(unsigned int) * NBUCKET, cudaMemcpyDeviceToHost, s));
        LABFM_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (hs[1] != 0) return fail(ctx, LABFM_ERR_ARG, "order[] has entries outside 1..8");
        std::vector<unsigned int> start(NBUCKET);
        int64_t cnt[KMAX + 1] = {0}, base[KMAX + 1] = {0};
        double degsum[KMAX + 1] = {0};
        unsigned int acc = 0;
        for (int b = 0; b < NBUCKET; b++) {
            start[b] = acc;
            acc += hist[b];
            const int k = KMAX - b / 256;
            if (k >= 1) {
                if (cnt[k] == 0 && hist[b]) base[k] = start[b];
                cnt[k] += hist[b];
                degsum[k] += (double)hist[b] * (255 - b % 256);
            }
        }
        LABFM_CUDA_TRY(ctx, ctx->status_tmp.reserve(sizeof(int32_t) * (n > 0 ? n : 1)));
        int32_t *list = ctx->status_tmp.as<int32_t>();
        LABFM_CUDA_TRY(ctx, cudaMemcpyAsync(d_cursor, start.data(), sizeof(unsigned int) * NBUCKET, cudaMemcpyHostToDevice, s));
        k_bucket_scatter<<<nb, 256, 0, s>>>(n, order, a.row_ptr, d_cursor, list);
        LABFM_CUDA_TRY(ctx, cudaGetLastError());
        // the FP64-routed orders: one persistent launch over their work items, costliest first
        OrderItems I{};
        int64_t items = 0;
        for (int k = KMAX; k >= 1; k--) {
            I.group[k] = 256;
            I.base[k] = base[k];
            I.item0[k] = items;
            if (!fp64_route(k) || !cnt[k]) continue;
            int G = 256;
            LABFM_CUDA_TRY(ctx, group_for(k, list + base[k], cnt[k], degsum[k] / (double)cnt[k], G));
            const int ng = BUILD_THREADS / G;
            I.group[k] = G;
            ctx->info_group[k] = G;
            I.cnt[k] = cnt[k];
            I.n_items[k] = (cnt[k] + ng - 1) / ng;
            items += I.n_items[k];
        }
        I.total = items;
        LABFM_CUDA_TRY(ctx, cudaMemsetAsync(dmisc, 0, sizeof(unsigned long long), s));  // the timing runs' flags
        if (items) {
            a.list = list;
            a.n_list = n;
            LABFM_CUDA_TRY(ctx, launch_persistent_build(k_build_fp64_items, items, ctx->num_sms, s, a, I));
        }
        // the mixed-built orders (MIXED_MIN_ORDER .. 8), highest first, each over its segment of the
        // bucketed list (one launch per order and phase: kernels shaped for each order were faster
        // than one launch per phase over all orders, which carries order 8's shared memory and
        // thread count for every node)
        for (int k = KMAX; k >= 1; k--)
            if (!fp64_route(k) && cnt[k])
                LABFM_CUDA_TRY(ctx, launch_mixed(k, list + base[k], cnt[k], degsum[k] / (double)cnt[k]));
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
        LABFM_CUDA_TRY(ctx, launch_persistent_build(k_build_fp64_any, nfb, ctx->num_sms, s, a, order, uniform_order));
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
