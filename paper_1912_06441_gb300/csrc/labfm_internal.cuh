// Internal declarations shared by the translation units of liblabfm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>

#include "labfm.h"

namespace labfm {

constexpr int KMAX = LABFM_MAX_ORDER;
constexpr int PMAX = LABFM_PMAX;
constexpr int MAX_OPS = LABFM_MAX_OPS;
// Lowest order a mixed-precision build runs through the mixed kernels; lower orders go to the
// FP64 kernel (small, well conditioned systems: faster there, and exact to the FP64 floor).
constexpr int MIXED_MIN_ORDER = 5;

__host__ __device__ constexpr int p_of_k(int k) { return (k * k + 3 * k) / 2; }

// Grow-only device buffer owned by a context.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t need);
    void release();
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// Cached CUDA graph of an RK4 run, with everything its launches were recorded with: it is
// replayed only while all of these are unchanged.
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    const void *u = nullptr;
    const void *v = nullptr;  // second field (Burgers' equation)
    const void *frozen = nullptr;
    int dtype = -1;
    double dt = 0;
    int64_t nsteps = 0;
    int64_t n = -1, nnz = -1;
    int wdtype = -1;
    const void *row_ptr = nullptr, *col = nullptr, *wc = nullptr, *acc = nullptr, *sa = nullptr, *sb = nullptr;
    void release();
};

}  // namespace labfm

struct labfm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::string err;

    // stencils
    int64_t n = 0;
    int64_t nnz = 0;
    int periodic = 0;
    double lo[2] = {0, 0}, hi[2] = {0, 0};
    labfm::DevBuf node_xy, node_h;  // context copies of the node positions and h
    labfm::DevBuf row_ptr, col;
    // scratch of the neighbour search
    labfm::DevBuf cell_of, cell_count, cell_start, cell_nodes, counts, scan_tmp, misc;

    // weights
    bool have_weights = false;
    int n_ops = 0;
    int wdtype = LABFM_F64;
    labfm::DevBuf w;
    labfm::DevBuf status_tmp;
    labfm::DevBuf wtilde;  // scratch of the mixed-precision build: unscaled weights in double
    labfm::DevBuf mscratch;  // scratch of the mixed-precision build: per-node matrices of one batch
    labfm::DevBuf mrecs;     // scratch of the mixed-precision build: per-entry preamble records
    labfm::DevBuf mwstore;   // scratch of the mixed-precision build: W of every entry (double-float)
    labfm::DevBuf mfallback; // scratch of the mixed-precision build: nodes rebuilt in FP64
    // statistics of the last labfm_build_weights (labfm_get_build_info)
    int64_t info_ref_hist[8] = {0};
    int64_t info_fp64_rebuilt = 0;
    int info_group[LABFM_MAX_ORDER + 1] = {0};  // threads per node of the FP64 kernel, per order built by it
    int info_inv_tpr[LABFM_MAX_ORDER + 1] = {0};  // threads per row of the mixed inversion, per order

    // RK4
    labfm::DevBuf wcomb, rk_acc, rk_stage_a, rk_stage_b;
    double beta_cached[LABFM_MAX_OPS] = {0};
    int wcomb_dtype = -1;
    bool wcomb_valid = false;
    labfm::StepGraph graph;
    cudaStream_t capture_stream = nullptr;  // private stream used only to record the RK4 graphs

    // RK4 of Burgers' equation: per entry (w^0, w^1, sum_{d>=2} beta_d w^d) in the weight type
    bool grad01 = false;  // operators 0 and 1 of the built weights are d/dx and d/dy
    labfm::DevBuf wburg, bu_acc, bu_stage_a, bu_stage_b;
    double beta_burg[LABFM_MAX_OPS] = {0};
    bool wburg_valid = false;
    labfm::StepGraph graph_burgers;

    // implicit solves (BiCGStab): operator weights as one FP64 stream, nine vectors, partial sums
    labfm::DevBuf sol_w, sol_vec, sol_part, sol_gmap, sol_wg;  // sol_gmap/sol_wg: Neumann ghost rows

    // launch shapes chosen by the apply / RK4 autotuner:
    // key (kind, n_ops, dtypes, size class of n, mean stencil size) -> (G << 8) | UNR
    std::unordered_map<uint64_t, uint32_t> tuned;

    // pinned host word for status read-back
    void *host_small = nullptr;
};

namespace labfm {

labfm_status fail(labfm_ctx *ctx, labfm_status st, const std::string &msg);
labfm_status cuda_fail(labfm_ctx *ctx, cudaError_t e, const char *where);

// Exclusive prefix sum of in[0..n) (int64) into out[0..n]; out[n] = total.  `tmp` is scratch.
cudaError_t exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, DevBuf &tmp, cudaStream_t s);
cudaError_t exclusive_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, DevBuf &tmp, cudaStream_t s);
// The same scan on a caller-provided workspace of tmp_elems int64 (at least scan_workspace_elems(n)).
size_t scan_workspace_elems(int64_t n);
cudaError_t exclusive_scan_i32_to_i64_ws(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, size_t tmp_elems,
                                         cudaStream_t s);

// Arguments of the mixed-precision build kernel (see build_mixed.cu).
struct MixedArgsPublic {
    int64_t n_list;
    const int32_t *list;
    const double *xy, *h;
    const int64_t *row_ptr;
    const int32_t *col;
    int periodic;
    double L[2], halfL[2];
    int rbf, n_ops, nref;
    int adaptive;                   // 1: refine each node until it converges, at most nref steps
    int32_t *fb_list;               // [n] nodes handed to the FP64 build (refinement diverged)
    unsigned long long *fb_count;   // device counter of fb_list
    unsigned long long *ref_hist;   // device [nref + 1]: nodes by refinement steps taken
    void *w;
    int wdtype;
    double *wt;
    int32_t *node_status;
    unsigned long long *n_bad;
    int lmax[MAX_OPS];
    double C[MAX_OPS * PMAX];
    int num_sms;
    int64_t batch_nodes;  // nodes per batch; `scratch` holds batch_nodes * mixed_scratch_bytes_per_node(k)
    void *scratch;
    void *recs;  // [nnz] per-entry records, mixed_record_bytes() each
    int tc;      // 1: moment matrices on the tensor cores (exact BF16 slices), 0: double-float
    int inv_tpr; // threads per matrix row in the inversion: 1 (rows in registers), 2 or 4
    unsigned long long *tc_timeout;  // device counter of tensor-core waits that gave up
    void *wstore;  // [nnz][p(k)] double-float W kept between the assembly and the weights, or null
};
// The mixed build of the listed nodes, all at order k (MIXED_MIN_ORDER <= k <= KMAX).
cudaError_t launch_build_mixed(int k, const MixedArgsPublic &p, cudaStream_t s);
size_t mixed_scratch_bytes_per_node(int k);
size_t mixed_record_bytes();

// Kernel launchers (each returns the launch error).
labfm_status run_neighbours(labfm_ctx *ctx, int64_t n, const double *xy, const double *h, int periodic,
                            const double lo[2], const double hi[2], int64_t *nnz_out);
labfm_status run_build(labfm_ctx *ctx, const int8_t *order, int uniform_order, int rbf, int n_ops, const double *C,
                       int precision, int weight_dtype, int32_t *node_status, int64_t *n_bad_out);
cudaError_t launch_apply(labfm_ctx *ctx, uint32_t op_mask, const void *f, int field_dtype, void *out);
// Neumann ghost rows of an implicit solve (Sec. 5.2); n_ghost = 0: none
struct SolveNeumann {
    int64_t n_ghost = 0;
    const int64_t *ghost = nullptr, *parent = nullptr;  // device [n_ghost]
    const double *normal = nullptr;                     // device [n_ghost][2]
    int op_x = 0, op_y = 0;
};
labfm_status run_solve(labfm_ctx *ctx, int op, const double *f, double *phi, const uint8_t *dirichlet,
                       const SolveNeumann &nm, double tol, int max_iter, int *iters_out, double *resid_out);
labfm_status run_step_burgers(labfm_ctx *ctx, const double *beta, void *u, void *v, int field_dtype, double dt,
                              int64_t nsteps, const uint8_t *frozen);
labfm_status run_step(labfm_ctx *ctx, const double *beta, void *u, int field_dtype, double dt, int64_t nsteps,
                      const uint8_t *frozen);

}  // namespace labfm

#define LABFM_CUDA_TRY(ctx, expr)                                   \
    do {                                                            \
        cudaError_t e_ = (expr);                                    \
        if (e_ != cudaSuccess) return labfm::cuda_fail(ctx, e_, #expr); \
    } while (0)
