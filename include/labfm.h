/*
 * labfm.h -- C ABI of the GB300 (sm_103a) implementation of the Local Anisotropic
 * Basis Function Method (LABFM) of King, Lind & Nasar, "High order difference
 * schemes using the Local Anisotropic Basis Function Method".
 *
 * The library computes, for every node i of a 2D node set, the stencil weights
 * w_ji^d of Eq. (w_abf) and applies the discrete operators L_i^d of
 * Eq. (general_do).  All compute runs in CUDA kernels of this library; the
 * caller supplies device memory (e.g. from PyTorch) and a CUDA stream.
 *
 * Conventions (every entry point):
 *  - Pointers named "device" must be device (or managed) memory readable by the
 *    context's device; pointers named "host" are ordinary host memory.
 *  - Caller-owned buffers are only read (or written where stated) during the
 *    call's stream-ordered work; the library keeps no reference to them.
 *  - Context-owned buffers (stencils, weights, scratch) live until the context is
 *    destroyed or the buffer is rebuilt.
 *  - Work is enqueued on the context stream.  Calls that return counts or
 *    statuses (labfm_build_neighbours, labfm_build_weights) synchronise that
 *    stream before returning; labfm_apply and labfm_step do not.
 *  - No C++ exception crosses the ABI; failures return a labfm_status and
 *    labfm_last_error() gives a message.  Invalid arguments are rejected on the
 *    host before any kernel is launched.
 *  - Per-node numerical failure is data, not an abort: see LABFM_NODE_*.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef LABFM_H
#define LABFM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct labfm_ctx labfm_ctx;

typedef enum {
    LABFM_OK = 0,
    LABFM_ERR_ARG = 1,      /* invalid argument, detected on the host */
    LABFM_ERR_CUDA = 2,     /* a CUDA runtime call failed */
    LABFM_ERR_NOMEM = 3,    /* device allocation failed */
    LABFM_ERR_CAPACITY = 4, /* a size limit of the library was exceeded (message says which) */
    LABFM_ERR_SINGULAR = 5, /* weights built, but >= 1 node was flagged (see node_status) */
    LABFM_ERR_TIMEOUT = 6,  /* a bounded device wait gave up */
    LABFM_ERR_STATE = 7,    /* call out of order (e.g. apply before build_weights) */
    LABFM_ERR_NOT_CONVERGED = 8 /* an iterative solve stopped short of its tolerance */
} labfm_status;

/* Fundamental RBFs W0(q), q = |r|/h, support [0, 2] (Sec. 3.2, Appendix A). */
enum {
    LABFM_RBF_WENDLAND_C2 = 0, /* 7/(4 pi) (1 - q/2)^4 (1 + 2q) (standard Wendland C2, normalised as Appendix A asks) */
    LABFM_RBF_QUADRATIC = 1,   /* 3/(16 pi) (q - 2)^2, Appendix A.1 */
    LABFM_RBF_CONE = 2,        /* 3/(4 pi) (1 - q/2), Sec. 3.2 */
    LABFM_RBF_WENDLAND_C6 = 3, /* 78/(28 pi) (1 - q/2)^8 (4q^3 + 6.25q^2 + 4q + 1), Appendix A.2 */
    LABFM_RBF_GAUSSIAN = 4     /* 9/pi exp(-9 q^2), Appendix A.3 */
};
#define LABFM_RBF_MASK 0xff

/* ABF form, OR-ed into the rbf argument of labfm_build_weights.
 * Default (0): the elements 1-9 (|alpha| <= 3) are the full chain rule of D(W0(|r|)) with
 * dW0/dr, d2W0/dr2 and d3W0/dr3, as printed in Appendix A; the elements >= 10 keep only
 * dW0/dr d^alpha|r| (Appendix A, truncation rule).
 * LABFM_ABF_DW0_ONLY: every element is dW0/dr d^alpha|r|, i.e. the higher RBF derivatives are
 * dropped for the elements 1-9 too.  Appendix A's truncation sentence names only elements >= 10,
 * but the stability results of Sec. 4.2 (the Laplacian's noise limits, a purely imaginary
 * convective spectrum on a regular lattice whenever dW0/dr vanishes at q = 2) are reproduced
 * by this form and not by the default one; explicit time stepping needs it. */
#define LABFM_ABF_DW0_ONLY 0x100

/* Arithmetic of the moment-matrix assembly (Eq. disc_form) and solve (Eq. lsys). */
enum {
    LABFM_PREC_FP64 = 0, /* everything in IEEE double */
    /* X and W in double; M, its inverse (Gauss-Jordan elimination with partial pivoting), Psi
     * and W . Psi in double-float
     * (pairs of FP32, ~48 bits, on the FP32 pipes); then iterative refinement on the
     * polynomial-reproduction residual C - sum_j X_j w_j computed in double (the moment
     * conditions of Sec. 3.1).  Default: adaptive per node.  With eta_t the relative size of the
     * t-th change of a node's weights (largest over its operators, eta_0 = 1), the node stops
     * after step t >= 1 once eta_t^2 / eta_(t-1) < 2^-44 (converged; one step for most nodes),
     * or once eta_t > eta_(t-1) / 2 (the corrections have reached the rounding level of the
     * FP64 residual), or after 6 steps.  A node whose corrections grow instead (eta_t above
     * both eta_(t-1) / 2 and 1e-3: M too ill-conditioned for the double-float inverse) is built
     * again by the FP64 path (LABFM_PREC_FP64).  labfm_get_build_info reports both counts. */
    LABFM_PREC_MIXED = 1,
    /* As LABFM_PREC_MIXED, with M formed on the tensor cores: X and W are scaled per row (a power
     * of two per chunk of <= 64 neighbours) and cut into seven 8-bit BF16 slices; the slice
     * products of each level a + b = 2..8 are summed exactly in FP32 (tcgen05.mma, accumulators
     * in tensor memory) and combined in double-float. */
    LABFM_PREC_MIXED_TC = 2
};
/* LABFM_PREC_MIXED with exactly n refinement steps, n = 0..4 (no adaptive rule, no FP64 rebuild) */
#define LABFM_PREC_MIXED_REFINE(n) (LABFM_PREC_MIXED | (((n) + 1) << 8))
/* LABFM_PREC_MIXED_TC with exactly n refinement steps, n = 0..4 */
#define LABFM_PREC_MIXED_TC_REFINE(n) (LABFM_PREC_MIXED_TC | (((n) + 1) << 8))

/* Storage type of weights and fields. */
enum { LABFM_F64 = 0, LABFM_F32 = 1 };

/* Per-node status written by labfm_build_weights. */
enum {
    LABFM_NODE_OK = 0,
    LABFM_NODE_SINGULAR = 1,     /* a pivot of the elimination was exactly zero or not finite */
    LABFM_NODE_UNDERSAMPLED = 2, /* fewer neighbours than p: M_i (a sum of N_i rank-one terms) is singular */
    LABFM_NODE_NONFINITE = 3     /* a weight came out NaN or infinite */
};

/* Limits of the library. */
#define LABFM_MAX_ORDER 8 /* k <= 8, p <= 44 */
#define LABFM_MAX_OPS 8   /* operators per build */
#define LABFM_PMAX 44     /* p(8) = (8^2 + 3*8)/2, Sec. 3.1 */

/* Create a context on CUDA device `device` that enqueues work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context.  Returns LABFM_ERR_CUDA if the device cannot be used. */
labfm_status labfm_create(labfm_ctx **out, int device, void *stream);

/* Release every context-owned buffer.  NULL is accepted. */
void labfm_destroy(labfm_ctx *ctx);

/* Message for the last failed call on this context ("" if none).  Valid until the next call. */
const char *labfm_last_error(const labfm_ctx *ctx);

/* Change the stream subsequent work is enqueued on. */
labfm_status labfm_set_stream(labfm_ctx *ctx, void *stream);

/*
 * Stencils (Sec. 2): for every node i, all j != i with |r_j - r_i| < 2 h_i.
 *   n        number of nodes, 1 <= n < 2^31
 *   xy       device double[2n], interleaved (x_0, y_0, x_1, y_1, ...)
 *   h        device double[n], h_i > 0 and finite
 *   periodic 1: the box [lo, hi)^2 wraps and offsets use the minimum image;
 *            0: no wrap.  Every node must lie in the closed box.
 *   box_lo, box_hi  host double[2]
 *   nnz_out  host, receives the total number of stencil entries
 * The predicate is evaluated exactly as written, in IEEE double without fused
 * multiply-add: dx = x_j - x_i (then +-L once if |dx| > L/2 in a periodic box),
 * r2 = dx*dx + dy*dy, accept r2 < (2 h_i)*(2 h_i).  Output is CSR, context-owned:
 * row_ptr int64[n+1], col int32[nnz], each row ascending in j.  Rebuilding
 * stencils invalidates any weights.  Errors: LABFM_ERR_ARG for a bad size, box,
 * h or a node outside the box; LABFM_ERR_CAPACITY if the cell grid would exceed
 * 2^28 cells.
 */
labfm_status labfm_build_neighbours(labfm_ctx *ctx, int64_t n, const double *xy, const double *h,
                                    int periodic, const double box_lo[2], const double box_hi[2],
                                    int64_t *nnz_out);

/* Context-owned device views of the stencils (valid until rebuilt or destroyed). */
labfm_status labfm_get_neighbours(labfm_ctx *ctx, const int64_t **row_ptr, const int32_t **col,
                                  int64_t *n, int64_t *nnz);

/*
 * Weights (Sec. 3.1-3.2): per node i, build M_i = sum_j X_ji (outer) W_ji
 * (Eq. disc_form) from the Taylor monomials X (Sec. 2) and the ABFs
 * W = D(W0)|r_ji (Sec. 3.2; elements >= 10 keep only the dW0/dr term, Appendix A),
 * solve M_i Psi^d = C^d (Eq. lsys) by Gaussian elimination with partial pivoting,
 * and set w_ji^d = W_ji . Psi^d (Eq. w_abf).  Offsets are taken in units of h_i
 * and C^d is scaled by h_i^-|alpha| (an exact similarity transform of M_i).
 *   order        device int8[n] per-node order k_i in 1..8, or NULL to use uniform_order
 *   uniform_order  1..8 when order == NULL
 *   rbf          LABFM_RBF_*, optionally OR-ed with LABFM_ABF_DW0_ONLY
 *   n_ops        number of operators, 1..LABFM_MAX_OPS
 *   C            host double[n_ops * 44]: row d is C^d in the derivative ordering D of
 *                Sec. 2 (d/dx, d/dy, d2/dx2, d2/dxdy, d2/dy2, d3/dx3, ...), physical units;
 *                entries beyond p(k_i) are ignored for node i
 *   precision    LABFM_PREC_*
 *   weight_dtype LABFM_F64 or LABFM_F32: storage of the context-owned weights,
 *                layout [nnz][n_ops] (entry e of the CSR, operator d at e*n_ops + d)
 *   node_status  device int32[n] receiving LABFM_NODE_* per node, or NULL
 *   n_bad_out    host, receives the number of flagged nodes (may be NULL)
 * The FP64 kernel builds a node with a group of 64, 128 or 256 threads (several small-order nodes
 * per CTA); the group size per order is chosen by timing the candidates once per (order, mean
 * stencil size, n_ops) on up to 16,384 of the order's nodes (not while `stream` is being captured,
 * nor below 4,096 nodes), and kept for the life of the context.  With per-node orders the nodes
 * are bucketed by (order, stencil size) and the FP64-built orders run in one persistent launch,
 * costliest nodes first.  The mixed builds build orders 1-4 with the FP64 kernel (small, well
 * conditioned systems: faster there and exact to the FP64 floor) and each order from 5 up with
 * the mixed kernels.
 * Flagged nodes get zero weights.  Returns LABFM_ERR_SINGULAR if any node was
 * flagged (the weights of all other nodes are valid), LABFM_ERR_STATE if no
 * stencils were built, LABFM_ERR_TIMEOUT if a bounded wait for the tensor cores
 * (LABFM_PREC_MIXED_TC) gave up (the weights are then undefined).
 */
labfm_status labfm_build_weights(labfm_ctx *ctx, const int8_t *order, int uniform_order, int rbf,
                                 int n_ops, const double *C, int precision, int weight_dtype,
                                 int32_t *node_status, int64_t *n_bad_out);

/* Statistics of the last successful labfm_build_weights on this context. */
typedef struct {
    /* mixed builds: nodes by the number of refinement steps they took (index 0..7; with the
     * default adaptive rule at most 6), the nodes then rebuilt in FP64 included; nodes flagged
     * before the refinement (undersampled, a zero pivot, a non-finite M) are not counted; all
     * zero after an FP64 build */
    int64_t refine_steps[8];
    /* mixed builds: nodes whose refinement diverged and that the FP64 build redid */
    int64_t fp64_rebuilt;
    /* per order k (index 1..8): threads that built one node in the FP64 kernel (64, 128: several
     * nodes per CTA; 256: one), as the build autotuner chose them; 0 for orders not built there */
    int32_t fp64_group_threads[LABFM_MAX_ORDER + 1];
    /* per order k (index 1..8): threads per matrix row of the mixed builds' double-float
     * inversion, as the build autotuner chose them (timed once per (order, mean stencil size,
     * n_ops, precision) like the FP64 group size): 1 = each row in the registers of one thread,
     * 2 or 4 = the matrix in shared memory; 0 for orders not built by the mixed kernels.  Builds
     * too small to time (an order with fewer than 4096 nodes) or recorded into a CUDA graph use 1.
     * The environment variable LABFM_MIXED_INVERSION = registers, shared2 or shared4, read at
     * each build, fixes the form instead (diagnostics). */
    int32_t mixed_inv_threads_per_row[LABFM_MAX_ORDER + 1];
} labfm_build_info;

/* Copy the statistics of the last weight build into *info.  LABFM_ERR_STATE before a build. */
labfm_status labfm_get_build_info(labfm_ctx *ctx, labfm_build_info *info);

/* Context-owned device view of the weights: *w points to [nnz][n_ops] of *dtype. */
labfm_status labfm_get_weights(labfm_ctx *ctx, const void **w, int *dtype, int *n_ops);

/*
 * Apply the discrete operators (Eq. general_do): out_d[i] = sum_j (f_j - f_i) w_ji^d
 * for every operator d selected by op_mask (bit d), written in increasing d.
 *   f           device [n] of field_dtype (LABFM_F64 or LABFM_F32)
 *   out         device [n_selected][n] of field_dtype, row-major by operator
 * Accumulation is in double for LABFM_F64 fields and in float for LABFM_F32 fields.
 * f and out must not overlap.
 * Launch shape: G lanes share a node and each lane keeps UNR stencil entries in flight,
 * (G, UNR) in {4, 8, 16, 32} x {2, 4, 8}.  The first call per (n_ops, field dtype, weight
 * dtype, floor(log2 n), mean stencil size) on a context (n >= 4096, stream not capturing)
 * times each shape once, writing out repeatedly, waits for the timings, and keeps the fastest
 * for the life of the context; later calls are asynchronous.
 * LABFM_ERR_STATE before labfm_build_weights.
 */
labfm_status labfm_apply(labfm_ctx *ctx, uint32_t op_mask, const void *f, int field_dtype, void *out);

/*
 * Explicit time stepping with the classical four-stage Runge-Kutta scheme (Sec. 5.1) of
 *   du/dt = F(u),  F(u)_i = sum_d beta_d L_i^d(u)
 * for nsteps steps of size dt.  The operators are combined once into one weight per
 * stencil entry, w_ji = sum_d beta_d w_ji^d (L^d is linear in w, summed in double), cached
 * while beta, the weights and the field type are unchanged.  It is kept in the weight type,
 * except for FP64 weights with FP32 fields: then it is kept as a double-float pair (two
 * floats, ~48 bits) and the stencil sums run in double-float arithmetic on the FP32 pipes.
 * The per-node stage update is in double (in float when weights and field are FP32).
 * Nodes with frozen[i] != 0 keep their value
 * (Dirichlet nodes, Sec. 5.1).  The nsteps x 4 stage launches are recorded once into a
 * CUDA graph and replayed; it is recorded again when an argument other than beta, the
 * stencil count or size, the weight type or a context buffer changes.  The stage's launch
 * shape is tuned as for labfm_apply, on first-stage launches that read u and write only
 * context-owned buffers (u is not changed by the tuning).
 *   beta    host double[n_ops]
 *   u       device [n] of field_dtype, updated in place
 *   frozen  device uint8[n] or NULL
 * Asynchronous.  LABFM_ERR_STATE before labfm_build_weights.
 */
labfm_status labfm_step(labfm_ctx *ctx, const double *beta, void *u, int field_dtype, double dt,
                        int64_t nsteps, const uint8_t *frozen);

/*
 * Explicit time stepping of the viscous Burgers' equation (Sec. 5.3, eq. burgers),
 * du/dt + (u . grad) u = (1/Re) nabla^2 u for the velocity u = (u, v), with the classical
 * four-stage Runge-Kutta scheme, in the form
 *   du/dt = -(u_i L^0_i(u) + v_i L^1_i(u)) + sum_{d>=2} beta_d L^d_i(u)
 *   dv/dt = -(u_i L^0_i(v) + v_i L^1_i(v)) + sum_{d>=2} beta_d L^d_i(v)
 * where operators 0 and 1 of the built weights must be d/dx and d/dy (their targets C^d the
 * unit vectors of the first two elements of D; LABFM_ERR_ARG otherwise) and the further
 * operators carry the linear terms: beta_2 = 1/Re on nabla^2, and e.g. a hyperviscosity
 * -alpha nabla^4 or alpha nabla^6 (Sec. 4.2) as another operator.  beta[0] and beta[1] are
 * not read.  The advection coefficients are the stage's own field values, so d/dx and d/dy
 * stay separate stencil sums; the linear operators are combined once into one weight per
 * entry (summed in double, kept in the weight type, cached while beta[2..] and the weights are
 * unchanged).  Sums run in double unless field and weights are both LABFM_F32.
 * Nodes with frozen[i] != 0 keep their values of u and v.  The nsteps x 4 stage launches are
 * recorded once into a CUDA graph and replayed, under the same rules as labfm_step; the
 * stage's launch shape is tuned on first-stage launches that read u and v and write only
 * context-owned buffers.
 *   beta    host double[n_ops]
 *   u, v    device [n] of field_dtype, distinct, updated in place
 *   frozen  device uint8[n] or NULL
 * Asynchronous.  LABFM_ERR_STATE before labfm_build_weights.
 */
labfm_status labfm_step_burgers(labfm_ctx *ctx, const double *beta, void *u, void *v, int field_dtype,
                                double dt, int64_t nsteps, const uint8_t *frozen);

/*
 * Solve the global linear system of Sec. 5.2 (eq. poisson_system), A Phi = F, whose rows are the
 * local operators of operator `op`: A_ij = w^op_ji for j != i and A_ii = -sum_j w^op_ji, so that
 * (A Phi)_i = L^op_i(Phi) (e.g. op = the Laplacian: Poisson's equation, eq. poisson).  Where
 * dirichlet[i] != 0 the row is replaced by the identity (Sec. 5.2, Dirichlet rows: A_ii = 1,
 * A_ij = 0, F_i = g_i), so that Phi_i = f[i] there.  The matrix is not formed: its products are
 * stencil sums over the context's stencils.  Stabilised bi-conjugate gradients (van der Vorst
 * 1992) with a Jacobi preconditioner (diag A), as in Sec. 5.2; all vectors and scalars in FP64 and
 * in device memory, iterations recorded in chunks of 16 into a CUDA graph with one host read of the
 * state per chunk.  The product's launch shape (lanes per node x entries in flight, 3 x 3 shapes)
 * is timed once per problem class (floor(log2 n), mean stencil size) on a context, as for
 * labfm_apply (n >= 4096, stream not capturing).
 * Stops when the recurrence residual ||r|| <= tol ||F||, or after max_iter iterations.  The
 * recurrence residual drifts from the true one ||F - A Phi|| in finite precision, so the true
 * residual is then formed; if it is above tol, the iteration restarts from the current Phi
 * (r = F - A Phi, shadow residual r^ = r).  A breakdown (rho = (r^, r), (r^, v) or omega
 * vanishing or not finite) with a finite Phi restarts the same way.  At most 8 restarts, within
 * max_iter iterations in total.
 * With a periodic node set A has the constants in its null space: fix at least one node with the
 * Dirichlet mask.
 *   op          operator index (0 <= op < n_ops), weights of either dtype
 *   f           device double[n]: F (the values g_i at Dirichlet nodes)
 *   phi         device double[n]: the initial guess in (its Dirichlet entries are set to f on
 *               entry, and then stay exact), the solution out (distinct from f)
 *   dirichlet   device uint8[n] or NULL
 *   tol         relative residual target, > 0;  max_iter >= 1
 *   iters_out   host, may be NULL: iterations taken (over all restarts)
 *   resid_out   host, may be NULL: the true relative residual ||F - A Phi|| / ||F|| at exit
 * Returns LABFM_OK only when that true residual is <= tol; LABFM_ERR_NOT_CONVERGED on a breakdown
 * that the restarts do not cure, when max_iter ends the iteration, or when the true residual stays
 * above tol after the restarts
 * (phi holds the last iterate).  Synchronises the context stream.  LABFM_ERR_STATE before labfm_build_weights.
 */
labfm_status labfm_solve(labfm_ctx *ctx, int op, const double *f, double *phi, const uint8_t *dirichlet,
                         double tol, int max_iter, int *iters_out, double *resid_out);

/*
 * labfm_solve with Neumann boundary rows (Sec. 5.2, the ghost-node treatment of a Neumann
 * boundary): for every boundary node b with a prescribed normal derivative g_b the node set holds
 * a ghost node g at r_b - n_b dr (n_b the unit normal into the domain), and the row of g is
 * replaced by the boundary normal derivative operator at b,
 *     A_gj = n_x w^(op_x)_jb + n_y w^(op_y)_jb  for every j in the stencil of b,
 *     A_gb = -(sum of those entries),           F_g = g_b,
 * so that the solution satisfies n . grad Phi = g_b at b while the ghost's value is free.  Every
 * other row is as in labfm_solve (operator op, identity rows where dirichlet is set).  The ghosts
 * are ordinary nodes of the stencil search and of the weight build (they complete the support of
 * the nodes near the wall; their own weights are not used).  The Jacobi scaling of a ghost row is
 * the inverse of its true diagonal, the entry of the ghost itself within the stencil of b (1 if
 * the ghost is not in that stencil).
 *   n_ghost        number of ghost rows, 0 <= n_ghost <= n (0: labfm_solve)
 *   ghost, parent  device int64[n_ghost]: the ghost's node index and its boundary node b
 *                  (distinct ghosts; ghost != parent; a ghost may not be a Dirichlet row)
 *   normal         device double[n_ghost][2]: (n_x, n_y), used as given (the paper's unit normal)
 *   op_x, op_y     operator indices of the weights giving d/dx and d/dy
 *   f              F as in labfm_solve, with F_g = g_b at each ghost row
 * The remaining arguments and the returns are those of labfm_solve; a bad index, a repeated
 * ghost, a ghost marked Dirichlet or a non-finite normal is LABFM_ERR_ARG (checked on the device
 * before the iteration).  Synchronises the context stream.
 */
labfm_status labfm_solve_neumann(labfm_ctx *ctx, int op, const double *f, double *phi, const uint8_t *dirichlet,
                                 int64_t n_ghost, const int64_t *ghost, const int64_t *parent, const double *normal,
                                 int op_x, int op_y, double tol, int max_iter, int *iters_out, double *resid_out);

/*
 * Stencil search that allocates nothing.  (The paper has no counterpart: this is an interface
 * for callers that cannot allocate device memory.)
 *
 * Some callers cannot call cudaMalloc: their device memory is owned entirely by another
 * allocator (a framework's caching pool, a fixed per-process budget on a shared GPU), or they
 * must not allocate once running (a latency-critical loop, where cudaMalloc may synchronise
 * the device).  This entry point computes the same stencils as labfm_build_neighbours
 * (identical predicate, identical CSR arrays, rows ascending in j) without a context and
 * without allocating: its scratch (the cell grid) lives in a fixed array of about 10 MB in the
 * library's device memory, which every GPU that loads the library holds until the process
 * exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 *   device          CUDA device to run on (made current for the call, then restored)
 *   stream          cudaStream_t the work is enqueued on (NULL = legacy default stream)
 *   n               number of nodes, 1 <= n <= LABFM_NOALLOC_MAX_NODES
 *   xy, h           device double[2n] (interleaved) and double[n], as in labfm_build_neighbours
 *   periodic, box_lo, box_hi   as in labfm_build_neighbours
 *   row_ptr         device int64[n+1], caller-owned, written
 *   col             device int32[col_capacity], caller-owned, written (may be NULL if 0)
 *   col_capacity    entries available in col
 *   nnz_out         host, receives the number of stencil entries (also on LABFM_ERR_CAPACITY,
 *                   so the caller can size col and call again)
 * Returns LABFM_ERR_ARG for bad arguments (as labfm_build_neighbours), LABFM_ERR_CAPACITY if
 * n > LABFM_NOALLOC_MAX_NODES or nnz > col_capacity (row_ptr is then valid, col untouched),
 * LABFM_ERR_CUDA on a CUDA error.  The call synchronises `stream` before returning.
 *
 * Every call looks up the device address of the fixed array with the device current (so a
 * reset of the device's primary context between calls is harmless); the first call on a device
 * also loads the library's device code there, so make it before any stream capture begins (the
 * call synchronises `stream` and cannot itself be captured).  All calls share the one array per
 * device: calls whose GPU work overlaps (on different streams or host threads) race on it and
 * must be serialised by the caller.  The array keeps the previous call's contents; every call
 * clears what it needs cleared.
 */
#define LABFM_NOALLOC_MAX_NODES 262144
labfm_status labfm_build_neighbours_noalloc(int device, void *stream, int64_t n, const double *xy, const double *h,
                                            int periodic, const double box_lo[2], const double box_hi[2],
                                            int64_t *row_ptr, int32_t *col, int64_t col_capacity, int64_t *nnz_out);

#ifdef __cplusplus
}
#endif

#endif /* LABFM_H */
