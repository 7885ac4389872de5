/*
 * labfm_oracle.c -- plain, slow, CPU reference of the LABFM weight build and
 * operator application (King, Lind & Nasar, "High order difference schemes
 * using the Local Anisotropic Basis Function Method").
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the timed CPU
 * baseline of the benchmark load this file; the library never does.  It shares
 * no code, header or table with the CUDA implementation.
 *
 * Every step follows the paper's definitions in the paper's order, with no
 * blocking, fusion or reordering:
 *   neighbours   all j != i with |r_ji| < 2 h_i, by brute force over j    (Sec. 2)
 *   X_ji         Taylor monomials x^a y^b / (a! b!), degree-major order    (Sec. 2, eq. X)
 *   W_ji         ABFs = D(W0) at r_ji (Sec. 3.2), full chain rule for the
 *                elements 1-9, only the dW0/dr term for elements >= 10
 *                (Appendix A, truncation rule)
 *   M_i          sum_j X_ji (outer) W_ji                                  (Eq. disc_form)
 *   Psi^d        Gaussian elimination with partial pivoting of M Psi = C^d (Eq. lsys)
 *   w_ji^d       W_ji . Psi^d                                             (Eq. w_abf)
 *   L_i^d(f)     sum_j (f_j - f_i) w_ji^d                                 (Eq. general_do)
 *   RK4          the classical four-stage scheme                          (Sec. 5.1)
 *   Burgers      RK4 of the viscous Burgers' equation                     (Sec. 5.3)
 *
 * Offsets are evaluated in units of h_i (rhat = r_ji / h_i) and C^d is scaled
 * by h_i^-|alpha| (Sec. 3.2: the elements of X scale with h^|alpha| and the
 * ABFs with h^-|alpha|).  This is the similarity transform
 * M = S Mhat S^-1, S = diag(h^|alpha|), so Psi = S Psihat and the physical
 * weights w = W . Psi = What . Psihat are identical in exact arithmetic.
 *
 * The derivatives of |r| used by the ABFs come from the Leibniz rule applied to
 * r * r = x^2 + y^2 at each point (an independent route from any table of
 * closed forms); the RBF derivatives come from expanding W0 as a polynomial in
 * t = 1 - q/2 (compact kernels) or as polynomial * exp(-9 q^2) (Gaussian) and
 * differentiating term by term.
 *
 * ORC_REAL selects the working precision: double (default), long double or
 * _Float128 (IEEE binary128, compiled with ORC_MANT_DIG=113); the wider ones are
 * used only to measure the rounding floor of the double build.
 * Compile with -ffp-contract=off so that no multiply-add is fused: the
 * neighbour predicate must round exactly as written.
 */
#include <float.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

#define ORC_KMAX 8
#define ORC_PMAX 44
#define ORC_PI 3.14159265358979323846264338327950288L

enum { RBF_WENDLAND_C2 = 0, RBF_QUADRATIC = 1, RBF_CONE = 2, RBF_WENDLAND_C6 = 3, RBF_GAUSSIAN = 4 };
enum { ST_OK = 0, ST_SINGULAR = 1, ST_UNDERSAMPLED = 2, ST_NONFINITE = 3 };

/* p = (k^2 + 3k)/2, Sec. 3.1 */
int orc_p_of_k(int k) { return (k * k + 3 * k) / 2; }

/* 0-based element e -> (a, b) of x^a y^b: degree n ascending, a from n down to 0 */
void orc_element_ab(int e, int *a, int *b)
{
    int n = 1;
    while (orc_p_of_k(n) <= e) n++;
    int pos = e - orc_p_of_k(n - 1); /* 0 .. n */
    *a = n - pos;
    *b = pos;
}

/* ---------------------------------------------------------------------------
 * Neighbour search: brute force over all j (Sec. 2: stencil radius 2h, j != i).
 * Minimum-image offsets in a periodic box.  r2 = dx*dx + dy*dy and the
 * acceptance r2 < (2 h_i)^2 are evaluated in double exactly as written.
 * queries: indices of the nodes whose stencils are wanted (NULL = all n).
 * Pass col == NULL to only count; row_ptr[nq+1] is always written.
 * Returns 0, or -1 when a stencil would exceed `cap` entries in total.
 * ------------------------------------------------------------------------- */
int orc_neighbours(int64_t n, const double *xy, const double *h, int periodic,
                   const double *lo, const double *hi, const int64_t *queries, int64_t nq,
                   int64_t *row_ptr, int32_t *col, int64_t cap)
{
    double L[2] = {hi[0] - lo[0], hi[1] - lo[1]};
    double halfL[2] = {0.5 * L[0], 0.5 * L[1]};
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int64_t q = 0; q < nq; q++) {
        int64_t i = queries ? queries[q] : q;
        double xi = xy[2 * i], yi = xy[2 * i + 1];
        double R = 2.0 * h[i];
        double R2 = R * R;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = xy[2 * j] - xi;
            double dy = xy[2 * j + 1] - yi;
            if (periodic) {
                if (dx > halfL[0]) dx -= L[0];
                else if (dx < -halfL[0]) dx += L[0];
                if (dy > halfL[1]) dy -= L[1];
                else if (dy < -halfL[1]) dy += L[1];
            }
            double r2 = dx * dx + dy * dy;
            if (r2 < R2) {
                if (col) {
                    if (nnz >= cap) return -1;
                    col[nnz] = (int32_t)j;
                }
                nnz++;
            }
        }
        row_ptr[q + 1] = nnz;
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Fundamental RBFs W0(q) (Sec. 3.2 and Appendix A) and their first three
 * derivatives d^m W0 / dq^m at q (m = 0..3).
 * ------------------------------------------------------------------------- */

/* polynomial helpers: c[0] + c[1] q + ... (degree < 16) */
typedef struct { int deg; real c[16]; } poly;

static poly poly_const(real v) { poly p; memset(&p, 0, sizeof p); p.deg = 0; p.c[0] = v; return p; }
static poly poly_lin(real c0, real c1) { poly p = poly_const(c0); p.deg = 1; p.c[1] = c1; return p; }
static poly poly_mul(poly a, poly b)
{
    poly r; memset(&r, 0, sizeof r);
    r.deg = a.deg + b.deg;
    for (int i = 0; i <= a.deg; i++)
        for (int j = 0; j <= b.deg; j++) r.c[i + j] += a.c[i] * b.c[j];
    return r;
}
static poly poly_pow(poly a, int e) { poly r = poly_const(1); for (int i = 0; i < e; i++) r = poly_mul(r, a); return r; }
static poly poly_der(poly a)
{
    poly r; memset(&r, 0, sizeof r);
    r.deg = a.deg > 0 ? a.deg - 1 : 0;
    for (int i = 1; i <= a.deg; i++) r.c[i - 1] = a.c[i] * (real)i;
    return r;
}
static real poly_eval(poly a, real q) { real v = 0; for (int i = a.deg; i >= 0; i--) v = v * q + a.c[i]; return v; }

/* P(a + b t) as a polynomial in t */
static poly poly_compose_lin(poly P, real a, real b)
{
    poly r = poly_const(0), pw = poly_const(1), lin = poly_lin(a, b);
    for (int i = 0; i <= P.deg; i++) {
        for (int j = 0; j <= pw.deg; j++) r.c[j] += P.c[i] * pw.c[j];
        if (pw.deg > r.deg) r.deg = pw.deg;
        pw = poly_mul(pw, lin);
    }
    return r;
}

/* The compactly supported kernels as polynomials in t = 1 - q/2 (q = 2 - 2t), so that
 * the factor (1 - q/2)^m is a plain power of t and no cancellation occurs near q = 2. */
static poly rbf_poly_t(int rbf)
{
    const real pi = (real)ORC_PI;
    poly t1 = poly_lin(0, 1); /* t */
    switch (rbf) {
    case RBF_WENDLAND_C2: /* 7/(4 pi) (1 - q/2)^4 (1 + 2q) */
        return poly_mul(poly_const(7 / (4 * pi)),
                        poly_mul(poly_pow(t1, 4), poly_compose_lin(poly_lin(1, 2), 2, -2)));
    case RBF_QUADRATIC: /* 3/(16 pi) (q - 2)^2, Appendix A.1 */
        return poly_mul(poly_const(3 / (16 * pi)), poly_pow(poly_compose_lin(poly_lin(-2, 1), 2, -2), 2));
    case RBF_CONE: /* 3/(4 pi) (1 - q/2), Sec. 3.2 */
        return poly_mul(poly_const(3 / (4 * pi)), t1);
    case RBF_WENDLAND_C6: { /* 78/(28 pi) (1 - q/2)^8 (4 q^3 + 6.25 q^2 + 4 q + 1), Appendix A.2 */
        poly b = poly_const(1); b.deg = 3; b.c[1] = 4; b.c[2] = 6.25; b.c[3] = 4;
        return poly_mul(poly_const(78 / (28 * pi)), poly_mul(poly_pow(t1, 8), poly_compose_lin(b, 2, -2)));
    }
    default:
        return poly_const(0);
    }
}

/* d[m] = d^m W0/dq^m (q), m = 0..3 */
void orc_rbf_derivs_r(int rbf, real q, real *d)
{
    if (rbf == RBF_GAUSSIAN) {
        /* W0 = 9/pi exp(-9 q^2), Appendix A.3.  d^m/dq^m exp(-9q^2) = P_m(q) exp(-9q^2)
         * with P_0 = 1 and P_{m+1} = P_m' - 18 q P_m. */
        const real pi = (real)ORC_PI;
        real e = (9 / pi) * exp(-9 * q * q);
        poly P = poly_const(1);
        for (int m = 0; m < 4; m++) {
            d[m] = poly_eval(P, q) * e;
            poly Pd = poly_der(P);
            poly t = poly_mul(poly_lin(0, -18), P);
            poly nx; memset(&nx, 0, sizeof nx);
            nx.deg = t.deg > Pd.deg ? t.deg : Pd.deg;
            for (int i = 0; i <= nx.deg; i++) nx.c[i] = t.c[i] + Pd.c[i];
            P = nx;
        }
        return;
    }
    /* d/dq = -1/2 d/dt */
    poly P = rbf_poly_t(rbf);
    real t = 1 - q / 2, sc = 1;
    for (int m = 0; m < 4; m++) {
        d[m] = (q < 2) ? sc * poly_eval(P, t) : 0;
        P = poly_der(P);
        sc *= (real)-0.5;
    }
}

void orc_rbf_derivs(int rbf, double q, double *d)
{
    real dr[4];
    orc_rbf_derivs_r(rbf, (real)q, dr);
    for (int m = 0; m < 4; m++) d[m] = (double)dr[m];
}

/* ---------------------------------------------------------------------------
 * Partial derivatives of r = |(x, y)|: dr[a][b] = d^(a+b) r / dx^a dy^b for
 * a + b <= kmax, by differentiating r * r = x^2 + y^2 (Leibniz rule):
 *   2 r d^alpha r = d^alpha(x^2 + y^2) - sum_{0 < beta < alpha} C(alpha, beta) d^beta r d^(alpha-beta) r
 * ------------------------------------------------------------------------- */
static real binom(int n, int k)
{
    real v = 1;
    for (int i = 1; i <= k; i++) v = v * (real)(n - k + i) / (real)i;
    return v;
}

static void dr_table(real x, real y, int kmax, real dr[ORC_KMAX + 1][ORC_KMAX + 1])
{
    real r = sqrt(x * x + y * y);
    dr[0][0] = r;
    for (int n = 1; n <= kmax; n++) {
        for (int a = n; a >= 0; a--) {
            int b = n - a;
            real rhs = 0;
            if (a == 1 && b == 0) rhs = 2 * x;
            if (a == 0 && b == 1) rhs = 2 * y;
            if ((a == 2 && b == 0) || (a == 0 && b == 2)) rhs = 2;
            for (int a2 = 0; a2 <= a; a2++)
                for (int b2 = 0; b2 <= b; b2++) {
                    if ((a2 == 0 && b2 == 0) || (a2 == a && b2 == b)) continue;
                    rhs -= binom(a, a2) * binom(b, b2) * dr[a2][b2] * dr[a - a2][b - b2];
                }
            dr[a][b] = rhs / (2 * r);
        }
    }
}

void orc_dr(double x, double y, int kmax, double *out /* [(kmax+1)^2], out[a*(kmax+1)+b] */)
{
    real t[ORC_KMAX + 1][ORC_KMAX + 1];
    dr_table((real)x, (real)y, kmax, t);
    for (int a = 0; a <= kmax; a++)
        for (int b = 0; b <= kmax - a; b++) out[a * (kmax + 1) + b] = (double)t[a][b];
}

/* ---------------------------------------------------------------------------
 * Monomials X (Sec. 2, eq. X): X_e = x^a y^b / (a! b!)
 * ------------------------------------------------------------------------- */
static void monomials_r(real x, real y, int k, real *X)
{
    int p = orc_p_of_k(k);
    for (int e = 0; e < p; e++) {
        int a, b;
        orc_element_ab(e, &a, &b);
        real v = 1;
        for (int t = 1; t <= a; t++) v = v * x / (real)t;
        for (int t = 1; t <= b; t++) v = v * y / (real)t;
        X[e] = v;
    }
}

void orc_monomials(double x, double y, int k, double *X)
{
    real t[ORC_PMAX];
    monomials_r((real)x, (real)y, k, t);
    for (int e = 0; e < orc_p_of_k(k); e++) X[e] = (double)t[e];
}

/* ---------------------------------------------------------------------------
 * ABFs W = D(W0(|r|)) at (x, y) with h = 1 (Sec. 3.2, Appendix A).
 * Elements 1..9 (|alpha| <= 3): the chain rule for W0(r(x, y)) with all of
 * W0', W0'', W0'''; elements >= 10 (|alpha| >= 4): W0'(r) d^alpha r only.
 * With ORC_ABF_DW0_ONLY set in rbf_form, the W0'' and W0''' terms are dropped
 * for the elements 1..9 as well, so that every element is W0'(r) d^alpha r.
 * ------------------------------------------------------------------------- */
#define ORC_ABF_DW0_ONLY 0x100
static void abfs_r(int rbf_form, real x, real y, int k, real *W)
{
    int p = orc_p_of_k(k);
    int rbf = rbf_form & 0xff;
    real dr[ORC_KMAX + 1][ORC_KMAX + 1];
    dr_table(x, y, k < 3 ? 3 : k, dr);
    real d[4];
    orc_rbf_derivs_r(rbf, dr[0][0], d);
    real f1 = d[1], f2 = d[2], f3 = d[3];
    if (rbf_form & ORC_ABF_DW0_ONLY) f2 = f3 = 0;
    real rx = dr[1][0], ry = dr[0][1];
    real rxx = dr[2][0], rxy = dr[1][1], ryy = dr[0][2];
    for (int e = 0; e < p; e++) {
        int a, b;
        orc_element_ab(e, &a, &b);
        int n = a + b;
        real v = f1 * dr[a][b];
        if (n == 2) {
            if (a == 2) v += f2 * rx * rx;
            if (a == 1) v += f2 * rx * ry;
            if (a == 0) v += f2 * ry * ry;
        } else if (n == 3) {
            if (a == 3) v += f3 * rx * rx * rx + f2 * 3 * rx * rxx;
            if (a == 2) v += f3 * rx * rx * ry + f2 * (ry * rxx + 2 * rx * rxy);
            if (a == 1) v += f3 * rx * ry * ry + f2 * (rx * ryy + 2 * ry * rxy);
            if (a == 0) v += f3 * ry * ry * ry + f2 * 3 * ry * ryy;
        }
        W[e] = v;
    }
}

void orc_abfs(int rbf, double x, double y, int k, double *W)
{
    real t[ORC_PMAX];
    abfs_r(rbf, (real)x, (real)y, k, t);
    for (int e = 0; e < orc_p_of_k(k); e++) W[e] = (double)t[e];
}

/* ---------------------------------------------------------------------------
 * Gaussian elimination with partial pivoting of A (p x p, row-major) on the
 * augmented right-hand sides B (p x nr, row-major); on return B holds the
 * solution.  Pivot: largest |A[r][c]|, r >= c, first one wins.
 * Returns 0, or 1 when a pivot is exactly zero or non-finite.
 * ------------------------------------------------------------------------- */
static int gauss_solve(int p, real *A, int nr, real *B, real *min_piv_ratio)
{
    real amax = 0;
    for (int t = 0; t < p * p; t++) if (fabs(A[t]) > amax) amax = fabs(A[t]);
    real minpiv = INFINITY;
    for (int c = 0; c < p; c++) {
        int piv = c;
        real best = fabs(A[c * p + c]);
        for (int r = c + 1; r < p; r++)
            if (fabs(A[r * p + c]) > best) { best = fabs(A[r * p + c]); piv = r; }
        if (!(best > 0) || !isfinite(best)) return 1;
        if (best < minpiv) minpiv = best;
        if (piv != c) {
            for (int t = 0; t < p; t++) { real s = A[c * p + t]; A[c * p + t] = A[piv * p + t]; A[piv * p + t] = s; }
            for (int t = 0; t < nr; t++) { real s = B[c * nr + t]; B[c * nr + t] = B[piv * nr + t]; B[piv * nr + t] = s; }
        }
        for (int r = c + 1; r < p; r++) {
            real l = A[r * p + c] / A[c * p + c];
            if (l == 0) continue;
            for (int t = c; t < p; t++) A[r * p + t] -= l * A[c * p + t];
            for (int t = 0; t < nr; t++) B[r * nr + t] -= l * B[c * nr + t];
        }
    }
    for (int c = p - 1; c >= 0; c--) {
        for (int t = 0; t < nr; t++) {
            real s = B[c * nr + t];
            for (int u = c + 1; u < p; u++) s -= A[c * p + u] * B[u * nr + t];
            B[c * nr + t] = s / A[c * p + c];
        }
    }
    if (min_piv_ratio) *min_piv_ratio = amax > 0 ? minpiv / amax : 0;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Weight build for a set of query nodes.
 *   row_ptr/col    the stencils of the queries (as orc_neighbours wrote them)
 *   order          per-node k (int8, indexed by node id) or NULL -> uniform_k
 *   C              n_ops x 44 target vectors in D ordering, physical units
 *   w              out, nnz x n_ops (row-major: w[e*n_ops + d]), physical units
 *   status         out, per query (ST_*)
 *   piv_ratio      out (may be NULL): min |pivot| / max |Mhat| per query
 *   mhat_out       out (may be NULL): per query the p x p Mhat, row-major, stride 44*44
 * ------------------------------------------------------------------------- */
static int build_one(int64_t i, const double *xy, const double *h, int periodic, const double *L,
                     const int32_t *nb, int64_t ni, int k, int rbf, int n_ops, const double *C,
                     double *w, double *piv_ratio, double *mhat_out)
{
    int p = orc_p_of_k(k);
    if (ni < p) {
        for (int64_t t = 0; t < ni * n_ops; t++) w[t] = 0;
        if (piv_ratio) *piv_ratio = 0;
        return ST_UNDERSAMPLED;
    }
    real hi = (real)h[i];
    real *X = (real *)malloc(sizeof(real) * ni * p);
    real *W = (real *)malloc(sizeof(real) * ni * p);
    real M[ORC_PMAX * ORC_PMAX];
    real B[ORC_PMAX * 16];
    for (int64_t j = 0; j < ni; j++) {
        int64_t jj = nb[j];
        double dx = xy[2 * jj] - xy[2 * i];
        double dy = xy[2 * jj + 1] - xy[2 * i + 1];
        if (periodic) {
            if (dx > 0.5 * L[0]) dx -= L[0];
            else if (dx < -0.5 * L[0]) dx += L[0];
            if (dy > 0.5 * L[1]) dy -= L[1];
            else if (dy < -0.5 * L[1]) dy += L[1];
        }
        real xh = (real)dx / hi, yh = (real)dy / hi;
        monomials_r(xh, yh, k, X + j * p);
        abfs_r(rbf, xh, yh, k, W + j * p);
    }
    /* M_i = sum_j X_ji (outer) W_ji : rows = monomials, columns = ABFs (Eq. disc_form) */
    for (int m = 0; m < p; m++)
        for (int c = 0; c < p; c++) {
            real s = 0;
            for (int64_t j = 0; j < ni; j++) s += X[j * p + m] * W[j * p + c];
            M[m * p + c] = s;
        }
    if (mhat_out)
        for (int t = 0; t < p * p; t++) mhat_out[t] = (double)M[t];
    /* a non-finite entry of M (e.g. a neighbour on top of node i, where the ABFs are
     * singular, Sec. 3.2) makes the node's weights meaningless */
    for (int t = 0; t < p * p; t++)
        if (!isfinite(M[t])) {
            for (int64_t u = 0; u < ni * n_ops; u++) w[u] = 0;
            if (piv_ratio) *piv_ratio = 0;
            free(X); free(W);
            return ST_NONFINITE;
        }
    /* scaled targets Chat_alpha = C_alpha h^-|alpha| */
    for (int m = 0; m < p; m++) {
        int a, b;
        orc_element_ab(m, &a, &b);
        real s = 1;
        for (int t = 0; t < a + b; t++) s /= hi;
        for (int d = 0; d < n_ops; d++) B[m * n_ops + d] = (real)C[d * ORC_PMAX + m] * s;
    }
    real pr = 0;
    int st = gauss_solve(p, M, n_ops, B, &pr);
    if (piv_ratio) *piv_ratio = (double)pr;
    if (st) {
        for (int64_t t = 0; t < ni * n_ops; t++) w[t] = 0;
        free(X); free(W);
        return ST_SINGULAR;
    }
    /* w_ji^d = W_ji . Psi^d (Eq. w_abf) */
    int bad = 0;
    for (int64_t j = 0; j < ni; j++)
        for (int d = 0; d < n_ops; d++) {
            real s = 0;
            for (int c = 0; c < p; c++) s += W[j * p + c] * B[c * n_ops + d];
            w[j * n_ops + d] = (double)s;
            if (!isfinite(w[j * n_ops + d])) bad = 1;
        }
    free(X); free(W);
    if (bad) {
        for (int64_t t = 0; t < ni * n_ops; t++) w[t] = 0;
        return ST_NONFINITE;
    }
    return ST_OK;
}

int orc_build_weights(const double *xy, const double *h, int periodic, const double *lo, const double *hi,
                      const int64_t *queries, int64_t nq, const int64_t *row_ptr, const int32_t *col,
                      const int8_t *order, int uniform_k, int rbf, int n_ops, const double *C,
                      double *w, int32_t *status, double *piv_ratio, double *mhat_out, int nthreads)
{
    if (n_ops < 1 || n_ops > 16) return -1;
    double L[2] = {hi[0] - lo[0], hi[1] - lo[1]};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t q = 0; q < nq; q++) {
        int64_t i = queries ? queries[q] : q;
        int k = order ? order[i] : uniform_k;
        int64_t b = row_ptr[q], e = row_ptr[q + 1];
        status[q] = build_one(i, xy, h, periodic, L, col + b, e - b, k, rbf, n_ops, C, w + b * n_ops,
                              piv_ratio ? piv_ratio + q : NULL,
                              mhat_out ? mhat_out + q * ORC_PMAX * ORC_PMAX : NULL);
    }
    (void)nthreads;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Operator application, Eq. general_do: out[d][q] = sum_j (f_j - f_i) w_ji^d.
 * ------------------------------------------------------------------------- */
void orc_apply(const int64_t *queries, int64_t nq, const int64_t *row_ptr, const int32_t *col,
               const double *w, int n_ops, const double *f, double *out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t q = 0; q < nq; q++) {
        int64_t i = queries ? queries[q] : q;
        for (int d = 0; d < n_ops; d++) {
            real s = 0;
            for (int64_t e = row_ptr[q]; e < row_ptr[q + 1]; e++)
                s += ((real)f[col[e]] - (real)f[i]) * (real)w[e * n_ops + d];
            out[d * nq + q] = (double)s;
        }
    }
    (void)nthreads;
}

/* ---------------------------------------------------------------------------
 * Classical RK4 (Sec. 5.1) for du/dt = F(u), F(u)_i = sum_d beta_d L_i^d(u),
 * over all n nodes (row_ptr/col/w cover every node).  Nodes with frozen[i]
 * set keep their value (Dirichlet nodes, Sec. 5.1): a fixed boundary value has
 * du/dt = 0, so F_i = 0 there in every stage.
 * ------------------------------------------------------------------------- */
static void rhs_eval(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w, int n_ops,
                     const double *beta, const real *u, real *F, const uint8_t *frozen)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; i++) {
        real s = 0;
        for (int d = 0; d < n_ops; d++) {
            real sd = 0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) sd += (u[col[e]] - u[i]) * (real)w[e * n_ops + d];
            s += (real)beta[d] * sd;
        }
        F[i] = (frozen && frozen[i]) ? 0 : s;
    }
}

int orc_rk4(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w, int n_ops,
            const double *beta, double *u_io, double dt, int64_t nsteps, const uint8_t *frozen, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    real *u = (real *)malloc(sizeof(real) * n), *ut = (real *)malloc(sizeof(real) * n);
    real *k1 = (real *)malloc(sizeof(real) * n), *k2 = (real *)malloc(sizeof(real) * n);
    real *k3 = (real *)malloc(sizeof(real) * n), *k4 = (real *)malloc(sizeof(real) * n);
    if (!u || !ut || !k1 || !k2 || !k3 || !k4) return -1;
    for (int64_t i = 0; i < n; i++) u[i] = (real)u_io[i];
    real hdt = (real)dt / 2, fdt = (real)dt;
    for (int64_t s = 0; s < nsteps; s++) {
        rhs_eval(n, row_ptr, col, w, n_ops, beta, u, k1, frozen);
        for (int64_t i = 0; i < n; i++) ut[i] = u[i] + hdt * k1[i];
        rhs_eval(n, row_ptr, col, w, n_ops, beta, ut, k2, frozen);
        for (int64_t i = 0; i < n; i++) ut[i] = u[i] + hdt * k2[i];
        rhs_eval(n, row_ptr, col, w, n_ops, beta, ut, k3, frozen);
        for (int64_t i = 0; i < n; i++) ut[i] = u[i] + fdt * k3[i];
        rhs_eval(n, row_ptr, col, w, n_ops, beta, ut, k4, frozen);
        for (int64_t i = 0; i < n; i++) u[i] = u[i] + fdt / 6 * (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]);
    }
    for (int64_t i = 0; i < n; i++) u_io[i] = (double)u[i];
    free(u); free(ut); free(k1); free(k2); free(k3); free(k4);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Classical RK4 for the viscous Burgers' equation (Sec. 5.3, eq. burgers),
 * du/dt + (u . grad) u = (1/Re) nabla^2 u with u = (u, v), written with the
 * discrete operators as
 *   du/dt = -(u_i L^0_i(u) + v_i L^1_i(u)) + sum_{d>=2} beta_d L^d_i(u)
 *   dv/dt = -(u_i L^0_i(v) + v_i L^1_i(v)) + sum_{d>=2} beta_d L^d_i(v)
 * where operators 0 and 1 are d/dx and d/dy (the caller builds them so) and
 * beta_2 = 1/Re multiplies the Laplacian.  Frozen nodes keep both values.
 * ------------------------------------------------------------------------- */
static real op_sum(const int64_t *row_ptr, const int32_t *col, const double *w, int n_ops, int d, const real *f,
                   int64_t i)
{
    real s = 0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) s += (f[col[e]] - f[i]) * (real)w[e * n_ops + d];
    return s;
}

static void burgers_rhs(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w, int n_ops,
                        const double *beta, const real *u, const real *v, real *Fu, real *Fv, const uint8_t *frozen)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; i++) {
        real fu = -(u[i] * op_sum(row_ptr, col, w, n_ops, 0, u, i) + v[i] * op_sum(row_ptr, col, w, n_ops, 1, u, i));
        real fv = -(u[i] * op_sum(row_ptr, col, w, n_ops, 0, v, i) + v[i] * op_sum(row_ptr, col, w, n_ops, 1, v, i));
        for (int d = 2; d < n_ops; d++) {
            fu += (real)beta[d] * op_sum(row_ptr, col, w, n_ops, d, u, i);
            fv += (real)beta[d] * op_sum(row_ptr, col, w, n_ops, d, v, i);
        }
        Fu[i] = (frozen && frozen[i]) ? 0 : fu;
        Fv[i] = (frozen && frozen[i]) ? 0 : fv;
    }
}

int orc_rk4_burgers(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w, int n_ops,
                    const double *beta, double *u_io, double *v_io, double dt, int64_t nsteps, const uint8_t *frozen,
                    int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    if (n_ops < 2) return -2;
    real *buf = (real *)malloc(sizeof(real) * n * 12);
    if (!buf) return -1;
    real *u = buf, *v = buf + n, *ut = buf + 2 * n, *vt = buf + 3 * n;
    real *k[4][2];
    for (int s = 0; s < 4; s++) {
        k[s][0] = buf + (4 + 2 * s) * n;
        k[s][1] = buf + (5 + 2 * s) * n;
    }
    for (int64_t i = 0; i < n; i++) {
        u[i] = (real)u_io[i];
        v[i] = (real)v_io[i];
    }
    const real hdt = (real)dt / 2, fdt = (real)dt;
    for (int64_t st = 0; st < nsteps; st++) {
        burgers_rhs(n, row_ptr, col, w, n_ops, beta, u, v, k[0][0], k[0][1], frozen);
        for (int64_t i = 0; i < n; i++) {
            ut[i] = u[i] + hdt * k[0][0][i];
            vt[i] = v[i] + hdt * k[0][1][i];
        }
        burgers_rhs(n, row_ptr, col, w, n_ops, beta, ut, vt, k[1][0], k[1][1], frozen);
        for (int64_t i = 0; i < n; i++) {
            ut[i] = u[i] + hdt * k[1][0][i];
            vt[i] = v[i] + hdt * k[1][1][i];
        }
        burgers_rhs(n, row_ptr, col, w, n_ops, beta, ut, vt, k[2][0], k[2][1], frozen);
        for (int64_t i = 0; i < n; i++) {
            ut[i] = u[i] + fdt * k[2][0][i];
            vt[i] = v[i] + fdt * k[2][1][i];
        }
        burgers_rhs(n, row_ptr, col, w, n_ops, beta, ut, vt, k[3][0], k[3][1], frozen);
        for (int64_t i = 0; i < n; i++) {
            u[i] = u[i] + fdt / 6 * (k[0][0][i] + 2 * k[1][0][i] + 2 * k[2][0][i] + k[3][0][i]);
            v[i] = v[i] + fdt / 6 * (k[0][1][i] + 2 * k[1][1][i] + 2 * k[2][1][i] + k[3][1][i]);
        }
    }
    for (int64_t i = 0; i < n; i++) {
        u_io[i] = (double)u[i];
        v_io[i] = (double)v[i];
    }
    free(buf);
    return 0;
}

/* precision of the real type this file was compiled with, in bits of significand */
#ifndef ORC_MANT_DIG
#define ORC_MANT_DIG (sizeof(real) == sizeof(double) ? DBL_MANT_DIG : LDBL_MANT_DIG)
#endif
int orc_real_mant_bits(void) { return ORC_MANT_DIG; }
