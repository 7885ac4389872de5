// Device evaluation of the Taylor monomials X (Sec. 2) and the anisotropic basis functions
// W = D(W0)|r (Sec. 3.2, Appendix A) at a scaled offset (x, y) = r_ji / h_i.
//
// Derivatives of |r|: d^alpha |r| = P_alpha(u, v) |r|^(1 - |alpha|), u = x/|r|, v = y/|r|,
// where P_alpha is a homogeneous polynomial of degree |alpha| with integer coefficients.
// Differentiating P |r|^(1-2n)... gives the recurrences (n = |alpha|)
//   P_{alpha+e_x} = (x^2 + y^2) dP/dx - (2n - 1) x P,
//   P_{alpha+e_y} = (x^2 + y^2) dP/dy - (2n - 1) y P,
// starting from P_(1,0) = x, P_(0,1) = y.  The table is built by a constexpr function, so it
// is a compile-time constant in constant memory.
#pragma once

#include "labfm_internal.cuh"

namespace labfm {

struct RPolyTable {
    // c[e][t]: coefficient of u^t v^(n-t) in P for element e (0-based, degree-major order)
    double c[PMAX][KMAX + 1];
};

__host__ __device__ constexpr int elem_degree(int e)
{
    int n = 1;
    while (p_of_k(n) <= e) n++;
    return n;
}
// power of x of element e
__host__ __device__ constexpr int elem_a(int e)
{
    int n = elem_degree(e);
    return n - (e - p_of_k(n - 1));
}
__host__ __device__ constexpr int elem_index(int a, int b) { return p_of_k(a + b - 1) + b; }

constexpr RPolyTable make_rpoly_table()
{
    RPolyTable T{};
    // degree 1
    T.c[elem_index(1, 0)][1] = 1.0;  // x
    T.c[elem_index(0, 1)][0] = 1.0;  // y
    for (int n = 1; n < KMAX; n++) {
        for (int a = n; a >= 0; a--) {
            int b = n - a;
            const double *p = T.c[elem_index(a, b)];
            // child via x: (a+1, b)
            {
                double *q = T.c[elem_index(a + 1, b)];
                bool set = false;
                for (int t = 0; t <= n + 1; t++) set |= (q[t] != 0.0);
                if (!set) {
                    for (int t = 0; t <= n; t++) {
                        double pt = p[t];
                        if (pt == 0.0) continue;
                        // (x^2 + y^2) * t x^(t-1) y^(n-t):  -> x^(t+1) y^(n-t) and x^(t-1) y^(n-t+2)
                        if (t >= 1) {
                            q[t + 1] += t * pt;
                            q[t - 1] += t * pt;
                        }
                        // -(2n-1) x * x^t y^(n-t) -> x^(t+1)
                        q[t + 1] -= (2 * n - 1) * pt;
                    }
                }
            }
            // child via y: (a, b+1), only needed for a == 0 (other elements come via x)
            if (a == 0) {
                double *q = T.c[elem_index(0, b + 1)];
                for (int t = 0; t <= n; t++) {
                    double pt = p[t];
                    if (pt == 0.0) continue;
                    // (x^2 + y^2) * (n-t) x^t y^(n-t-1) -> x^(t+2) y^(n-t-1) and x^t y^(n-t+1)
                    if (n - t >= 1) {
                        q[t + 2] += (n - t) * pt;
                        q[t] += (n - t) * pt;
                    }
                    q[t] -= (2 * n - 1) * pt;
                }
            }
        }
    }
    return T;
}

// d^m W0/dq^m, m = 1..3, at q in [0, 2) for the kernels of labfm.h.  rbf_form is a
// LABFM_RBF_* value, optionally with LABFM_ABF_DW0_ONLY: then d2 = d3 = 0, which reduces the
// chain rule of the elements 1..9 to dW0/dq d^alpha|r| (the form of the elements >= 10).
__device__ __forceinline__ void rbf_derivs(int rbf_form, double q, double &d1, double &d2, double &d3)
{
    const double PI = 3.141592653589793238462643383279502884;
    double t = 1.0 - 0.5 * q;
    switch (rbf_form & LABFM_RBF_MASK) {
    case LABFM_RBF_WENDLAND_C2: {  // W = c t^4 (1 + 2q)
        const double c = 7.0 / (4.0 * PI);
        d1 = -5.0 * c * q * t * t * t;
        d2 = -5.0 * c * t * t * (1.0 - 2.0 * q);
        d3 = 15.0 * c * t * (1.0 - q);
        break;
    }
    case LABFM_RBF_QUADRATIC: {  // W = c (q - 2)^2
        const double c = 3.0 / (16.0 * PI);
        d1 = 2.0 * c * (q - 2.0);
        d2 = 2.0 * c;
        d3 = 0.0;
        break;
    }
    case LABFM_RBF_CONE: {  // W = c (1 - q/2)
        const double c = 3.0 / (4.0 * PI);
        d1 = -0.5 * c;
        d2 = 0.0;
        d3 = 0.0;
        break;
    }
    case LABFM_RBF_WENDLAND_C6: {  // W = c T B, T = t^8, B = 4q^3 + 6.25q^2 + 4q + 1
        const double c = 78.0 / (28.0 * PI);
        double t2 = t * t, t4 = t2 * t2, t5 = t4 * t, t6 = t4 * t2, t7 = t6 * t, t8 = t4 * t4;
        double T0 = t8, T1 = -4.0 * t7, T2 = 14.0 * t6, T3 = -42.0 * t5;
        double B0 = ((4.0 * q + 6.25) * q + 4.0) * q + 1.0;
        double B1 = (12.0 * q + 12.5) * q + 4.0;
        double B2 = 24.0 * q + 12.5;
        double B3 = 24.0;
        d1 = c * (T1 * B0 + T0 * B1);
        d2 = c * (T2 * B0 + 2.0 * T1 * B1 + T0 * B2);
        d3 = c * (T3 * B0 + 3.0 * T2 * B1 + 3.0 * T1 * B2 + T0 * B3);
        break;
    }
    default: {  // Gaussian W = c exp(-9 q^2)
        const double c = 9.0 / PI;
        double W = c * exp(-9.0 * q * q);
        d1 = -18.0 * q * W;
        d2 = (324.0 * q * q - 18.0) * W;
        d3 = (972.0 * q - 5832.0 * q * q * q) * W;
        break;
    }
    }
    if (rbf_form & LABFM_ABF_DW0_ONLY) d2 = d3 = 0.0;
}

namespace {

__constant__ RPolyTable c_rpoly = make_rpoly_table();
__constant__ double c_invfact[KMAX + 1] = {1.0,       1.0,        0.5,         1.0 / 6.0,   1.0 / 24.0,
                                           1.0 / 120, 1.0 / 720., 1.0 / 5040., 1.0 / 40320.};

// 1 / (a! b!) as the product of the two reciprocals above, rounded once (the value a product of
// the two entries of c_invfact gives at run time)
struct InvFact2 {
    double v[KMAX + 1][KMAX + 1];
};
constexpr InvFact2 make_invfact2()
{
    const double f[KMAX + 1] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120, 1.0 / 720., 1.0 / 5040., 1.0 / 40320.};
    InvFact2 T{};
    for (int a = 0; a <= KMAX; a++)
        for (int b = 0; b <= KMAX; b++) T.v[a][b] = f[a] * f[b];
    return T;
}
__constant__ InvFact2 c_invfact2 = make_invfact2();

// The coefficients of the |r|-polynomials on the scaled monomials: P_(a,b)(x, y) =
// sum_t c[e][t] x^t y^(n-t) = sum_t c[e][t] t! (n-t)! X_(t,n-t), exact integers in double
// (below 2^26 at order 8)
constexpr RPolyTable make_rpolyf_table()
{
    RPolyTable T = make_rpoly_table();
    double f[KMAX + 1] = {1, 1, 2, 6, 24, 120, 720, 5040, 40320};
    for (int e = 0; e < PMAX; e++) {
        const int n = elem_degree(e);
        for (int t = 0; t <= n; t++) T.c[e][t] *= f[t] * f[n - t];
    }
    return T;
}
__constant__ RPolyTable c_rpolyf = make_rpolyf_table();

// Monomials and ABFs of one scaled offset (x, y), written to X[0..P), W[0..P).  With
// q = |(x, y)| and degree n = a + b:
//   X_(a,b) = x^a y^b / (a! b!)        d^(a,b)|r| = q^(1-2n) P_(a,b)(x, y)
// (P_(a,b) homogeneous of degree n), and P_(a,b)(x, y) = sum_t c~[e][t] X_(t,n-t) on the
// monomials of the same degree, so that one multiply per element forms X and serves W: on GB300
// every FP64 multiply takes the FP64 pipe's time.  d^(a,b)|r| has the parity of a in x (|r| is
// even in x and y), so P_(a,b) has only the terms of t of the parity of a: the others are skipped
// (their coefficients are exactly zero).  Results go straight to shared memory to keep the
// register footprint small.
template <int K>
__device__ __forceinline__ void eval_xw(double x, double y, int rbf, double *__restrict__ X, double *__restrict__ W)
{
    double q = sqrt(x * x + y * y);
    double iq = 1.0 / q;
    double d1, d2, d3;
    rbf_derivs(rbf, q, d1, d2, d3);
    // x^a / a!, y^b / b!
    double xs[K + 1], ys[K + 1];
    xs[0] = ys[0] = 1.0;
    {
        double xp = 1.0, yp = 1.0;
#pragma unroll
        for (int t = 1; t <= K; t++) {
            xp *= x;
            yp *= y;
            xs[t] = xp * c_invfact2.v[t][0];
            ys[t] = yp * c_invfact2.v[t][0];
        }
    }
    const double iq2 = iq * iq;
    double g = iq;  // q^(1-2n)
    double rxx = 0.0, rxy = 0.0, ryy = 0.0, u = 0.0, v = 0.0;
    if (K >= 2) {
        u = x * iq;
        v = y * iq;
    }
#pragma unroll
    for (int n = 1; n <= K; n++) {
        if (n > 1) g *= iq2;
        const double d1g = d1 * g;  // W = d1 q^(1-2n) P for n >= 4
        double mono[K + 1];          // X of this degree: mono[t] = X_(t, n-t)
#pragma unroll
        for (int t = 0; t <= n; t++) mono[t] = xs[t] * ys[n - t];
#pragma unroll
        for (int a = n; a >= 0; a--) {
            const int e = p_of_k(n - 1) + (n - a);
            X[e] = mono[a];
            double s = 0.0;
#pragma unroll
            for (int t = a & 1; t <= n; t += 2) s = fma(c_rpolyf.c[e][t], mono[t], s);
            double wv;
            // chain rule for |alpha| <= 3 (all radial derivatives), W0' only for |alpha| >= 4 (Appendix A)
            if (n <= 3) {
                const double dr = s * g;
                wv = d1 * dr;
                if (n == 2) {
                    if (a == 2) { rxx = dr; wv = fma(d2, u * u, wv); }
                    if (a == 1) { rxy = dr; wv = fma(d2, u * v, wv); }
                    if (a == 0) { ryy = dr; wv = fma(d2, v * v, wv); }
                } else if (n == 3) {
                    if (a == 3) wv = fma(d3, u * u * u, fma(d2, 3.0 * u * rxx, wv));
                    if (a == 2) wv = fma(d3, u * u * v, fma(d2, v * rxx + 2.0 * u * rxy, wv));
                    if (a == 1) wv = fma(d3, u * v * v, fma(d2, u * ryy + 2.0 * v * rxy, wv));
                    if (a == 0) wv = fma(d3, v * v * v, fma(d2, 3.0 * v * ryy, wv));
                }
            } else {
                wv = s * d1g;
            }
            W[e] = wv;
        }
    }
}

}  // namespace

}  // namespace labfm
