/*
 * FP64 CPU oracle, part 2: the fourth-order equilibrium of Coelho & Doria
 * (arXiv 1710.09472, Sec. 3 and Sec. 4) and a one-dimensional thermal model
 * on the D1V5 / D1V7 lattices of App. A.
 *
 * TEST INFRASTRUCTURE ONLY, like lbm_oracle.c: only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code with the CUDA library.
 *
 *   or_coefficients4   Sec. 3: c_K (K = 0..4), c'_K, cbar_K (K = 2..4),
 *                      d_4, d'_4, dbar_4 with Delta_2K, J_2K and delta_L
 *   or_polynomials     Sec. 3: P_0 .. P_4 as dense tensors
 *   or_projections     Sec. 4: A_0 .. A_4 of an isotropic EDF shifted by u
 *   or_edf             Eq. feq-4order-01: w_a sum_{N<=order} A_N . P_N / N!
 *   or_lattice1d       Table lattices-tab (D1V5 a/b) and App. A (D1V7)
 *   or_thermal_*       the 1D thermal model (see below)
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - the thermal model keeps the whole fourth-order EDF with the local
 *     reduced temperature thetabar(x), found from the energy moment
 *     sum_a f_a xi_a^2 = rho (D thetabar + u^2), and with the fourth-moment
 *     factor g of Eq. int-2nd-coeff-eq held at the weight's own value
 *     g = I_0 I_4 / I_2^2 (the fugacity of the weight);
 *   - the D1V7 reference speed is a positive root of the cubic of App. A;
 *     root 0 is the one of its printed closed form (the largest), roots 1
 *     and 2 the next smaller positive ones;
 *   - a force acts by the velocity shift u* = u + tau E of Sec. 7 (Eq.
 *     u-update-force-term-eq); the box is periodic (no solid cells).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR4_MAXQ 7

/* ------------------------------------------------------------------------- */
/* Sec. 3 coefficients.  I[0..4] = I_0, I_2, I_4, I_6, I_8.                  */
/* out[0..4]  c_0 .. c_4                c_K = I_2K^{-1/2}                    */
/* out[5..7]  c'_2, c'_3, c'_4          c'_K = -c_K (I_{2K-2}/I_{2K-4}) Delta_{2K-2} */
/* out[8..10] cbar_2, cbar_3, cbar_4    cbar_K = c_K (Delta_{2K-2} - 1)/(D+2K-4) */
/* out[11..13] d_4, d'_4, dbar_4                                              */
/* out[14..16] Delta_2, Delta_4, Delta_6                                      */
/*   Delta_2K = sqrt(2 / ((D+2K) - J_2K (D+2K-2))), J_2K = I_2K^2/(I_{2K+2} I_{2K-2}) */
/*   delta_L = 2 I_{L+2} I_{L-2} / Delta_L^2                                  */
/*   d_4^2 = 8 delta_4^2 I_4 / (delta_2 [delta_2 delta_6 (D+4) - delta_4^2 D]) */
/*   d'_4 = -(d_4/D)[I_0/I_2 + I_4 delta_2/(I_2 delta_4)] + 2 c_4 I_6 Delta_6/(D I_4) */
/*   dbar_4 = d_4 delta_2/(D(D+2) delta_4) + c_4 [D - 2(D+2) Delta_6]/(D(D+2)(D+4)) */
/* Returns 0, or -1 when a square root has a negative argument.              */
/* ------------------------------------------------------------------------- */
int or_coefficients4(int D, const double* I, double* out) {
    double Delta[4], J[4], delta[4], c[5], d4sq;
    int K;
    if (D < 1 || D > 3) return -1;
    for (K = 0; K <= 4; ++K) {
        if (!(I[K] > 0.0)) return -1;
        c[K] = 1.0 / sqrt(I[K]);
    }
    for (K = 1; K <= 3; ++K) {
        double arg;
        J[K] = I[K] * I[K] / (I[K + 1] * I[K - 1]);
        arg = 2.0 / ((D + 2.0 * K) - J[K] * (D + 2.0 * K - 2.0));
        if (!(arg > 0.0)) return -1;
        Delta[K] = sqrt(arg);
        delta[K] = 2.0 * I[K + 1] * I[K - 1] / (Delta[K] * Delta[K]);
    }
    for (K = 0; K <= 4; ++K) out[K] = c[K];
    for (K = 2; K <= 4; ++K) {
        out[5 + K - 2] = -c[K] * (I[K - 1] / I[K - 2]) * Delta[K - 1];
        out[8 + K - 2] = c[K] * (Delta[K - 1] - 1.0) / (D + 2.0 * K - 4.0);
    }
    d4sq = 8.0 * delta[2] * delta[2] * I[2] / (delta[1] * (delta[1] * delta[3] * (D + 4.0) - delta[2] * delta[2] * D));
    if (!(d4sq > 0.0)) return -1;
    out[11] = sqrt(d4sq);
    out[12] = -(out[11] / D) * (I[0] / I[1] + I[2] * delta[1] / (I[1] * delta[2])) +
              2.0 * c[4] * I[3] * Delta[3] / (D * I[2]);
    out[13] = out[11] * delta[1] / (D * (D + 2.0) * delta[2]) +
              c[4] * (D - 2.0 * (D + 2.0) * Delta[3]) / (D * (D + 2.0) * (D + 4.0));
    out[14] = Delta[1];
    out[15] = Delta[2];
    out[16] = Delta[3];
    return 0;
}

/* Dense tensors over index tuples (i1, .., iN), i in [0, D): flat index
 * ((i1 D + i2) D + ..) iN; rank N has D^N entries. */
static int or4_pow(int D, int N) {
    int r = 1, k;
    for (k = 0; k < N; ++k) r *= D;
    return r;
}
static void or4_unflat(int D, int N, int flat, int* idx) {
    int k;
    for (k = N - 1; k >= 0; --k) {
        idx[k] = flat % D;
        flat /= D;
    }
}
static double or4_d(int i, int j) { return i == j ? 1.0 : 0.0; }

/* ------------------------------------------------------------------------- */
/* Polynomials P_0 .. P_4 of Sec. 3 at xi (D components), with              */
/*   f_K(xi) = cbar_K xi^2 + c'_K (K = 2, 3, 4), g_4 = dbar_4 xi^4 + d'_4 xi^2 + d_4: */
/*   P_0 = c_0;  P_i = c_1 xi_i;  P_ij = c_2 xi_i xi_j + f_2 delta_ij;       */
/*   P_ijk = c_3 xi_i xi_j xi_k + f_3 (xi_i d_jk + xi_j d_ik + xi_k d_ij);   */
/*   P_ijkl = c_4 xi_i xi_j xi_k xi_l + f_4 (six xi xi delta terms)          */
/*            + g_4 (d_ij d_kl + d_ik d_jl + d_il d_jk).                     */
/* P[0] = P_0, P + 1 = P_i, P + 1 + D = P_ij, ... (1 + D + D^2 + D^3 + D^4) */
/* ------------------------------------------------------------------------- */
void or_polynomials(int D, const double* co, const double* xi, double* P) {
    double x2 = 0.0, f2, f3, f4, g4;
    double *P1, *P2, *P3, *P4;
    int d, f, idx[4];
    for (d = 0; d < D; ++d) x2 += xi[d] * xi[d];
    f2 = co[8] * x2 + co[5];
    f3 = co[9] * x2 + co[6];
    f4 = co[10] * x2 + co[7];
    g4 = co[13] * x2 * x2 + co[12] * x2 + co[11];
    P1 = P + 1;
    P2 = P1 + D;
    P3 = P2 + D * D;
    P4 = P3 + D * D * D;
    P[0] = co[0];
    for (d = 0; d < D; ++d) P1[d] = co[1] * xi[d];
    for (f = 0; f < or4_pow(D, 2); ++f) {
        int i, j;
        or4_unflat(D, 2, f, idx);
        i = idx[0];
        j = idx[1];
        P2[f] = co[2] * xi[i] * xi[j] + f2 * or4_d(i, j);
    }
    for (f = 0; f < or4_pow(D, 3); ++f) {
        int i, j, k;
        or4_unflat(D, 3, f, idx);
        i = idx[0];
        j = idx[1];
        k = idx[2];
        P3[f] = co[3] * xi[i] * xi[j] * xi[k] + f3 * (xi[i] * or4_d(j, k) + xi[j] * or4_d(i, k) + xi[k] * or4_d(i, j));
    }
    for (f = 0; f < or4_pow(D, 4); ++f) {
        int i, j, k, l;
        double six, d4t;
        or4_unflat(D, 4, f, idx);
        i = idx[0];
        j = idx[1];
        k = idx[2];
        l = idx[3];
        six = xi[i] * xi[j] * or4_d(k, l) + xi[i] * xi[k] * or4_d(j, l) + xi[i] * xi[l] * or4_d(j, k) +
              xi[j] * xi[k] * or4_d(i, l) + xi[j] * xi[l] * or4_d(i, k) + xi[k] * xi[l] * or4_d(i, j);
        d4t = or4_d(i, j) * or4_d(k, l) + or4_d(i, k) * or4_d(j, l) + or4_d(i, l) * or4_d(j, k);
        P4[f] = co[4] * xi[i] * xi[j] * xi[k] * xi[l] + f4 * six + g4 * d4t;
    }
}

/* ------------------------------------------------------------------------- */
/* Projections of Sec. 4 for an isotropic EDF with density rho, reduced     */
/* temperature thetabar and fourth-moment factor g (Eq. int-2nd-coeff-eq),  */
/* shifted by u.  Same tensor packing as or_polynomials.                     */
/*   A_0 = c_0 rho;  A_i = rho c_1 u_i;                                      */
/*   A_ij = rho [(c_2 thb + c'_2) d_ij + c_2 u_i u_j + cbar_2 (D thb + u^2) d_ij]; */
/*   A_ijk = rho [(c_3 thb + cbar_3 thb (D+2) + c'_3 + cbar_3 u^2)            */
/*                (u_i d_jk + u_k d_ij + u_j d_ik) + c_3 u_i u_j u_k];        */
/*   A_ijkl = rho { d_ijkl [c_4 thb^2 g + 2 (c'_4 + cbar_4 u^2) thb           */
/*              + 2 cbar_4 thb^2 g (D+2) + d_4 + d'_4 (D thb + u^2)           */
/*              + dbar_4 (thb^2 g D (D+2) + 2 u^2 thb D + 4 u^2 thb + u^4)]   */
/*            + (six d u u terms)(c_4 thb + c'_4 + cbar_4 u^2 + cbar_4 thb D  */
/*              + 4 cbar_4 thb) + c_4 u_i u_j u_k u_l }.                      */
/* ------------------------------------------------------------------------- */
void or_projections(int D, const double* co, double rho, const double* u, double thb, double g, double* A) {
    double u2 = 0.0, s3, s4a, s4b;
    double *A1, *A2, *A3, *A4;
    int d, f, idx[4];
    for (d = 0; d < D; ++d) u2 += u[d] * u[d];
    A1 = A + 1;
    A2 = A1 + D;
    A3 = A2 + D * D;
    A4 = A3 + D * D * D;
    A[0] = co[0] * rho;
    for (d = 0; d < D; ++d) A1[d] = rho * co[1] * u[d];
    for (f = 0; f < or4_pow(D, 2); ++f) {
        int i, j;
        or4_unflat(D, 2, f, idx);
        i = idx[0];
        j = idx[1];
        A2[f] = rho * ((co[2] * thb + co[5]) * or4_d(i, j) + co[2] * u[i] * u[j] + co[8] * (D * thb + u2) * or4_d(i, j));
    }
    s3 = co[3] * thb + co[9] * thb * (D + 2.0) + co[6] + co[9] * u2;
    for (f = 0; f < or4_pow(D, 3); ++f) {
        int i, j, k;
        or4_unflat(D, 3, f, idx);
        i = idx[0];
        j = idx[1];
        k = idx[2];
        A3[f] = rho * (s3 * (u[i] * or4_d(j, k) + u[k] * or4_d(i, j) + u[j] * or4_d(i, k)) + co[3] * u[i] * u[j] * u[k]);
    }
    s4a = co[4] * thb * thb * g + 2.0 * (co[7] + co[10] * u2) * thb + 2.0 * co[10] * thb * thb * g * (D + 2.0) +
          co[11] + co[12] * (D * thb + u2) +
          co[13] * (thb * thb * g * D * (D + 2.0) + 2.0 * u2 * thb * D + 4.0 * u2 * thb + u2 * u2);
    s4b = co[4] * thb + co[7] + co[10] * u2 + co[10] * thb * D + 4.0 * co[10] * thb;
    for (f = 0; f < or4_pow(D, 4); ++f) {
        int i, j, k, l;
        double six, d4t;
        or4_unflat(D, 4, f, idx);
        i = idx[0];
        j = idx[1];
        k = idx[2];
        l = idx[3];
        d4t = or4_d(i, j) * or4_d(k, l) + or4_d(i, k) * or4_d(j, l) + or4_d(i, l) * or4_d(j, k);
        six = or4_d(i, j) * u[k] * u[l] + or4_d(i, k) * u[j] * u[l] + or4_d(i, l) * u[j] * u[k] +
              or4_d(j, k) * u[i] * u[l] + or4_d(j, l) * u[i] * u[k] + or4_d(k, l) * u[i] * u[j];
        A4[f] = rho * (d4t * s4a + six * s4b + co[4] * u[i] * u[j] * u[k] * u[l]);
    }
}

/* Eq. feq-4order-01 at one lattice vector: the quadrature weight w_a times
 * sum_{N = 0}^{order} (1/N!) A_{i1..iN} P_{i1..iN}(xi_a) (full contraction). */
double or_edf(int D, int order, const double* co, double w_a, const double* xi_a, double rho, const double* u,
              double thb, double g) {
    double A[1 + 3 + 9 + 27 + 81], P[1 + 3 + 9 + 27 + 81], s = 0.0;
    static const double inv_fact[5] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0};
    int N, off = 0, f;
    or_projections(D, co, rho, u, thb, g, A);
    or_polynomials(D, co, xi_a, P);
    for (N = 0; N <= order && N <= 4; ++N) {
        double t = 0.0;
        int n = or4_pow(D, N);
        for (f = 0; f < n; ++f) t += A[off + f] * P[off + f];
        s += inv_fact[N] * t;
        off += n;
    }
    return w_a * s;
}

/* ------------------------------------------------------------------------- */
/* One-dimensional lattices for higher-order EDFs.                           */
/*   kind 0: D1V5 root a (e = 0, +-1, +-3; c_s^2 with the + sign)            */
/*   kind 1: D1V5 root b (the - sign)            (Table lattices-tab)        */
/*   kind 2, 3, 4: D1V7 (e = 0, +-1, +-2, +-3) with root 0, 1, 2 of the cubic */
/*            12 I_2 - 49 I_4 x + 70 I_6 x^2 - 35 I_8 x^3 = 0, x = c_s^2,     */
/*            positive roots in decreasing order (root 0 is the one of the    */
/*            printed closed form)                                  (App. A)  */
/* Velocity order: rest, then opposite pairs.  Returns Q, -1 (bad input or   */
/* no such root) or -2 (a weight or c_s not positive, Sec. 8).               */
/* ------------------------------------------------------------------------- */
static double or4_cubic(const double* I, double x) {
    return 12.0 * I[1] - 49.0 * I[2] * x + 70.0 * I[3] * x * x - 35.0 * I[4] * x * x * x;
}

/* positive roots of the D1V7 cubic by sign changes on a fine grid, then
 * bisection to round-off; returns their number, largest first */
static int or4_cubic_roots(const double* I, double* roots) {
    /* all roots lie below the Cauchy bound 1 + max|a_k / a_3| */
    double a3 = 35.0 * I[4], b = 1.0, xmax, h, x0, f0;
    int n = 0, k, steps = 200000;
    if (fabs(12.0 * I[1] / a3) > b) b = fabs(12.0 * I[1] / a3);
    if (fabs(49.0 * I[2] / a3) > b) b = fabs(49.0 * I[2] / a3);
    if (fabs(70.0 * I[3] / a3) > b) b = fabs(70.0 * I[3] / a3);
    xmax = 1.0 + b;
    h = xmax / steps;
    x0 = 0.0;
    f0 = or4_cubic(I, x0);
    for (k = 1; k <= steps && n < 3; ++k) {
        double x1 = k * h, f1 = or4_cubic(I, x1);
        if ((f0 < 0.0) != (f1 < 0.0)) {
            double lo = x0, hi = x1, flo = f0;
            int it;
            for (it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi), fm = or4_cubic(I, mid);
                if (mid == lo || mid == hi) break;
                if ((fm < 0.0) == (flo < 0.0)) {
                    lo = mid;
                    flo = fm;
                } else {
                    hi = mid;
                }
            }
            roots[n++] = 0.5 * (lo + hi);
        }
        x0 = x1;
        f0 = f1;
    }
    /* largest first */
    for (k = 0; k < n / 2; ++k) {
        double t = roots[k];
        roots[k] = roots[n - 1 - k];
        roots[n - 1 - k] = t;
    }
    return n;
}

int or_lattice1d(int kind, const double* I, int* e, double* w, double* cs_out) {
    double I0 = I[0], I2 = I[1], I4 = I[2], I6 = I[3], x;
    int q, a;
    if (kind == 0 || kind == 1) {
        double disc = 100.0 * I4 * I4 - 60.0 * I6 * I2;
        if (disc < 0.0) return -1;
        x = (10.0 * I4 + (kind == 0 ? 1.0 : -1.0) * sqrt(disc)) / (10.0 * I6);
        if (!(x > 0.0)) return -2;
        q = 5;
        e[0] = 0;
        e[1] = 1;
        e[2] = -1;
        e[3] = 3;
        e[4] = -3;
        w[0] = I0 - 10.0 * I2 * x / 9.0 + I4 * x * x / 3.0;
        w[1] = w[2] = 9.0 * I2 * x / 16.0 - 3.0 * I4 * x * x / 16.0;
        w[3] = w[4] = 3.0 * I4 * x * x / 144.0 - I2 * x / 144.0;
    } else if (kind >= 2 && kind <= 4) {
        double roots[3];
        int n = or4_cubic_roots(I, roots), r = kind - 2;
        if (r >= n) return -1;
        x = roots[r];
        q = 7;
        e[0] = 0;
        e[1] = 1;
        e[2] = -1;
        e[3] = 2;
        e[4] = -2;
        e[5] = 3;
        e[6] = -3;
        w[0] = (360.0 * I0 - 150.0 * I6 * x * x * x + 420.0 * I4 * x * x - 490.0 * I2 * x) / 360.0;
        w[1] = w[2] = (-13.0 * I4 * x * x + 5.0 * I6 * x * x * x + 12.0 * I2 * x) / 16.0;
        w[3] = w[4] = (30.0 * I4 * x * x - 15.0 * I6 * x * x * x - 9.0 * I2 * x) / 120.0;
        w[5] = w[6] = (15.0 * I6 * x * x * x - 15.0 * I4 * x * x + 4.0 * I2 * x) / 720.0;
    } else {
        return -1;
    }
    *cs_out = sqrt(x);
    for (a = 0; a < q; ++a)
        if (!(w[a] > 0.0)) return -2;
    return q;
}

/* ------------------------------------------------------------------------- */
/* The 1D thermal model.  Per cell: rho = sum f, rho u = sum f xi,           */
/* rho (thetabar + u^2) = sum f xi^2 (D = 1); the EDF is Eq. feq-4order-01    */
/* with (rho, u*, thetabar, g), u* = u + tau E (Sec. 7 velocity shift); BGK   */
/* relaxation f* = f - (f - f^eq)/tau, then streaming f_a(x + e_a) = f*_a(x)  */
/* in a periodic box.                                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    int Q, order;
    int e[OR4_MAXQ];
    double w[OR4_MAXQ], xi[OR4_MAXQ];
    double cs, tau, E, g;
    double I[5];
    double co[17];
} or_thermal;

int or_thermal_size(void) { return (int)sizeof(or_thermal); }

extern int or_weight_integrals(int D, int stat, double theta, double mu, int nmax, double* I);

/* Returns 0, -1 (bad argument) or -2 (unstable lattice). */
int or_thermal_init(or_thermal* m, int kind, int stat, double theta, double mu, double tau, double E, int order) {
    int q, a;
    memset(m, 0, sizeof(*m));
    if (!(tau > 0.5) || order < 0 || order > 4) return -1;
    if (or_weight_integrals(1, stat, theta, mu, 4, m->I) != 0) return -1;
    if (or_coefficients4(1, m->I, m->co) != 0) return -1;
    q = or_lattice1d(kind, m->I, m->e, m->w, &m->cs);
    if (q < 0) return q;
    m->Q = q;
    m->order = order;
    for (a = 0; a < q; ++a) m->xi[a] = m->e[a] / m->cs;
    m->tau = tau;
    m->E = E;
    m->g = m->I[0] * m->I[2] / (m->I[1] * m->I[1]);
    return 0;
}

/* constants: I_0..I_8, c_s, g, coefficients (17), weights (Q) */
int or_thermal_constants(const or_thermal* m, double* out) {
    int k;
    for (k = 0; k < 5; ++k) out[k] = m->I[k];
    out[5] = m->cs;
    out[6] = m->g;
    for (k = 0; k < 17; ++k) out[7 + k] = m->co[k];
    for (k = 0; k < m->Q; ++k) out[24 + k] = m->w[k];
    return m->Q;
}

void or_thermal_equilibrium(const or_thermal* m, double rho, double u, double thb, double* feq) {
    int a;
    for (a = 0; a < m->Q; ++a) feq[a] = or_edf(1, m->order, m->co, m->w[a], &m->xi[a], rho, &u, thb, m->g);
}

/* rho, u, thetabar of one cell */
void or_thermal_cell_moments(const or_thermal* m, const double* f, double* rho, double* u, double* thb) {
    double r = 0.0, j = 0.0, e2 = 0.0;
    int a;
    for (a = 0; a < m->Q; ++a) {
        r += f[a];
        j += f[a] * m->xi[a];
        e2 += f[a] * m->xi[a] * m->xi[a];
    }
    *rho = r;
    *u = j / r;
    *thb = e2 / r - (*u) * (*u);
}

void or_thermal_collide_cell(const or_thermal* m, const double* f, double Ecell, double* out) {
    double rho, u, thb, feq[OR4_MAXQ];
    int a;
    or_thermal_cell_moments(m, f, &rho, &u, &thb);
    or_thermal_equilibrium(m, rho, u + m->tau * Ecell, thb, feq);
    for (a = 0; a < m->Q; ++a) out[a] = f[a] - (f[a] - feq[a]) / m->tau;
}

/* f[a * n + x]; Efield[n] per-cell E (NULL: the uniform E) */
void or_thermal_step(const or_thermal* m, int64_t n, const double* Efield, double* f, double* tmp, int64_t nsteps) {
    int64_t t, x;
    int a;
    for (t = 0; t < nsteps; ++t) {
        for (x = 0; x < n; ++x) {
            double fc[OR4_MAXQ], fo[OR4_MAXQ];
            for (a = 0; a < m->Q; ++a) fc[a] = f[a * n + x];
            or_thermal_collide_cell(m, fc, Efield ? Efield[x] : m->E, fo);
            for (a = 0; a < m->Q; ++a) tmp[a * n + x] = fo[a];
        }
        for (x = 0; x < n; ++x)
            for (a = 0; a < m->Q; ++a) {
                int64_t src = ((x - m->e[a]) % n + n) % n;
                f[a * n + x] = tmp[a * n + src];
            }
    }
}

/* f(x, 0) = f^eq(rho(x), u(x), thetabar(x)) (no force shift) */
void or_thermal_init_state(const or_thermal* m, int64_t n, const double* rho, const double* u, const double* thb,
                           double* f) {
    int64_t x;
    int a;
    for (x = 0; x < n; ++x) {
        double feq[OR4_MAXQ];
        or_thermal_equilibrium(m, rho[x], u ? u[x] : 0.0, thb[x], feq);
        for (a = 0; a < m->Q; ++a) f[a * n + x] = feq[a];
    }
}

/* per-cell rho, j = rho u, energy e = sum f xi^2 = rho (thetabar + u^2), and
 * the totals (sum rho, sum j, sum e) */
void or_thermal_moments(const or_thermal* m, int64_t n, const double* f, double* rho, double* j, double* en,
                        double* totals) {
    int64_t x;
    int a;
    totals[0] = totals[1] = totals[2] = 0.0;
    for (x = 0; x < n; ++x) {
        double r = 0.0, jj = 0.0, e2 = 0.0;
        for (a = 0; a < m->Q; ++a) {
            r += f[a * n + x];
            jj += f[a * n + x] * m->xi[a];
            e2 += f[a * n + x] * m->xi[a] * m->xi[a];
        }
        if (rho) rho[x] = r;
        if (j) j[x] = jj;
        if (en) en[x] = e2;
        totals[0] += r;
        totals[1] += jj;
        totals[2] += e2;
    }
}

/* ------------------------------------------------------------------------- */
/* Density and chemical potential of the FD/BE equilibrium (Sec. 4 before    */
/* Eq. rho-fd-be-eq; Sec. 9.1 Eq. rho-def-eq and the inverse of Sec. 9.1.2). */
/*   g_nu(z) = 1/Gamma(nu) int_0^inf x^{nu-1} / (z^{-1} e^x + s) dx,          */
/*   s = +1 (FD) or -1 (BE), z = e^eta; with x = t^2                          */
/*   g_nu = 2/Gamma(nu) int_0^inf t^{2 nu - 1} / (e^{t^2 - eta} + s) dt.      */
/*   rho(mu) = (pi theta)^{D/2} g_{D/2}(e^{mu/theta}) for the non-dimensional  */
/*   EDF of Eq. fd-dist-non-dim-eq (exponent (xi - u)^2 / theta).             */
/* ------------------------------------------------------------------------- */
typedef struct {
    double nu, eta;
    int s;
} or4_gnu;

static double or4_gnu_f(const or4_gnu* p, double t) {
    double y = t * t - p->eta, den;
    if (p->s > 0) { /* 1/(e^y + 1) without overflow */
        if (y > 0.0) {
            double e = exp(-y);
            return pow(t, 2.0 * p->nu - 1.0) * e / (1.0 + e);
        }
        return pow(t, 2.0 * p->nu - 1.0) / (exp(y) + 1.0);
    }
    den = expm1(y); /* BE: eta < 0 so y > 0 */
    return pow(t, 2.0 * p->nu - 1.0) / den;
}

/* composite 16-point Gauss-Legendre on panels of width <= 0.01 in t, which
 * resolve the Fermi edge (width about 1/(2 sqrt(eta)) in t) to round-off */
extern void or_gauss_legendre16(double* x, double* w);

/* stat 0 = FD, 1 = BE (eta < 0); returns NaN for bad arguments */
double or_fd_integral(double nu, double eta, int stat) {
    or4_gnu p;
    double x[16], w[16], top, h, s = 0.0;
    int k, i, n;
    if (!(nu > 0.0) || (stat == 1 && !(eta < 0.0)) || stat < 0 || stat > 1) return NAN;
    or_gauss_legendre16(x, w);
    p.nu = nu;
    p.eta = eta;
    p.s = stat == 0 ? 1 : -1;
    top = sqrt((eta > 0.0 ? eta : 0.0) + 800.0);
    n = (int)ceil(top / 0.01);
    h = top / n;
    for (k = 0; k < n; ++k) {
        double a = k * h, m = a + 0.5 * h, ps = 0.0;
        for (i = 0; i < 16; ++i) ps += w[i] * or4_gnu_f(&p, m + 0.5 * h * x[i]);
        s += 0.5 * h * ps;
    }
    return 2.0 * s / tgamma(nu);
}

double or_density_of_mu(int D, int stat, double theta, double mu) {
    if (D < 1 || D > 3 || !(theta > 0.0)) return NAN;
    return pow(M_PI * theta, 0.5 * D) * or_fd_integral(0.5 * D, mu / theta, stat);
}

/* the inverse by bisection on eta = mu / theta (rho increases with eta) */
double or_mu_of_density(int D, int stat, double theta, double rho) {
    double lo = -60.0, hi = stat == 1 ? -1e-12 : 1.0;
    int it;
    if (D < 1 || D > 3 || !(theta > 0.0) || !(rho > 0.0)) return NAN;
    /* 100 halvings of a bracket of width <= 2^23 reach the spacing of doubles */
    if (!(or_density_of_mu(D, stat, theta, lo * theta) < rho)) return NAN;
    if (stat == 1) {
        if (!(or_density_of_mu(D, stat, theta, hi * theta) > rho)) return NAN;
    } else {
        while (!(or_density_of_mu(D, stat, theta, hi * theta) > rho)) {
            hi *= 2.0;
            if (hi > 1e7) return NAN;
        }
    }
    for (it = 0; it < 100; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (or_density_of_mu(D, stat, theta, mid * theta) < rho)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi) * theta;
}
