/*
 * FP64 CPU oracle for the semiclassical lattice Boltzmann method of
 * Coelho & Doria, "Lattice Boltzmann method for semiclassical fluids"
 * (arXiv 1710.09472).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously-correct
 * restatement of the paper in double precision.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant generator with the CUDA library.
 *
 * Conventions (the paper's notation):
 *   D      dimension; Q number of lattice vectors
 *   e_a    integer lattice vectors; xi_a = e_a / c_s  (Sec. 8)
 *   w_a    quadrature weights, sum w_a = I_0           (Sec. 8, Table A)
 *   I_2N   weight integrals                             (Sec. 3, Eq. i2n-cont2)
 *   populations f[a*N + cell], cell = (z*Ny + y)*Nx + x, x fastest.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - moments are rho = sum_a f_a and rho*u = sum_a f_a xi_a; the w_a printed
 *     in Eq. mac-fields-model-sec-eq is read as a typo (it would break
 *     sum_a f^eq_a = rho for the EDF of Eq. feq-reduced-applied-...).
 *   - collide, then stream; halfway bounce-back on links into solid cells;
 *     the box is periodic in every direction and walls come from the mask.
 *   - the explicit forcing term is +a.grad_u f^eq (Sec. 7, Eq.
 *     forcing-term-integrals-eq with its sign read so that its first moment
 *     is +rho*a), evaluated per direction with a_a = E + xi_a x B.
 *   - the velocity-shift forcing (Sec. 7, Eq. u-update-force-term-eq) uses
 *     a = E + u x B with the pre-shift velocity u.
 *
 * Parity pins for every function live in tests/ (printed tables, closed
 * forms, moment identities, analytic flows and finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXQ 27

/* ------------------------------------------------------------------------- */
/* Weight functions (Sec. 2, Eq. be-fd-dist-eq; Sec. 9.1, Eqs.               */
/* fd-dist-non-dim-eq and weight-func-isotherm-eq; Hermite weight Eq.        */
/* hermite-weight-eq / MB EDF).                                              */
/*   stat 0 = Fermi-Dirac  omega = 1/(exp((xi^2-mu)/theta)+1)                */
/*   stat 1 = Bose-Einstein omega = 1/(exp((xi^2-mu)/theta)-1), mu < 0       */
/*   stat 2 = Maxwell-Boltzmann omega = (2 pi theta)^(-D/2) exp(-xi^2/2theta)*/
/*            (theta = 1 gives the Hermite weight, I_2N = 1)                 */
/* ------------------------------------------------------------------------- */
typedef struct {
    int stat, D;
    double theta, mu;
    int power; /* integrand is omega(xi) * xi^power */
} or_integrand;

static double or_omega(const or_integrand* p, double xi) {
    double x;
    if (p->stat == 2) {
        return pow(2.0 * M_PI * p->theta, -0.5 * p->D) * exp(-xi * xi / (2.0 * p->theta));
    }
    x = (xi * xi - p->mu) / p->theta;
    if (p->stat == 0) {
        if (x > 0.0) {
            double e = exp(-x);
            return e / (1.0 + e);
        }
        return 1.0 / (exp(x) + 1.0);
    }
    return 1.0 / expm1(x);
}

static double or_integrand_eval(const or_integrand* p, double xi) {
    return or_omega(p, xi) * pow(xi, (double)p->power);
}

/* Gauss-Legendre nodes on [-1,1] by Newton iteration on P_n. */
#define OR_GL_N 16
static double or_gl_x[OR_GL_N], or_gl_w[OR_GL_N];
static int or_gl_ready = 0;

static void or_gl_init(void) {
    int n = OR_GL_N, i, k, it;
    if (or_gl_ready) return;
    for (i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5)), p0, p1, dp = 1.0;
        for (it = 0; it < 100; ++it) {
            double dx;
            p0 = 1.0;
            p1 = x;
            for (k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        p0 = 1.0;
        p1 = x;
        for (k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        or_gl_x[i] = x;
        or_gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    or_gl_ready = 1;
}

/* the 16 Gauss-Legendre nodes and weights on [-1, 1] (also used by the FD
 * integrals of lbm_oracle4.c) */
void or_gauss_legendre16(double* x, double* w) {
    int i;
    or_gl_init();
    for (i = 0; i < OR_GL_N; ++i) {
        x[i] = or_gl_x[i];
        w[i] = or_gl_w[i];
    }
}

static double or_gl_panel(const or_integrand* p, double a, double b) {
    double h = 0.5 * (b - a), m = 0.5 * (a + b), s = 0.0;
    int i;
    for (i = 0; i < OR_GL_N; ++i) s += or_gl_w[i] * or_integrand_eval(p, m + h * or_gl_x[i]);
    return s * h;
}

/* Adaptive bisection: accept a panel when the one-panel and two-half-panel
 * Gauss-Legendre results agree to an absolute tolerance tied to the size of
 * the whole integral (the per-panel tolerance is not shrunk with depth, so
 * the recursion ends once panels are resolved to round-off). */
static double or_adapt(const or_integrand* p, double a, double b, double whole, double tol, int depth) {
    double m = 0.5 * (a + b);
    double l = or_gl_panel(p, a, m), r = or_gl_panel(p, m, b);
    if (depth >= 40 || fabs(l + r - whole) <= tol) return l + r;
    return or_adapt(p, a, m, l, tol, depth + 1) + or_adapt(p, m, b, r, tol, depth + 1);
}

static double or_integrate(const or_integrand* p, double a, double b) {
    /* a first estimate of the size of the integral sets the tolerance */
    double est = 0.0, h = (b - a) / 64.0;
    int i;
    for (i = 0; i < 64; ++i) est += fabs(or_gl_panel(p, a + i * h, a + (i + 1) * h));
    if (est == 0.0) return 0.0;
    return or_adapt(p, a, b, or_gl_panel(p, a, b), 1e-16 * est, 0);
}

/* I_{2N} = pi^{D/2} / (2^{N-1} Gamma(N + D/2)) * int_0^inf omega xi^{2N+D-1}
 * (Sec. 3, Eq. i2n-cont2).  Returns I_0, I_2, ..., I_{2*nmax} in I[0..nmax]. */
int or_weight_integrals(int D, int stat, double theta, double mu, int nmax, double* I) {
    or_integrand p;
    int N;
    double xmax, edge;
    if (D < 1 || D > 3 || theta <= 0.0 || nmax < 0 || nmax > 8) return -1;
    if (stat == 1 && mu >= 0.0) return -1;
    if (stat < 0 || stat > 2) return -1;
    or_gl_init();
    p.stat = stat;
    p.D = D;
    p.theta = theta;
    p.mu = mu;
    if (stat == 2) {
        xmax = sqrt(2.0 * theta * 800.0);
        edge = sqrt(theta);
    } else {
        xmax = sqrt((mu > 0 ? mu : 0.0) + 800.0 * theta);
        edge = mu > 0 ? sqrt(mu) : sqrt(theta);
    }
    for (N = 0; N <= nmax; ++N) {
        double pref, s;
        p.power = 2 * N + D - 1;
        s = or_integrate(&p, 0.0, edge) + or_integrate(&p, edge, xmax);
        pref = pow(M_PI, 0.5 * D) / (pow(2.0, N - 1.0) * tgamma(N + 0.5 * D));
        I[N] = pref * s;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Polynomial coefficients (Sec. 3): c_K = I_2K^{-1/2};                      */
/* J_2K = I_2K^2/(I_{2K+2} I_{2K-2}); Delta_2K = sqrt(2/((D+2K)-J_2K(D+2K-2)))*/
/* c'_K = -c_K (I_{2K-2}/I_{2K-4}) Delta_{2K-2};                             */
/* cbar_K = c_K (Delta_{2K-2}-1)/(D+2K-4).  thetabar = I_2/I_0 (Sec. 9.1).  */
/* out: c0 c1 c2 cbar2 cprime2 thetabar J2 Delta2                            */
/* ------------------------------------------------------------------------- */
int or_coefficients(int D, const double* I, double* out) {
    double I0 = I[0], I2 = I[1], I4 = I[2];
    double J2 = I2 * I2 / (I4 * I0);
    double Delta2 = sqrt(2.0 / ((D + 2.0) - J2 * D));
    double c2 = 1.0 / sqrt(I4);
    out[0] = 1.0 / sqrt(I0);
    out[1] = 1.0 / sqrt(I2);
    out[2] = c2;
    out[3] = c2 * (Delta2 - 1.0) / D;
    out[4] = -c2 * (I2 / I0) * Delta2;
    out[5] = I2 / I0;
    out[6] = J2;
    out[7] = Delta2;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Lattices (Sec. 8 and Table lattices-tab in App. A).                       */
/*   vel 0 = D1V3, 1 = D2V9, 2 = D3V15, 3 = D3V19, 4 = D3V27                 */
/* Velocity order: rest first, then opposite pairs (a odd, a+1 = -e_a).      */
/* ------------------------------------------------------------------------- */
static int or_push(int* e, int* q, int ex, int ey, int ez) {
    e[3 * (*q) + 0] = ex;
    e[3 * (*q) + 1] = ey;
    e[3 * (*q) + 2] = ez;
    (*q)++;
    e[3 * (*q) + 0] = -ex;
    e[3 * (*q) + 1] = -ey;
    e[3 * (*q) + 2] = -ez;
    (*q)++;
    return 0;
}

/* Fills e[3*Q], w[Q], opp[Q]; returns Q, or -1 for bad input, -2 when a
 * weight or c_s is not positive (Sec. 8: both must be positive). */
int or_lattice(int vel, const double* I, int* e, double* w, int* opp, double* cs_out) {
    double I0 = I[0], I2 = I[1], I4 = I[2], I6 = I[3];
    double J2 = I2 * I2 / (I4 * I0);
    double cs = sqrt(I2 / (3.0 * I4));
    int q = 0, a, i;
    memset(e, 0, sizeof(int) * 3 * OR_MAXQ);
    e[0] = e[1] = e[2] = 0;
    q = 1;
    switch (vel) {
        case 0: /* D1V3 */
            or_push(e, &q, 1, 0, 0);
            w[0] = I0 * (1.0 - J2 / 3.0);
            w[1] = w[2] = I0 * J2 / 6.0;
            break;
        case 1: /* D2V9 */
            or_push(e, &q, 1, 0, 0);
            or_push(e, &q, 0, 1, 0);
            or_push(e, &q, 1, 1, 0);
            or_push(e, &q, 1, -1, 0);
            w[0] = I0 * (1.0 - 5.0 * J2 / 9.0);
            for (a = 1; a <= 4; ++a) w[a] = I0 * J2 / 9.0;
            for (a = 5; a <= 8; ++a) w[a] = I0 * J2 / 36.0;
            break;
        case 2: /* D3V15 */
            or_push(e, &q, 1, 0, 0);
            or_push(e, &q, 0, 1, 0);
            or_push(e, &q, 0, 0, 1);
            or_push(e, &q, 1, 1, 1);
            or_push(e, &q, 1, 1, -1);
            or_push(e, &q, 1, -1, 1);
            or_push(e, &q, -1, 1, 1);
            w[0] = I0 * (1.0 - 7.0 * J2 / 9.0);
            for (a = 1; a <= 6; ++a) w[a] = I0 * J2 / 9.0;
            for (a = 7; a <= 14; ++a) w[a] = I0 * J2 / 72.0;
            break;
        case 3: /* D3V19 */
            or_push(e, &q, 1, 0, 0);
            or_push(e, &q, 0, 1, 0);
            or_push(e, &q, 0, 0, 1);
            or_push(e, &q, 1, 1, 0);
            or_push(e, &q, 1, -1, 0);
            or_push(e, &q, 1, 0, 1);
            or_push(e, &q, 1, 0, -1);
            or_push(e, &q, 0, 1, 1);
            or_push(e, &q, 0, 1, -1);
            w[0] = I0 * (1.0 - 2.0 * J2 / 3.0);
            for (a = 1; a <= 6; ++a) w[a] = I0 * J2 / 18.0;
            for (a = 7; a <= 18; ++a) w[a] = I0 * J2 / 36.0;
            break;
        case 4: /* D3V27 */
            or_push(e, &q, 1, 0, 0);
            or_push(e, &q, 0, 1, 0);
            or_push(e, &q, 0, 0, 1);
            or_push(e, &q, 1, 1, 0);
            or_push(e, &q, 1, -1, 0);
            or_push(e, &q, 1, 0, 1);
            or_push(e, &q, 1, 0, -1);
            or_push(e, &q, 0, 1, 1);
            or_push(e, &q, 0, 1, -1);
            or_push(e, &q, 1, 1, 1);
            or_push(e, &q, 1, 1, -1);
            or_push(e, &q, 1, -1, 1);
            or_push(e, &q, -1, 1, 1);
            w[0] = I0 - 2.0 * I2 * I2 / (3.0 * I4) - I6 * I2 * I2 * I2 / (27.0 * I4 * I4 * I4);
            for (a = 1; a <= 6; ++a)
                w[a] = (3.0 * I2 * I2 * I4 * I4 + I6 * I2 * I2 * I2) / (54.0 * I4 * I4 * I4);
            for (a = 7; a <= 18; ++a)
                w[a] = (3.0 * I4 * I4 * I2 * I2 - I6 * I2 * I2 * I2) / (108.0 * I4 * I4 * I4);
            for (a = 19; a <= 26; ++a) w[a] = I2 * I2 * I2 * I6 / (216.0 * I4 * I4 * I4);
            break;
        default:
            return -1;
    }
    for (a = 0; a < q; ++a) {
        opp[a] = (a == 0) ? 0 : ((a % 2 == 1) ? a + 1 : a - 1);
    }
    *cs_out = cs;
    if (!(cs > 0.0)) return -2;
    for (i = 0; i < q; ++i)
        if (!(w[i] > 0.0)) return -2;
    return q;
}

/* ------------------------------------------------------------------------- */
/* Model: everything the step needs, in the paper's symbols.                 */
/* ------------------------------------------------------------------------- */
typedef struct {
    int D, Q;
    int e[3 * OR_MAXQ];
    int opp[OR_MAXQ];
    double w[OR_MAXQ];
    double cs;
    double I0, I2, I4;
    double c0, c1, c2, cbar2, cprime2, thetabar, J2, Delta2;
    double xi[3 * OR_MAXQ]; /* xi_a = e_a / c_s */
    double tau;
    double E[3], B[3];
    int force_mode; /* 0 = velocity shift (Eq. u-update-force-term-eq), 1 = explicit term */
} or_model;

/* Build a model.  Returns 0, -1 (bad argument) or -2 (unstable lattice). */
int or_model_size(void) { return (int)sizeof(or_model); }

int or_model_init(or_model* m, int vel, int stat, double theta, double mu, double tau,
                  const double* E, const double* B, int force_mode) {
    double I[5], co[8];
    int D, q, a, d;
    static const int dims[5] = {1, 2, 3, 3, 3};
    if (vel < 0 || vel > 4 || !(tau > 0.5)) return -1;
    memset(m, 0, sizeof(*m));
    D = dims[vel];
    if (or_weight_integrals(D, stat, theta, mu, 4, I) != 0) return -1;
    q = or_lattice(vel, I, m->e, m->w, m->opp, &m->cs);
    if (q < 0) return q;
    or_coefficients(D, I, co);
    m->D = D;
    m->Q = q;
    m->I0 = I[0];
    m->I2 = I[1];
    m->I4 = I[2];
    m->c0 = co[0];
    m->c1 = co[1];
    m->c2 = co[2];
    m->cbar2 = co[3];
    m->cprime2 = co[4];
    m->thetabar = co[5];
    m->J2 = co[6];
    m->Delta2 = co[7];
    for (a = 0; a < q; ++a)
        for (d = 0; d < 3; ++d) m->xi[3 * a + d] = m->e[3 * a + d] / m->cs;
    m->tau = tau;
    for (d = 0; d < 3; ++d) {
        m->E[d] = E ? E[d] : 0.0;
        m->B[d] = B ? B[d] : 0.0;
    }
    if (D < 3) { /* in 2D only B_z acts on in-plane velocities; E_z is unused */
        m->E[2] = 0.0;
        m->B[0] = m->B[1] = 0.0;
    }
    if (D < 2) {
        m->E[1] = 0.0;
        m->B[2] = 0.0;
    }
    m->force_mode = force_mode;
    return 0;
}

/* Reads back the scalar constants: I0 I2 I4 c0 c1 c2 cbar2 cprime2 thetabar
 * J2 Delta2 cs, then w[0..Q-1]. */
int or_model_constants(const or_model* m, double* out) {
    int a;
    out[0] = m->I0;
    out[1] = m->I2;
    out[2] = m->I4;
    out[3] = m->c0;
    out[4] = m->c1;
    out[5] = m->c2;
    out[6] = m->cbar2;
    out[7] = m->cprime2;
    out[8] = m->thetabar;
    out[9] = m->J2;
    out[10] = m->Delta2;
    out[11] = m->cs;
    for (a = 0; a < m->Q; ++a) out[12 + a] = m->w[a];
    return m->Q;
}

int or_model_velocities(const or_model* m, int* e, int* opp) {
    int a;
    for (a = 0; a < 3 * m->Q; ++a) e[a] = m->e[a];
    for (a = 0; a < m->Q; ++a) opp[a] = m->opp[a];
    return m->Q;
}

static double or_dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void or_cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Discrete second-order EDF actually simulated (Sec. 9.1, Eq.
 * feq-reduced-applied-electrons-in-metals-eq):
 *   f^eq_a = rho w_a { c0^2 + c1^2 (xi_a.u) + c2^2/2 (xi_a.u)^2
 *            + 1/2 c2 cbar2 u^2 xi_a^2 + 1/2 (cbar2 xi_a^2 + c'2)(c2 + D cbar2) u^2 } */
void or_equilibrium(const or_model* m, double rho, const double* u, double* feq) {
    int a;
    double u2 = or_dot3(u, u);
    for (a = 0; a < m->Q; ++a) {
        const double* xi = &m->xi[3 * a];
        double xu = or_dot3(xi, u), x2 = or_dot3(xi, xi);
        feq[a] = rho * m->w[a] *
                 (m->c0 * m->c0 + m->c1 * m->c1 * xu + 0.5 * m->c2 * m->c2 * xu * xu +
                  0.5 * m->c2 * m->cbar2 * u2 * x2 +
                  0.5 * (m->cbar2 * x2 + m->cprime2) * (m->c2 + m->D * m->cbar2) * u2);
    }
}

/* The same discrete EDF before the constant-thetabar approximation of Sec.
 * 9.1, Eq. feq-exp-2nd-order-eq, with the reduced temperature thetabar as an
 * argument (the local model of the weight's own EDF with the cell's chemical
 * potential, Sec. 5 Eq. omega-feq, on the fixed lattice of the weight):
 *   f^eq_a = rho w_a { c0^2 + c1^2 (xi_a.u) + 1/2 c2 (c2 thetabar + c'2) xi_a^2
 *            + c2^2/2 (xi_a.u)^2 + 1/2 c2 cbar2 (D thetabar + u^2) xi_a^2
 *            + 1/2 (cbar2 xi_a^2 + c'2) [D (c2 thetabar + c'2) + c2 u^2
 *                                        + D cbar2 (D thetabar + u^2)] } */
void or_equilibrium_thetabar(const or_model* m, double rho, const double* u, double thetabar, double* feq) {
    int a;
    const double D = m->D, c2 = m->c2, cb = m->cbar2, cp = m->cprime2;
    double u2 = or_dot3(u, u);
    for (a = 0; a < m->Q; ++a) {
        const double* xi = &m->xi[3 * a];
        double xu = or_dot3(xi, u), x2 = or_dot3(xi, xi);
        feq[a] = rho * m->w[a] *
                 (m->c0 * m->c0 + m->c1 * m->c1 * xu + 0.5 * c2 * (c2 * thetabar + cp) * x2 +
                  0.5 * c2 * c2 * xu * xu + 0.5 * c2 * cb * (D * thetabar + u2) * x2 +
                  0.5 * (cb * x2 + cp) * (D * (c2 * thetabar + cp) + c2 * u2 + D * cb * (D * thetabar + u2)));
    }
}

/* Explicit forcing term S_a = a_a . grad_u f^eq_a written with the weight
 * integrals (Sec. 7, Eq. forcing-term-integrals-eq):
 *   S_a = rho w_a [ xi_a.a/I2 + (xi_a.u)(xi_a.a)/I4
 *                   + (Delta2^2-1) xi_a^2 (u.a)/(I4 D) - I2 Delta2^2 (u.a)/(I0 I4) ]
 * with a_a = E + xi_a x B (Sec. 7: a_E = E, a_B = xi x B). */
void or_force_term(const or_model* m, double rho, const double* u, const double* E, double* S) {
    int a;
    double D2 = m->Delta2 * m->Delta2;
    for (a = 0; a < m->Q; ++a) {
        const double* xi = &m->xi[3 * a];
        double xb[3], acc[3];
        or_cross3(xi, m->B, xb);
        acc[0] = E[0] + xb[0];
        acc[1] = E[1] + xb[1];
        acc[2] = E[2] + xb[2];
        S[a] = rho * m->w[a] *
               (or_dot3(xi, acc) / m->I2 + or_dot3(xi, u) * or_dot3(xi, acc) / m->I4 +
                (D2 - 1.0) * or_dot3(xi, xi) * or_dot3(u, acc) / (m->I4 * m->D) -
                m->I2 * D2 * or_dot3(u, acc) / (m->I0 * m->I4));
    }
}

/* Moments of one cell (reading of Eq. mac-fields-model-sec-eq):
 * rho = sum_a f_a, j = rho u = sum_a f_a xi_a. */
void or_cell_moments(const or_model* m, const double* fc, double* rho, double* j) {
    int a;
    *rho = 0.0;
    j[0] = j[1] = j[2] = 0.0;
    for (a = 0; a < m->Q; ++a) {
        *rho += fc[a];
        j[0] += fc[a] * m->xi[3 * a + 0];
        j[1] += fc[a] * m->xi[3 * a + 1];
        j[2] += fc[a] * m->xi[3 * a + 2];
    }
}

/* BGK collision of one cell, Delta t = 1 (Sec. 9.1, discrete Boltzmann):
 *   f*_a = f_a - (f_a - f^eq_a)/tau (+ S_a for the explicit force term). */
/* thb: NULL for the simulated EDF of Eq. feq-reduced-..., else a pointer to
 * the cell's thetabar for Eq. feq-exp-2nd-order-eq.  The thetabar terms of the
 * latter do not depend on u, so the forcing term S_a is the same for both. */
static void or_collide_cell_th(const or_model* m, const double* fc, const double* E, const double* thb,
                               double* fout) {
    double rho, j[3], u[3], ueq[3], feq[OR_MAXQ], S[OR_MAXQ];
    int a;
    or_cell_moments(m, fc, &rho, j);
    u[0] = j[0] / rho;
    u[1] = j[1] / rho;
    u[2] = j[2] / rho;
    if (m->force_mode == 0) {
        double uxb[3];
        or_cross3(u, m->B, uxb);
        ueq[0] = u[0] + m->tau * (E[0] + uxb[0]);
        ueq[1] = u[1] + m->tau * (E[1] + uxb[1]);
        ueq[2] = u[2] + m->tau * (E[2] + uxb[2]);
        if (thb)
            or_equilibrium_thetabar(m, rho, ueq, *thb, feq);
        else
            or_equilibrium(m, rho, ueq, feq);
        for (a = 0; a < m->Q; ++a) fout[a] = fc[a] - (fc[a] - feq[a]) / m->tau;
    } else {
        if (thb)
            or_equilibrium_thetabar(m, rho, u, *thb, feq);
        else
            or_equilibrium(m, rho, u, feq);
        or_force_term(m, rho, u, E, S);
        for (a = 0; a < m->Q; ++a) fout[a] = fc[a] - (fc[a] - feq[a]) / m->tau + S[a];
    }
}

void or_collide_cell(const or_model* m, const double* fc, const double* E, double* fout) {
    or_collide_cell_th(m, fc, E, NULL, fout);
}

/* One cell with its own thetabar (Eq. feq-exp-2nd-order-eq). */
void or_collide_cell_thetabar(const or_model* m, const double* fc, const double* E, double thetabar,
                              double* fout) {
    or_collide_cell_th(m, fc, E, &thetabar, fout);
}

/* ------------------------------------------------------------------------- */
/* Grid helpers.                                                             */
/* ------------------------------------------------------------------------- */
static int64_t or_neighbor(const int64_t* n, int64_t cell, const int* e, int sign) {
    int64_t x = cell % n[0], y = (cell / n[0]) % n[1], z = cell / (n[0] * n[1]);
    x = ((x + sign * e[0]) % n[0] + n[0]) % n[0];
    y = ((y + sign * e[1]) % n[1] + n[1]) % n[1];
    z = ((z + sign * e[2]) % n[2] + n[2]) % n[2];
    return (z * n[1] + y) * n[0] + x;
}

static void or_cell_E(const or_model* m, const double* Efield, int64_t N, int64_t cell, double* E) {
    int d;
    for (d = 0; d < 3; ++d) E[d] = m->E[d];
    if (Efield) {
        for (d = 0; d < m->D; ++d) E[d] = Efield[d * N + cell];
    }
}

/* f(x,0) = f^eq(rho(x), u(x)) on fluid cells, 0 on solid cells.
 * rho[N], u[3*N] as u[d*N + cell] (xi units). */
void or_init_equilibrium(const or_model* m, const int64_t* n, const uint8_t* solid, const double* rho,
                         const double* u, double* f) {
    int64_t N = n[0] * n[1] * n[2], c;
    int a;
    for (c = 0; c < N; ++c) {
        double feq[OR_MAXQ], uc[3] = {0, 0, 0};
        int d;
        if (solid && solid[c]) {
            for (a = 0; a < m->Q; ++a) f[a * N + c] = 0.0;
            continue;
        }
        for (d = 0; d < m->D; ++d) uc[d] = u ? u[d * N + c] : 0.0;
        or_equilibrium(m, rho[c], uc, feq);
        for (a = 0; a < m->Q; ++a) f[a * N + c] = feq[a];
    }
}

/* One or more time steps: collide every fluid cell, then stream with
 * halfway bounce-back: f_a(x, t+1) = f*_a(x - e_a) if x - e_a is fluid,
 * else f*_{abar}(x).  f[Q*N] is updated in place (tmp[Q*N] is scratch).
 * Efield is NULL (uniform m->E) or [D][N]. */
static void or_step_th(const or_model* m, const int64_t* n, const uint8_t* solid, const double* Efield,
                       const double* thetabar, double* f, double* tmp, int64_t nsteps);

void or_step(const or_model* m, const int64_t* n, const uint8_t* solid, const double* Efield, double* f,
             double* tmp, int64_t nsteps) {
    or_step_th(m, n, solid, Efield, NULL, f, tmp, nsteps);
}

/* One step with a per-cell thetabar[N] (Eq. feq-exp-2nd-order-eq in every
 * fluid cell); the caller evaluates thetabar from the cells' densities. */
void or_step_thetabar(const or_model* m, const int64_t* n, const uint8_t* solid, const double* Efield,
                      const double* thetabar, double* f, double* tmp) {
    or_step_th(m, n, solid, Efield, thetabar, f, tmp, 1);
}

static void or_step_th(const or_model* m, const int64_t* n, const uint8_t* solid, const double* Efield,
                       const double* thetabar, double* f, double* tmp, int64_t nsteps) {
    int64_t N = n[0] * n[1] * n[2], t;
    for (t = 0; t < nsteps; ++t) {
        int64_t c;
#pragma omp parallel for schedule(static)
        for (c = 0; c < N; ++c) {
            double fc[OR_MAXQ], fo[OR_MAXQ], E[3];
            int a;
            if (solid && solid[c]) {
                for (a = 0; a < m->Q; ++a) tmp[a * N + c] = 0.0;
                continue;
            }
            for (a = 0; a < m->Q; ++a) fc[a] = f[a * N + c];
            or_cell_E(m, Efield, N, c, E);
            or_collide_cell_th(m, fc, E, thetabar ? &thetabar[c] : NULL, fo);
            for (a = 0; a < m->Q; ++a) tmp[a * N + c] = fo[a];
        }
#pragma omp parallel for schedule(static)
        for (c = 0; c < N; ++c) {
            int a;
            if (solid && solid[c]) {
                for (a = 0; a < m->Q; ++a) f[a * N + c] = 0.0;
                continue;
            }
            for (a = 0; a < m->Q; ++a) {
                int64_t src = or_neighbor(n, c, &m->e[3 * a], -1);
                if (solid && solid[src])
                    f[a * N + c] = tmp[m->opp[a] * N + c];
                else
                    f[a * N + c] = tmp[a * N + src];
            }
        }
    }
}

/* Per-cell moments (rho[N], j[D*N]) and FP64 totals over fluid cells. */
void or_moments(const or_model* m, const int64_t* n, const uint8_t* solid, const double* f, double* rho,
                double* j, double* totals) {
    int64_t N = n[0] * n[1] * n[2], c;
    int d;
    for (d = 0; d < 4; ++d) totals[d] = 0.0;
    for (c = 0; c < N; ++c) {
        double fc[OR_MAXQ], r = 0.0, jc[3] = {0, 0, 0};
        int a;
        if (!(solid && solid[c])) {
            for (a = 0; a < m->Q; ++a) fc[a] = f[a * N + c];
            or_cell_moments(m, fc, &r, jc);
            totals[0] += r;
            for (d = 0; d < 3; ++d) totals[1 + d] += jc[d];
        }
        if (rho) rho[c] = r;
        if (j)
            for (d = 0; d < m->D; ++d) j[d * N + c] = jc[d];
    }
}

/* ------------------------------------------------------------------------- */
/* Adjoint.  Forward map per step: f_{t+1} = Stream(Collide(f_t)).           */
/* Loss L = sum_{t in (t_begin, t_end]} sum_x [wr(x) rho_t(x) + wj(x).j_t(x)] */
/* with the state f_t after t steps and T = t_end steps in total.            */
/* Reverse sweep: lam_T = dl_T/df_T; for t = T-1..0:                          */
/*   lamt = Stream^T lam_{t+1}:  lamt_a(y) = lam_a(y+e_a) or lam_abar(y)      */
/*   parameter gradients from lamt and f_t;                                  */
/*   lam_t = Collide'(f_t)^T lamt + dl_t/df_t.                               */
/* The collision derivatives below are the chain rule through               */
/* rho = sum f, j = sum f xi, u = j/rho of the model in or_collide_cell.    */
/* ------------------------------------------------------------------------- */

/* d f^eq_a / d u (at velocity v), from Eq. feq-reduced-...:
 * rho w_a [ c1^2 xi_a + c2^2 (xi_a.v) xi_a + (c2 cbar2 xi_a^2 + (cbar2 xi_a^2 + c'2)(c2 + D cbar2)) v ] */
static void or_dfeq_du(const or_model* m, int a, double rho, const double* v, double* g) {
    const double* xi = &m->xi[3 * a];
    double xv = or_dot3(xi, v), x2 = or_dot3(xi, xi);
    double kv = m->c2 * m->cbar2 * x2 + (m->cbar2 * x2 + m->cprime2) * (m->c2 + m->D * m->cbar2);
    int d;
    for (d = 0; d < 3; ++d)
        g[d] = rho * m->w[a] * (m->c1 * m->c1 * xi[d] + m->c2 * m->c2 * xv * xi[d] + kv * v[d]);
}

/* d f^eq_a / d thetabar of Eq. feq-exp-2nd-order-eq (its thetabar terms, term
 * by term): rho w_a [ 1/2 c2^2 xi^2 + 1/2 c2 cbar2 D xi^2
 *                     + 1/2 (cbar2 xi^2 + c'2) (D c2 + D^2 cbar2) ] */
static double or_dfeq_dthetabar(const or_model* m, int a, double rho) {
    const double* xi = &m->xi[3 * a];
    const double D = m->D, c2 = m->c2, cb = m->cbar2, x2 = or_dot3(xi, xi);
    return rho * m->w[a] *
           (0.5 * c2 * c2 * x2 + 0.5 * c2 * cb * D * x2 + 0.5 * (cb * x2 + m->cprime2) * (D * c2 + D * D * cb));
}

/* Adjoint of one cell's collision.  fc = pre-collision populations, lt =
 * adjoint of the post-collision populations.  Writes lam (adjoint of fc),
 * adds this cell's contributions to gE[3], gB[3], gtau[1].  thb: NULL for the
 * simulated EDF, else the cell's thetabar for Eq. feq-exp-2nd-order-eq with
 * dthb = d thetabar / d rho (thetabar a function of the cell's density). */
static void or_collide_cell_adjoint_th(const or_model* m, const double* fc, const double* E, const double* lt,
                                       const double* thb, double dthb, double* lam, double* gE, double* gB,
                                       double* gtau) {
    double rho, j[3], u[3], feq[OR_MAXQ];
    double rho_bar = 0.0, u_bar[3] = {0, 0, 0};
    double D2 = m->Delta2 * m->Delta2;
    int a, d;
    or_cell_moments(m, fc, &rho, j);
    for (d = 0; d < 3; ++d) u[d] = j[d] / rho;
    if (thb) /* the thetabar terms of f^eq through thetabar(rho) */
        for (a = 0; a < m->Q; ++a) rho_bar += lt[a] * or_dfeq_dthetabar(m, a, rho) * dthb / m->tau;
    if (m->force_mode == 0) {
        double uxb[3], acc[3], ue[3], ue_bar[3] = {0, 0, 0}, tmp[3];
        or_cross3(u, m->B, uxb);
        for (d = 0; d < 3; ++d) {
            acc[d] = E[d] + uxb[d];
            ue[d] = u[d] + m->tau * acc[d];
        }
        if (thb)
            or_equilibrium_thetabar(m, rho, ue, *thb, feq);
        else
            or_equilibrium(m, rho, ue, feq);
        for (a = 0; a < m->Q; ++a) {
            double g[3];
            /* f*_a = (1-1/tau) f_a + f^eq_a(rho, ue)/tau */
            rho_bar += lt[a] * feq[a] / (m->tau * rho);
            or_dfeq_du(m, a, rho, ue, g);
            for (d = 0; d < 3; ++d) ue_bar[d] += lt[a] * g[d] / m->tau;
            *gtau += lt[a] * (fc[a] - feq[a]) / (m->tau * m->tau);
        }
        /* ue = u + tau (E + u x B) */
        *gtau += or_dot3(ue_bar, acc);
        for (d = 0; d < 3; ++d) gE[d] += m->tau * ue_bar[d];
        or_cross3(ue_bar, u, tmp); /* d(u x B)/dB transposed */
        for (d = 0; d < 3; ++d) gB[d] += m->tau * tmp[d];
        or_cross3(m->B, ue_bar, tmp); /* d(u x B)/du transposed */
        for (d = 0; d < 3; ++d) u_bar[d] += ue_bar[d] + m->tau * tmp[d];
    } else {
        double S[OR_MAXQ];
        if (thb)
            or_equilibrium_thetabar(m, rho, u, *thb, feq);
        else
            or_equilibrium(m, rho, u, feq);
        or_force_term(m, rho, u, E, S);
        for (a = 0; a < m->Q; ++a) {
            const double* xi = &m->xi[3 * a];
            double g[3], xb[3], acc[3], dS_du[3], dS_da[3], abar[3], tmp[3];
            double x2 = or_dot3(xi, xi), xa, xu;
            or_cross3(xi, m->B, xb);
            for (d = 0; d < 3; ++d) acc[d] = E[d] + xb[d];
            xa = or_dot3(xi, acc);
            xu = or_dot3(xi, u);
            /* f*_a = (1-1/tau) f_a + f^eq_a(rho,u)/tau + S_a(rho,u,a_a) */
            rho_bar += lt[a] * (feq[a] / m->tau + S[a]) / rho;
            or_dfeq_du(m, a, rho, u, g);
            for (d = 0; d < 3; ++d) {
                dS_du[d] = rho * m->w[a] *
                           (xi[d] * xa / m->I4 + (D2 - 1.0) * x2 * acc[d] / (m->I4 * m->D) -
                            m->I2 * D2 * acc[d] / (m->I0 * m->I4));
                dS_da[d] = rho * m->w[a] *
                           (xi[d] / m->I2 + xu * xi[d] / m->I4 + (D2 - 1.0) * x2 * u[d] / (m->I4 * m->D) -
                            m->I2 * D2 * u[d] / (m->I0 * m->I4));
                u_bar[d] += lt[a] * (g[d] / m->tau + dS_du[d]);
                abar[d] = lt[a] * dS_da[d];
                gE[d] += abar[d];
            }
            or_cross3(abar, xi, tmp); /* a_a = E + xi_a x B: d/dB transposed */
            for (d = 0; d < 3; ++d) gB[d] += tmp[d];
            *gtau += lt[a] * (fc[a] - feq[a]) / (m->tau * m->tau);
        }
    }
    /* u = j / rho */
    rho_bar -= or_dot3(u_bar, u) / rho;
    for (a = 0; a < m->Q; ++a) {
        const double* xi = &m->xi[3 * a];
        lam[a] = (1.0 - 1.0 / m->tau) * lt[a] + rho_bar + or_dot3(u_bar, xi) / rho;
    }
}

void or_collide_cell_adjoint(const or_model* m, const double* fc, const double* E, const double* lt,
                             double* lam, double* gE, double* gB, double* gtau) {
    or_collide_cell_adjoint_th(m, fc, E, lt, NULL, 0.0, lam, gE, gB, gtau);
}

/* Full adjoint over a stored trajectory.
 * states: (T+1) consecutive arrays of Q*N doubles, states[t] = f_t.
 * wr[N] (may be NULL) and wj[D*N] (may be NULL): loss weights per cell.
 * Outputs: lam0[Q*N] = dL/df_0 (may be NULL), gE[D*N] per-cell dL/dE(x)
 * (may be NULL), gB[3], gtau[1]; loss[1] = L (evaluated on the trajectory). */
static void or_adjoint_th(const or_model* m, const int64_t* n, const uint8_t* solid, const double* Efield,
                          const double* states, const double* thb, const double* dthb, int64_t t_begin,
                          int64_t t_end, const double* wr, const double* wj, double* lam0, double* gE, double* gB,
                          double* gtau, double* loss);

void or_adjoint(const or_model* m, const int64_t* n, const uint8_t* solid, const double* Efield,
                const double* states, int64_t t_begin, int64_t t_end, const double* wr, const double* wj,
                double* lam0, double* gE, double* gB, double* gtau, double* loss) {
    or_adjoint_th(m, n, solid, Efield, states, NULL, NULL, t_begin, t_end, wr, wj, lam0, gE, gB, gtau, loss);
}

/* The same for the local-thetabar model: thb[t * N + c] and dthb[t * N + c]
 * are thetabar and d thetabar / d rho of cell c in state t (t = 0..t_end). */
void or_adjoint_thetabar(const or_model* m, const int64_t* n, const uint8_t* solid, const double* Efield,
                         const double* states, const double* thb, const double* dthb, int64_t t_begin,
                         int64_t t_end, const double* wr, const double* wj, double* lam0, double* gE, double* gB,
                         double* gtau, double* loss) {
    or_adjoint_th(m, n, solid, Efield, states, thb, dthb, t_begin, t_end, wr, wj, lam0, gE, gB, gtau, loss);
}

static void or_adjoint_th(const or_model* m, const int64_t* n, const uint8_t* solid, const double* Efield,
                          const double* states, const double* thb, const double* dthb, int64_t t_begin,
                          int64_t t_end, const double* wr, const double* wj, double* lam0, double* gE, double* gB,
                          double* gtau, double* loss) {
    int64_t N = n[0] * n[1] * n[2], T = t_end, t, c;
    size_t QN = (size_t)m->Q * (size_t)N;
    double* lam = (double*)calloc(QN, sizeof(double));
    double* lt = (double*)calloc(QN, sizeof(double));
    int a, d;
    gB[0] = gB[1] = gB[2] = 0.0;
    *gtau = 0.0;
    *loss = 0.0;
    if (gE) memset(gE, 0, sizeof(double) * (size_t)m->D * (size_t)N);
    /* lam_T = dl_T/df_T, and the loss itself */
    for (t = T; t >= 0; --t) {
        const double* ft = states + (size_t)t * QN;
        int in_window = (t > t_begin && t <= t_end);
        if (t < T) {
            /* lamt = Stream^T lam_{t+1} */
            for (c = 0; c < N; ++c) {
                if (solid && solid[c]) {
                    for (a = 0; a < m->Q; ++a) lt[a * N + c] = 0.0;
                    continue;
                }
                for (a = 0; a < m->Q; ++a) {
                    int64_t dst = or_neighbor(n, c, &m->e[3 * a], +1);
                    if (solid && solid[dst])
                        lt[a * N + c] = lam[m->opp[a] * N + c];
                    else
                        lt[a * N + c] = lam[a * N + dst];
                }
            }
            /* lam_t = Collide'^T lamt, with the parameter gradients */
            for (c = 0; c < N; ++c) {
                double fc[OR_MAXQ], ltc[OR_MAXQ], lc[OR_MAXQ], E[3], ge[3] = {0, 0, 0};
                if (solid && solid[c]) {
                    for (a = 0; a < m->Q; ++a) lam[a * N + c] = 0.0;
                    continue;
                }
                for (a = 0; a < m->Q; ++a) {
                    fc[a] = ft[a * N + c];
                    ltc[a] = lt[a * N + c];
                }
                or_cell_E(m, Efield, N, c, E);
                if (thb)
                    or_collide_cell_adjoint_th(m, fc, E, ltc, &thb[t * N + c], dthb[t * N + c], lc, ge, gB, gtau);
                else
                    or_collide_cell_adjoint_th(m, fc, E, ltc, NULL, 0.0, lc, ge, gB, gtau);
                for (a = 0; a < m->Q; ++a) lam[a * N + c] = lc[a];
                if (gE)
                    for (d = 0; d < m->D; ++d) gE[d * N + c] += ge[d];
            }
        }
        if (in_window) {
            for (c = 0; c < N; ++c) {
                double fc[OR_MAXQ], r, jc[3];
                if (solid && solid[c]) continue;
                for (a = 0; a < m->Q; ++a) fc[a] = ft[a * N + c];
                or_cell_moments(m, fc, &r, jc);
                for (a = 0; a < m->Q; ++a) {
                    double g = wr ? wr[c] : 0.0;
                    if (wj)
                        for (d = 0; d < m->D; ++d) g += wj[d * N + c] * m->xi[3 * a + d];
                    lam[a * N + c] += g;
                }
                if (wr) *loss += wr[c] * r;
                if (wj)
                    for (d = 0; d < m->D; ++d) *loss += wj[d * N + c] * jc[d];
            }
        }
    }
    if (lam0) memcpy(lam0, lam, QN * sizeof(double));
    free(lam);
    free(lt);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
