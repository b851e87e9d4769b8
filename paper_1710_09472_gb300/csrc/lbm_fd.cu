// Density <-> chemical potential of the Fermi-Dirac equilibrium as GPU field
// conversions: rho = (pi theta)^{D/2} g_{D/2}(e^{mu/theta}) (Sec. 9.1, Eq.
// rho-def-eq) and its inverse mu = theta ln g_{D/2}^{-1}(rho / (pi theta)^{D/2})
// (Sec. 9.1.2), with the complete FD integral
//   g_nu(e^eta) = 1/Gamma(nu) int_0^inf x^{nu-1} / (e^{x - eta} + 1) dx.
// Per element in FP64: eta <= -30, the classical series z - z^2/2^nu + z^3/3^nu
// (z = e^eta); eta >= 60, the Sommerfeld series of Eq. sommerfeld-approx-eq
// with four corrections (the next term and the exponentially small part are
// below 1e-13 there); in between, cubic Hermite interpolation of G = ln g_nu
// and G' = g_{nu-1}/g_nu tabulated every 0.01 in eta.  The table is built on
// the GPU (16-point Gauss-Legendre in t = sqrt(x)) the first time a device
// and a dimension are used, and kept until the process exits.
#include <cmath>
#include <mutex>

#include "lbm_internal.h"

namespace {

constexpr double kEtaLo = -30.0, kEtaHi = 60.0, kStep = 0.01;
constexpr int kNodes = 9001;  // (kEtaHi - kEtaLo) / kStep + 1
constexpr int kMaxDev = 64;

struct GL16 {
    double x[16], w[16];
};

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_16).
GL16 gauss_legendre16() {
    GL16 g;
    const int n = 16;
    for (int i = 0; i < n; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return g;
}

// Table node k: G = ln g_nu(e^eta), G' = d G / d eta, eta = kEtaLo + k kStep.
// g_nu = 2/Gamma(nu) int t^{2nu-1} F(t^2 - eta) dt with F(y) = 1/(e^y + 1),
// dg/deta = 2/Gamma(nu) int t^{2nu-1} F (1 - F) dt; panels of 0.05 in t (the
// Fermi edge is at least 0.065 wide for eta <= 60), up to t^2 = eta + 40.
__global__ void k_fd_table(double nu, GL16 gl, double* __restrict__ G, double* __restrict__ Gp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNodes) return;
    const double eta = kEtaLo + k * kStep;
    const double top = sqrt((eta > 0.0 ? eta : 0.0) + 40.0);
    const int np = (int)ceil(top / 0.05);
    const double h = top / np;
    double s = 0.0, sd = 0.0;
    for (int q = 0; q < np; ++q) {
        const double m = (q + 0.5) * h;
        double ps = 0.0, pd = 0.0;
        for (int i = 0; i < 16; ++i) {
            const double t = m + 0.5 * h * gl.x[i];
            const double y = t * t - eta;
            const double F = y > 0.0 ? exp(-y) / (1.0 + exp(-y)) : 1.0 / (exp(y) + 1.0);
            const double tp = pow(t, 2.0 * nu - 1.0);
            ps += gl.w[i] * tp * F;
            pd += gl.w[i] * tp * F * (1.0 - F);
        }
        s += 0.5 * h * ps;
        sd += 0.5 * h * pd;
    }
    G[k] = log(s) + log(2.0 / tgamma(nu));
    Gp[k] = sd / s;
}

struct FdTable {
    const double* G;
    const double* Gp;
    double nu, lgam1;  // nu and ln Gamma(nu + 1)
};

// G(eta) = ln g_nu(e^eta) and its derivative, by region.
__device__ __forceinline__ void lng(const FdTable& T, double eta, double& G, double& Gp) {
    const double nu = T.nu;
    if (eta <= kEtaLo) {
        const double z = exp(eta), a = exp2(-nu), b = exp(-nu * log(3.0));
        const double g = z * (1.0 - z * a + z * z * b), d = z * (1.0 - 2.0 * z * a + 3.0 * z * z * b);
        G = log(g);
        Gp = d / g;
    } else if (eta >= kEtaHi) {
        // Sommerfeld: 1 + sum_k 2 (1 - 2^{1-2k}) zeta(2k) nu (nu-1) .. (nu-2k+1) eta^{-2k}
        const double zeta2k[4] = {1.6449340668482264, 1.0823232337111382, 1.0173430619844491, 1.0040773561979443};
        double s = 1.0, ds = 0.0, fall = 1.0, ie2 = 1.0 / (eta * eta);
        double pw = 1.0;
        for (int k = 1; k <= 4; ++k) {
            fall *= (nu - (2 * k - 2)) * (nu - (2 * k - 1));
            pw *= ie2;
            const double c = 2.0 * (1.0 - exp2(1.0 - 2.0 * k)) * zeta2k[k - 1] * fall;
            s += c * pw;
            ds -= 2.0 * k * c * pw / eta;
        }
        G = nu * log(eta) - T.lgam1 + log(s);
        Gp = nu / eta + ds / s;
    } else {
        const double u = (eta - kEtaLo) / kStep;
        int k = (int)floor(u);
        if (k > kNodes - 2) k = kNodes - 2;
        const double t = u - k, t2 = t * t, t3 = t2 * t;
        const double g0 = T.G[k], g1 = T.G[k + 1], d0 = T.Gp[k] * kStep, d1 = T.Gp[k + 1] * kStep;
        G = (2 * t3 - 3 * t2 + 1) * g0 + (t3 - 2 * t2 + t) * d0 + (-2 * t3 + 3 * t2) * g1 + (t3 - t2) * d1;
        Gp = ((6 * t2 - 6 * t) * g0 + (3 * t2 - 4 * t + 1) * d0 + (-6 * t2 + 6 * t) * g1 + (3 * t2 - 2 * t) * d1) /
             kStep;
    }
}

__global__ void k_density_from_mu(FdTable T, double inv_theta, double lnpref, const float* __restrict__ mu,
                                  float* __restrict__ rho, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double G, Gp;
    lng(T, (double)mu[i] * inv_theta, G, Gp);
    rho[i] = (float)exp(lnpref + G);
}

// Solve G(eta) = target: G increases with eta.  Newton from the classical or
// the degenerate estimate, kept inside a bracket that every step narrows.
__device__ double eta_of_G(const FdTable& T, double target) {
    double lo = -800.0, hi = 1e9;
    double eta = target < 0.0 ? target : exp((target + T.lgam1) / T.nu);
    for (int it = 0; it < 100; ++it) {
        double G, Gp;
        lng(T, eta, G, Gp);
        const double f = G - target;
        if (f < 0.0)
            lo = eta;
        else
            hi = eta;
        if (fabs(f) <= 1e-15 * fmax(1.0, fabs(target))) break;
        double next = eta - f / Gp;
        if (!(next > lo && next < hi)) next = hi < 1e9 ? 0.5 * (lo + hi) : 2.0 * fmax(eta, 1.0);
        if (next == eta) break;
        eta = next;
    }
    return eta;
}

__global__ void k_mu_from_density(FdTable T, double theta, double lnpref, const float* __restrict__ rho,
                                  float* __restrict__ mu, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = (double)rho[i];
    if (!(r > 0.0) || isinf(r)) {
        mu[i] = nanf("");
        return;
    }
    mu[i] = (float)(eta_of_G(T, log(r) - lnpref) * theta);
}

// Local chemical-potential table: thetabar = I_2/I_0 = (theta/2) g_{nu+1} / g_nu
// (Sec. 9.1, nu = D/2) at the eta with ln g_nu(e^eta) = ln r + ln g_nu(e^eta_w)
// (rho proportional to g_nu, Eq. rho-def-eq), and its r-derivative
// dthetabar/dr = thetabar (G'_{nu+1} - G'_nu) / (r G'_nu).
__global__ void k_lmu_table(FdTable Tn, FdTable Tn1, double theta, double eta_w, int n, int k1, double dr,
                            float2* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double Gw, Gpw, G1w, G1pw;
    lng(Tn, eta_w, Gw, Gpw);
    lng(Tn1, eta_w, G1w, G1pw);
    const double th1 = 0.5 * theta * exp(G1w - Gw);
    const double r = 1.0 + (k - k1) * dr;
    const double eta = k == k1 ? eta_w : eta_of_G(Tn, log(r) + Gw);
    double G, Gp, G1, G1p;
    lng(Tn, eta, G, Gp);
    lng(Tn1, eta, G1, G1p);
    const double th = 0.5 * theta * exp(G1 - G);
    const double dth = th * (G1p - Gp) / (r * Gp);
    out[k] = make_float2((float)(th - th1), (float)(dth * dr));
}

std::mutex g_mu;
double* g_tab[kMaxDev][6] = {};  // per device and 2 nu = 1..5: G then G' (2 kNodes doubles)

// The table of nu = D/2 (D = 1..5: the densities of D = 1..3 dimensions and
// the g_{D/2+1} of thetabar).
lbm_status table_for(int D, cudaStream_t s, FdTable* T) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    double*& tab = g_tab[dev][D];
    T->nu = 0.5 * D;
    T->lgam1 = std::lgamma(T->nu + 1.0);
    if (!tab) {
        double* p = nullptr;
        cudaError_t e = cudaMalloc((void**)&p, sizeof(double) * 2 * kNodes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
        }
        k_fd_table<<<(kNodes + 127) / 128, 128, 0, s>>>(T->nu, gauss_legendre16(), p, p + kNodes);
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            cudaFree(p);
            return LBM_ERR_CUDA;
        }
        tab = p;
    }
    T->G = tab;
    T->Gp = tab + kNodes;
    return LBM_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

lbm_status convert(int D, double theta, const float* in, float* out, int64_t n, void* stream, bool to_mu) {
    if (D < 1 || D > 3 || !(theta > 0.0) || !std::isfinite(theta) || n < 0 || (n > 0 && (!in || !out)))
        return LBM_ERR_INVALID_ARG;
    if (n == 0) return LBM_OK;
    if (!on_device(in) || !on_device(out)) return LBM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FdTable T;
    lbm_status st = table_for(D, s, &T);
    if (st != LBM_OK) return st;
    const double lnpref = 0.5 * D * std::log(M_PI * theta);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (to_mu)
        k_mu_from_density<<<blocks, 256, 0, s>>>(T, theta, lnpref, in, out, n);
    else
        k_density_from_mu<<<blocks, 256, 0, s>>>(T, 1.0 / theta, lnpref, in, out, n);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace

namespace lbm {

lbm_status build_local_mu_table(int D, double theta, double mu_w, int n, int k1, double dr, float2* out,
                                cudaStream_t s) {
    if (D < 1 || D > 3 || !(theta > 0.0) || !std::isfinite(mu_w) || n < 2 || k1 < 0 || k1 >= n || !(dr > 0.0) ||
        !out)
        return LBM_ERR_INVALID_ARG;
    FdTable Tn, Tn1;
    lbm_status st = table_for(D, s, &Tn);
    if (st == LBM_OK) st = table_for(D + 2, s, &Tn1);
    if (st != LBM_OK) return st;
    k_lmu_table<<<(n + 127) / 128, 128, 0, s>>>(Tn, Tn1, theta, mu_w / theta, n, k1, dr, out);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

}  // namespace lbm

extern "C" {

lbm_status lbm_density_from_mu(int D, double theta, const float* mu, float* rho, int64_t n, void* stream) {
    return convert(D, theta, mu, rho, n, stream, false);
}

lbm_status lbm_mu_from_density(int D, double theta, const float* rho, float* mu, int64_t n, void* stream) {
    return convert(D, theta, rho, mu, n, stream, true);
}

}  // extern "C"
