// One-dimensional thermal model of the semiclassical LBM: the fourth-order
// equilibrium of Sec. 4 (Eq. feq-4order-01, projections A_0..A_4 on the
// polynomials P_0..P_4 of Sec. 3) with the local reduced temperature
// thetabar(x), on the D1V5 and D1V7 lattices of App. A and Table
// lattices-tab.  Host constants, kernels and the lbm_thermal_* entry points.
//
// Storage is the deviation h_a = f_a - rho0 w_a / I0 (FP32, or FP16 scaled
// by 2^12, or BF16), as for the main model; the collision is FP32.  In 1D the
// projections are scalars.  Around the weight's own state (u = 0, thetabar =
// I2/I0 = thw, the fourth-moment factor g of Eq. int-2nd-coeff-eq at the
// weight's value I0 I4 / I2^2) A_2 and A_4 vanish (Sec. 9.1 identity
// c2 thw + c'2 + D cbar2 thw = 0 and its fourth-order analogue), so the
// kernel evaluates them from the deviations dth = thetabar - thw and u:
//   A_2 = rho (c2 + cbar2)(dth + u^2),
//   A_3 = rho [3 K3 u + c3 u^3],  K3 = K3_0 + (c3 + 3 cbar3) dth + cbar3 u^2,
//   A_4 = rho [3 S + 6 u^2 T + c4 u^4] with
//         S = a4 dth (2 thw + dth) + b4 dth + S_0 + u^2 ((2 cbar4 + 6 dbar4) thetabar + d'4) + dbar4 u^4,
//         T = T_0 + (c4 + 5 cbar4) dth + cbar4 u^2,
//   a4 = g (c4 + 6 cbar4 + 3 dbar4), b4 = 2 c'4 + d'4 (the D = 1 case of the
//   printed A_ijk and A_ijkl), and dth = sum_a h_a (xi_a^2 - thw) / rho - u^2
//   taken straight from the stored deviations.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "lbm_device.cuh"

namespace {

constexpr int kTQ = 7;
constexpr int kTBlock = 256;

struct TParams {
    int nx, Q, order;
    int e[kTQ];
    float xi[kTQ], xim[kTQ];   // xi_a, xi_a^2 - thw
    float W[5][kTQ];           // w_a P_N(xi_a) / N!  (N = 0: w_a c0^2), as hi + lo pairs:
    float Wlo[5][kTQ];         // an FP32-rounded table breaks sum_a xi_a^k W_N,a by ~1e-7, a
                               // drift of momentum and energy that compounds step by step
    float f0[kTQ];             // rho0 w_a / I0
    float c1, c22, c3, cb3, K30, c4, cb4, db4, dp4, a4, b4, S0, T0, c45, thw;
    float rho0, omega, tau, E, scale, inv_scale;
    uint32_t step, seed;
    uint32_t skey;        // t_hash(step * 0x9E3779B9 + seed): the step's rounding key
    int64_t off[kTQ];     // a nx - e_a: the pull of direction a, away from the row's ends
    int64_t plane[kTQ];   // a nx: the store of direction a
};

// The lowbias32 integer hash (C. Wellons) and one 32-bit LCG step per pair of
// stores (Numerical Recipes constants) give the stochastic-rounding words.
__host__ __device__ __forceinline__ uint32_t t_hash(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// x - e for |e| <= 3 in a periodic row of nx >= 1 cells (a row shorter than
// 3 cells can need more than one wrap)
__device__ __forceinline__ int wrapx(int x, int nx) {
    while (x < 0) x += nx;
    while (x >= nx) x -= nx;
    return x;
}

// Lattice velocities as compile-time constants: rest, then opposite pairs
// (D1V5: 0, +-1, +-3; D1V7: 0, +-1, +-2, +-3), as lbm_thermal_create sets them.
template <int Q>
__host__ __device__ constexpr int t_e(int a) {
    return a == 0 ? 0 : ((a & 1) ? 1 : -1) * (Q == 5 ? (a <= 2 ? 1 : 3) : (a + 1) / 2);
}
// x - e_a with periodic wrap, for rows of at least 3 cells
template <int Q>
__device__ __forceinline__ int t_src(int x, int a, int nx) {
    int s = x - t_e<Q>(a);
    s = s < 0 ? s + nx : s;
    return s >= nx ? s - nx : s;
}

// The equilibrium deviations heq~_a (scaled) of one cell (a < Q).  The
// lattice pairs a, a + 1 have xi_{a+1} = -xi_a, so W_N,a+1 = (-1)^N W_N,a
// (checked on the host): heq_a = even + odd and heq_{a+1} = even - odd with
// even = sum over N = 0, 2, 4 and odd = sum over N = 1, 3; the rest
// population has no odd part.  With kLo the hi + lo weight pairs are used.
template <int Q, bool kLo>
__device__ __forceinline__ void t_equilibrium(const TParams& p, float drho, float rho, float us, float dth,
                                              float* heq) {
    const float srho = p.scale * rho;
    const float u2 = us * us;
    const float A1 = srho * p.c1 * us;
    const float A2 = p.order >= 2 ? srho * p.c22 * (dth + u2) : 0.f;
    float A3 = 0.f, A4 = 0.f;
    if (p.order >= 3) {
        const float K3 = p.K30 + (p.c3 + 3.f * p.cb3) * dth + p.cb3 * u2;
        A3 = srho * (3.f * K3 * us + p.c3 * u2 * us);
    }
    if (p.order >= 4) {
        const float th = p.thw + dth;
        const float S = p.a4 * dth * (2.f * p.thw + dth) + p.b4 * dth + p.S0 +
                        u2 * ((2.f * p.cb4 + 6.f * p.db4) * th + p.dp4) + p.db4 * u2 * u2;
        const float T = p.T0 + p.c45 * dth + p.cb4 * u2;
        A4 = srho * (3.f * S + 6.f * u2 * T + p.c4 * u2 * u2);
    }
    const float A[5] = {drho, A1, A2, A3, A4};
    auto term = [&](int N, int a) { return kLo ? fmaf(p.Wlo[N][a], A[N], p.W[N][a] * A[N]) : p.W[N][a] * A[N]; };
    heq[0] = term(0, 0) + term(2, 0) + term(4, 0);
#pragma unroll
    for (int a = 1; a < Q; a += 2) {
        const float even = term(0, a) + term(2, a) + term(4, a);
        const float odd = term(1, a) + term(3, a);
        heq[a] = even + odd;
        heq[a + 1] = even - odd;
    }
}

// Error-free sum and product (Knuth TwoSum, FMA TwoProd) for the moment sums.
__device__ __forceinline__ void t_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void t_acc(float& hi, float& lo, float a, float b) {  // hi + lo += a b
    const float p = a * b, pe = fmaf(a, b, -p);
    float e;
    t_two_sum(hi, p, hi, e);
    lo += e + pe;
}

template <class S, bool SR, int Q>
__global__ void __launch_bounds__(kTBlock) k_thermal_step(const typename S::T* __restrict__ Pin,
                                                          typename S::T* __restrict__ Pout, TParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    // FP32 storage: the moments as double-float sums (the first FP32
    // rounding of a moment would otherwise recur in every step) and the
    // hi + lo equilibrium weights; 16-bit storage rounds far coarser, so
    // there plain FP32 sums over the pairs a, a + 1 suffice.
    constexpr bool kExact = sizeof(typename S::T) == 4;
    float h[Q], heq[Q];
    float dh = 0.f, dl = 0.f, jh = 0.f, jl = 0.f, mh = 0.f, ml = 0.f;
    // a block whose cells are all at least 3 cells from both ends of the row
    // pulls without the periodic wrap, at fixed offsets from its own cell
    const bool inner = (int)blockIdx.x * kTBlock >= 3 && ((int)blockIdx.x + 1) * kTBlock + 3 <= p.nx;
    if (inner) {
        const typename S::T* px = Pin + x;
#pragma unroll
        for (int a = 0; a < Q; ++a) h[a] = S::cvt(px[p.off[a]]);
    } else {
#pragma unroll
        for (int a = 0; a < Q; ++a)
            h[a] = S::cvt(Pin[(int64_t)a * p.nx + (p.nx >= 3 ? t_src<Q>(x, a, p.nx) : wrapx(x - p.e[a], p.nx))]);
    }
    if (kExact) {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            float e;
            t_two_sum(dh, h[a], dh, e);
            dl += e;
            t_acc(jh, jl, h[a], p.xi[a]);
            t_acc(mh, ml, h[a], p.xim[a]);
        }
    } else {
        dh = h[0];
        mh = p.xim[0] * h[0];
#pragma unroll
        for (int a = 1; a < Q; a += 2) {
            const float sa = h[a] + h[a + 1], da = h[a] - h[a + 1];
            dh += sa;
            jh = fmaf(p.xi[a], da, jh);
            mh = fmaf(p.xim[a], sa, mh);
        }
    }
    const float drho = dh + dl, j = jh + jl, m2 = mh + ml;
    const float rho = p.rho0 + drho * p.inv_scale;
    float u, dth;
    if (kExact) {
        u = j * p.inv_scale / rho;
        dth = m2 * p.inv_scale / rho - u * u;
    } else {
        const float ir = p.inv_scale / rho;
        u = j * ir;
        dth = m2 * ir - u * u;
    }
    t_equilibrium<Q, kExact>(p, drho, rho, u + p.tau * p.E, dth, heq);
    const float omm = 1.f - p.omega;
    float rest = dh;
    uint32_t r = 0;
    if (SR) r = t_hash((uint32_t)x ^ p.skey);
    typename S::T* py = Pout + x;
#pragma unroll
    for (int a = 1; a < Q; a += 2) {
        const float ha = fmaf(omm, h[a], p.omega * heq[a]);
        const float hb = fmaf(omm, h[a + 1], p.omega * heq[a + 1]);
        rest -= ha + hb;
        typename S::T ta, tb;
        if (SR) {
            r = r * 1664525u + 1013904223u;
            S::sr2(ha, hb, r ^ (r >> 16), ta, tb);
        } else {
            S::put(&ta, ha);
            S::put(&tb, hb);
        }
        py[p.plane[a]] = ta;
        py[p.plane[a + 1]] = tb;
    }
    rest += dl;
    typename S::T t0, unused;
    if (SR) {
        r = r * 1664525u + 1013904223u;
        S::sr2(rest, rest, r ^ (r >> 16), t0, unused);
    } else {
        S::put(&t0, rest);
    }
    Pout[x] = t0;
}

// f(x, 0) = f^eq(rho(x), u(x), thetabar(x)): P_a(y) holds f_a(y + e_a, 0).
template <class S, int Q>
__global__ void __launch_bounds__(kTBlock) k_thermal_init(typename S::T* __restrict__ P, const float* __restrict__ rho,
                                                          const float* __restrict__ u, const float* __restrict__ th,
                                                          TParams p) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= p.nx) return;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int x = wrapx(y + p.e[a], p.nx);
        const float r = rho ? rho[x] : p.rho0;
        const float uu = u ? u[x] : 0.f;
        const float dth = th ? th[x] - p.thw : 0.f;
        float heq[Q];
        t_equilibrium<Q, sizeof(typename S::T) == 4>(p, (r - p.rho0) * p.scale, r, uu, dth, heq);
        S::put(P + (int64_t)a * p.nx + y, heq[a]);
    }
}

// rho, j = sum f xi, energy = sum f xi^2 per cell; FP64 block partials of the three
template <class S, int Q>
__global__ void __launch_bounds__(kTBlock) k_thermal_moments(const typename S::T* __restrict__ P, float* rho_out,
                                                             float* j_out, float* e_out, float* f_out, int deviation,
                                                             double* partials, TParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[3] = {0.0, 0.0, 0.0};
    if (x < p.nx) {
        float drho = 0.f, j = 0.f, e2 = 0.f;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const float h = S::cvt(P[(int64_t)a * p.nx + wrapx(x - p.e[a], p.nx)]) * p.inv_scale;
            drho += h;
            j += h * p.xi[a];
            e2 += h * p.xi[a] * p.xi[a];
            if (f_out) f_out[(int64_t)a * p.nx + x] = deviation ? h : p.f0[a] + h;
        }
        const float rho = p.rho0 + drho;
        const float en = p.rho0 * p.thw + e2;  // sum_a f0_a xi_a^2 = rho0 thw
        if (rho_out) rho_out[x] = rho;
        if (j_out) j_out[x] = j;
        if (e_out) e_out[x] = en;
        acc[0] = rho;
        acc[1] = j;
        acc[2] = en;
    }
    if (!partials) return;
    __shared__ double sh[kTBlock / 32][3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 3; ++k) acc[k] = lbm::dev::warp_sum(acc[k]);
    if (lane == 0)
        for (int k = 0; k < 3; ++k) sh[wid][k] = acc[k];
    __syncthreads();
    if (wid == 0) {
        for (int k = 0; k < 3; ++k) {
            double v = lane < (int)(blockDim.x / 32) ? sh[lane][k] : 0.0;
            v = lbm::dev::warp_sum(v);
            if (lane == 0) partials[(int64_t)blockIdx.x * 3 + k] = v;
        }
    }
}

template <class F>
int by_storage(int storage, F&& f) {
    if (storage == LBM_F16_DEV) return f(lbm::StoreF16{});
    if (storage == LBM_BF16_DEV) return f(lbm::StoreBF16{});
    return f(lbm::StoreF32{});
}

template <int Q>
struct QTag {
    static constexpr int value = Q;
};
// storage type and lattice size (5 or 7) as compile-time tags
template <class F>
int by_storage_q(int storage, int Q, F&& f) {
    return by_storage(storage, [&](auto st) { return Q == 5 ? f(st, QTag<5>{}) : f(st, QTag<7>{}); });
}

// ---------------------------------------------------------------------------
// Host constants (FP64).
// ---------------------------------------------------------------------------
// Sec. 3 coefficients up to K = 4 for dimension D from I[k] = I_2k, k = 0..4:
// c[K], cp[K] (c'_K), cb[K] (cbar_K) for K = 2..4, and d4, d4p, d4b.
struct Coef4 {
    double c[5], cp[5], cb[5], d4, d4p, d4b;
};

bool coefficients4(int D, const double* I, Coef4* k) {
    std::memset(k, 0, sizeof *k);
    double Dl[4] = {0, 0, 0, 0}, dl[4] = {0, 0, 0, 0};  // Delta_2K and delta_2K, K = 1..3
    for (int K = 0; K <= 4; ++K) {
        if (!(I[K] > 0.0)) return false;
        k->c[K] = 1.0 / std::sqrt(I[K]);
    }
    for (int K = 1; K <= 3; ++K) {
        const double J = I[K] * I[K] / (I[K + 1] * I[K - 1]);
        const double den = (D + 2.0 * K) - J * (D + 2.0 * K - 2.0);
        if (!(den > 0.0)) return false;
        Dl[K] = std::sqrt(2.0 / den);
        dl[K] = 2.0 * I[K + 1] * I[K - 1] / (Dl[K] * Dl[K]);
    }
    for (int K = 2; K <= 4; ++K) {
        k->cp[K] = -k->c[K] * Dl[K - 1] * I[K - 1] / I[K - 2];
        k->cb[K] = k->c[K] * (Dl[K - 1] - 1.0) / (D + 2.0 * K - 4.0);
    }
    const double num = 8.0 * dl[2] * dl[2] * I[2];
    const double den = dl[1] * (dl[1] * dl[3] * (D + 4.0) - dl[2] * dl[2] * D);
    if (!(num / den > 0.0)) return false;
    k->d4 = std::sqrt(num / den);
    k->d4p = 2.0 * k->c[4] * I[3] * Dl[3] / (D * I[2]) - k->d4 / D * (I[0] / I[1] + I[2] * dl[1] / (I[1] * dl[2]));
    k->d4b = k->c[4] * (D - 2.0 * (D + 2.0) * Dl[3]) / (D * (D + 2.0) * (D + 4.0)) + k->d4 * dl[1] / (D * (D + 2.0) * dl[2]);
    return true;
}

// Positive roots (descending) of the App. A cubic in x = c_s^2,
// 35 I8 x^3 - 70 I6 x^2 + 49 I4 x - 12 I2 = 0, by the trigonometric
// solution of the depressed cubic (three real roots) or Cardano (one).
int d1v7_roots(const double* I, double* out) {
    const double a = 35.0 * I[4], b = -70.0 * I[3], c = 49.0 * I[2], d = -12.0 * I[1];
    const double p = (3.0 * a * c - b * b) / (3.0 * a * a);
    const double q = (2.0 * b * b * b - 9.0 * a * b * c + 27.0 * a * a * d) / (27.0 * a * a * a);
    const double shift = -b / (3.0 * a);
    double r[3];
    int n = 0;
    const double disc = q * q / 4.0 + p * p * p / 27.0;
    if (disc > 0.0) {
        const double s = std::sqrt(disc);
        r[n++] = std::cbrt(-q / 2.0 + s) + std::cbrt(-q / 2.0 - s) + shift;
    } else {
        const double m = 2.0 * std::sqrt(-p / 3.0);
        const double th = std::acos(std::fmax(-1.0, std::fmin(1.0, 3.0 * q / (p * m)))) / 3.0;
        for (int k = 0; k < 3; ++k) r[n++] = m * std::cos(th - 2.0 * M_PI * k / 3.0) + shift;
    }
    // one Newton polish each, keep positive roots, sort descending
    int m = 0;
    for (int k = 0; k < n; ++k) {
        double x = r[k];
        const double f = ((a * x + b) * x + c) * x + d, fp = (3.0 * a * x + 2.0 * b) * x + c;
        if (fp != 0.0) x -= f / fp;
        if (x > 0.0) out[m++] = x;
    }
    for (int i = 0; i < m; ++i)
        for (int k = i + 1; k < m; ++k)
            if (out[k] > out[i]) std::swap(out[i], out[k]);
    return m;
}

}  // namespace

struct lbm_thermal {
    cudaStream_t stream = nullptr;
    int64_t nx = 0;
    int Q = 0, order = 4, storage = 0;
    int e[kTQ] = {};
    double w[kTQ] = {}, cs = 0, g = 0, thw = 0, tau = 1, E = 0, rho0 = 1, scale = 1;
    double I[5] = {};
    Coef4 k{};
    bool stochastic = false;
    uint32_t seed = 0;
    void* pop[2] = {nullptr, nullptr};
    int cur = 0;
    double* partials = nullptr;
    double* totals_dev = nullptr;
    double* totals_host = nullptr;
    float* stage = nullptr;
    int64_t steps = 0, launches = 0;
    bool has_state = false;
    std::string err;
};

namespace {

lbm_status tfail(lbm_thermal* t, lbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (t) t->err = buf;
    return s;
}

lbm_status tcuda(lbm_thermal* t, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LBM_OK;
    cudaGetLastError();
    return tfail(t, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

TParams tparams(const lbm_thermal* t) {
    TParams p;
    std::memset(&p, 0, sizeof p);
    p.nx = (int)t->nx;
    p.Q = t->Q;
    p.order = t->order;
    const Coef4& k = t->k;
    const double fact[5] = {1.0, 1.0, 2.0, 6.0, 24.0};
    for (int a = 0; a < t->Q; ++a) {
        const double xi = t->e[a] / t->cs, x2 = xi * xi;
        const double f2 = k.cb[2] * x2 + k.cp[2], f3 = k.cb[3] * x2 + k.cp[3], f4 = k.cb[4] * x2 + k.cp[4];
        const double g4 = (k.d4b * x2 + k.d4p) * x2 + k.d4;
        // 1D polynomials: delta_11 = 1, three xi delta terms = 3 xi, six xi xi delta terms = 6 xi^2, delta_1111 = 3
        const double P[5] = {k.c[0], k.c[1] * xi, k.c[2] * x2 + f2, k.c[3] * x2 * xi + 3.0 * f3 * xi,
                             k.c[4] * x2 * x2 + 6.0 * f4 * x2 + 3.0 * g4};
        p.e[a] = t->e[a];
        p.xi[a] = (float)xi;
        p.xim[a] = (float)(x2 - t->thw);
        for (int N = 0; N <= 4; ++N) {
            const double W = N == 0 ? t->w[a] / t->I[0] : t->w[a] * P[N] / fact[N];
            p.W[N][a] = (float)W;
            p.Wlo[N][a] = (float)(W - (double)p.W[N][a]);
        }
        p.f0[a] = (float)(t->rho0 * t->w[a] / t->I[0]);
    }
    const double thw = t->thw, g = t->g;
    p.c1 = (float)k.c[1];
    p.c22 = (float)(k.c[2] + k.cb[2]);
    p.c3 = (float)k.c[3];
    p.cb3 = (float)k.cb[3];
    p.K30 = (float)((k.c[3] + 3.0 * k.cb[3]) * thw + k.cp[3]);
    p.c4 = (float)k.c[4];
    p.cb4 = (float)k.cb[4];
    p.db4 = (float)k.d4b;
    p.dp4 = (float)k.d4p;
    const double a4 = g * (k.c[4] + 6.0 * k.cb[4] + 3.0 * k.d4b), b4 = 2.0 * k.cp[4] + k.d4p;
    p.a4 = (float)a4;
    p.b4 = (float)b4;
    p.S0 = (float)(a4 * thw * thw + b4 * thw + k.d4);
    p.T0 = (float)((k.c[4] + 5.0 * k.cb[4]) * thw + k.cp[4]);
    p.c45 = (float)(k.c[4] + 5.0 * k.cb[4]);
    p.thw = (float)thw;
    p.rho0 = (float)t->rho0;
    p.omega = (float)(1.0 / t->tau);
    p.tau = (float)t->tau;
    p.E = (float)t->E;
    p.scale = (float)t->scale;
    p.inv_scale = (float)(1.0 / t->scale);
    p.step = (uint32_t)t->steps;
    p.seed = t->seed;
    p.skey = t_hash(p.step * 0x9E3779B9u + p.seed);
    for (int a = 0; a < t->Q; ++a) {
        p.plane[a] = (int64_t)a * t->nx;
        p.off[a] = p.plane[a] - t->e[a];
    }
    return p;
}

bool is_dev(const void* ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

unsigned tgrid(int64_t nx) { return (unsigned)((nx + kTBlock - 1) / kTBlock); }

}  // namespace

extern "C" {

lbm_status lbm_thermal_create(lbm_thermal** out, int lattice, int stat, double theta, double mu, int64_t nx,
                              double tau, double E, int order, int storage, void* stream) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (lattice < LBM_T_D1V5A || lattice > LBM_T_D1V7_R2 || nx < 1 || nx > (1ll << 30) || !(tau > 0.5) ||
        order < 2 || order > 4 || storage < LBM_F32 || storage > LBM_BF16_DEV || !std::isfinite(E))
        return LBM_ERR_INVALID_ARG;
    lbm_thermal* t = new lbm_thermal();
    t->stream = (cudaStream_t)stream;
    t->nx = nx;
    t->tau = tau;
    t->E = E;
    t->order = order;
    t->storage = storage;
    t->scale = storage == LBM_F16_DEV ? 4096.0 : 1.0;
    t->stochastic = storage != LBM_F32;
    lbm_status st = lbm_weight_integrals(1, stat, theta, mu, t->I);
    if (st != LBM_OK || !coefficients4(1, t->I, &t->k)) {
        delete t;
        return LBM_ERR_INVALID_ARG;
    }
    double x = 0.0;
    const double I0 = t->I[0], I2 = t->I[1], I4 = t->I[2], I6 = t->I[3];
    if (lattice <= LBM_T_D1V5B) {
        const double disc = 100.0 * I4 * I4 - 60.0 * I6 * I2;
        if (disc < 0.0) {
            delete t;
            return LBM_ERR_UNSTABLE_LATTICE;
        }
        x = (10.0 * I4 + (lattice == LBM_T_D1V5A ? 1.0 : -1.0) * std::sqrt(disc)) / (10.0 * I6);
        const int ev[5] = {0, 1, -1, 3, -3};
        t->Q = 5;
        std::memcpy(t->e, ev, sizeof ev);
        t->w[0] = I0 - 10.0 * I2 * x / 9.0 + I4 * x * x / 3.0;
        t->w[1] = t->w[2] = 9.0 * I2 * x / 16.0 - 3.0 * I4 * x * x / 16.0;
        t->w[3] = t->w[4] = 3.0 * I4 * x * x / 144.0 - I2 * x / 144.0;
    } else {
        double roots[3];
        const int n = d1v7_roots(t->I, roots), r = lattice - LBM_T_D1V7;
        if (r >= n) {
            delete t;
            return LBM_ERR_UNSTABLE_LATTICE;
        }
        x = roots[r];
        const int ev[7] = {0, 1, -1, 2, -2, 3, -3};
        t->Q = 7;
        std::memcpy(t->e, ev, sizeof ev);
        const double x2 = x * x, x3 = x2 * x;
        t->w[0] = I0 - (490.0 * I2 * x - 420.0 * I4 * x2 + 150.0 * I6 * x3) / 360.0;
        t->w[1] = t->w[2] = (12.0 * I2 * x - 13.0 * I4 * x2 + 5.0 * I6 * x3) / 16.0;
        t->w[3] = t->w[4] = (-9.0 * I2 * x + 30.0 * I4 * x2 - 15.0 * I6 * x3) / 120.0;
        t->w[5] = t->w[6] = (4.0 * I2 * x - 15.0 * I4 * x2 + 15.0 * I6 * x3) / 720.0;
    }
    bool ok = x > 0.0;
    for (int a = 0; a < t->Q; ++a) ok = ok && t->w[a] > 0.0;
    for (int a = 0; a < t->Q; ++a)  // the kernels' compile-time velocities
        ok = ok && t->e[a] == (t->Q == 5 ? t_e<5>(a) : t_e<7>(a));
    if (!ok) {
        delete t;
        return LBM_ERR_UNSTABLE_LATTICE;
    }
    t->cs = std::sqrt(x);
    t->thw = I2 / I0;
    t->g = I0 * I4 / (I2 * I2);
    {  // the pair symmetry the equilibrium kernel relies on: W_N,a+1 = (-1)^N W_N,a, no odd rest term
        const TParams tp = tparams(t);
        bool sym = tp.W[1][0] == 0.f && tp.W[3][0] == 0.f && tp.Wlo[1][0] == 0.f && tp.Wlo[3][0] == 0.f;
        for (int a = 1; a < t->Q; a += 2)
            for (int N = 0; N <= 4; ++N) {
                const float sg = (N & 1) ? -1.f : 1.f;
                sym = sym && tp.W[N][a + 1] == sg * tp.W[N][a] && tp.Wlo[N][a + 1] == sg * tp.Wlo[N][a];
            }
        if (!sym) {
            delete t;
            return LBM_ERR_INVALID_ARG;
        }
    }
    const size_t elem = storage == LBM_F32 ? 4 : 2;
    const size_t bytes = (size_t)t->Q * (size_t)nx * elem;
    const int64_t nb = tgrid(nx);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&t->pop[k], bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->partials, sizeof(double) * 3 * (size_t)nb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->totals_dev, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&t->totals_host, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&t->stage, sizeof(float) * 3 * (size_t)nx);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lbm_thermal_destroy(t);
        return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    }
    *out = t;
    return LBM_OK;
}

void lbm_thermal_destroy(lbm_thermal* t) {
    if (!t) return;
    for (int k = 0; k < 2; ++k)
        if (t->pop[k]) cudaFree(t->pop[k]);
    if (t->partials) cudaFree(t->partials);
    if (t->totals_dev) cudaFree(t->totals_dev);
    if (t->totals_host) cudaFreeHost(t->totals_host);
    if (t->stage) cudaFree(t->stage);
    delete t;
}

lbm_status lbm_thermal_constants(const lbm_thermal* t, double* out, int n) {
    if (!t || !out || n < 24 + t->Q) return LBM_ERR_INVALID_ARG;
    const Coef4& k = t->k;
    const double v[24] = {t->I[0], t->I[1], t->I[2], t->I[3], t->I[4], t->cs, t->g, k.c[0], k.c[1], k.c[2], k.c[3],
                          k.c[4], k.cp[2], k.cp[3], k.cp[4], k.cb[2], k.cb[3], k.cb[4], k.d4, k.d4p, k.d4b,
                          t->thw, (double)t->Q, t->tau};
    std::memcpy(out, v, sizeof v);
    for (int a = 0; a < t->Q; ++a) out[24 + a] = t->w[a];
    return LBM_OK;
}

lbm_status lbm_thermal_set_rounding(lbm_thermal* t, int stochastic, uint32_t seed) {
    if (!t) return LBM_ERR_INVALID_ARG;
    if (stochastic && t->storage == LBM_F32)
        return tfail(t, LBM_ERR_INVALID_ARG, "stochastic rounding applies to FP16/BF16 storage only");
    t->stochastic = stochastic != 0;
    t->seed = seed;
    return LBM_OK;
}

lbm_status lbm_thermal_init(lbm_thermal* t, const float* rho, const float* u, const float* thetabar) {
    if (!t) return LBM_ERR_INVALID_ARG;
    const float* f[3] = {rho, u, thetabar};
    const float* d[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) {
        if (!f[k]) continue;
        if (is_dev(f[k])) {
            d[k] = f[k];
        } else {
            float* dst = t->stage + (size_t)k * t->nx;
            lbm_status s = tcuda(t, cudaMemcpyAsync(dst, f[k], sizeof(float) * t->nx, cudaMemcpyHostToDevice,
                                                    t->stream), "lbm_thermal_init copy");
            if (s != LBM_OK) return s;
            d[k] = dst;
        }
    }
    const TParams p = tparams(t);
    t->launches += by_storage_q(t->storage, t->Q, [&](auto st, auto q) {
        using S = decltype(st);
        k_thermal_init<S, decltype(q)::value>
            <<<tgrid(t->nx), kTBlock, 0, t->stream>>>((typename S::T*)t->pop[0], d[0], d[1], d[2], p);
        return 1;
    });
    t->cur = 0;
    t->steps = 0;
    t->has_state = true;
    return tcuda(t, cudaGetLastError(), "lbm_thermal_init");
}

lbm_status lbm_thermal_step(lbm_thermal* t, int64_t n) {
    if (!t || n < 0) return LBM_ERR_INVALID_ARG;
    if (!t->has_state) return tfail(t, LBM_ERR_STATE, "lbm_thermal_step before lbm_thermal_init");
    for (int64_t s = 0; s < n; ++s) {
        const TParams p = tparams(t);
        const bool sr = t->stochastic;
        t->launches += by_storage_q(t->storage, t->Q, [&](auto st, auto q) {
            using S = decltype(st);
            using T = typename S::T;
            constexpr int Q = decltype(q)::value;
            if (sr && S::kBytes == 2)
                k_thermal_step<S, true, Q><<<tgrid(t->nx), kTBlock, 0, t->stream>>>((const T*)t->pop[t->cur],
                                                                                    (T*)t->pop[t->cur ^ 1], p);
            else
                k_thermal_step<S, false, Q><<<tgrid(t->nx), kTBlock, 0, t->stream>>>((const T*)t->pop[t->cur],
                                                                                     (T*)t->pop[t->cur ^ 1], p);
            return 1;
        });
        t->cur ^= 1;
        ++t->steps;
    }
    return tcuda(t, cudaGetLastError(), "lbm_thermal_step");
}

lbm_status lbm_thermal_moments(lbm_thermal* t, float* rho, float* j, float* energy, double totals[3]) {
    if (!t) return LBM_ERR_INVALID_ARG;
    if (!t->has_state) return tfail(t, LBM_ERR_STATE, "lbm_thermal_moments before lbm_thermal_init");
    for (const float* q : {rho, j, energy})
        if (q && !is_dev(q)) return tfail(t, LBM_ERR_INVALID_ARG, "lbm_thermal_moments: fields must be device memory");
    const TParams p = tparams(t);
    t->launches += by_storage_q(t->storage, t->Q, [&](auto st, auto q) {
        using S = decltype(st);
        k_thermal_moments<S, decltype(q)::value><<<tgrid(t->nx), kTBlock, 0, t->stream>>>(
            (const typename S::T*)t->pop[t->cur], rho, j, energy, nullptr, 0, totals ? t->partials : nullptr, p);
        return 1;
    });
    if (totals) {
        t->launches += lbm::launch_reduce_slots(t->partials, tgrid(t->nx), 3, t->totals_dev, t->stream);
        lbm_status s = tcuda(t, cudaMemcpyAsync(t->totals_host, t->totals_dev, sizeof(double) * 3,
                                                cudaMemcpyDeviceToHost, t->stream), "lbm_thermal_moments totals");
        if (s != LBM_OK) return s;
        s = tcuda(t, cudaStreamSynchronize(t->stream), "lbm_thermal_moments");
        if (s != LBM_OK) return s;
        for (int k = 0; k < 3; ++k) totals[k] = t->totals_host[k];
        if (!(std::isfinite(totals[0]) && std::isfinite(totals[1]) && std::isfinite(totals[2])))
            return tfail(t, LBM_ERR_NONFINITE, "non-finite totals");
    }
    return tcuda(t, cudaGetLastError(), "lbm_thermal_moments");
}

lbm_status lbm_thermal_populations(lbm_thermal* t, float* f, int deviation) {
    if (!t || !f) return LBM_ERR_INVALID_ARG;
    if (!t->has_state) return tfail(t, LBM_ERR_STATE, "lbm_thermal_populations before lbm_thermal_init");
    if (!is_dev(f)) return tfail(t, LBM_ERR_INVALID_ARG, "lbm_thermal_populations: f must be device memory");
    const TParams p = tparams(t);
    t->launches += by_storage_q(t->storage, t->Q, [&](auto st, auto q) {
        using S = decltype(st);
        k_thermal_moments<S, decltype(q)::value><<<tgrid(t->nx), kTBlock, 0, t->stream>>>(
            (const typename S::T*)t->pop[t->cur], nullptr, nullptr, nullptr, f, deviation, nullptr, p);
        return 1;
    });
    return tcuda(t, cudaGetLastError(), "lbm_thermal_populations");
}

const char* lbm_thermal_last_error(const lbm_thermal* t) { return t ? t->err.c_str() : "null context"; }

int64_t lbm_thermal_launch_count(const lbm_thermal* t) { return t ? t->launches : 0; }

}  // extern "C"
