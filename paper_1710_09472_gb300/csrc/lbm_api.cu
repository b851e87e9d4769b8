// Host side of the C ABI declared in include/lbm.h: context lifetime, FP64
// derivation of the model constants (weight integrals, EDF coefficients,
// lattice weights), argument marshalling and kernel launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <functional>
#include <vector>

#include "lbm_internal.h"

using lbm::KParams;
using lbm::make_params;

namespace {

// ---------------------------------------------------------------------------
// Weight integrals I_2N = pi^{D/2} / (2^{N-1} Gamma(N + D/2)) int_0^inf omega
// xi^{2N+D-1} dxi (Sec. 3, Eq. i2n-cont2), by adaptive Simpson quadrature
// with Richardson correction, split at the Fermi edge xi = sqrt(mu).
// ---------------------------------------------------------------------------
struct Weight {
    int stat, D, power;
    double theta, mu;
    double operator()(double xi) const {
        double om;
        if (stat == LBM_MB) {
            om = std::pow(2.0 * M_PI * theta, -0.5 * D) * std::exp(-0.5 * xi * xi / theta);
        } else {
            const double x = (xi * xi - mu) / theta;
            if (stat == LBM_FD)
                om = x > 0 ? std::exp(-x) / (1.0 + std::exp(-x)) : 1.0 / (std::exp(x) + 1.0);
            else
                om = 1.0 / std::expm1(x);
        }
        double pw = 1.0;
        for (int k = 0; k < power; ++k) pw *= xi;
        return om * pw;
    }
};

bool simpson(const Weight& f, double a, double b, double* result) {
    struct Seg {
        double a, b, fa, fm, fb, whole;
        int depth;
    };
    // size estimate on a fixed grid sets the absolute tolerance
    double est = 0.0;
    const int n0 = 256;
    for (int i = 0; i <= n0; ++i) est += std::fabs(f(a + (b - a) * i / n0)) * (b - a) / n0;
    if (est == 0.0) {
        *result = 0.0;
        return true;
    }
    const double tol = 2e-18 * est;
    std::vector<Seg> stack;
    const double fa = f(a), fb = f(b), fm = f(0.5 * (a + b));
    stack.push_back({a, b, fa, fm, fb, (b - a) / 6.0 * (fa + 4 * fm + fb), 0});
    double total = 0.0, comp = 0.0;  // Kahan-compensated sum of accepted panels
    long evals = 3;
    while (!stack.empty()) {
        Seg s = stack.back();
        stack.pop_back();
        const double m = 0.5 * (s.a + s.b);
        const double lm = 0.5 * (s.a + m), rm = 0.5 * (m + s.b);
        const double flm = f(lm), frm = f(rm);
        evals += 2;
        const double left = (m - s.a) / 6.0 * (s.fa + 4 * flm + s.fm);
        const double right = (s.b - m) / 6.0 * (s.fm + 4 * frm + s.fb);
        const double diff = left + right - s.whole;
        if (std::fabs(diff) <= 15.0 * tol || s.depth >= 48) {
            const double y = (left + right + diff / 15.0) - comp;
            const double t = total + y;
            comp = (t - total) - y;
            total = t;
        } else {
            stack.push_back({s.a, m, s.fa, flm, s.fm, left, s.depth + 1});
            stack.push_back({m, s.b, s.fm, frm, s.fb, right, s.depth + 1});
        }
        if (evals > 50000000L) return false;
    }
    *result = total;
    return true;
}

bool weight_integrals(int D, int stat, double theta, double mu, double* I /* [5] */) {
    Weight f{stat, D, 0, theta, mu};
    double edge, top;
    if (stat == LBM_MB) {
        edge = std::sqrt(theta);
        top = std::sqrt(1600.0 * theta);
    } else {
        edge = mu > 0 ? std::sqrt(mu) : std::sqrt(theta);
        top = std::sqrt((mu > 0 ? mu : 0.0) + 800.0 * theta);
    }
    for (int N = 0; N <= 4; ++N) {
        f.power = 2 * N + D - 1;
        double s1, s2;
        if (!simpson(f, 0.0, edge, &s1) || !simpson(f, edge, top, &s2)) return false;
        const double pref = std::pow(M_PI, 0.5 * D) / (std::pow(2.0, N - 1.0) * std::tgamma(N + 0.5 * D));
        I[N] = pref * (s1 + s2);
    }
    return true;
}

lbm_status fail(lbm_ctx* c, lbm_status st, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

lbm_status cuda_check(lbm_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LBM_OK;
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define LBM_CUDA(ctx, call)                                   \
    do {                                                      \
        lbm_status _st = cuda_check((ctx), (call), #call);    \
        if (_st != LBM_OK) return _st;                        \
    } while (0)

// After a stream synchronisation: a kernel whose bounded wait ran out has
// written a nonzero code into the mapped status word; report it once.
lbm_status device_status(lbm_ctx* c) {
    volatile int* w = c->status_host;
    if (!w || *w == 0) return LBM_OK;
    const int code = *w;
    *w = 0;
    return fail(c, LBM_ERR_TIMEOUT, "a device-side wait ran out (code %d); the state is invalid", code);
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t pop_elem_bytes(int storage) { return storage == LBM_F32 ? 4 : 2; }

// |e_a|^2 of direction a of a lattice (the velocity tables of lbm_internal.h)
int lattice_esq(int vel, int a) {
    switch (vel) {
        case LBM_D2V9: return lbm::esq_of<lbm::LatD2V9>(a);
        case LBM_D3V27: return lbm::esq_of<lbm::LatD3V27>(a);
        case LBM_D1V3: return lbm::esq_of<lbm::LatD1V3>(a);
        default: return lbm::esq_of<lbm::LatD3V19>(a);
    }
}

}  // namespace

// Local chemical-potential table: nodes r = rho / rho0 = 1 + (k - kLmuK1) kLmuDr,
// k = 0 .. kLmuNodes - 1, i.e. r from 1/4 to 4 in steps of 1/1024.
constexpr int kLmuK1 = 768, kLmuNodes = 3841;
constexpr double kLmuDr = 1.0 / 1024.0;

lbm::KParams lbm::make_params(const lbm_ctx* c) {
    KParams p;
    std::memset(&p, 0, sizeof p);
    p.nx = (int)c->nx;
    p.ny = (int)c->ny;
    p.nz = (int)c->nz;
    p.N = c->N;
    p.omega = (float)(1.0 / c->tau);
    p.tau = (float)c->tau;
    p.rho0 = (float)c->lat.rho0;
    p.A = (float)c->A;
    p.Bp = (float)(c->Bc / c->cs);
    p.Cp = (float)(c->Cc / (c->cs * c->cs));
    p.Gp = (float)(c->G / (c->cs * c->cs));
    p.H = (float)c->H;
    p.cs = (float)c->cs;
    p.cs_inv = (float)(1.0 / c->cs);
    for (int a = 0; a < c->Q; ++a) {
        const int e2 = lattice_esq(c->lat.vel, a);
        p.w[a] = (float)c->w[a];
        p.k2[a] = (float)(c->G * e2 / (c->cs * c->cs) + c->H);
        // W1_a = w_a Bp / c_s = w_a / (I2 c_s^2) as a double-float pair
        const double W1 = c->w[a] * c->Bc / (c->cs * c->cs);
        p.W1hi[a] = (float)W1;
        p.W1lo[a] = (float)(W1 - (double)p.W1hi[a]);
        p.f0[a] = (float)(c->lat.rho0 * c->w[a] * c->A);
    }
    for (int d = 0; d < 3; ++d) {
        p.E[d] = (float)c->E[d];
        p.B[d] = (float)c->B[d];
    }
    p.scale = (float)c->scale;
    p.inv_scale = (float)(1.0 / c->scale);
    p.gofs = c->gofs;
    p.lbase = c->lbase;
    p.rowG = c->rowG;
    p.ldesc = c->ldesc;
    p.max_row_links = c->max_row_links;
    p.rorder = c->rorder;
    p.lorder = c->lorder;
    p.lgofs = 0;
    p.status = c->status_dev;
    p.seed = c->rseed;
    if (c->lmu_tab) {
        // table coordinate (rho / rho0 - 1) / dr + k1 from the scaled deviation drho~
        p.lmu_tab = c->lmu_tab;
        p.lmu_n = kLmuNodes;
        p.lmu_a = (float)(1.0 / (c->scale * c->lat.rho0 * kLmuDr));
        p.lmu_b = (float)kLmuK1;
        const double g = c->c2 + c->D * c->cbar2;
        for (int sh = 0; sh <= 3; ++sh)  // shell 0: the rest population (the reverse step uses it)
            p.lmu_K[sh] = (float)(0.5 * g * (g * sh / (c->cs * c->cs) + c->D * c->cprime2));
    }
    return p;
}

namespace {

void sanitize_fields(lbm_ctx* c) {
    if (c->D == 2) {  // only in-plane E and B_z act in 2D
        c->E[2] = 0.0;
        c->B[0] = c->B[1] = 0.0;
    }
    if (c->D == 1) {  // only E_x acts in 1D (xi x B has no x component)
        c->E[1] = c->E[2] = 0.0;
        c->B[0] = c->B[1] = c->B[2] = 0.0;
    }
}

// Device staging for a host-pointer argument of `bytes` bytes.
lbm_status stage(lbm_ctx* c, size_t bytes) {
    if (c->stage_bytes >= bytes) return LBM_OK;
    if (c->stage) cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    LBM_CUDA(c, cudaMalloc((void**)&c->stage, bytes));
    c->stage_bytes = bytes;
    return LBM_OK;
}

lbm_status after_launch(lbm_ctx* c, int n) {
    c->launches += n;
    return cuda_check(c, cudaGetLastError(), "kernel launch");
}

uint32_t checksum(const unsigned char* p, size_t n) {  // FNV-1a
    uint32_t h = 2166136261u;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 16777619u;
    }
    return h;
}

struct StateHeader {
    char magic[8];
    int32_t vel, storage;
    int64_t nx, ny, nz;
    int64_t steps;
    uint64_t payload;
    uint32_t crc;
    uint32_t pad;
};

// Frees the adjoint workspace (after the stream has drained).
void ws_release(lbm_ctx* c) {
    AdjWorkspace& w = c->ws;
    if (w.states.empty() && !w.lam[0] && !w.lam[1] && !w.slots && !w.red && !w.wstage && !w.gpart) return;
    cudaStreamSynchronize(c->stream);
    for (void* q : w.states) cudaFree(q);
    w.states.clear();
    cudaFree(w.lam[0]);
    cudaFree(w.lam[1]);
    cudaFree(w.slots);
    cudaFree(w.red);
    cudaFree(w.wstage);
    cudaFree(w.gpart);
    w = AdjWorkspace();
}

// Link-buffer layout for the current link masks, then state buffers sized
// for populations + links (contents undefined until lbm_init_equilibrium).
lbm_status build_links_and_state(lbm_ctx* c) {
    KParams p = make_params(c);
    size_t temp_bytes = 0;
    if (lbm::launch_build_links(c->lat.vel, c->nbr, c->lbase, c->rowG, nullptr, &temp_bytes, p, c->stream) != 0)
        return fail(c, LBM_ERR_CUDA, "link layout: scan size query failed");
    void* temp = nullptr;
    LBM_CUDA(c, cudaMalloc(&temp, temp_bytes > 0 ? temp_bytes : 16));
    c->launches += lbm::launch_build_links(c->lat.vel, c->nbr, c->lbase, c->rowG, temp, &temp_bytes, p, c->stream);
    lbm_status st = cuda_check(c, cudaGetLastError(), "link layout kernels");
    const int64_t R = c->ny * c->nz;
    std::vector<uint32_t> rowG((size_t)R + 1);
    if (st == LBM_OK)
        st = cuda_check(c, cudaMemcpyAsync(rowG.data(), c->rowG, sizeof(uint32_t) * (R + 1), cudaMemcpyDeviceToHost,
                                           c->stream), "copy row link offsets");
    if (st == LBM_OK) st = cuda_check(c, cudaStreamSynchronize(c->stream), "link layout");
    cudaFree(temp);
    if (st != LBM_OK) return st;
    c->n_links = rowG[R];
    int mx = 0;
    for (int64_t r = 0; r < R; ++r) mx = std::max(mx, (int)(rowG[r + 1] - rowG[r]));
    c->max_row_links = mx;
    // link descriptors (x | b << 24), one per slot
    cudaFree(c->ldesc);
    c->ldesc = nullptr;
    LBM_CUDA(c, cudaMalloc((void**)&c->ldesc, sizeof(uint32_t) * ((size_t)c->n_links + 4)));
    p.ldesc = c->ldesc;
    c->launches += lbm::launch_build_link_desc(c->lat.vel, c->nbr, c->lbase, c->ldesc, p, c->stream);
    LBM_CUDA(c, cudaGetLastError());
    // per-row cell order of the row-staged kernels (entries are 16-bit x)
    if (!c->rorder && c->nx <= 65535) {
        c->lorder = 8 + (int)((c->nx + 7) / 8) * 8;
        LBM_CUDA(c, cudaMalloc((void**)&c->rorder, sizeof(uint16_t) * (size_t)R * (size_t)c->lorder));
        p.lorder = c->lorder;
    }
    if (c->rorder) {
        p.rorder = c->rorder;
        c->launches += lbm::launch_build_row_order(c->nbr, c->rorder, p, c->stream);
        LBM_CUDA(c, cudaGetLastError());
    }
    const size_t eb = pop_elem_bytes(c->storage);
    const size_t pbytes = (size_t)c->Q * (size_t)c->N * eb;
    c->gofs = (pbytes + 255) & ~(size_t)255;
    const size_t need = c->gofs + ((((size_t)c->n_links * eb) + 16 + 255) & ~(size_t)255);
    if (need != c->state_bytes || c->ws.lam_bytes) ws_release(c);  // sizes follow the links
    if (need != c->state_bytes) {
        cudaFree(c->pop[0]);
        cudaFree(c->pop[1]);
        c->pop[0] = c->pop[1] = nullptr;
        c->state_bytes = 0;
        LBM_CUDA(c, cudaMalloc(&c->pop[0], need));
        LBM_CUDA(c, cudaMalloc(&c->pop[1], need));
        c->state_bytes = need;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_ERR_INVALID_ARG: return "invalid argument";
        case LBM_ERR_UNSTABLE_LATTICE: return "unstable lattice (a weight or c_s is not positive)";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_OOM: return "out of memory";
        case LBM_ERR_NONFINITE: return "non-finite value";
        case LBM_ERR_TIMEOUT: return "timeout";
        case LBM_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

lbm_status lbm_weight_integrals(int D, int stat, double theta, double mu, double I[5]) {
    if (!I || D < 1 || D > 3 || stat < LBM_FD || stat > LBM_MB || !(theta > 0.0)) return LBM_ERR_INVALID_ARG;
    if (stat == LBM_BE && !(mu < 0.0)) return LBM_ERR_INVALID_ARG;
    return weight_integrals(D, stat, theta, mu, I) ? LBM_OK : LBM_ERR_INVALID_ARG;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t lbm_launch_count(const lbm_ctx* c) { return c ? c->launches : 0; }

lbm_status lbm_create(lbm_ctx** out, const lbm_lattice* lat, const int64_t dims[3], double tau, const double E[3],
                      const double B[3], int storage, void* cuda_stream) {
    if (!out || !lat || !dims) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (lat->vel != LBM_D2V9 && lat->vel != LBM_D3V19 && lat->vel != LBM_D3V27 && lat->vel != LBM_D1V3)
        return LBM_ERR_INVALID_ARG;
    if (lat->stat < LBM_FD || lat->stat > LBM_MB) return LBM_ERR_INVALID_ARG;
    if (lat->force != LBM_FORCE_SHIFT && lat->force != LBM_FORCE_TERM) return LBM_ERR_INVALID_ARG;
    if (storage < LBM_F32 || storage > LBM_BF16_DEV) return LBM_ERR_INVALID_ARG;
    if (!(lat->theta > 0.0) || !(tau > 0.5) || !std::isfinite(tau) || !(lat->rho0 > 0.0)) return LBM_ERR_INVALID_ARG;
    if (lat->stat == LBM_BE && !(lat->mu < 0.0)) return LBM_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (dims[d] < 1 || dims[d] > (1 << 20)) return LBM_ERR_INVALID_ARG;
    if (lat->vel == LBM_D2V9 && dims[2] != 1) return LBM_ERR_INVALID_ARG;
    if (lat->vel == LBM_D1V3 && (dims[1] != 1 || dims[2] != 1)) return LBM_ERR_INVALID_ARG;
    if (dims[1] * dims[2] > 0x7fffffffLL || dims[0] > 0x7fffffffLL) return LBM_ERR_INVALID_ARG;

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_OOM;
    c->lat = *lat;
    c->D = lat->vel == LBM_D2V9 ? 2 : (lat->vel == LBM_D1V3 ? 1 : 3);
    c->Q = lat->vel == LBM_D2V9 ? 9 : (lat->vel == LBM_D1V3 ? 3 : (lat->vel == LBM_D3V27 ? 27 : 19));
    c->nx = dims[0];
    c->ny = dims[1];
    c->nz = dims[2];
    c->N = dims[0] * dims[1] * dims[2];
    c->n_fluid = c->N;
    c->storage = storage;
    c->tau = tau;
    c->stream = (cudaStream_t)cuda_stream;
    for (int d = 0; d < 3; ++d) {
        c->E[d] = E ? E[d] : 0.0;
        c->B[d] = B ? B[d] : 0.0;
    }
    sanitize_fields(c);
    c->scale = storage == LBM_F16_DEV ? 4096.0 : 1.0;
    c->stochastic = storage != LBM_F32;

    // --- constants (Sec. 3, 5.1, 8, 9.1) ---
    if (!weight_integrals(c->D, lat->stat, lat->theta, lat->mu, c->I)) {
        lbm_destroy(c);
        return LBM_ERR_INVALID_ARG;
    }
    const double I0 = c->I[0], I2 = c->I[1], I4 = c->I[2];
    const int D = c->D;
    c->J2 = I2 * I2 / (I4 * I0);
    const double Delta2sq = 2.0 / ((D + 2.0) - c->J2 * D);
    if (!(Delta2sq > 0.0)) {
        lbm_destroy(c);
        return LBM_ERR_UNSTABLE_LATTICE;
    }
    c->Delta2 = std::sqrt(Delta2sq);
    c->c0 = 1.0 / std::sqrt(I0);
    c->c1 = 1.0 / std::sqrt(I2);
    c->c2 = 1.0 / std::sqrt(I4);
    c->cbar2 = c->c2 * (c->Delta2 - 1.0) / D;
    c->cprime2 = -c->c2 * (I2 / I0) * c->Delta2;
    c->thetabar = I2 / I0;
    // direct N = 2 EDF (Sec. 5.1): rho w [1/I0 + xi.u/I2 + (xi.u)^2/(2 I4)
    //   + u^2 xi^2 (Delta2^2 - 1)/(2 D I4) - u^2 I2 Delta2^2/(2 I0 I4)]
    c->A = 1.0 / I0;
    c->Bc = 1.0 / I2;
    c->Cc = 1.0 / (2.0 * I4);
    c->G = (Delta2sq - 1.0) / (2.0 * D * I4);
    c->H = -I2 * Delta2sq / (2.0 * I0 * I4);
    // lattice (Sec. 8.1 D1V3, Sec. 8.2 D2V9, Table lattices-tab D3V19 and
    // D3V27); c_s = sqrt(I2/(3 I4)) for all four
    c->cs = std::sqrt(I2 / (3.0 * I4));
    if (lat->vel == LBM_D2V9) {
        c->w[0] = I0 * (1.0 - 5.0 * c->J2 / 9.0);
        for (int a = 1; a <= 4; ++a) c->w[a] = I0 * c->J2 / 9.0;
        for (int a = 5; a <= 8; ++a) c->w[a] = I0 * c->J2 / 36.0;
    } else if (lat->vel == LBM_D1V3) {
        c->w[0] = I0 * (1.0 - c->J2 / 3.0);
        c->w[1] = c->w[2] = I0 * c->J2 / 6.0;
    } else if (lat->vel == LBM_D3V27) {
        // the shells' weights need I6 (fourth-order isotropy on three shells)
        const double I6 = c->I[3], I4c = I4 * I4 * I4;
        c->w[0] = I0 - 2.0 * I2 * I2 / (3.0 * I4) - I6 * I2 * I2 * I2 / (27.0 * I4c);
        for (int a = 1; a <= 6; ++a) c->w[a] = (3.0 * I2 * I2 * I4 * I4 + I6 * I2 * I2 * I2) / (54.0 * I4c);
        for (int a = 7; a <= 18; ++a) c->w[a] = (3.0 * I4 * I4 * I2 * I2 - I6 * I2 * I2 * I2) / (108.0 * I4c);
        for (int a = 19; a <= 26; ++a) c->w[a] = I2 * I2 * I2 * I6 / (216.0 * I4c);
    } else {
        c->w[0] = I0 * (1.0 - 2.0 * c->J2 / 3.0);
        for (int a = 1; a <= 6; ++a) c->w[a] = I0 * c->J2 / 18.0;
        for (int a = 7; a <= 18; ++a) c->w[a] = I0 * c->J2 / 36.0;
    }
    bool stable = c->cs > 0.0;
    for (int a = 0; a < c->Q; ++a) stable = stable && c->w[a] > 0.0;
    if (!stable) {
        lbm_destroy(c);
        return LBM_ERR_UNSTABLE_LATTICE;
    }

    // --- device buffers ---
    lbm_status st = LBM_OK;
    cudaGetDevice(&c->device);
    const size_t pop_bytes = (size_t)c->Q * (size_t)c->N * pop_elem_bytes(storage);
    KParams p = make_params(c);
    c->partials_cap = lbm::moments_partial_count(p);
    (void)pop_bytes;
    if ((st = cuda_check(c, cudaMalloc((void**)&c->nbr, sizeof(uint32_t) * c->N), "cudaMalloc neighbours")) !=
            LBM_OK ||
        (st = cuda_check(c, cudaMalloc((void**)&c->lbase, sizeof(uint32_t) * c->N), "cudaMalloc link bases")) !=
            LBM_OK ||
        (st = cuda_check(c, cudaMalloc((void**)&c->rowG, sizeof(uint32_t) * (c->ny * c->nz + 1)),
                         "cudaMalloc row links")) != LBM_OK ||
        (st = cuda_check(c, cudaMalloc((void**)&c->mask_dev, c->N), "cudaMalloc mask")) != LBM_OK ||
        (st = cuda_check(c, cudaMalloc((void**)&c->partials, sizeof(double) * 4 * c->partials_cap),
                         "cudaMalloc partials")) != LBM_OK ||
        (st = cuda_check(c, cudaMalloc((void**)&c->totals_dev, sizeof(double) * 4), "cudaMalloc totals")) !=
            LBM_OK ||
        (st = cuda_check(c, cudaMalloc((void**)&c->count_dev, sizeof(unsigned long long)), "cudaMalloc count")) !=
            LBM_OK ||
        (st = cuda_check(c, cudaMallocHost((void**)&c->totals_host, sizeof(double) * 4), "cudaMallocHost")) !=
            LBM_OK ||
        (st = cuda_check(c, cudaHostAlloc((void**)&c->status_host, sizeof(int), cudaHostAllocMapped),
                         "cudaHostAlloc status")) != LBM_OK ||
        (st = cuda_check(c, cudaHostGetDevicePointer((void**)&c->status_dev, c->status_host, 0),
                         "status device pointer")) != LBM_OK) {
        lbm_destroy(c);
        return st;
    }
    // cudaHostAlloc does not clear the word (a reused pinned page keeps the
    // bytes of its previous owner), and a nonzero word reports a timeout
    *(volatile int*)c->status_host = 0;
    // default geometry: all fluid
    if ((st = cuda_check(c, cudaMemsetAsync(c->mask_dev, 0, c->N, c->stream), "memset mask")) != LBM_OK) {
        lbm_destroy(c);
        return st;
    }
    cudaMemsetAsync(c->count_dev, 0, sizeof(unsigned long long), c->stream);
    c->launches += lbm::launch_build_neighbors(c->lat.vel, c->mask_dev, c->nbr, c->count_dev, p, c->stream);
    if ((st = cuda_check(c, cudaGetLastError(), "neighbour kernel")) != LBM_OK ||
        (st = build_links_and_state(c)) != LBM_OK) {
        lbm_destroy(c);
        return st;
    }
    c->geometry_counted = false;
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    ws_release(c);
    cudaFree(c->pop[0]);
    cudaFree(c->pop[1]);
    cudaFree(c->lmu_tab);
    cudaFree(c->nbr);
    cudaFree(c->lbase);
    cudaFree(c->rowG);
    cudaFree(c->ldesc);
    cudaFree(c->rorder);
    cudaFree(c->mask_dev);
    cudaFree(c->Efield);
    cudaFree(c->partials);
    cudaFree(c->totals_dev);
    cudaFree(c->count_dev);
    cudaFree(c->stage);
    if (c->totals_host) cudaFreeHost(c->totals_host);
    if (c->status_host) cudaFreeHost(c->status_host);
    delete c;
}

lbm_status lbm_constants(const lbm_ctx* c, double* out, int n) {
    if (!c || !out || n < 12 + c->Q) return LBM_ERR_INVALID_ARG;
    const double v[12] = {c->I[0], c->I[1], c->I[2], c->c0, c->c1, c->c2, c->cbar2, c->cprime2,
                          c->thetabar, c->J2, c->Delta2, c->cs};
    for (int k = 0; k < 12; ++k) out[k] = v[k];
    for (int a = 0; a < c->Q; ++a) out[12 + a] = c->w[a];
    return LBM_OK;
}

lbm_status lbm_info(const lbm_ctx* cc, int64_t* out, int n) {
    lbm_ctx* c = const_cast<lbm_ctx*>(cc);
    if (!c || !out || n < 9) return LBM_ERR_INVALID_ARG;
    if (!c->geometry_counted) {
        unsigned long long cnt = 0;
        LBM_CUDA(c, cudaMemcpyAsync(&cnt, c->count_dev, sizeof cnt, cudaMemcpyDeviceToHost, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
        c->n_fluid = (int64_t)cnt;
        c->geometry_counted = true;
    }
    const int64_t v[9] = {c->D, c->Q, c->nx, c->ny, c->nz, c->N, c->n_fluid, c->steps,
                          (int64_t)pop_elem_bytes(c->storage)};
    for (int k = 0; k < 9; ++k) out[k] = v[k];
    return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx* c, const uint8_t* mask) {
    if (!c || !mask) return fail(c, LBM_ERR_INVALID_ARG, "lbm_set_geometry: null argument");
    const cudaMemcpyKind kind = is_device_ptr(mask) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LBM_CUDA(c, cudaMemcpyAsync(c->mask_dev, mask, c->N, kind, c->stream));
    LBM_CUDA(c, cudaMemsetAsync(c->count_dev, 0, sizeof(unsigned long long), c->stream));
    KParams p = make_params(c);
    lbm_status st = after_launch(c, lbm::launch_build_neighbors(c->lat.vel, c->mask_dev, c->nbr, c->count_dev, p,
                                                                 c->stream));
    c->geometry_counted = false;
    c->has_state = false;
    if (st != LBM_OK) return st;
    return build_links_and_state(c);
}

lbm_status lbm_set_E_field(lbm_ctx* c, const float* E) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!E) {
        c->use_Efield = false;
        return LBM_OK;
    }
    const size_t bytes = sizeof(float) * (size_t)c->D * (size_t)c->N;
    if (!c->Efield) LBM_CUDA(c, cudaMalloc((void**)&c->Efield, bytes));
    const cudaMemcpyKind kind = is_device_ptr(E) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LBM_CUDA(c, cudaMemcpyAsync(c->Efield, E, bytes, kind, c->stream));
    c->use_Efield = true;
    return LBM_OK;
}

lbm_status lbm_set_rounding(lbm_ctx* c, int stochastic) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (stochastic && c->storage == LBM_F32)
        return fail(c, LBM_ERR_INVALID_ARG, "stochastic rounding applies to FP16/BF16 storage only");
    c->stochastic = stochastic != 0;
    return LBM_OK;
}

lbm_status lbm_set_rounding_seed(lbm_ctx* c, uint32_t seed) {
    if (!c) return LBM_ERR_INVALID_ARG;
    c->rseed = seed;
    return LBM_OK;
}

lbm_status lbm_set_local_mu(lbm_ctx* c, int enable) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!enable) {
        cudaFree(c->lmu_tab);
        c->lmu_tab = nullptr;
        return LBM_OK;
    }
    if (c->lat.vel != LBM_D2V9 && c->lat.vel != LBM_D3V19)
        return fail(c, LBM_ERR_INVALID_ARG, "lbm_set_local_mu: built for D2V9 and D3V19 only");
    if (c->lat.stat == LBM_BE)
        return fail(c, LBM_ERR_INVALID_ARG, "lbm_set_local_mu: built for the FD and MB weights only");
    if (c->lmu_tab) return LBM_OK;
    float2* tab = nullptr;
    cudaError_t e = cudaMalloc((void**)&tab, sizeof(float2) * kLmuNodes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "lbm_set_local_mu: %s",
                    cudaGetErrorString(e));
    }
    lbm_status st = LBM_OK;
    if (c->lat.stat == LBM_MB) {  // thetabar = theta whatever mu: the table is zero
        e = cudaMemsetAsync(tab, 0, sizeof(float2) * kLmuNodes, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = LBM_ERR_CUDA;
        }
    } else {
        st = lbm::build_local_mu_table(c->D, c->lat.theta, c->lat.mu, kLmuNodes, kLmuK1, kLmuDr, tab, c->stream);
    }
    if (st != LBM_OK) {
        cudaFree(tab);
        return fail(c, st, "lbm_set_local_mu: table build failed");
    }
    c->lmu_tab = tab;
    return LBM_OK;
}

lbm_status lbm_set_params(lbm_ctx* c, double tau, const double E[3], const double B[3]) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(c, LBM_ERR_INVALID_ARG, "tau must be > 1/2");
    c->tau = tau;
    for (int d = 0; d < 3; ++d) {
        if (E) c->E[d] = E[d];
        if (B) c->B[d] = B[d];
    }
    sanitize_fields(c);
    return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_ctx* c, const float* rho, const float* u) {
    if (!c) return LBM_ERR_INVALID_ARG;
    const size_t nN = (size_t)c->N;
    const float* rho_d = rho;
    const float* u_d = u;
    const bool rho_host = rho && !is_device_ptr(rho);
    const bool u_host = u && !is_device_ptr(u);
    if (rho_host || u_host) {
        lbm_status st = stage(c, sizeof(float) * nN * (1 + c->D));
        if (st != LBM_OK) return st;
        if (rho_host) {
            LBM_CUDA(c, cudaMemcpyAsync(c->stage, rho, sizeof(float) * nN, cudaMemcpyHostToDevice, c->stream));
            rho_d = c->stage;
        }
        if (u_host) {
            LBM_CUDA(c, cudaMemcpyAsync(c->stage + nN, u, sizeof(float) * nN * c->D, cudaMemcpyHostToDevice,
                                        c->stream));
            u_d = c->stage + nN;
        }
    }
    KParams p = make_params(c);
    c->cur = 0;
    lbm_status st = after_launch(c, lbm::launch_init(c->lat.vel, c->storage, c->pop[0], c->nbr, rho_d, u_d, p,
                                                      c->stream));
    if (st != LBM_OK) return st;
    c->has_state = true;
    c->steps = 0;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int64_t n) {
    if (!c || n < 0) return fail(c, LBM_ERR_INVALID_ARG, "lbm_step: bad argument");
    if (!c->has_state) return fail(c, LBM_ERR_STATE, "lbm_step before lbm_init_equilibrium");
    KParams p = make_params(c);
    const bool ef = c->use_Efield;
    for (int64_t t = 0; t < n; ++t) {
        p.step = (uint32_t)(c->steps + t);
        c->launches += lbm::launch_step(c->lat.vel, c->storage, c->lat.force, ef, c->stochastic, c->pop[c->cur],
                                        c->pop[c->cur ^ 1], c->nbr, c->Efield, p, c->stream);
        c->cur ^= 1;
    }
    c->steps += n;
    return cuda_check(c, cudaGetLastError(), "lbm_step launch");
}

lbm_status lbm_moments(lbm_ctx* c, float* rho, float* j, double* total_rho, double total_j[3]) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!c->has_state) return fail(c, LBM_ERR_STATE, "lbm_moments before lbm_init_equilibrium");
    const size_t nN = (size_t)c->N;
    const bool rho_host = rho && !is_device_ptr(rho);
    const bool j_host = j && !is_device_ptr(j);
    float* rho_d = rho;
    float* j_d = j;
    if (rho_host || j_host) {
        lbm_status st = stage(c, sizeof(float) * nN * (1 + c->D));
        if (st != LBM_OK) return st;
        if (rho_host) rho_d = c->stage;
        if (j_host) j_d = c->stage + nN;
    }
    const bool want_totals = total_rho || total_j;
    KParams p = make_params(c);
    int64_t np = 0;
    lbm_status st = after_launch(c, lbm::launch_moments(c->lat.vel, c->storage, c->pop[c->cur], c->nbr, rho_d, j_d,
                                                         want_totals ? c->partials : nullptr, &np, p, c->stream));
    if (st != LBM_OK) return st;
    if (want_totals) {
        st = after_launch(c, lbm::launch_reduce_partials(c->partials, np, c->totals_dev, c->stream));
        if (st != LBM_OK) return st;
        LBM_CUDA(c, cudaMemcpyAsync(c->totals_host, c->totals_dev, sizeof(double) * 4, cudaMemcpyDeviceToHost,
                                    c->stream));
    }
    if (rho_host)
        LBM_CUDA(c, cudaMemcpyAsync(rho, rho_d, sizeof(float) * nN, cudaMemcpyDeviceToHost, c->stream));
    if (j_host)
        LBM_CUDA(c, cudaMemcpyAsync(j, j_d, sizeof(float) * nN * c->D, cudaMemcpyDeviceToHost, c->stream));
    if (want_totals || rho_host || j_host) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (want_totals || rho_host || j_host) {
        lbm_status _ds = device_status(c);
        if (_ds != LBM_OK) return _ds;
    }
    if (want_totals) {
        for (int k = 0; k < 4; ++k)
            if (!std::isfinite(c->totals_host[k])) return fail(c, LBM_ERR_NONFINITE, "non-finite total moment");
        if (total_rho) *total_rho = c->totals_host[0];
        if (total_j)
            for (int d = 0; d < 3; ++d) total_j[d] = c->totals_host[1 + d];
    }
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* c, float* f, int deviation) {
    if (!c || !f) return fail(c, LBM_ERR_INVALID_ARG, "lbm_get_populations: null argument");
    if (!c->has_state) return fail(c, LBM_ERR_STATE, "lbm_get_populations before lbm_init_equilibrium");
    const size_t bytes = sizeof(float) * (size_t)c->Q * (size_t)c->N;
    const bool host = !is_device_ptr(f);
    float* fd = f;
    if (host) {
        lbm_status st = stage(c, bytes);
        if (st != LBM_OK) return st;
        fd = c->stage;
    }
    KParams p = make_params(c);
    lbm_status st = after_launch(c, lbm::launch_populations(c->lat.vel, c->storage, c->pop[c->cur], c->nbr, fd,
                                                             deviation != 0, p, c->stream));
    if (st != LBM_OK) return st;
    if (host) {
        LBM_CUDA(c, cudaMemcpyAsync(f, fd, bytes, cudaMemcpyDeviceToHost, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
        {
            lbm_status _ds = device_status(c);
            if (_ds != LBM_OK) return _ds;
        }
    }
    return LBM_OK;
}

lbm_status lbm_save_state(lbm_ctx* c, void* host_buf, size_t cap, size_t* used) {
    if (!c || !used) return LBM_ERR_INVALID_ARG;
    const size_t payload = c->state_bytes;
    const size_t total = sizeof(StateHeader) + payload;
    *used = total;
    if (!host_buf) return LBM_OK;
    if (cap < total) return fail(c, LBM_ERR_INVALID_ARG, "lbm_save_state: buffer too small");
    if (!c->has_state) return fail(c, LBM_ERR_STATE, "lbm_save_state without a state");
    StateHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "LBMSTAT", 8);
    h.vel = c->lat.vel;
    h.storage = c->storage;
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.steps = c->steps;
    h.payload = payload;
    unsigned char* dst = (unsigned char*)host_buf + sizeof(StateHeader);
    LBM_CUDA(c, cudaMemcpyAsync(dst, c->pop[c->cur], payload, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    {
        lbm_status _ds = device_status(c);
        if (_ds != LBM_OK) return _ds;
    }
    h.crc = checksum(dst, payload);
    std::memcpy(host_buf, &h, sizeof h);
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_ctx* c, const void* host_buf, size_t len) {
    if (!c || !host_buf) return LBM_ERR_INVALID_ARG;
    if (len < sizeof(StateHeader)) return fail(c, LBM_ERR_INVALID_ARG, "lbm_load_state: short buffer");
    StateHeader h;
    std::memcpy(&h, host_buf, sizeof h);
    const size_t payload = c->state_bytes;
    if (std::memcmp(h.magic, "LBMSTAT", 8) != 0 || h.vel != c->lat.vel || h.storage != c->storage || h.nx != c->nx ||
        h.ny != c->ny || h.nz != c->nz || h.payload != payload)
        return fail(c, LBM_ERR_INVALID_ARG, "lbm_load_state: header does not match this context");
    if (len < sizeof(StateHeader) + payload) return fail(c, LBM_ERR_INVALID_ARG, "lbm_load_state: short buffer");
    const unsigned char* src = (const unsigned char*)host_buf + sizeof(StateHeader);
    if (checksum(src, payload) != h.crc) return fail(c, LBM_ERR_INVALID_ARG, "lbm_load_state: checksum mismatch");
    LBM_CUDA(c, cudaMemcpyAsync(c->pop[c->cur], src, payload, cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    *(volatile int*)c->status_host = 0;  // the state that a timed-out wait left is replaced
    c->steps = h.steps;
    c->has_state = true;
    return LBM_OK;
}


lbm_status lbm_window_totals(lbm_ctx* c, int64_t t_begin, int64_t t_end, double out[4]) {
    if (!c || !out) return fail(c, LBM_ERR_INVALID_ARG, "lbm_window_totals: null argument");
    if (!c->has_state) return fail(c, LBM_ERR_STATE, "lbm_window_totals before lbm_init_equilibrium");
    if (t_end < 0 || t_begin < -1 || t_begin > t_end)
        return fail(c, LBM_ERR_INVALID_ARG, "lbm_window_totals: need -1 <= t_begin <= t_end");
    KParams p = make_params(c);
    LBM_CUDA(c, cudaMemsetAsync(c->totals_dev, 0, sizeof(double) * 4, c->stream));
    int64_t np = 0;
    if (t_begin < 0) {  // the start state itself is in the window
        c->launches += lbm::launch_moments(c->lat.vel, c->storage, c->pop[c->cur], c->nbr, nullptr, nullptr,
                                           c->partials, &np, p, c->stream);
        c->launches += lbm::launch_accumulate_totals(c->partials, np, c->totals_dev, c->stream);
    }
    for (int64_t t = 1; t <= t_end; ++t) {
        p.step = (uint32_t)(c->steps + t - 1);
        c->launches += lbm::launch_step(c->lat.vel, c->storage, c->lat.force, c->use_Efield, c->stochastic,
                                        c->pop[c->cur], c->pop[c->cur ^ 1], c->nbr, c->Efield, p, c->stream);
        c->cur ^= 1;
        if (t > t_begin) {
            c->launches += lbm::launch_moments(c->lat.vel, c->storage, c->pop[c->cur], c->nbr, nullptr, nullptr,
                                               c->partials, &np, p, c->stream);
            c->launches += lbm::launch_accumulate_totals(c->partials, np, c->totals_dev, c->stream);
        }
    }
    c->steps += t_end;
    LBM_CUDA(c, cudaGetLastError());
    LBM_CUDA(c, cudaMemcpyAsync(c->totals_host, c->totals_dev, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    {
        lbm_status _ds = device_status(c);
        if (_ds != LBM_OK) return _ds;
    }
    for (int k = 0; k < 4; ++k) {
        if (!std::isfinite(c->totals_host[k])) return fail(c, LBM_ERR_NONFINITE, "non-finite window total");
        out[k] = c->totals_host[k];
    }
    return LBM_OK;
}

lbm_status lbm_set_memory_budget(lbm_ctx* c, uint64_t bytes) {
    if (!c) return LBM_ERR_INVALID_ARG;
    c->mem_budget = (size_t)bytes;
    return LBM_OK;
}

lbm_status lbm_release_workspace(lbm_ctx* c) {
    if (!c) return LBM_ERR_INVALID_ARG;
    ws_release(c);
    return LBM_OK;
}

lbm_status lbm_adjoint_stats(const lbm_ctx* c, int64_t out[5]) {
    if (!c || !out) return LBM_ERR_INVALID_ARG;
    for (int k = 0; k < 4; ++k) out[k] = c->adj_stats[k];
    out[4] = (int64_t)c->state_bytes;
    return LBM_OK;
}

lbm_status lbm_selftest_wait_timeout(lbm_ctx* c, int64_t clocks) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (clocks < 1 || clocks > (1ll << 31))
        return fail(c, LBM_ERR_INVALID_ARG, "lbm_selftest_wait_timeout: need 1 <= clocks <= 2^31");
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    {
        lbm_status _ds = device_status(c);  // an earlier timeout is reported first
        if (_ds != LBM_OK) return _ds;
    }
    c->launches += lbm::launch_wait_probe(c->status_dev, (long long)clocks, c->stream);
    LBM_CUDA(c, cudaGetLastError());
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return device_status(c);
}

lbm_status lbm_adjoint(lbm_ctx* c, const float* w_rho, const float* w_j, int64_t t_begin, int64_t t_end,
                       int64_t checkpoint_every, double* dL_dE, double dL_dB[3], double* dL_dtau, double* loss,
                       float* dL_df0) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (!c->has_state) return fail(c, LBM_ERR_STATE, "lbm_adjoint before lbm_init_equilibrium");
    if (t_end < 1 || t_begin < -1 || t_begin >= t_end)
        return fail(c, LBM_ERR_INVALID_ARG, "lbm_adjoint: need -1 <= t_begin < t_end and t_end >= 1");

    if ((dL_dE && !is_device_ptr(dL_dE)) || (dL_df0 && !is_device_ptr(dL_df0)))
        return fail(c, LBM_ERR_INVALID_ARG, "lbm_adjoint: dL_dE and dL_df0 must be device pointers");
    const int64_t T = t_end;
    int64_t K = checkpoint_every < 0 ? 0 : checkpoint_every;
    if (K == 0) {
        K = 1;
        while (K * K < T) ++K;
    }
    if (K > T) K = T;
    const int64_t nseg = (T + K - 1) / K;
    const size_t pop_bytes = c->state_bytes;  // populations + link buffer
    // adjoint field: lam in population layout, then its link buffer (one FP32
    // per bounce-back link) at a 256-byte aligned offset
    const size_t lam_bytes = sizeof(float) * (size_t)c->Q * (size_t)c->N;
    const size_t lgofs = (lam_bytes + 255) & ~(size_t)255;
    const size_t lam_alloc = lgofs + ((sizeof(float) * (size_t)c->n_links + 16 + 255) & ~(size_t)255);
    KParams p = make_params(c);
    p.lgofs = lgofs;
    const int64_t nslot = lbm::adjoint_slot_count(p);

    // --- memory and schedule ---
    // Fixed: two adjoint fields, the gradient slots, staged loss weights.
    // States: the segment schedule (K > 0, or K = 0 when it fits) keeps
    // ceil(T/K) checkpoints and K - 1 replay states; the binomial schedule
    // keeps the initial state, one work buffer and s snapshots.  Buffers held
    // in the context's workspace from earlier calls count as free.
    AdjWorkspace& ws = c->ws;
    if ((ws.state_bytes && ws.state_bytes != pop_bytes) || (ws.lam_bytes && ws.lam_bytes != lam_alloc) ||
        (ws.nslot && ws.nslot != nslot))
        ws_release(c);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    free_b += ws.held();
    const size_t gpart_bytes = dL_dE ? sizeof(float) * (size_t)c->D * (size_t)c->N : 0;
    const size_t fixed =
        2 * lam_alloc + sizeof(double) * (nslot + 8) + sizeof(float) * (size_t)c->N * (1 + c->D) + gpart_bytes;
    // bytes for the kept forward states: the budget, or 95% of what the fixed part leaves free
    const size_t avail = free_b > fixed ? free_b - fixed : 0;
    const size_t budget = c->mem_budget ? std::min(c->mem_budget, avail) : avail - avail / 20;
    const int64_t states_fit = (int64_t)(budget / pop_bytes);
    bool binomial = checkpoint_every < 0 || (checkpoint_every == 0 && nseg + K - 1 > states_fit);
    // K = 0 and room for every state: keep them all during the one forward
    // sweep (no replay); the state at t = 0 is the context's current buffer
    const bool store_all = checkpoint_every == 0 && T - 1 <= states_fit;
    if (store_all) {
        binomial = false;
        K = T;
    }
    int64_t nsnap = 0;  // binomial: snapshots besides the initial state and the work buffer
    if (checkpoint_every < 0) {
        nsnap = std::min<int64_t>(-checkpoint_every, T);
        if ((size_t)(nsnap + 2) * pop_bytes + fixed > free_b)
            return fail(c, LBM_ERR_OOM, "lbm_adjoint: %lld snapshots need %.2f GB, %.2f GB free", (long long)nsnap,
                        ((size_t)(nsnap + 2) * pop_bytes + fixed) / 1e9, free_b / 1e9);
    } else if (binomial) {
        nsnap = std::min<int64_t>(states_fit - 2, T);
        if (nsnap < 0)
            return fail(c, LBM_ERR_OOM, "lbm_adjoint: the budget of %.2f GB holds fewer than 2 states of %.2f GB",
                        budget / 1e9, pop_bytes / 1e9);
    } else if ((size_t)(nseg + K - 1) * pop_bytes + fixed > free_b) {
        return fail(c, LBM_ERR_OOM, "lbm_adjoint: needs %.2f GB of device memory, %.2f GB free; choose "
                    "checkpoint_every near sqrt(t_end), or 0 for a schedule sized to the memory budget",
                    ((size_t)(nseg + K - 1) * pop_bytes + fixed) / 1e9, free_b / 1e9);
    }
    const int64_t nstates = binomial ? nsnap + 2 : (store_all ? T - 1 : nseg + K - 1);
    lbm_status st = LBM_OK;
#define ADJ_CHECK(call)                                        \
    do {                                                       \
        st = cuda_check(c, (call), #call);                     \
        if (st != LBM_OK) {                                    \
            cudaStreamSynchronize(c->stream);                  \
            return st;                                         \
        }                                                      \
    } while (0)
    // grow the workspace to this call's needs (buffers are reused as they are)
    ws.state_bytes = pop_bytes;
    while ((int64_t)ws.states.size() < nstates) {
        void* q = nullptr;
        ADJ_CHECK(cudaMalloc(&q, pop_bytes));
        ws.states.push_back(q);
    }
    if (!ws.lam[0]) {
        ADJ_CHECK(cudaMalloc(&ws.lam[0], lam_alloc));
        ADJ_CHECK(cudaMalloc(&ws.lam[1], lam_alloc));
        ws.lam_bytes = lam_alloc;
    }
    if (!ws.slots) {
        ADJ_CHECK(cudaMalloc((void**)&ws.slots, sizeof(double) * nslot));
        ws.nslot = nslot;
    }
    if (!ws.red) ADJ_CHECK(cudaMalloc((void**)&ws.red, sizeof(double) * 8));
    if (gpart_bytes && ws.gpart_bytes != gpart_bytes) {
        cudaFree(ws.gpart);
        ws.gpart = nullptr;
        ws.gpart_bytes = 0;
        ADJ_CHECK(cudaMalloc((void**)&ws.gpart, gpart_bytes));
        ws.gpart_bytes = gpart_bytes;
    }
    // the schedule's views of the state buffers
    std::vector<void*> ckpt, seg, snaps;
    void* base = nullptr;   // binomial: the state at t = 0
    void* work1 = nullptr;  // binomial: second work buffer
    {
        size_t k = 0;
        if (binomial) {
            base = ws.states[k++];
            work1 = ws.states[k++];
            for (int64_t i = 0; i < nsnap; ++i) snaps.push_back(ws.states[k++]);
        } else {
            if (!store_all)
                for (int64_t i = 0; i < nseg; ++i) ckpt.push_back(ws.states[k++]);
            seg.assign((size_t)K, nullptr);
            for (int64_t i = 1; i < K; ++i) seg[i] = ws.states[k++];
        }
    }
    float* lam[2] = {(float*)ws.lam[0], (float*)ws.lam[1]};
    double* slots = ws.slots;
    double* red = ws.red;
    ADJ_CHECK(cudaMemsetAsync(slots, 0, sizeof(double) * nslot, c->stream));
    // loss weights: device, or staged from the host
    const float* wr_d = w_rho;
    const float* wj_d = w_j;
    if ((w_rho && !is_device_ptr(w_rho)) || (w_j && !is_device_ptr(w_j))) {
        if (!ws.wstage) {
            ADJ_CHECK(cudaMalloc((void**)&ws.wstage, sizeof(float) * (size_t)c->N * (1 + c->D)));
            ws.wstage_bytes = sizeof(float) * (size_t)c->N * (1 + c->D);
        }
        float* wstage = ws.wstage;
        if (w_rho && !is_device_ptr(w_rho)) {
            ADJ_CHECK(cudaMemcpyAsync(wstage, w_rho, sizeof(float) * c->N, cudaMemcpyHostToDevice, c->stream));
            wr_d = wstage;
        }
        if (w_j && !is_device_ptr(w_j)) {
            ADJ_CHECK(cudaMemcpyAsync(wstage + c->N, w_j, sizeof(float) * c->N * c->D, cudaMemcpyHostToDevice,
                                      c->stream));
            wj_d = wstage + c->N;
        }
    }
    if (dL_dE) {
        ADJ_CHECK(cudaMemsetAsync(dL_dE, 0, sizeof(double) * (size_t)c->D * c->N, c->stream));
        ADJ_CHECK(cudaMemsetAsync(ws.gpart, 0, gpart_bytes, c->stream));
    }
    // dL/dE: each reverse step adds into FP32 partials, folded into the FP64
    // gradient every kFoldEvery reverse steps (counted from t_end, so every
    // schedule folds after the same steps) and at the end
    constexpr int64_t kFoldEvery = 32;
    float* gpart = dL_dE ? ws.gpart : nullptr;
    int64_t rsteps = 0;

    const int vel = c->lat.vel, sto = c->storage, force = c->lat.force;
    const bool ef = c->use_Efield, sr = c->stochastic;
    const int64_t step0 = c->steps;
    int li = 0;
    int64_t fwd_steps = 0;
    // one forward step of global index step0 + t, in -> out
    auto fstep = [&](int64_t t, const void* in, void* out) {
        p.step = (uint32_t)(step0 + t);
        c->launches += lbm::launch_step(vel, sto, force, ef, sr, in, out, c->nbr, c->Efield, p, c->stream);
        ++fwd_steps;
    };
    // one reverse step at t from the state at t: lam_{t+1} -> lam_t
    auto rstep = [&](int64_t t, const void* state) {
        const bool win = t > t_begin && t <= t_end;
        c->launches += lbm::launch_adjoint_step(vel, sto, force, ef, win, state, lam[li], lam[li ^ 1], c->nbr,
                                                c->Efield, wr_d, wj_d, gpart, slots, p, c->stream);
        li ^= 1;
        if (gpart && ++rsteps % kFoldEvery == 0)
            c->launches += lbm::launch_fold_partials(gpart, dL_dE, (int64_t)c->D * c->N, c->stream);
    };
    auto seed = [&](const void* state_T) {
        c->launches += lbm::launch_adjoint_seed(vel, sto, state_T, c->nbr, wr_d, wj_d, lam[li], slots,
                                                T > t_begin && T <= t_end, p, c->stream);
    };
    if (store_all) {
        // --- one forward sweep keeping every state, then the reverse sweep ---
        seg[0] = c->pop[c->cur];
        for (int64_t t = 0; t < T; ++t) fstep(t, seg[t], t + 1 < T ? seg[t + 1] : c->pop[c->cur ^ 1]);
        ADJ_CHECK(cudaGetLastError());
        seed(c->pop[c->cur ^ 1]);
        for (int64_t t = T - 1; t >= 0; --t) rstep(t, seg[t]);
        ADJ_CHECK(cudaGetLastError());
        seg[0] = nullptr;
        c->cur ^= 1;  // the context's current state is the state at T
    } else if (!binomial) {
        // --- forward with checkpoints every K steps ---
        for (int64_t t = 0; t < T; ++t) {
            if (t % K == 0)
                ADJ_CHECK(
                    cudaMemcpyAsync(ckpt[t / K], c->pop[c->cur], pop_bytes, cudaMemcpyDeviceToDevice, c->stream));
            fstep(t, c->pop[c->cur], c->pop[c->cur ^ 1]);
            c->cur ^= 1;
        }
        ADJ_CHECK(cudaGetLastError());
        seed(c->pop[c->cur]);
        // --- reverse sweep, one segment at a time: replay storing every state ---
        for (int64_t s = nseg - 1; s >= 0; --s) {
            const int64_t t0 = s * K, t1 = std::min(t0 + K, T);
            seg[0] = ckpt[s];
            for (int64_t t = t0; t < t1 - 1; ++t) fstep(t, seg[t - t0], seg[t - t0 + 1]);
            for (int64_t t = t1 - 1; t >= t0; --t) rstep(t, seg[t - t0]);
            ADJ_CHECK(cudaGetLastError());
        }
        seg[0] = nullptr;
    } else {
        // --- binomial schedule (the recursion of Griewank's revolve): with s
        // free snapshots, a span of n steps is split so that the right part
        // [m, t1) is reversed first with s - 1 snapshots and the left part
        // [t0, m) after it with s; with r the smallest number of sweeps such
        // that C(s + r, s) >= n, the left part takes C(s + r - 1, s) steps.
        // Each forward state is recomputed bit for bit (the rounding stream
        // depends only on the global step index), so every schedule gives the
        // same gradients.  The state at T ends in the context's other buffer.
        ADJ_CHECK(cudaMemcpyAsync(base, c->pop[c->cur], pop_bytes, cudaMemcpyDeviceToDevice, c->stream));
        void* work[2] = {c->pop[c->cur], work1};
        void* final_state = c->pop[c->cur ^ 1];
        bool seeded = false;
        auto binom = [](int64_t n, int64_t k) {  // C(n, k), saturating
            double v = 1.0;
            for (int64_t i = 1; i <= k; ++i) {
                v = v * (double)(n - k + i) / (double)i;
                if (v > 4e18) return (int64_t)4e18;
            }
            return (int64_t)(v + 0.5);
        };
        // state at t0 + n from `from` (at t0): the last step writes `dst`
        auto advance_to = [&](const void* from, int64_t t0, int64_t n, void* dst) {
            const void* in = from;
            for (int64_t k = 0; k < n; ++k) {
                void* out = (k == n - 1) ? dst : work[k & 1];
                fstep(t0 + k, in, out);
                in = out;
            }
        };
        // state at t0 + n in a work buffer (or `from` itself when n = 0)
        auto advance_w = [&](const void* from, int64_t t0, int64_t n) {
            const void* in = from;
            for (int64_t k = 0; k < n; ++k) {
                fstep(t0 + k, in, work[k & 1]);
                in = work[k & 1];
            }
            return in;
        };
        std::vector<void*> pool = snaps;
        // reverses [t0, t1) with the state at t0 in `at`; recursion depth <= s + 1
        std::function<void(int64_t, int64_t, const void*)> reverse = [&](int64_t t0, int64_t t1, const void* at) {
            while (t1 > t0) {
                const int64_t n = t1 - t0;
                if (!seeded) {  // the first leaf is the rightmost: make the state at T and seed lam_T
                    if (n == 1 || pool.empty()) {
                        advance_to(at, t0, n, final_state);
                        seed(final_state);
                        seeded = true;
                    }
                }
                if (n == 1) {
                    rstep(t0, at);
                    return;
                }
                if (pool.empty()) {  // no snapshot left: recompute from t0 for every step
                    for (int64_t t = t1 - 1; t >= t0; --t) rstep(t, advance_w(at, t0, t - t0));
                    return;
                }
                const int64_t sfree = (int64_t)pool.size();
                int64_t r = 1;
                while (binom(sfree + r, sfree) < n) ++r;
                const int64_t left = std::max<int64_t>(1, std::min<int64_t>(binom(sfree + r - 1, sfree), n - 1));
                void* snap = pool.back();
                pool.pop_back();
                advance_to(at, t0, left, snap);
                reverse(t0 + left, t1, snap);
                pool.push_back(snap);
                t1 = t0 + left;  // then the left part, with the snapshot free again
            }
        };
        reverse(0, T, base);
        ADJ_CHECK(cudaGetLastError());
        c->cur ^= 1;  // the context's current state is the state at T
    }
    if (gpart && rsteps % kFoldEvery != 0)  // the last partials
        c->launches += lbm::launch_fold_partials(gpart, dL_dE, (int64_t)c->D * c->N, c->stream);
    c->adj_stats[0] = store_all ? 2 : (binomial ? 1 : 0);
    c->adj_stats[1] = store_all ? T + 1 : (binomial ? 2 + nsnap : nseg + K - 1);
    c->adj_stats[2] = fwd_steps;
    c->adj_stats[3] = T;
    if (dL_df0) {
        c->launches += lbm::launch_unslot(c->lat.vel, lam[li], dL_df0, p, c->stream);
        ADJ_CHECK(cudaGetLastError());
    }
    c->launches += lbm::launch_reduce_slots(slots, nslot / 5, 5, red, c->stream);
    double host[5];
    ADJ_CHECK(cudaMemcpyAsync(host, red, sizeof(double) * 5, cudaMemcpyDeviceToHost, c->stream));
    ADJ_CHECK(cudaStreamSynchronize(c->stream));
#undef ADJ_CHECK
    {
        lbm_status _ds = device_status(c);
        if (_ds != LBM_OK) return _ds;
    }
    c->steps += T;
    for (int k = 0; k < 5; ++k)
        if (!std::isfinite(host[k])) return fail(c, LBM_ERR_NONFINITE, "lbm_adjoint: non-finite gradient or loss");
    if (dL_dB) {
        dL_dB[0] = host[0];
        dL_dB[1] = host[1];
        dL_dB[2] = host[2];
        if (c->D == 2) dL_dB[0] = dL_dB[1] = 0.0;
    }
    if (dL_dtau) *dL_dtau = host[3];
    if (loss) *loss = host[4];
    return LBM_OK;
}

}  // extern "C"
