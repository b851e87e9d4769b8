// Step kernels of the semiclassical LBM (templates): the fused pull-stream +
// BGK collision + Lorentz forcing update of Sec. 9.1, a general one-thread-
// per-cell kernel and a row-staged persistent kernel, plus their launcher.
// Included by one translation unit per storage type.
#pragma once

#include <mutex>

#include "lbm_device.cuh"

namespace lbm {
namespace stepk {

using dev::Cell;
using dev::kBlock;

// ---------------------------------------------------------------------------
// The fused step.  f(x, t) is pulled, its moments taken, the force applied,
// f^eq formed and the BGK relaxation written (Sec. 9.1), all in scaled
// deviations h~ = s (f - f0):
//   h~*_a = (1 - w) h~_a + w heq~_a + S~_a,  w = 1/tau,
//   heq~_a = w_a [A drho~ + s rho (Cp (e.u)^2 + k2_a u^2)] + W1_a (e_a . j~)   (+ shift part)
// FORCE 0: velocity shift u* = u + tau (E + u x B) (Sec. 7, Eq.
//          u-update-force-term-eq): the odd part uses j~ + s c_s rho tau a.
// FORCE 1: S_a = a_a . grad_u f^eq_a with a_a = E + xi_a x B (Sec. 7, Eq.
//          forcing-term-integrals-eq):
//          S~_a = s rho w_a [2 Cp (e.u)(e.E) + 2 k2_a u.E]                  (even)
//               + W1_a (e . s c_s rho E) + 2 s rho w_a k2_a (e.(B x u))/c_s (odd).
// Opposite directions share the even part and negate the odd part, so the
// work is done once per pair; the rest population closes the mass balance
// exactly: h~*_0 = sum_a h~_a - sum_{a>0} h~*_a.
// ---------------------------------------------------------------------------
// The weights w_a, k2_a and W1_a depend on the shell |e_a|^2 only (axis 1,
// face diagonal 2, corner 3; each lattice has some of them), so the per-cell
// factors are folded per shell first:
//   even_a = w_s (c0 + k2_s Ku) + w_s Cp s rho (e.u*) (w (e.u*) + 2 (e.E)),
//            c0 = w A drho~, Ku = s rho (w u*^2 + 2 u.E)        (the E terms: FORCE 1)
//   odd_a  = e_a . V_s,  V_s = W1_s v + 2 s rho w_s k2_s (B x u) / c_s  (B term: FORCE 1),
// with v = w j~ + s c_s rho E (FORCE 1) or w j~ + s c_s rho a (FORCE 0), and
// W1_s applied as its double-float pair once per cell.
// Arithmetic helpers of the value type V of collide_emit (float here).
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vdiv(float c, float x) { return c / x; }

template <class L, class V>
__device__ __forceinline__ V vedot(int a, const V* v) {
    V r(0.f);
    if (L::c(a, 0) > 0) r += v[0];
    if (L::c(a, 0) < 0) r -= v[0];
    if (L::c(a, 1) > 0) r += v[1];
    if (L::c(a, 1) < 0) r -= v[1];
    if (L::D == 3) {
        if (L::c(a, 2) > 0) r += v[2];
        if (L::c(a, 2) < 0) r -= v[2];
    }
    return r;
}

// Local chemical-potential model (LMU): the EDF of Sec. 9.1, Eq.
// feq-exp-2nd-order-eq, keeps its thetabar terms with the cell's own
// thetabar(rho) instead of the weight's thetabar_w; they add
// rho w_a K_a (thetabar - thetabar_w) with K_a a constant of the shell
// |e_a|^2 (KParams::lmu_K), no u dependence (so neither forcing form changes)
// and sum_a w_a K_a = 0 (the rest population's share follows from the mass
// closure).  lmu_kd returns w s rho (thetabar - thetabar_w) from the table.
__device__ __forceinline__ float lmu_kd(const KParams& p, float drho, float rho) {
    // (r - 1) / dr relative to the node of r = 1 (index lmu_b), so that the
    // fraction t keeps FP32's relative precision near r = 1
    float x = drho * p.lmu_a;
    x = fminf(fmaxf(x, -p.lmu_b), (float)(p.lmu_n - 1) - p.lmu_b);  // also maps NaN to node 0
    const float fl = floorf(x);
    int i = (int)fl + (int)p.lmu_b;
    float t = x - fl;
    if (i > p.lmu_n - 2) {  // x at the last node
        i = p.lmu_n - 2;
        t = 1.f;
    }
    const float t2 = t * t, t3 = t2 * t;
    const float2 a = __ldg(p.lmu_tab + i), b = __ldg(p.lmu_tab + i + 1);
    const float d = (2.f * t3 - 3.f * t2 + 1.f) * a.x + (t3 - 2.f * t2 + t) * a.y + (3.f * t2 - 2.f * t3) * b.x +
                    (t3 - t2) * b.y;
    return p.omega * p.scale * rho * d;
}

// The post-collision values go to emit(a, h*_a, h*_a+1) pair by pair (a odd)
// and then to emit_rest(h*_0), so a caller can round and store each pair as
// soon as it exists instead of holding all Q values.
template <class L, int FORCE, bool LMU = false, class V, class Emit, class EmitRest>
__device__ __forceinline__ void collide_emit(const V* h, const V* E, const KParams& p, Emit&& emit,
                                             EmitRest&& emit_rest) {
    constexpr int kR1 = shell_first<L>(1), kR2 = shell_first<L>(2), kR3 = shell_first<L>(3);
    V drho = h[0], j[3] = {V(0.f), V(0.f), V(0.f)};
#pragma unroll
    for (int a = 1; a < L::Q; a += 2) {
        const V sum = h[a] + h[a + 1], dif = h[a] - h[a + 1];
        drho += sum;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (L::c(a, d) > 0) j[d] += dif;
            if (L::c(a, d) < 0) j[d] -= dif;
        }
    }
    const V rho = vfma(drho, V(p.inv_scale), V(p.rho0));
    const V q = vdiv(p.inv_scale * p.cs_inv, rho);  // u = j~ q  (xi units)
    const V u[3] = {j[0] * q, j[1] * q, j[2] * q};
    const V srho = V(p.scale) * rho;
    const V om(p.omega), omm(1.0f - p.omega);
    const V scr = srho * V(p.cs);  // s c_s rho
    V ue[3], v[3], bu[3] = {V(0.f), V(0.f), V(0.f)}, Ku, cq;
    if (FORCE == 0) {
        const V a0 = E[0] + (u[1] * V(p.B[2]) - u[2] * V(p.B[1]));
        const V a1 = E[1] + (u[2] * V(p.B[0]) - u[0] * V(p.B[2]));
        const V a2 = (L::D == 3) ? E[2] + (u[0] * V(p.B[1]) - u[1] * V(p.B[0])) : V(0.f);
        ue[0] = vfma(V(p.tau), a0, u[0]);
        ue[1] = vfma(V(p.tau), a1, u[1]);
        ue[2] = vfma(V(p.tau), a2, u[2]);
        // odd part of w heq~ at u*: W1 (e . (w j~ + s c_s rho a))
        v[0] = vfma(om, j[0], scr * a0);
        v[1] = vfma(om, j[1], scr * a1);
        v[2] = vfma(om, j[2], scr * a2);
        Ku = om * srho * (ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2]);
        cq = om * srho * V(p.Cp);
    } else {
        ue[0] = u[0];
        ue[1] = u[1];
        ue[2] = u[2];
        v[0] = vfma(om, j[0], scr * E[0]);
        v[1] = vfma(om, j[1], scr * E[1]);
        v[2] = vfma(om, j[2], scr * E[2]);
        const V uE = u[0] * E[0] + u[1] * E[1] + u[2] * E[2];
        const V tb = V(2.f * p.cs_inv) * srho;  // 2 s rho / c_s times (B x u)
        bu[0] = tb * (V(p.B[1]) * u[2] - V(p.B[2]) * u[1]);
        bu[1] = tb * (V(p.B[2]) * u[0] - V(p.B[0]) * u[2]);
        bu[2] = tb * (V(p.B[0]) * u[1] - V(p.B[1]) * u[0]);
        Ku = srho * vfma(om, u[0] * u[0] + u[1] * u[1] + u[2] * u[2], V(2.f) * uE);
        cq = srho * V(p.Cp);
    }
    const V c0 = V(p.omega * p.A) * drho;
    V kd(0.f);
    if constexpr (LMU) kd = lmu_kd(p, drho, rho);
    V rest = drho;
    if constexpr (kR1 > 0 && kR2 > 0 && kR3 < 0) {
        // two moving shells (D2V9, D3V19): axis and diagonal
        constexpr int kAx = kR1, kDg = kR2;
        const V c0a = LMU ? vfma(V(p.lmu_K[1]), kd, c0) : c0, c0d = LMU ? vfma(V(p.lmu_K[2]), kd, c0) : c0;
        // per shell: the even constant, the (e.u) coefficient and the odd vector
        const V e0a = V(p.w[kAx]) * vfma(V(p.k2[kAx]), Ku, c0a), e0d = V(p.w[kDg]) * vfma(V(p.k2[kDg]), Ku, c0d);
        const V cqa = V(p.w[kAx]) * cq, cqd = V(p.w[kDg]) * cq;
        V Va[3], Vd[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Va[d] = vfma(V(p.W1lo[kAx]), v[d], V(p.W1hi[kAx]) * v[d]);
            Vd[d] = vfma(V(p.W1lo[kDg]), v[d], V(p.W1hi[kDg]) * v[d]);
            if (FORCE == 1) {
                Va[d] = vfma(V(p.w[kAx] * p.k2[kAx]), bu[d], Va[d]);
                Vd[d] = vfma(V(p.w[kDg] * p.k2[kDg]), bu[d], Vd[d]);
            }
        }
#pragma unroll
        for (int a = 1; a < L::Q; a += 2) {
            const bool ax = esq_of<L>(a) == 1;
            const V eu = vedot<L>(a, ue);
            const V g = (FORCE == 1) ? vfma(om, eu, V(2.f) * vedot<L>(a, E)) : eu;
            const V even = vfma(ax ? cqa : cqd, eu * g, ax ? e0a : e0d);
            const V odd = vedot<L>(a, ax ? Va : Vd);
            const V ha = vfma(omm, h[a], even) + odd;
            const V hb = vfma(omm, h[a + 1], even) - odd;
            rest -= ha + hb;
            emit(a, ha, hb);
        }
    } else {
        // per shell s (index s = |e|^2): the even constant, the (e.u) coefficient and the odd vector
        V e0[4], cqs[4], Vs[4][3];
#pragma unroll
        for (int sh = 1; sh <= 3; ++sh) {
            const int r = sh == 1 ? kR1 : (sh == 2 ? kR2 : kR3);
            if (r < 0) continue;
            e0[sh] = V(p.w[r]) * vfma(V(p.k2[r]), Ku, LMU ? vfma(V(p.lmu_K[sh]), kd, c0) : c0);
            cqs[sh] = V(p.w[r]) * cq;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                Vs[sh][d] = vfma(V(p.W1lo[r]), v[d], V(p.W1hi[r]) * v[d]);
                if (FORCE == 1) Vs[sh][d] = vfma(V(p.w[r] * p.k2[r]), bu[d], Vs[sh][d]);
            }
        }
#pragma unroll
        for (int a = 1; a < L::Q; a += 2) {
            const int sh = esq_of<L>(a);
            const V eu = vedot<L>(a, ue);
            const V g = (FORCE == 1) ? vfma(om, eu, V(2.f) * vedot<L>(a, E)) : eu;
            const V even = vfma(cqs[sh], eu * g, e0[sh]);
            const V odd = vedot<L>(a, Vs[sh]);
            const V ha = vfma(omm, h[a], even) + odd;
            const V hb = vfma(omm, h[a + 1], even) - odd;
            rest -= ha + hb;
            emit(a, ha, hb);
        }
    }
    emit_rest(rest);
}

template <class L, int FORCE, bool LMU = false>
__device__ __forceinline__ void collide(const float* h, const float* E, const KParams& p, float* out) {
    collide_emit<L, FORCE, LMU>(
        h, E, p,
        [&](int a, float ha, float hb) {
            out[a] = ha;
            out[a + 1] = hb;
        },
        [&](float rest) { out[0] = rest; });
}

// Error-free transformations (Knuth TwoSum, FMA TwoProd) for the compensated
// FP32 collision below.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = __fmaf_rn(a, b, -p);
}

// Compensated collision for FP32 storage.  Same formulas as collide(), but the
// moments and the momentum-carrying odd parts (w j~ + s c_s rho E, times W1,
// and e_a . V) are carried as double-float (hi + lo); the final combination
// (1 - w) h + even + odd is plain FP32.  With plain FP32 moments and momentum
// chain each collision adds roundings of size eps |h| to the momentum, which
// over thousands of steps exceed the 1e-5 target for FP32 storage (measured:
// 5.9e-5 after 5000 Poiseuille steps, 7.8e-5 after 2000 Riemann steps); with
// both compensated the errors are 6e-7 and 6e-6, within 1.1x of also
// compensating the final sum, which costs another 28% of the step.
template <class L, int FORCE, bool LMU = false>
__device__ __forceinline__ void collide_acc(const float* h, const float* E, const KParams& p, float* out) {
    constexpr int kR1 = shell_first<L>(1), kR2 = shell_first<L>(2), kR3 = shell_first<L>(3);
    float drho = h[0], drho_lo = 0.f, j[3] = {0.f, 0.f, 0.f}, jl[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 1; a < L::Q; a += 2) {
        float sum, es, dif, ed, e;
        two_sum(h[a], h[a + 1], sum, es);
        two_sum(h[a], -h[a + 1], dif, ed);
        two_sum(drho, sum, drho, e);
        drho_lo += e + es;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (L::c(a, d) > 0) {
                two_sum(j[d], dif, j[d], e);
                jl[d] += e + ed;
            }
            if (L::c(a, d) < 0) {
                two_sum(j[d], -dif, j[d], e);
                jl[d] += e - ed;
            }
        }
    }
    const float drho_f = drho + drho_lo;
    const float rho = p.rho0 + drho_f * p.inv_scale;
    const float jf[3] = {j[0] + jl[0], j[1] + jl[1], j[2] + jl[2]};
    const float q = p.inv_scale * p.cs_inv / rho;
    const float u[3] = {jf[0] * q, jf[1] * q, jf[2] * q};
    const float srho = p.scale * rho;
    const float om = p.omega, omm = 1.0f - p.omega;
    const float scr = srho * p.cs;
    float ue[3], F[3], uE = 0.f, bu[3] = {0.f, 0.f, 0.f};
    if (FORCE == 0) {
        F[0] = E[0] + (u[1] * p.B[2] - u[2] * p.B[1]);
        F[1] = E[1] + (u[2] * p.B[0] - u[0] * p.B[2]);
        F[2] = (L::D == 3) ? E[2] + (u[0] * p.B[1] - u[1] * p.B[0]) : 0.f;
        ue[0] = u[0] + p.tau * F[0];
        ue[1] = u[1] + p.tau * F[1];
        ue[2] = u[2] + p.tau * F[2];
    } else {
        F[0] = E[0];
        F[1] = E[1];
        F[2] = E[2];
        ue[0] = u[0];
        ue[1] = u[1];
        ue[2] = u[2];
        uE = u[0] * E[0] + u[1] * E[1] + u[2] * E[2];
        const float tb = 2.f * srho * p.cs_inv;
        bu[0] = tb * (p.B[1] * u[2] - p.B[2] * u[1]);
        bu[1] = tb * (p.B[2] * u[0] - p.B[0] * u[2]);
        bu[2] = tb * (p.B[0] * u[1] - p.B[1] * u[0]);
    }
    // v = w j~ + s c_s rho F as hi + lo
    float vh[3], vl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float pp, ep, e;
        two_prod(om, j[d], pp, ep);
        two_sum(pp, scr * F[d], vh[d], e);
        vl[d] = e + ep + om * jl[d];
    }
    // per shell s = |e|^2: V_s = W1_s v as a double-float product, plus the
    // B term 2 s rho w_s k2_s (B x u) / c_s (FORCE 1) in the low part; the
    // even constant and the (e.u) coefficient, as in collide()
    float Vh[4][3], Vl[4][3];
#pragma unroll
    for (int sh = 1; sh <= 3; ++sh) {
        const int r = sh == 1 ? kR1 : (sh == 2 ? kR2 : kR3);
        if (r < 0) continue;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float e;
            two_prod(p.W1hi[r], vh[d], Vh[sh][d], e);
            Vl[sh][d] = e + p.W1hi[r] * vl[d] + p.W1lo[r] * vh[d];
            if (FORCE == 1) Vl[sh][d] += p.w[r] * p.k2[r] * bu[d];
        }
    }
    const float u2 = ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2];
    const float c0 = om * p.A * drho_f;
    const float Ku = (FORCE == 1) ? srho * (om * u2 + 2.f * uE) : om * srho * u2;
    const float cq = (FORCE == 1) ? srho * p.Cp : om * srho * p.Cp;
    float e0[4], cqs[4], kd = 0.f;
    if constexpr (LMU) kd = lmu_kd(p, drho_f, rho);
#pragma unroll
    for (int sh = 1; sh <= 3; ++sh) {
        const int r = sh == 1 ? kR1 : (sh == 2 ? kR2 : kR3);
        if (r < 0) continue;
        e0[sh] = p.w[r] * ((LMU ? fmaf(p.lmu_K[sh], kd, c0) : c0) + p.k2[r] * Ku);
        cqs[sh] = p.w[r] * cq;
    }
    float rest = drho;
    const float rest_lo = drho_lo;
#pragma unroll
    for (int a = 1; a < L::Q; a += 2) {
        const int sh = esq_of<L>(a);
        const float eu = dev::edot<L>(a, ue);
        const float g = (FORCE == 1) ? fmaf(om, eu, 2.f * dev::edot<L>(a, E)) : eu;
        const float even = fmaf(cqs[sh], eu * g, e0[sh]);
        // odd = e . V_s in double-float
        float oh = 0.f, ol = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float e;
            if (L::c(a, d) > 0) {
                two_sum(oh, Vh[sh][d], oh, e);
                ol += e + Vl[sh][d];
            }
            if (L::c(a, d) < 0) {
                two_sum(oh, -Vh[sh][d], oh, e);
                ol += e - Vl[sh][d];
            }
        }
        // (1 - w) h + even +/- odd
        const float o = oh + ol;
        const float ha = fmaf(omm, h[a], even) + o;
        const float hb = fmaf(omm, h[a + 1], even) - o;
        out[a] = ha;
        out[a + 1] = hb;
        rest -= ha + hb;
    }
    out[0] = rest + rest_lo;
}

// The "lowbias32" integer hash of C. Wellons (seeds the rounding stream).
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Random stream for stochastic rounding: one hash of (cell, step) per cell,
// then per pair of stores one step of a 32-bit LCG (Numerical Recipes
// constants) folded as x ^ (x >> 16), so that the low bits of each 16-bit half
// (the bits the conversion consumes) mix in the LCG's strong high bits.  A
// replayed step reproduces its stores bit for bit.
struct Rng {
    uint32_t x;
    __device__ __forceinline__ Rng(uint32_t cell, const KParams& p)
        : x(hash32(cell ^ hash32(p.step * 0x9E3779B9u + p.seed))) {}
    __device__ __forceinline__ uint32_t pair() {
        x = x * 1664525u + 1013904223u;
        return x ^ (x >> 16);
    }
};

// Rounds the Q post-collision values to storage: the opposite pairs (a, a + 1),
// then out[0] (converted as a pair with itself), stochastically when SR.
template <class L, class S, bool SR>
__device__ __forceinline__ void round_all(const float* out, uint32_t cell, const KParams& p, typename S::T* t) {
    if (SR) {
        Rng rng(cell, p);
        typename S::T unused;
#pragma unroll
        for (int a = 1; a < L::Q; a += 2) S::sr2(out[a], out[a + 1], rng.pair(), t[a], t[a + 1]);
        S::sr2(out[0], out[0], rng.pair(), t[0], unused);
    } else {
#pragma unroll
        for (int a = 0; a < L::Q; ++a) S::put(&t[a], out[a]);
    }
}

template <class L>
__device__ __forceinline__ void load_E(const float* __restrict__ Ef, bool ef, const KParams& p, uint32_t cell,
                                       float* E) {
    if (ef) {
        E[0] = __ldg(Ef + cell);
        E[1] = (L::D >= 2) ? __ldg(Ef + p.N + cell) : 0.f;
        E[2] = (L::D == 3) ? __ldg(Ef + 2 * p.N + cell) : 0.f;
    } else {
        E[0] = p.E[0];
        E[1] = p.E[1];
        E[2] = p.E[2];
    }
}

template <class L, class S, int FORCE, bool LMU = false>
__device__ __forceinline__ void collide_any(const float* h, const float* E, const KParams& p, float* out) {
    if (S::kBytes == 4)
        collide_acc<L, FORCE, LMU>(h, E, p, out);
    else
        collide<L, FORCE, LMU>(h, E, p, out);
}

// General step kernel: one thread per cell, pulls straight from global memory
// and writes every own slot (solid cells write zeros, so that every sector is
// written whole); links into solid cells also store into their link slot.
template <class L, class S, int FORCE, bool EF, bool SR>
__global__ void __launch_bounds__(kBlock) k_step(const typename S::T* __restrict__ Pin, typename S::T* __restrict__ Pout,
                                                 const uint32_t* __restrict__ nbr, const float* __restrict__ Ef,
                                                 KParams p) {
    Cell c;
    if (!dev::cell_of_thread(p, c)) return;
    const uint32_t m = __ldg(nbr + c.cell);
    if (m & kSolidBit) {
#pragma unroll
        for (int a = 0; a < L::Q; ++a) S::put(Pout + dev::pop_at<L>(p, c, a, 0), 0.f);
        return;
    }
    float h[L::Q];
    dev::pull<L, S>(Pin, p, m, c, h);
    float E[3];
    load_E<L>(Ef, EF, p, c.cell, E);
    float out[L::Q];
    // the local-mu model is built for D2V9 and D3V19 (the host refuses others)
    constexpr bool kLmu = L::Q == 9 || L::Q == 19;
    if (kLmu && p.lmu_tab)
        collide_any<L, S, FORCE, kLmu>(h, E, p, out);
    else
        collide_any<L, S, FORCE>(h, E, p, out);
    typename S::T t[L::Q];
    round_all<L, S, SR>(out, c.cell, p, t);
    typename S::T* Gout = reinterpret_cast<typename S::T*>(reinterpret_cast<char*>(Pout) + p.gofs);
    const uint32_t o = outgoing<L::Q>(m);
    const uint32_t base = m ? __ldg(p.lbase + c.cell) : 0u;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        Pout[dev::pop_at<L>(p, c, a, 0)] = t[a];
        if (a != 0 && ((o >> a) & 1u)) Gout[link_slot(base, o, a)] = t[a];
    }
}

// ---------------------------------------------------------------------------
// Row-staged step kernel (used when a whole x-row of one direction is a
// whole number of 16-byte chunks and the stages fit shared memory).  A
// persistent block walks rows r = blockIdx.x, blockIdx.x + gridDim.x, ...:
//  - the Q source rows P_a(y - e_ay, z - e_az, :) of the row (one contiguous
//    block of consecutive slots per neighbouring row, at most 9 copies), its
//    cell order and its ranges of the link buffer and of the link
//    descriptors arrive by bulk asynchronous copies into a ring of STAGES
//    stages, STAGES - 1 rows ahead of the row being computed.  One thread,
//    lane 0 of the last warp, arms the stage's mbarrier with the byte count
//    and issues the copies.  A bulk copy holds its issuing thread for many
//    cycles, so the issuer is the warp with the least cell work (the order
//    puts the solid cells, and the cells of a second pass, on the first
//    warps);
//  - one pass over the row's links writes each bounced value f*_b(x) into the
//    staged slot that the pull of direction bbar at x reads (the slot of the
//    solid neighbour), so the cells pull without link logic;
//  - thread i takes the i-th cell of the row's order (the fluid cells first,
//    fixed by the geometry), so the collision runs on full warps; solid cells
//    only write zeros;
//  - f_a(x) is read from the ring at x - e_ax (periodic wrap in x is a
//    shared-memory index); results go into a shared-memory output row set
//    that leaves by one bulk store (the row's Q slots are contiguous);
//  - one pass over the row's links copies the outgoing values f*_b(x) from
//    the output rows into the row's contiguous range of the link buffer.
// Two block barriers per row; a stage is refilled after the first barrier of
// the row that follows its own.  Every wait on an mbarrier is bounded; one that
// runs out writes a code to p.status, the block stops issuing copies, and the
// kernel carries on (its results are then invalid, but it ends and no access
// leaves its buffers).
// ---------------------------------------------------------------------------

// Shared-memory layout of one stage: the Q source rows in slot order (row s
// at s rs, rs = nx, so that consecutive slots of one neighbouring row land
// with one copy), the row's cell order (lorder 16-bit entries), its range of
// the link buffer (gcap bytes) and of the link descriptors (dcap bytes), both
// as 16-byte aligned windows.
template <class L, class S>
struct StageLayout {
    int nx, rs, lorder, gcap, dcap;  // row length, shared-memory row stride (elements), order entries
    __device__ __forceinline__ int rows_bytes() const { return L::Q * rs * S::kBytes; }
    __device__ __forceinline__ int bytes() const { return rows_bytes() + 2 * lorder + gcap + dcap; }
    __device__ __forceinline__ typename S::T* rows(unsigned char* st) const {
        return reinterpret_cast<typename S::T*>(st);
    }
    __device__ __forceinline__ uint16_t* order(unsigned char* st) const {
        return reinterpret_cast<uint16_t*>(st + rows_bytes());
    }
    __device__ __forceinline__ typename S::T* links(unsigned char* st) const {
        return reinterpret_cast<typename S::T*>(st + rows_bytes() + 2 * lorder);
    }
    __device__ __forceinline__ uint32_t* descs(unsigned char* st) const {
        return reinterpret_cast<uint32_t*>(st + rows_bytes() + 2 * lorder + gcap);
    }
};

// One thread: arms a stage's mbarrier with the byte count of row `row`
// (links [g0, g1)), records the first elements of its two windows, and issues
// the row's copies into stage st, all completing on bar: per neighbouring row
// (y - e_ay, z - e_az) the block of slots of the directions with that
// (e_ay, e_az), the cell order, the link window and the descriptor window.  The window
// starts are written before the barrier is armed, so the arrive releases them
// to the waiting threads.
template <class L, class S>
__device__ __forceinline__ void stage_row(unsigned char* st, const StageLayout<L, S>& lay, uint64_t* bar,
                                          const typename S::T* __restrict__ Pin, int row, uint32_t g0, uint32_t g1,
                                          uint32_t* gstart, uint32_t* dstart, const KParams& p) {
    const uint32_t row_bytes = (uint32_t)p.nx * S::kBytes;
    uint64_t gb0, gb1, db0, db1;
    dev::window_bytes(g0, g1, S::kBytes, gb0, gb1);
    dev::window_bytes(g0, g1, 4, db0, db1);
    *gstart = (uint32_t)(gb0 / S::kBytes);
    *dstart = (uint32_t)(db0 / 4);
    dev::mbar_expect_tx(bar, L::Q * row_bytes + 2u * (uint32_t)lay.lorder + (uint32_t)(gb1 - gb0) +
                                 (uint32_t)(db1 - db0));
    const int y = row % p.ny, z = row / p.ny;
    const int yp = y == p.ny - 1 ? 0 : y + 1, ym = y == 0 ? p.ny - 1 : y - 1;
    const int zp = z == p.nz - 1 ? 0 : z + 1, zm = z == 0 ? p.nz - 1 : z - 1;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        if (key_count<L>(k) == 0) continue;
        // slots key_first(k) .. of source row (y - e_y, z - e_z), periodic
        const int ey = k / 3 - 1, ez = k % 3 - 1, s0 = key_first<L>(k);
        const int ys = ey > 0 ? ym : (ey < 0 ? yp : y);
        const int zs = ez > 0 ? zm : (ez < 0 ? zp : z);
        dev::bulk_load(lay.rows(st) + s0 * lay.rs, Pin + ((int64_t)(zs * p.ny + ys) * L::Q + s0) * p.nx,
                       (uint32_t)key_count<L>(k) * row_bytes, bar);
    }
    dev::bulk_load(lay.order(st), p.rorder + (int64_t)row * lay.lorder, 2u * (uint32_t)lay.lorder, bar);
    if (gb1 > gb0)
        dev::bulk_load(lay.links(st), reinterpret_cast<const unsigned char*>(Pin) + p.gofs + gb0,
                       (uint32_t)(gb1 - gb0), bar);
    if (db1 > db0)
        dev::bulk_load(lay.descs(st), reinterpret_cast<const unsigned char*>(p.ldesc) + db0, (uint32_t)(db1 - db0),
                       bar);
}

// FP32 storage with 256-cell rows writes each row's outputs over its own
// stage after a block barrier (one cell per thread, 256 threads) instead of
// into separate output rows: 46 instead of 66 KB of shared memory, four
// blocks per SM instead of three, 0.458 against 0.468 ms per 256^3 step.  The
// stage is refilled only after the row's bulk store has read it and every
// thread has passed its link copies (the first barrier of the next row).  For
// FP16 the extra barrier and the 256-thread blocks cost more than the freed
// memory gains (0.321 against 0.258 ms), so 16-bit storage keeps output rows.
template <class S, int RS, bool LMU>
constexpr bool kInPlaceOut = S::kBytes == 4 && RS == 256 && !LMU;

template <class L, class S, int FORCE, bool EF, bool SR, int STAGES, int RS, bool LMU = false>
__global__ void __launch_bounds__(256) k_step_rows(const typename S::T* __restrict__ Pin,
                                                   typename S::T* __restrict__ Pout, const float* __restrict__ Ef,
                                                   int gcap, int dcap, KParams p) {
    using T = typename S::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nx = p.nx;
    const int rs = RS ? RS : nx;  // shared-memory row stride (= nx): a constant for the common row lengths
    // FP32 rows of 256 cells write their outputs over the row's own stage
    // (no output rows: four blocks per SM instead of three); see kInPlaceOut
    constexpr bool kInPlace = kInPlaceOut<S, RS, LMU>;
    const StageLayout<L, S> lay{nx, rs, p.lorder, gcap, dcap};
    const int sbytes = lay.bytes();
    T* outrow = reinterpret_cast<T*>(smem_raw + STAGES * sbytes);
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ uint32_t gstart[STAGES], dstart[STAGES];
    T* Gout = reinterpret_cast<T*>(reinterpret_cast<char*>(Pout) + p.gofs);
    const uint32_t row_bytes = (uint32_t)nx * S::kBytes;
    const int R = p.ny * p.nz;
    const int G = gridDim.x;
    const bool leader = threadIdx.x == 0;
    const bool issuer = (int)threadIdx.x == (int)blockDim.x - 32;  // lane 0 of the last warp
    auto range = [&](int row, uint32_t& g0, uint32_t& g1) {
        g0 = g1 = 0u;
        if (row < R) {
            g0 = __ldg(p.rowG + row);
            g1 = __ldg(p.rowG + row + 1);
        }
    };
    if (leader) {
#pragma unroll
        for (int k = 0; k < STAGES; ++k) dev::mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (issuer) {
#pragma unroll
        for (int k = 0; k < STAGES - 1; ++k) {
            const int rk = blockIdx.x + k * G;
            if (rk < R) {
                uint32_t g0, g1;
                range(rk, g0, g1);
                stage_row<L, S>(smem_raw + k * sbytes, lay, &bar[k], Pin, rk, g0, g1, &gstart[k], &dstart[k], p);
            }
        }
    }
    int it = 0;
    bool ok = true;  // false once a wait has run out (the same in every thread after the first barrier)
    for (int r = blockIdx.x; r < R; r += G, ++it) {
        const int cs = it % STAGES;
        const int rn = r + (STAGES - 1) * G;       // the row refilled during this one ...
        const int sn = (it + STAGES - 1) % STAGES;  // ... into the stage of the previous row
        uint32_t g0, g1;  // this row's links
        range(r, g0, g1);
        if (ok && !dev::mbar_wait(&bar[cs], (uint32_t)(it / STAGES) & 1u)) {
            ok = false;
            if (p.status) atomicExch(p.status, 1);
            dev::pause_cycles(1ll << 22);  // let this block's copies in flight land
        }
        unsigned char* st = smem_raw + cs * sbytes;
        T* buf = lay.rows(st);
        T* orow = kInPlace ? buf : outrow;  // where this row's outputs go
        const uint16_t* ord = lay.order(st);
        const uint32_t* desc = lay.descs(st);
        const uint32_t d0 = dstart[cs];
        dev::patch_links<L, true>(buf, nx, rs, lay.links(st), gstart[cs], g0, g1, desc, d0);
        dev::bulk_wait_read();  // this thread's bulk stores of the previous row have read the output rows
        // bounced values in place, output rows free; a timeout anywhere in
        // the block stops the copies
        ok = __syncthreads_and(ok) != 0;
        if (issuer && ok && rn < R) {
            // refill the stage of the previous row: every thread is past its
            // last reads of it (the link pass that follows the output) and
            // its wait on that stage's barrier
            uint32_t n0, n1;
            range(rn, n0, n1);
            stage_row<L, S>(smem_raw + sn * sbytes, lay, &bar[sn], Pin, rn, n0, n1, &gstart[sn], &dstart[sn], p);
        }
        const int nf = ord[0];
        const uint32_t rowbase = (uint32_t)r * (uint32_t)nx;
        if constexpr (kInPlace) {
            // one cell per thread (the launcher sets blockDim.x = nx): every
            // pull first, then a barrier, then the outputs over the stage
            const int i = threadIdx.x;
            const int x = (int)ord[8 + i];
            const bool fluid = i < nf;
            const uint32_t cell = rowbase + (uint32_t)x;
            float h[L::Q];
            if (fluid) {
                const int xm = x == 0 ? nx - 1 : x - 1;
                const int xp = x == nx - 1 ? 0 : x + 1;
#pragma unroll
                for (int a = 0; a < L::Q; ++a) {
                    const int ex = L::c(a, 0);
                    h[a] = S::cvt(buf[pop_slot<L>(a) * rs + (ex > 0 ? xm : (ex < 0 ? xp : x))]);
                }
            }
            __syncthreads();  // no thread overwrites a slot another has still to pull
            if (fluid) {
                float E[3];
                load_E<L>(Ef, EF, p, cell, E);
                float out[L::Q];
                collide_any<L, S, FORCE, LMU>(h, E, p, out);
                typename S::T t[L::Q];
                round_all<L, S, SR>(out, cell, p, t);
#pragma unroll
                for (int a = 0; a < L::Q; ++a) orow[pop_slot<L>(a) * rs + x] = t[a];
            } else {
#pragma unroll
                for (int a = 0; a < L::Q; ++a) S::put(orow + a * rs + x, 0.f);
            }
        } else
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int x = (int)ord[8 + i];
            if (i < nf) {
                const uint32_t cell = rowbase + (uint32_t)x;
                const int xm = x == 0 ? nx - 1 : x - 1;
                const int xp = x == nx - 1 ? 0 : x + 1;
                float h[L::Q];
#pragma unroll
                for (int a = 0; a < L::Q; ++a) {
                    const int ex = L::c(a, 0);
                    h[a] = S::cvt(buf[pop_slot<L>(a) * rs + (ex > 0 ? xm : (ex < 0 ? xp : x))]);
                }
                float E[3];
                load_E<L>(Ef, EF, p, cell, E);
                if (S::kBytes == 4) {
                    // FP32 storage: compensated collision
                    float out[L::Q];
                    collide_any<L, S, FORCE, LMU>(h, E, p, out);
                    typename S::T t[L::Q];
                    round_all<L, S, SR>(out, cell, p, t);
#pragma unroll
                    for (int a = 0; a < L::Q; ++a) outrow[pop_slot<L>(a) * rs + x] = t[a];
                } else {
                    // 16-bit storage: each pair is rounded and stored as soon as it exists
                    Rng rng(cell, p);
                    collide_emit<L, FORCE, LMU>(
                        h, E, p,
                        [&](int a, float ha, float hb) {
                            T ta, tb;
                            if (SR) {
                                S::sr2(ha, hb, rng.pair(), ta, tb);
                            } else {
                                S::put(&ta, ha);
                                S::put(&tb, hb);
                            }
                            outrow[pop_slot<L>(a) * rs + x] = ta;
                            outrow[pop_slot<L>(a + 1) * rs + x] = tb;
                        },
                        [&](float rest) {
                            T t0, unused;
                            if (SR)
                                S::sr2(rest, rest, rng.pair(), t0, unused);
                            else
                                S::put(&t0, rest);
                            outrow[pop_slot<L>(0) * rs + x] = t0;
                        });
                }
            } else {
#pragma unroll
                for (int a = 0; a < L::Q; ++a) S::put(outrow + a * rs + x, 0.f);
            }
        }
        dev::fence_proxy_async();  // this thread's shared-memory writes before the bulk copies
        __syncthreads();           // output rows complete; the stage is free for its refill
        if (threadIdx.x == 0) {
            // the row's Q slots, one contiguous block
            dev::bulk_store(Pout + (int64_t)rowbase * L::Q, orow, L::Q * row_bytes);
            dev::bulk_commit();
        }
        // outgoing links: slot k of (x, b) takes f*_b(x)
        for (uint32_t k = g0 + threadIdx.x; k < g1; k += blockDim.x) {
            const uint32_t d = desc[k - d0];
            Gout[k] = orow[slot_of<L>((int)(d >> 24)) * rs + (int)(d & 0xFFFFFFu)];
        }
    }
    dev::bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Launch policy.  The row-staged kernel runs when a row of one direction is a
// multiple of 16 bytes and STAGES rows of all directions fit the shared-memory
// budget; otherwise the general kernel runs.  The persistent grid is the
// number of co-resident blocks (occupancy API) times the SM count, capped by
// the number of rows.
// ---------------------------------------------------------------------------
constexpr int kStages = 2;
constexpr int kRowThreads = 256;
constexpr size_t kSmemBudget = 160 * 1024;

// Block size and persistent grid of the row-staged kernel.  A block walks
// whole rows, so any multiple of 32 threads up to the row length works; the
// choice is the one with the most co-resident blocks per SM (occupancy API),
// the larger block on a tie: more rows in flight per SM hide the per-row
// copy latency.  256-cell FP16 rows: 192 threads (six blocks per SM) take
// 0.258 ms per 256^3 step, against 0.268 at 160, 0.277 at 224 and 0.278 at
// 256 threads.  fixed_threads != 0 takes that block size (the in-place FP32
// rows need one thread per cell).
struct Shape {
    int threads, blocks;
};
template <class K>
Shape launch_shape(K kernel, int nx, size_t smem, int fixed_threads = 0) {
    static std::mutex mu;
    static const void* last_k = nullptr;
    static size_t last_smem = 0;
    static int last_nx = 0;
    static Shape last{0, 0};
    std::lock_guard<std::mutex> lock(mu);
    if ((const void*)kernel != last_k || smem != last_smem || nx != last_nx) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int tmax = fixed_threads ? fixed_threads : (nx >= kRowThreads ? kRowThreads : ((nx + 31) / 32) * 32);
        const int tmin = fixed_threads ? fixed_threads : tmax / 2;
        Shape best{tmax, 0};
        int best_per_sm = -1;
        for (int t = tmax; t >= 32 && t >= tmin; t -= 32) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, t, smem);
            if (per_sm > best_per_sm) {
                best_per_sm = per_sm;
                best.threads = t;
            }
        }
        best.blocks = best_per_sm > 0 ? best_per_sm * sms : 0;
        last_k = (const void*)kernel;
        last_smem = smem;
        last_nx = nx;
        last = best;
    }
    return last;
}

template <class L, class S, int FORCE, bool EF, bool SR, int RS, bool LMU = false>
bool launch_rows(const S*, const void* fin, void* fout, const uint32_t* nbr, const float* Ef, const KParams& p,
                 cudaStream_t s) {
    using T = typename S::T;
    if (RS && RS != p.nx) return false;  // the stage rows are exactly nx long
    const int rs = p.nx;
    const size_t row_bytes = (size_t)p.nx * S::kBytes, srow = (size_t)rs * S::kBytes;
    const int gcap = dev::window_cap(p.max_row_links, S::kBytes);
    const int dcap = dev::window_cap(p.max_row_links, 4);
    const size_t stage_bytes = (size_t)L::Q * srow + 2 * (size_t)p.lorder + gcap + dcap;
    constexpr bool kInPlace = kInPlaceOut<S, RS, LMU>;
    const size_t smem = (size_t)kStages * stage_bytes + (kInPlace ? 0 : (size_t)L::Q * srow);
    if (!p.rorder || row_bytes % 16 != 0 || smem > kSmemBudget || p.nx < 32 || p.nx % 4 != 0) return false;
    auto kern = k_step_rows<L, S, FORCE, EF, SR, kStages, RS, LMU>;
    // one cell per thread in place: exactly nx (= 256) threads
    const Shape sh = launch_shape(kern, p.nx, smem, kInPlace ? p.nx : 0);
    const int threads = sh.threads, blocks = sh.blocks;
    if (blocks <= 0) return false;
    const int rows = p.ny * p.nz;
    kern<<<blocks < rows ? blocks : rows, threads, smem, s>>>((const T*)fin, (T*)fout, Ef, gcap, dcap, p);
    return true;
}

// Row-staged kernel when the rows qualify, with the shared-memory row stride
// (the row length) a compile-time constant for rows of 256 or 512 cells (the
// indexing then folds into immediate offsets); otherwise the general kernel.
template <class L, class S, int FORCE, bool EF, bool SR>
int launch_one(const void* fin, void* fout, const uint32_t* nbr, const float* Ef, const KParams& p, cudaStream_t s) {
    using T = typename S::T;
    const S* tag = nullptr;
    bool done;
    // the compile-time strides only for the benchmarked lattices (D2V9, D3V19);
    // the others take the run-time stride (fewer instantiations to compile)
    constexpr bool kFixed = L::Q == 9 || L::Q == 19;
    if (p.lmu_tab)  // the local-mu model (D2V9, D3V19 only): run-time row stride
        done = kFixed && launch_rows<L, S, FORCE, EF, SR, 0, kFixed>(tag, fin, fout, nbr, Ef, p, s);
    else if (kFixed && p.nx == 256)
        done = launch_rows<L, S, FORCE, EF, SR, kFixed ? 256 : 0>(tag, fin, fout, nbr, Ef, p, s);
    else if (kFixed && p.nx == 512)
        done = launch_rows<L, S, FORCE, EF, SR, kFixed ? 512 : 0>(tag, fin, fout, nbr, Ef, p, s);
    else
        done = launch_rows<L, S, FORCE, EF, SR, 0>(tag, fin, fout, nbr, Ef, p, s);
    if (done) return 1;
    const int bx = p.nx >= kBlock ? kBlock : ((p.nx + 31) / 32) * 32;
    const dim3 grid((unsigned)(p.ny * p.nz), (unsigned)((p.nx + bx - 1) / bx));
    k_step<L, S, FORCE, EF, SR><<<grid, bx, 0, s>>>((const T*)fin, (T*)fout, nbr, Ef, p);
    return 1;
}

template <class L, class S, bool SR>
int launch_lat(int force, bool efield, const void* fin, void* fout, const uint32_t* nbr, const float* Ef,
               const KParams& p, cudaStream_t s) {
    if (force == LBM_FORCE_SHIFT)
        return efield ? launch_one<L, S, 0, true, SR>(fin, fout, nbr, Ef, p, s)
                      : launch_one<L, S, 0, false, SR>(fin, fout, nbr, Ef, p, s);
    return efield ? launch_one<L, S, 1, true, SR>(fin, fout, nbr, Ef, p, s)
                  : launch_one<L, S, 1, false, SR>(fin, fout, nbr, Ef, p, s);
}

// GROUP 0: D2V9 and D3V19; GROUP 1: D3V27 and D1V3 (compiled in translation
// units of their own, so that the build runs them in parallel)
template <class S, bool HAS_SR, int GROUP>
int launch_storage(int vel, int force, bool efield, bool sr, const void* fin, void* fout, const uint32_t* nbr,
                   const float* Ef, const KParams& p, cudaStream_t s) {
    if constexpr (GROUP == 0) {
        if (HAS_SR && sr) {
            if (vel == LBM_D2V9) return launch_lat<LatD2V9, S, HAS_SR>(force, efield, fin, fout, nbr, Ef, p, s);
            return launch_lat<LatD3V19, S, HAS_SR>(force, efield, fin, fout, nbr, Ef, p, s);
        }
        if (vel == LBM_D2V9) return launch_lat<LatD2V9, S, false>(force, efield, fin, fout, nbr, Ef, p, s);
        return launch_lat<LatD3V19, S, false>(force, efield, fin, fout, nbr, Ef, p, s);
    } else {
        if (HAS_SR && sr) {
            if (vel == LBM_D1V3) return launch_lat<LatD1V3, S, HAS_SR>(force, efield, fin, fout, nbr, Ef, p, s);
            return launch_lat<LatD3V27, S, HAS_SR>(force, efield, fin, fout, nbr, Ef, p, s);
        }
        if (vel == LBM_D1V3) return launch_lat<LatD1V3, S, false>(force, efield, fin, fout, nbr, Ef, p, s);
        return launch_lat<LatD3V27, S, false>(force, efield, fin, fout, nbr, Ef, p, s);
    }
}

}  // namespace stepk
}  // namespace lbm
