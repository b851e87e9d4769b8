// Adjoint (reverse-mode) kernels of the fused semiclassical-LBM step
// (templates; included by one translation unit per storage type).
//
// Forward map per step: f_{t+1} = Stream(Collide(f_t)) (Sec. 9.1), with the
// collision of Sec. 9.1 and the forcing of Sec. 7.  For a loss
//   L = sum_{t in window} sum_x [w_rho(x) rho_t(x) + w_j(x) . j_t(x)]
// one reverse step maps lam_{t+1} = dL/df_{t+1} to lam_t = dL/df_t:
//   lamt_a(y) = lam_{t+1,a}(y + e_a)        (y + e_a fluid)
//             = lam_{t+1,abar}(y)           (y + e_a solid: transpose of bounce-back)
//   lam_t = (dCollide/df_t)^T lamt + [t in window] (w_rho + w_j . xi_a),
// and accumulates dL/dE(x), dL/dB, dL/dtau from lamt and f_t.  The collision
// Jacobian is applied through the chain rule over rho = sum f,
// j = sum f xi, u = j / rho; the formulas are the derivatives of the forward
// kernel's own expressions (direct N = 2 EDF of Sec. 5.1, forcing term of
// Sec. 7), so the reverse step is consistent with the FP32 forward.
//
// An adjoint field is lam[a * N + cell] (f-space, population layout) followed,
// at byte offset p.lgofs, by a link buffer: for every link of a fluid cell y
// into a solid cell (outgoing direction b) the slot of (y, b) in the forward's
// link numbering holds lam_bbar(y).  The bounced gather lamt_b(y) =
// lam_{t+1,bbar}(y) is then one contiguous range per row, as in the forward's
// pull.
//
// f_t is rebuilt by pulling the stored state of the forward replay.
// Parameter gradients: dL/dE(x) is accumulated per cell in FP32 partials
// that the driver folds into FP64 every few reverse steps; dL/dB,
// dL/dtau and the loss are block-reduced into per-block FP64 slots that each
// block owns (deterministic for a fixed launch shape).
#pragma once

#include <mutex>

#include "lbm_device.cuh"

namespace lbm {
namespace adjk {

using dev::Cell;
using dev::cross3;
using dev::edot;
using dev::kBlock;
using dev::warp_sum;
constexpr int kSlots = 5;         // gB[3], gtau, loss

// Adds the block's sums of acc[kSlots] into slots[block * kSlots + k].
__device__ __forceinline__ void block_accumulate(double* acc, double* __restrict__ slots, int64_t block) {
    __shared__ double sh[32][kSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) acc[k] = warp_sum(acc[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kSlots; ++k) sh[wid][k] = acc[k];
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) / 32;
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
            double v = lane < nw ? sh[lane][k] : 0.0;
            v = warp_sum(v);
            if (lane == 0) slots[block * kSlots + k] += v;
        }
    }
}

// Local chemical-potential model (KParams::lmu_*): dth = thetabar - thetabar_w
// and d dth / d rho at the unscaled density deviation drho, from the same
// cubic Hermite table as the forward step (node and fraction taken relative
// to the node r = 1; outside the table the end value, slope 0).
__device__ __forceinline__ void lmu_table(const KParams& p, float drho, float& dth, float& ddth) {
    const float a = p.lmu_a * p.scale;  // table units per unit of unscaled deviation
    float x = drho * a;
    const float lo = -p.lmu_b, hi = (float)(p.lmu_n - 1) - p.lmu_b;
    const bool inside = x > lo && x < hi;
    x = fminf(fmaxf(x, lo), hi);  // also maps NaN to node 0
    const float fl = floorf(x);
    int i = (int)fl + (int)p.lmu_b;
    float t = x - fl;
    if (i > p.lmu_n - 2) {
        i = p.lmu_n - 2;
        t = 1.f;
    }
    const float t2 = t * t, t3 = t2 * t;
    const float2 A = __ldg(p.lmu_tab + i), B = __ldg(p.lmu_tab + i + 1);
    dth = (2.f * t3 - 3.f * t2 + 1.f) * A.x + (t3 - 2.f * t2 + t) * A.y + (3.f * t2 - 2.f * t3) * B.x +
          (t3 - t2) * B.y;
    const float dx = (6.f * t2 - 6.f * t) * A.x + (3.f * t2 - 4.f * t + 1.f) * A.y + (6.f * t - 6.f * t2) * B.x +
                     (3.f * t2 - 2.f * t) * B.y;
    ddth = inside ? dx * a : 0.f;
}

template <class L, bool EF>
__device__ __forceinline__ void load_E(const float* __restrict__ Ef, const KParams& p, uint32_t cell, float* E) {
    if (EF) {
        E[0] = __ldg(Ef + cell);
        E[1] = (L::D >= 2) ? __ldg(Ef + p.N + cell) : 0.f;
        E[2] = (L::D == 3) ? __ldg(Ef + 2 * p.N + cell) : 0.f;
    } else {
        E[0] = p.E[0];
        E[1] = p.E[1];
        E[2] = p.E[2];
    }
}

template <class L, bool WIN>
__device__ __forceinline__ void load_weights(const float* __restrict__ w_rho, const float* __restrict__ w_j,
                                             const KParams& p, uint32_t cell, float& wr, float* wj) {
    wr = 0.f;
    wj[0] = wj[1] = wj[2] = 0.f;
    if (WIN) {
        wr = w_rho ? __ldg(w_rho + cell) : 0.f;
#pragma unroll
        for (int d = 0; d < L::D; ++d) wj[d] = w_j ? __ldg(w_j + (int64_t)d * p.N + cell) : 0.f;
    }
}


// The reverse step at one fluid cell.  h: unscaled deviations of f_t at the
// cell; lt: lamt; E: the field there; wr, wj: its loss weights (used when WIN).
// Writes lam = lam_t at the cell and gEc = its dL/dE term; adds
// {dL/dB, dL/dtau, loss} into acc[0..4].
//
// Every sum over directions that the chain rule needs is a moment of
// mu_a = lt_a w_a: with the forcing-free part F_a = rho w_a [A + Bp (e.v) +
// Cp (e.v)^2 + k2_a v^2] and the term S_a = rho w_a [Bp (e.E) + 2 Cp (e.u)(e.E)
// + 2 k2_a (u.E + u.(e x B)/c_s)] of the forward step,
//   sum lt F   = rho [A M0 + Bp M1.v + Cp v.M2.v + v^2 K0],
//   d/dv       = rho [Bp M1 + 2 Cp M2 v + 2 K0 v],
//   sum lt S   = rho [Bp M1.E + 2 Cp u.M2.E + 2 K0 u.E + 2 u.(K1 x B)/c_s],
// with M0 = sum mu, M1 = sum mu e, M2 = sum mu e e^T, K0 = sum mu k2,
// K1 = sum mu k2 e.  Since w_a and k2_a are constant on each shell (|e|^2 =
// 1, 2, 3: axes, face diagonals, corners), the per-direction work is only
// the unweighted shell moments of lt.
template <class L, int FORCE, bool WIN, bool LMU = false>
__device__ __forceinline__ void adjoint_cell(const float* h, const float* lt, const float* E, const KParams& p,
                                             float wr, const float* wj, float* lam, float* gEc, double* acc) {
    constexpr int kR1 = shell_first<L>(1), kR2 = shell_first<L>(2), kR3 = shell_first<L>(3);
    // forward moments of f_t
    float drho = 0.f, j[3] = {0.f, 0.f, 0.f}, lth = 0.f;
    float rho, inv_rho, u[3], M0, K0, M1[3], K1[3], Mxx, Myy, Mzz, Mxy, Mxz, Myz;
    if constexpr (kR1 > 0 && kR2 > 0 && kR3 < 0) {
        // two moving shells (D2V9, D3V19): axis and diagonal
        constexpr int kAx = kR1, kDg = kR2;
        // shell moments of lt: axis (1) and diagonal (2); the rest shell adds to M0 only
        float L0a = 0.f, L0d = 0.f, L1a[3] = {0.f, 0.f, 0.f}, L1d[3] = {0.f, 0.f, 0.f};
        float L2a[3] = {0.f, 0.f, 0.f};                     // axis shell: diagonal of sum lt e e^T
        float L2d[3] = {0.f, 0.f, 0.f}, L2o[3] = {0.f, 0.f, 0.f};  // diagonal shell: diagonal; (xy, xz, yz)
#pragma unroll
        for (int a = 0; a < L::Q; ++a) {
            const int ex = L::c(a, 0), ey = L::c(a, 1), ez = L::c(a, 2);
            drho += h[a];
            j[0] += ex * h[a];
            j[1] += ey * h[a];
            j[2] += ez * h[a];
            lth = fmaf(lt[a], h[a], lth);
            const int sh = esq_of<L>(a);
            if (sh == 1) {
                L0a += lt[a];
                if (ex) { L1a[0] += ex * lt[a]; L2a[0] += lt[a]; }
                if (ey) { L1a[1] += ey * lt[a]; L2a[1] += lt[a]; }
                if (ez) { L1a[2] += ez * lt[a]; L2a[2] += lt[a]; }
            } else if (sh == 2) {
                L0d += lt[a];
                if (ex) { L1d[0] += ex * lt[a]; L2d[0] += lt[a]; }
                if (ey) { L1d[1] += ey * lt[a]; L2d[1] += lt[a]; }
                if (ez) { L1d[2] += ez * lt[a]; L2d[2] += lt[a]; }
                if (ex * ey) L2o[0] += ex * ey * lt[a];
                if (ex * ez) L2o[1] += ex * ez * lt[a];
                if (ey * ez) L2o[2] += ey * ez * lt[a];
            }
        }
        j[0] *= p.cs_inv;
        j[1] *= p.cs_inv;
        j[2] = (L::D == 3) ? j[2] * p.cs_inv : 0.f;
        rho = p.rho0 + drho;
        inv_rho = 1.0f / rho;
        u[0] = j[0] * inv_rho;
        u[1] = j[1] * inv_rho;
        u[2] = j[2] * inv_rho;
        // weighted moments
        const float w0 = p.w[0], w1 = p.w[kAx], w2 = p.w[kDg];
        const float k1 = p.k2[kAx], k2d = p.k2[kDg];
        M0 = w0 * lt[0] + w1 * L0a + w2 * L0d;
        K0 = w0 * p.k2[0] * lt[0] + w1 * k1 * L0a + w2 * k2d * L0d;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            M1[d] = w1 * L1a[d] + w2 * L1d[d];
            K1[d] = w1 * k1 * L1a[d] + w2 * k2d * L1d[d];
        }
        // M2 = w1 diag(L2a) + w2 [L2d on the diagonal, L2o off it]
        Mxx = w1 * L2a[0] + w2 * L2d[0];
        Myy = w1 * L2a[1] + w2 * L2d[1];
        Mzz = w1 * L2a[2] + w2 * L2d[2];
        Mxy = w2 * L2o[0];
        Mxz = w2 * L2o[1];
        Myz = w2 * L2o[2];
    } else {
        // unweighted moments of lt per shell s = |e|^2: sum lt, sum lt e, the
        // diagonal of sum lt e e^T, and its (xy, xz, yz) entries; the rest
        // direction adds to M0 and K0 only
        float L0[4] = {0.f, 0.f, 0.f, 0.f}, L1[4][3] = {}, L2[4][3] = {}, L2o[4][3] = {};
#pragma unroll
        for (int a = 0; a < L::Q; ++a) {
            const int ex = L::c(a, 0), ey = L::c(a, 1), ez = L::c(a, 2);
            drho += h[a];
            j[0] += ex * h[a];
            j[1] += ey * h[a];
            j[2] += ez * h[a];
            lth = fmaf(lt[a], h[a], lth);
            const int sh = esq_of<L>(a);
            if (sh == 0) continue;
            L0[sh] += lt[a];
            if (ex) { L1[sh][0] += ex * lt[a]; L2[sh][0] += lt[a]; }
            if (ey) { L1[sh][1] += ey * lt[a]; L2[sh][1] += lt[a]; }
            if (ez) { L1[sh][2] += ez * lt[a]; L2[sh][2] += lt[a]; }
            if (ex * ey) L2o[sh][0] += ex * ey * lt[a];
            if (ex * ez) L2o[sh][1] += ex * ez * lt[a];
            if (ey * ez) L2o[sh][2] += ey * ez * lt[a];
        }
        j[0] *= p.cs_inv;
        j[1] *= p.cs_inv;
        j[2] = (L::D == 3) ? j[2] * p.cs_inv : 0.f;
        rho = p.rho0 + drho;
        inv_rho = 1.0f / rho;
        u[0] = j[0] * inv_rho;
        u[1] = j[1] * inv_rho;
        u[2] = j[2] * inv_rho;
        // weighted moments: shell s contributes with w_s and w_s k2_s
        M0 = p.w[0] * lt[0];
        K0 = p.w[0] * p.k2[0] * lt[0];
        M1[0] = M1[1] = M1[2] = 0.f;
        K1[0] = K1[1] = K1[2] = 0.f;
        Mxx = Myy = Mzz = Mxy = Mxz = Myz = 0.f;
#pragma unroll
        for (int sh = 1; sh <= 3; ++sh) {
            const int r = sh == 1 ? kR1 : (sh == 2 ? kR2 : kR3);
            if (r < 0) continue;
            const float ws = p.w[r], wk = p.w[r] * p.k2[r];
            M0 += ws * L0[sh];
            K0 += wk * L0[sh];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                M1[d] += ws * L1[sh][d];
                K1[d] += wk * L1[sh][d];
            }
            Mxx += ws * L2[sh][0];
            Myy += ws * L2[sh][1];
            Mzz += ws * L2[sh][2];
            Mxy += ws * L2o[sh][0];
            Mxz += ws * L2o[sh][1];
            Myz += ws * L2o[sh][2];
        }
    }
    auto m2v = [&](const float* v, float* out) {
        out[0] = Mxx * v[0] + Mxy * v[1] + Mxz * v[2];
        out[1] = Mxy * v[0] + Myy * v[1] + Myz * v[2];
        out[2] = Mxz * v[0] + Myz * v[1] + Mzz * v[2];
    };
    float acc_f[3], ue[3];
    if (FORCE == 0) {
        float uxb[3];
        cross3(u, p.B, uxb);
        acc_f[0] = E[0] + uxb[0];
        acc_f[1] = E[1] + uxb[1];
        acc_f[2] = (L::D == 3) ? E[2] + uxb[2] : 0.f;
        ue[0] = u[0] + p.tau * acc_f[0];
        ue[1] = u[1] + p.tau * acc_f[1];
        ue[2] = u[2] + p.tau * acc_f[2];
    } else {
        ue[0] = u[0];
        ue[1] = u[1];
        ue[2] = u[2];
    }
    const float u2 = ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2];
    float M2v[3];
    m2v(ue, M2v);
    const float M1v = M1[0] * ue[0] + M1[1] * ue[1] + M1[2] * ue[2];
    const float vM2v = M2v[0] * ue[0] + M2v[1] * ue[1] + M2v[2] * ue[2];
    const float inv_tau = p.omega;
    // sum_a lt_a F_a / rho and sum_a lt_a heq_a
    const float ltF = p.A * M0 + p.Bp * M1v + p.Cp * vM2v + u2 * K0;
    const float ltHeq = p.A * drho * M0 + rho * (p.Bp * M1v + p.Cp * vM2v + u2 * K0);
    float gtau = (lth - ltHeq) * inv_tau * inv_tau;
    // dF/dv summed against mu: rho [Bp M1 + 2 Cp M2 v + 2 K0 v]
    float dF[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) dF[d] = rho * (p.Bp * M1[d] + 2.f * p.Cp * M2v[d] + 2.f * K0 * ue[d]);
    float rho_bar, u_bar[3], gBc[3];
    if (FORCE == 0) {
        rho_bar = ltF * inv_tau;
        const float ue_bar[3] = {dF[0] * inv_tau, dF[1] * inv_tau, dF[2] * inv_tau};
        gtau += ue_bar[0] * acc_f[0] + ue_bar[1] * acc_f[1] + ue_bar[2] * acc_f[2];
        float t1[3], t2[3];
        cross3(ue_bar, u, t1);    // d(u x B)/dB transposed
        cross3(p.B, ue_bar, t2);  // d(u x B)/du transposed
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            gEc[d] = p.tau * ue_bar[d];
            gBc[d] = p.tau * t1[d];
            u_bar[d] = ue_bar[d] + p.tau * t2[d];
        }
    } else {
        float M2E[3], K1xB[3];
        m2v(E, M2E);
        cross3(K1, p.B, K1xB);
        const float uE = u[0] * E[0] + u[1] * E[1] + u[2] * E[2];
        const float ltS = p.Bp * (M1[0] * E[0] + M1[1] * E[1] + M1[2] * E[2]) +
                          2.f * p.Cp * (u[0] * M2E[0] + u[1] * M2E[1] + u[2] * M2E[2]) +
                          2.f * (K0 * uE + (u[0] * K1xB[0] + u[1] * K1xB[1] + u[2] * K1xB[2]) * p.cs_inv);
        rho_bar = ltF * inv_tau + ltS;
        // d(sum lt S)/du = rho [2 Cp M2 E + 2 K0 E + 2 (K1 x B)/c_s]; d/dE = dF; d/dB = (2 rho / c_s) u x K1
        float uxK[3];
        cross3(u, K1, uxK);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            u_bar[d] = dF[d] * inv_tau + rho * (2.f * p.Cp * M2E[d] + 2.f * (K0 * E[d] + K1xB[d] * p.cs_inv));
            gEc[d] = dF[d];
            gBc[d] = 2.f * rho * p.cs_inv * uxK[d];
        }
    }
    if constexpr (LMU && kR1 > 0 && kR2 > 0 && kR3 < 0) {
        // local-mu model (D2V9, D3V19): the collision adds w rho w_a K_a dth(rho),
        // whose rho-derivative feeds rho_bar and whose w-derivative dL/dtau.
        // K_a = K_0 + (K_1 - K_0) |e_a|^2 is affine in |e_a|^2, so
        // sum_a lt_a w_a K_a = K_0 M0 + (K_1 - K_0) trace(M2).
        {
            const float KM = p.lmu_K[0] * M0 + (p.lmu_K[1] - p.lmu_K[0]) * (Mxx + Myy + Mzz);
            float dth, ddth;
            lmu_table(p, drho, dth, ddth);
            rho_bar += inv_tau * (dth + rho * ddth) * KM;
            gtau -= inv_tau * inv_tau * rho * dth * KM;
        }
    }
    rho_bar -= (u_bar[0] * u[0] + u_bar[1] * u[1] + u_bar[2] * u[2]) * inv_rho;
    const float ub[3] = {u_bar[0] * inv_rho * p.cs_inv, u_bar[1] * inv_rho * p.cs_inv,
                         u_bar[2] * inv_rho * p.cs_inv};
    float wjs[3] = {0.f, 0.f, 0.f};
    if (WIN) {
#pragma unroll
        for (int d = 0; d < L::D; ++d) wjs[d] = wj[d] * p.cs_inv;
        acc[4] += (double)wr * (double)rho + (double)wj[0] * (double)j[0] + (double)wj[1] * (double)j[1] +
                  (double)wj[2] * (double)j[2];
    }
    const float omm = 1.0f - p.omega;
#pragma unroll
    for (int b = 0; b < L::Q; ++b) {
        float v = omm * lt[b] + rho_bar + edot<L>(b, ub);
        if (WIN) v += wr + edot<L>(b, wjs);
        lam[b] = v;
    }
    acc[0] += gBc[0];
    acc[1] += gBc[1];
    acc[2] += gBc[2];
    acc[3] += gtau;
}

// The link-buffer copies of a fluid cell's lam_t: slot (y, b) = lam_bbar(y)
// for every outgoing direction b into a solid cell.
template <class L>
__device__ __forceinline__ void store_lam_links(float* __restrict__ lamG, uint32_t o, uint32_t lb, const float* lam) {
#pragma unroll
    for (int b = 1; b < L::Q; ++b)
        if ((o >> b) & 1u) lamG[link_slot(lb, o, b)] = lam[opposite(b)];
}

__device__ __forceinline__ float* link_part(float* lam, const KParams& p) {
    return reinterpret_cast<float*>(reinterpret_cast<char*>(lam) + p.lgofs);
}
__device__ __forceinline__ const float* link_part(const float* lam, const KParams& p) {
    return reinterpret_cast<const float*>(reinterpret_cast<const char*>(lam) + p.lgofs);
}

// ---------------------------------------------------------------------------
// lam_T = dl_T/df_T (zero outside the window) and the loss term of step T.
// ---------------------------------------------------------------------------
template <class L, class S>
__global__ void __launch_bounds__(kBlock) k_adjoint_seed(const typename S::T* __restrict__ P,
                                                         const uint32_t* __restrict__ nbr,
                                                         const float* __restrict__ w_rho,
                                                         const float* __restrict__ w_j, float* __restrict__ lam,
                                                         double* __restrict__ slots, int in_window, KParams p) {
    Cell c;
    double acc[kSlots] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (dev::cell_of_thread(p, c)) {
        const uint32_t m = nbr[c.cell];
        if (m & kSolidBit) {
#pragma unroll
            for (int a = 0; a < L::Q; ++a) lam[dev::pop_at<L>(p, c, a, 0)] = 0.f;
        } else {
            float wr = 0.f, wj[3] = {0.f, 0.f, 0.f};
            if (in_window) {
                wr = w_rho ? w_rho[c.cell] : 0.f;
#pragma unroll
                for (int d = 0; d < L::D; ++d) wj[d] = w_j ? w_j[(int64_t)d * p.N + c.cell] * p.cs_inv : 0.f;
                // loss of step T: w_rho rho + w_j . j
                float h[L::Q];
                dev::pull<L, S>(P, p, m, c, h);
                float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
                for (int a = 0; a < L::Q; ++a) {
                    const float ha = h[a] * p.inv_scale;
                    drho += ha;
                    jx += L::c(a, 0) * ha;
                    jy += L::c(a, 1) * ha;
                    jz += L::c(a, 2) * ha;
                }
                acc[4] = (double)wr * (double)(p.rho0 + drho) + (double)wj[0] * jx + (double)wj[1] * jy +
                         (double)wj[2] * jz;
            }
            float lm[L::Q];
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                lm[a] = wr + edot<L>(a, wj);
                lam[dev::pop_at<L>(p, c, a, 0)] = lm[a];
            }
            const uint32_t o = outgoing<L::Q>(m);
            if (o) store_lam_links<L>(link_part(lam, p), o, __ldg(p.lbase + c.cell), lm);
        }
    }
    block_accumulate(acc, slots, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------------------
// One reverse step, general kernel: one thread per cell, direct global loads.
// ---------------------------------------------------------------------------
template <class L, class S, int FORCE, bool EF, bool WIN>
__global__ void __launch_bounds__(kBlock) k_adjoint_step(
    const typename S::T* __restrict__ P,  // stored state of the forward replay at step t
    const float* __restrict__ lam_in,     // lam_{t+1}
    float* __restrict__ lam_out,          // lam_t
    const uint32_t* __restrict__ nbr, const float* __restrict__ Ef, const float* __restrict__ w_rho,
    const float* __restrict__ w_j, float* __restrict__ gE, double* __restrict__ slots, KParams p) {
    Cell c;
    double acc[kSlots] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (dev::cell_of_thread(p, c)) {
        const uint32_t m = __ldg(nbr + c.cell);
        if (m & kSolidBit) {
#pragma unroll
            for (int a = 0; a < L::Q; ++a) lam_out[dev::pop_at<L>(p, c, a, 0)] = 0.f;
        } else {
            // f_t(y): pull of the stored state; lamt(y): gather from downstream
            float h[L::Q], lt[L::Q];
            dev::pull<L, S>(P, p, m, c, h);
            const uint32_t o = outgoing<L::Q>(m);
            const uint32_t lb = m ? __ldg(p.lbase + c.cell) : 0u;
            const float* lamG_in = link_part(lam_in, p);
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                h[a] *= p.inv_scale;
                if (a != 0 && ((o >> a) & 1u))
                    lt[a] = __ldg(lamG_in + link_slot(lb, o, a));
                else
                    lt[a] = __ldg(lam_in + dev::pop_at<L>(p, c, a, +1));
            }
            float E[3], wr, wj[3], lam[L::Q], gEc[3];
            load_E<L, EF>(Ef, p, c.cell, E);
            load_weights<L, WIN>(w_rho, w_j, p, c.cell, wr, wj);
            // the local-mu model is built for D2V9 and D3V19 (the host refuses others)
            constexpr bool kLmu = L::Q == 9 || L::Q == 19;
            if (kLmu && p.lmu_tab)
                adjoint_cell<L, FORCE, WIN, kLmu>(h, lt, E, p, wr, wj, lam, gEc, acc);
            else
                adjoint_cell<L, FORCE, WIN>(h, lt, E, p, wr, wj, lam, gEc, acc);
#pragma unroll
            for (int b = 0; b < L::Q; ++b) lam_out[dev::pop_at<L>(p, c, b, 0)] = lam[b];
            if (o) store_lam_links<L>(link_part(lam_out, p), o, lb, lam);
            if (gE) {
#pragma unroll
                for (int d = 0; d < L::D; ++d) gE[(int64_t)d * p.N + c.cell] += gEc[d];
            }
        }
    }
    block_accumulate(acc, slots, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------------------
// Row-staged reverse step (persistent; block b takes rows b, b + G, ...).
// One stage holds, for the row (y, z):
//   - with dL/dE, the row's D rows of its FP32 partials (accumulated in place
//     and stored back after the row); with a per-cell field, its D rows of E;
//   - the Q pull rows of the forward state P_t in slot order: direction a
//     from row (y - e_ay, z - e_az), read at x - e_ax (one copy per
//     neighbouring row: its block of consecutive slots);
//   - the row's cell order (fluid cells first, ascending x);
//   - its window of P_t's link buffer (bounced pulls);
//   - the Q gather rows of lam_{t+1} in slot order: direction a from row
//     (y + e_ay, z + e_az), read at x + e_ax (again one copy per row);
//   - its windows of lam_{t+1}'s link buffer (bounced gathers) and of the
//     link descriptors;
// all by bulk asynchronous copies, completing on the stage's mbarrier, armed
// and issued by lane 0 of the last warp (as in the forward's row-staged
// kernel; waits are bounded).  One pass over the
// row's links patches both bounced reads into the staged rows (the solid
// neighbour's slot, read by that cell alone), so cells read their rows
// without link logic.  Thread i takes the i-th cell of the row's order, so
// each thread's FP64 sums see the same cells in the same order on every run.
// lam_t goes through shared-memory output rows (zeros for solid cells) that
// leave by one bulk store (lam has the populations' slot layout), and one
// pass over the links copies lam_bbar(x) into the row's range of the new
// link buffer.  dL/dB, dL/dtau and the loss stay
// in registers until the block's single reduction at the end.
// ---------------------------------------------------------------------------
template <class L, class S>
struct AdjLayout {
    int nx, rs, lorder, gcapP, gcapL;  // row length, shared-memory row stride (elements), order entries;
                                       // gcapL also bounds the descriptor window (4-byte elements)
    int gerow, efrow;                  // bytes of the staged dL/dE rows and E rows (FP32), 0 when absent
    __device__ __host__ int prow() const { return L::Q * rs * S::kBytes; }
    __device__ __host__ int lrow() const { return L::Q * rs * 4; }
    __device__ __host__ int bytes() const {
        return gerow + prow() + 2 * lorder + gcapP + lrow() + 2 * gcapL + efrow;
    }
    __device__ unsigned char* gerows(unsigned char* st) const { return st; }
    __device__ unsigned char* prows(unsigned char* st) const { return st + gerow; }
    __device__ unsigned char* order(unsigned char* st) const { return st + gerow + prow(); }
    __device__ unsigned char* plinks(unsigned char* st) const { return order(st) + 2 * lorder; }
    __device__ unsigned char* lrows(unsigned char* st) const { return plinks(st) + gcapP; }
    __device__ unsigned char* llinks(unsigned char* st) const { return lrows(st) + lrow(); }
    __device__ unsigned char* descs(unsigned char* st) const { return llinks(st) + gcapL; }
    __device__ unsigned char* efrows(unsigned char* st) const { return descs(st) + gcapL; }
};

// One thread: arms a stage's mbarrier with the byte count of row `row`
// (links [g0, g1)), records where its windows start (ws[0]: P_t's link
// window; ws[1]: lam's link window and the descriptor window, which start at
// the same element), and issues the row's copies into stage st, all
// completing on bar.  With gE, the row's dL/dE (accumulated in place, stored
// back after the row); with Ef, its E.
template <class L, class S>
__device__ __forceinline__ void adj_stage(unsigned char* st, const AdjLayout<L, S>& lay, uint64_t* bar,
                                          const typename S::T* P, const float* lam, const float* gE, const float* Ef,
                                          int row, uint32_t g0, uint32_t g1, uint32_t* ws, const KParams& p) {
    const uint32_t prb = (uint32_t)p.nx * S::kBytes, lrb = (uint32_t)p.nx * 4u;
    const int rs = lay.rs;
    uint64_t pb0, pb1, lb0, lb1;
    dev::window_bytes(g0, g1, S::kBytes, pb0, pb1);
    dev::window_bytes(g0, g1, 4, lb0, lb1);
    ws[0] = (uint32_t)(pb0 / S::kBytes);
    ws[1] = (uint32_t)(lb0 / 4);
    dev::mbar_expect_tx(bar, L::Q * (prb + lrb) + 2u * (uint32_t)lay.lorder + (uint32_t)(pb1 - pb0) +
                                 2u * (uint32_t)(lb1 - lb0) + (lay.gerow ? L::D * (uint32_t)p.nx * 4u : 0u) +
                                 (lay.efrow ? L::D * (uint32_t)p.nx * 4u : 0u));
    const int y = row % p.ny, z = row / p.ny;
    const int yp = y == p.ny - 1 ? 0 : y + 1, ym = y == 0 ? p.ny - 1 : y - 1;
    const int zp = z == p.nz - 1 ? 0 : z + 1, zm = z == 0 ? p.nz - 1 : z - 1;
    unsigned char* pr = lay.prows(st);
    unsigned char* lr = lay.lrows(st);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        if (key_count<L>(k) == 0) continue;
        // the slots key_first(k) .. of the directions with (e_y, e_z): from pull
        // row (y - e_y, z - e_z) of P_t and gather row (y + e_y, z + e_z) of lam_{t+1}
        const int ey = k / 3 - 1, ez = k % 3 - 1, s0 = key_first<L>(k), n = key_count<L>(k);
        const int ysP = ey > 0 ? ym : (ey < 0 ? yp : y), zsP = ez > 0 ? zm : (ez < 0 ? zp : z);
        const int ysL = ey > 0 ? yp : (ey < 0 ? ym : y), zsL = ez > 0 ? zp : (ez < 0 ? zm : z);
        dev::bulk_load(pr + s0 * rs * S::kBytes, P + ((int64_t)(zsP * p.ny + ysP) * L::Q + s0) * p.nx,
                       (uint32_t)n * prb, bar);
        dev::bulk_load(lr + s0 * rs * 4, lam + ((int64_t)(zsL * p.ny + ysL) * L::Q + s0) * p.nx, (uint32_t)n * lrb,
                       bar);
    }
    dev::bulk_load(lay.order(st), p.rorder + (int64_t)row * lay.lorder, 2u * (uint32_t)lay.lorder, bar);
    if (pb1 > pb0)
        dev::bulk_load(lay.plinks(st), reinterpret_cast<const unsigned char*>(P) + p.gofs + pb0, (uint32_t)(pb1 - pb0),
                       bar);
    if (lb1 > lb0) {
        dev::bulk_load(lay.llinks(st), reinterpret_cast<const unsigned char*>(lam) + p.lgofs + lb0,
                       (uint32_t)(lb1 - lb0), bar);
        dev::bulk_load(lay.descs(st), reinterpret_cast<const unsigned char*>(p.ldesc) + lb0, (uint32_t)(lb1 - lb0),
                       bar);
    }
    if (lay.gerow) {
#pragma unroll
        for (int d = 0; d < L::D; ++d)
            dev::bulk_load(lay.gerows(st) + d * rs * 4, gE + (int64_t)d * p.N + (int64_t)row * p.nx,
                           (uint32_t)p.nx * 4u, bar);
    }
    if (lay.efrow) {
#pragma unroll
        for (int d = 0; d < L::D; ++d)
            dev::bulk_load(lay.efrows(st) + d * rs * 4, Ef + (int64_t)d * p.N + (int64_t)row * p.nx,
                           (uint32_t)p.nx * 4u, bar);
    }
}

template <class L, class S, int FORCE, bool EF, bool WIN, int STAGES, int RS, bool LMU = false>
__global__ void __launch_bounds__(256, 2) k_adjoint_rows(const typename S::T* __restrict__ P,
                                                         const float* __restrict__ lam_in,
                                                         float* __restrict__ lam_out,
                                                         const float* __restrict__ Ef,
                                                         const float* __restrict__ w_rho,
                                                         const float* __restrict__ w_j, float* __restrict__ gE,
                                                         double* __restrict__ slots, int gcapP, int gcapL, KParams p) {
    using T = typename S::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nx = p.nx;
    const int rs = RS ? RS : nx;  // shared-memory row stride (= nx): a constant for the common row lengths
    const AdjLayout<L, S> lay{nx, rs, p.lorder, gcapP, gcapL, gE ? L::D * rs * 4 : 0, EF ? L::D * rs * 4 : 0};
    const int sbytes = lay.bytes();
    float* outrow = reinterpret_cast<float*>(smem_raw + STAGES * sbytes);
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ uint32_t wstart[STAGES][2];
    float* lamG_out = link_part(lam_out, p);
    const int R = p.ny * p.nz;
    const int G = gridDim.x;
    const bool leader = threadIdx.x == 0;
    const int warp = (int)(threadIdx.x >> 5), nw = (int)(blockDim.x >> 5), lane = (int)(threadIdx.x & 31);
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
                adj_stage<L, S>(smem_raw + k * sbytes, lay, &bar[k], P, lam_in, gE, Ef, rk, g0, g1, wstart[k], p);
            }
        }
    }
    double acc[kSlots] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int it = 0;
    bool ok = true;  // false once a wait has run out (the same in every thread after the first barrier)
    for (int r = blockIdx.x; r < R; r += G, ++it) {
        const int cs = it % STAGES;
        const int rn = r + (STAGES - 1) * G;       // the row refilled during this one ...
        const int sn = (it + STAGES - 1) % STAGES;  // ... into the stage of the previous row
        uint32_t g0, g1;
        range(r, g0, g1);
        if (ok && !dev::mbar_wait(&bar[cs], (uint32_t)(it / STAGES) & 1u)) {
            ok = false;
            if (p.status) atomicExch(p.status, 2);
            dev::pause_cycles(1ll << 22);  // let this block's copies in flight land
        }
        unsigned char* st = smem_raw + cs * sbytes;
        T* prow = reinterpret_cast<T*>(lay.prows(st));
        float* ge_s = reinterpret_cast<float*>(lay.gerows(st));
        const float* ef_s = reinterpret_cast<const float*>(lay.efrows(st));
        float* lrow = reinterpret_cast<float*>(lay.lrows(st));
        const uint16_t* ord = reinterpret_cast<const uint16_t*>(lay.order(st));
        const uint32_t* desc = reinterpret_cast<const uint32_t*>(lay.descs(st));
        const uint32_t d0 = wstart[cs][1];
        dev::patch_links<L, true>(prow, nx, rs, reinterpret_cast<const T*>(lay.plinks(st)), wstart[cs][0], g0, g1,
                                  desc, d0);
        dev::patch_links<L, false>(lrow, nx, rs, reinterpret_cast<const float*>(lay.llinks(st)), d0, g0, g1, desc,
                                   d0);
        dev::bulk_wait_read();  // this thread's bulk stores of the previous row have read their sources
        // bounced values in place, output rows free; a timeout anywhere in
        // the block stops the copies
        ok = __syncthreads_and(ok) != 0;
        if (issuer && ok && rn < R) {
            // refill the stage of the previous row (every thread is past its
            // reads of it and its wait on that stage's barrier)
            uint32_t n0, n1;
            range(rn, n0, n1);
            adj_stage<L, S>(smem_raw + sn * sbytes, lay, &bar[sn], P, lam_in, gE, Ef, rn, n0, n1, wstart[sn], p);
        }
        const int nf = ord[0];
        const uint32_t rowbase = (uint32_t)r * (uint32_t)nx;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int x = (int)ord[8 + i];
            if (i < nf) {
                const uint32_t cell = rowbase + (uint32_t)x;
                const int xm = x == 0 ? nx - 1 : x - 1;
                const int xp = x == nx - 1 ? 0 : x + 1;
                float h[L::Q], lt[L::Q];
#pragma unroll
                for (int a = 0; a < L::Q; ++a) {
                    const int ex = L::c(a, 0);
                    h[a] = S::cvt(prow[pop_slot<L>(a) * rs + (ex > 0 ? xm : (ex < 0 ? xp : x))]) * p.inv_scale;
                    lt[a] = lrow[pop_slot<L>(a) * rs + (ex > 0 ? xp : (ex < 0 ? xm : x))];
                }
                float E[3], wr, wj[3], lam[L::Q], gEc[3];
                if (EF) {
                    E[0] = ef_s[x];
                    E[1] = ef_s[rs + x];
                    E[2] = (L::D == 3) ? ef_s[2 * rs + x] : 0.f;
                } else {
                    load_E<L, false>(Ef, p, cell, E);
                }
                load_weights<L, WIN>(w_rho, w_j, p, cell, wr, wj);
                adjoint_cell<L, FORCE, WIN, LMU>(h, lt, E, p, wr, wj, lam, gEc, acc);
#pragma unroll
                for (int b = 0; b < L::Q; ++b) outrow[pop_slot<L>(b) * rs + x] = lam[b];
                if (gE) {
#pragma unroll
                    for (int d = 0; d < L::D; ++d) ge_s[d * rs + x] += gEc[d];
                }
            } else {
#pragma unroll
                for (int b = 0; b < L::Q; ++b) outrow[b * rs + x] = 0.f;
            }
        }
        dev::fence_proxy_async();
        __syncthreads();  // output rows complete
        {
            // lane l of warp w takes piece w + l nw: the row's Q output slots
            // (one block), then its D updated dL/dE rows back from the stage
            // (which is refilled only after the issuing threads' reads are done)
            const int k = warp + lane * nw;
            if (k == 0) {
                dev::bulk_store(lam_out + (int64_t)rowbase * L::Q, outrow, (uint32_t)(L::Q * nx) * 4u);
                dev::bulk_commit();
            } else if (gE && k <= L::D) {
                const int d = k - 1;
                dev::bulk_store(gE + (int64_t)d * p.N + rowbase, ge_s + d * rs, (uint32_t)nx * 4u);
                dev::bulk_commit();
            }
        }
        // link copies of lam_t: slot k of (x, b) takes lam_bbar(x)
        for (uint32_t k = g0 + threadIdx.x; k < g1; k += blockDim.x) {
            const uint32_t d = desc[k - d0];
            lamG_out[k] = outrow[slot_of<L>(opposite((int)(d >> 24))) * rs + (int)(d & 0xFFFFFFu)];
        }
    }
    dev::bulk_wait_all();
    block_accumulate(acc, slots, blockIdx.x);
}

inline Launch grid_of(const KParams& p) {
    Launch l;
    const int bx = p.nx >= kBlock ? kBlock : ((p.nx + 31) / 32) * 32;
    l.block = dim3(bx);
    l.grid = dim3((unsigned)(p.ny * p.nz), (unsigned)((p.nx + bx - 1) / bx));
    return l;
}

// GROUP 0: D2V9 and D3V19; GROUP 1: D3V27 and D1V3 (separate translation units)
template <int GROUP, class F>
int dispatch_lattice(int vel, F&& f) {
    if constexpr (GROUP == 0 || GROUP == 2) {
        if (vel == LBM_D2V9) return f(LatD2V9{});
        return f(LatD3V19{});
    } else {
        if (vel == LBM_D1V3) return f(LatD1V3{});
        return f(LatD3V27{});
    }
}


// ---------------------------------------------------------------------------
// Launch policy of the reverse step: the row-staged kernel when a row of one
// direction of the state is a multiple of 16 bytes, nx >= 32, nx % 4 == 0 and
// the stages fit the shared-memory budget; otherwise the general kernel.
// ---------------------------------------------------------------------------
constexpr int kAdjStages = 2;
constexpr int kAdjThreads = 256;
constexpr size_t kAdjSmemBudget = 200 * 1024;

template <class L, class S, int FORCE, bool EF, bool WIN, int RS, bool LMU = false>
bool launch_rows_rs(const void* P, const float* lam_in, float* lam_out, const uint32_t* nbr, const float* Ef,
                 const float* w_rho, const float* w_j, float* gE, double* slots, int64_t slot_blocks,
                 const KParams& p, cudaStream_t s) {
    if (!p.rorder || (p.nx * S::kBytes) % 16 != 0 || p.nx % 4 != 0 || p.nx < 32) return false;
    if (reinterpret_cast<uintptr_t>(gE) % 16 != 0) return false;  // dL/dE rows move by bulk copies
    const int gcapP = dev::window_cap(p.max_row_links, S::kBytes);
    const int gcapL = dev::window_cap(p.max_row_links, 4);
    if (RS && RS != p.nx) return false;  // the stage rows are exactly nx long
    const int rs = p.nx;
    const size_t stage =
        (size_t)AdjLayout<L, S>{p.nx, rs, p.lorder, gcapP, gcapL, gE ? L::D * rs * 4 : 0, EF ? L::D * rs * 4 : 0}
            .bytes();
    const size_t smem = kAdjStages * stage + (size_t)L::Q * rs * 4;
    // the kernel choice and the persistent grid are taken for the layout with
    // dL/dE rows, whether or not this call has them, so that the blocks (and
    // with them the order of the FP64 gradient sums) are the same either way
    const size_t smem_ref =
        kAdjStages *
            (size_t)AdjLayout<L, S>{p.nx, rs, p.lorder, gcapP, gcapL, L::D * rs * 4, EF ? L::D * rs * 4 : 0}.bytes() +
        (size_t)L::Q * rs * 4;
    if (smem_ref > kAdjSmemBudget) return false;
    const int threads = p.nx >= kAdjThreads ? kAdjThreads : ((p.nx + 31) / 32) * 32;
    auto kern = k_adjoint_rows<L, S, FORCE, EF, WIN, kAdjStages, RS, LMU>;
    // persistent grid: co-resident blocks per SM (occupancy API) x SMs,
    // cached per instantiation and shared-memory size
    static std::mutex mu;
    static size_t last_smem = 0;
    static int last_threads = 0, last_blocks = 0;
    int blocks;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (smem_ref != last_smem || threads != last_threads) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (smem_ref > 48 * 1024)
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ref);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem_ref);
            last_smem = smem_ref;
            last_threads = threads;
            last_blocks = per_sm > 0 ? per_sm * sms : 0;
        }
        blocks = last_blocks;
    }
    const int rows = p.ny * p.nz;
    if (blocks > rows) blocks = rows;
    if (blocks <= 0 || blocks > slot_blocks) return false;
    kern<<<blocks, threads, smem, s>>>((const typename S::T*)P, lam_in, lam_out, Ef, w_rho, w_j, gE, slots,
                                       gcapP, gcapL, p);
    return true;
}

// The shared-memory row stride (the row length) is a compile-time constant
// for rows of 256 or 512 cells (as in the step kernel).
template <class L, class S, int FORCE, bool EF, bool WIN>
bool launch_rows(const void* P, const float* lam_in, float* lam_out, const uint32_t* nbr, const float* Ef,
                 const float* w_rho, const float* w_j, float* gE, double* slots, int64_t slot_blocks,
                 const KParams& p, cudaStream_t s) {
    // the compile-time strides only for the benchmarked lattices (D2V9, D3V19)
    constexpr bool kFixed = L::Q == 9 || L::Q == 19;
    if (kFixed && p.nx == 256)
        return launch_rows_rs<L, S, FORCE, EF, WIN, kFixed ? 256 : 0>(P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE,
                                                                       slots, slot_blocks, p, s);
    if (kFixed && p.nx == 512)
        return launch_rows_rs<L, S, FORCE, EF, WIN, kFixed ? 512 : 0>(P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE,
                                                                       slots, slot_blocks, p, s);
    return launch_rows_rs<L, S, FORCE, EF, WIN, 0>(P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE, slots, slot_blocks,
                                                    p, s);
}

// Launchers for one storage type (instantiated in one translation unit per
// storage).
template <class S, int GROUP>
int seed_storage(int vel, const void* P, const uint32_t* nbr, const float* w_rho, const float* w_j, float* lam,
                 double* slots, bool in_window, const KParams& p, cudaStream_t s) {
    Launch l = grid_of(p);
    return dispatch_lattice<GROUP>(vel, [&](auto lat) {
        using L = decltype(lat);
        k_adjoint_seed<L, S><<<l.grid, l.block, 0, s>>>((const typename S::T*)P, nbr, w_rho, w_j, lam, slots,
                                                       in_window ? 1 : 0, p);
        return 1;
    });
}

template <class S, int GROUP>
int step_storage(int vel, int force, bool efield, bool in_window, const void* P, const float* lam_in,
                 float* lam_out, const uint32_t* nbr, const float* Ef, const float* w_rho, const float* w_j,
                 float* gE, double* slots, const KParams& p, cudaStream_t s) {
    Launch l = grid_of(p);
    const int64_t slot_blocks = (int64_t)l.grid.x * l.grid.y;
    return dispatch_lattice<GROUP>(vel, [&](auto lat) {
        using L = decltype(lat);
        const auto* Pt = (const typename S::T*)P;
// GROUP 2: the local-mu model (D2V9, D3V19), whose staged reverse kernel is
// an instantiation of its own with the run-time row stride
#define LBM_ADJ(F, EFV, W)                                                                                    \
    do {                                                                                                      \
        bool staged;                                                                                          \
        if constexpr (GROUP == 2)                                                                             \
            staged = launch_rows_rs<L, S, F, EFV, W, 0, true>(P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE,    \
                                                              slots, slot_blocks, p, s);                      \
        else                                                                                                  \
            staged = launch_rows<L, S, F, EFV, W>(P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE, slots,         \
                                                  slot_blocks, p, s);                                         \
        if (!staged)                                                                                          \
            k_adjoint_step<L, S, F, EFV, W>                                                                   \
                <<<l.grid, l.block, 0, s>>>(Pt, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE, slots, p);          \
    } while (0)
        if (force == LBM_FORCE_SHIFT) {
            if (efield) {
                if (in_window) LBM_ADJ(0, true, true); else LBM_ADJ(0, true, false);
            } else {
                if (in_window) LBM_ADJ(0, false, true); else LBM_ADJ(0, false, false);
            }
        } else {
            if (efield) {
                if (in_window) LBM_ADJ(1, true, true); else LBM_ADJ(1, true, false);
            } else {
                if (in_window) LBM_ADJ(1, false, true); else LBM_ADJ(1, false, false);
            }
        }
#undef LBM_ADJ
        return 1;
    });
}

}  // namespace adjk
}  // namespace lbm
