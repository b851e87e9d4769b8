// Adjoint (reverse-mode) kernels of the fused semiclassical-LBM step.
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
// f_t is rebuilt by pulling the stored buffer P_t of the forward replay.
// Parameter gradients: dL/dE(x) is accumulated per cell in FP64; dL/dB,
// dL/dtau and the loss are block-reduced into per-block FP64 slots that each
// block owns (one read-modify-write per block per launch, deterministic).
#include "lbm_device.cuh"

namespace lbm {
namespace {

using dev::Cell;
using dev::cross3;
using dev::edot;
using dev::esq;
using dev::kBlock;
using dev::warp_sum;
constexpr int kSlots = 5;  // gB[3], gtau, loss

// Adds the block's sums of acc[kSlots] into slots[block * kSlots + k].
__device__ __forceinline__ void block_accumulate(double* acc, double* __restrict__ slots) {
    __shared__ double sh[kBlock / 32][kSlots];
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
        const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
            double v = lane < nw ? sh[lane][k] : 0.0;
            v = warp_sum(v);
            if (lane == 0) slots[b * kSlots + k] += v;
        }
    }
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
            for (int a = 0; a < L::Q; ++a) lam[(int64_t)a * p.N + c.cell] = 0.f;
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
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                const float g = wr + edot<L>(a, wj);
                lam[(int64_t)a * p.N + c.cell] = g;
            }
        }
    }
    block_accumulate(acc, slots);
}

// ---------------------------------------------------------------------------
// One reverse step.
// ---------------------------------------------------------------------------
template <class L, class S, int FORCE, bool EF, bool WIN>
__global__ void __launch_bounds__(kBlock) k_adjoint_step(
    const typename S::T* __restrict__ P,       // stored buffer of the forward replay at step t
    const float* __restrict__ lam_in,          // lam_{t+1}
    float* __restrict__ lam_out,               // lam_t
    const uint32_t* __restrict__ nbr, const float* __restrict__ Ef, const float* __restrict__ w_rho,
    const float* __restrict__ w_j, double* __restrict__ gE, double* __restrict__ slots, KParams p) {
    Cell c;
    double acc[kSlots] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (dev::cell_of_thread(p, c)) {
        const uint32_t m = __ldg(nbr + c.cell);
        if (m & kSolidBit) {
#pragma unroll
            for (int a = 0; a < L::Q; ++a) lam_out[(int64_t)a * p.N + c.cell] = 0.f;
        } else {
            // f_t(y): pull of the stored buffer; lamt(y): gather from downstream,
            // lamt_a(y) = lam_a(y + e_a), or lam_abar(y) when y + e_a is solid
            // (y + e_a = y - e_abar: bit abar of the link mask)
            float h[L::Q], lt[L::Q];
            dev::pull<L, S>(P, p, m, c, h);
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                h[a] *= p.inv_scale;
                int64_t lidx;
                if (a == 0)
                    lidx = c.cell;
                else
                    lidx = ((m >> opposite(a)) & 1u) ? (int64_t)opposite(a) * p.N + c.cell
                                                     : (int64_t)a * p.N + dev::shifted<L>(c, a, +1);
                lt[a] = __ldg(lam_in + lidx);
            }
            // forward quantities
            float drho = 0.f, j[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                drho += h[a];
                j[0] += L::c(a, 0) * h[a];
                j[1] += L::c(a, 1) * h[a];
                j[2] += L::c(a, 2) * h[a];
            }
            j[0] *= p.cs_inv;
            j[1] *= p.cs_inv;
            j[2] = (L::D == 3) ? j[2] * p.cs_inv : 0.f;
            const float rho = p.rho0 + drho;
            const float inv_rho = 1.0f / rho;
            const float u[3] = {j[0] * inv_rho, j[1] * inv_rho, j[2] * inv_rho};
            float E[3];
            if (EF) {
                E[0] = __ldg(Ef + c.cell);
                E[1] = __ldg(Ef + p.N + c.cell);
                E[2] = (L::D == 3) ? __ldg(Ef + 2 * p.N + c.cell) : 0.f;
            } else {
                E[0] = p.E[0];
                E[1] = p.E[1];
                E[2] = p.E[2];
            }
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
            const float Adr = p.A * drho;
            const float inv_tau = p.omega;

            float rho_bar = 0.f;
            float gtau = 0.f;
            // sums over a of lt_a w_a X for the vector derivatives
            float s_e[3] = {0.f, 0.f, 0.f};   // sum lt w e
            float s_eue[3] = {0.f, 0.f, 0.f}; // sum lt w (e.ue) e
            float s_k2 = 0.f;                 // sum lt w k2
            float s_eE_e[3] = {0.f, 0.f, 0.f};  // sum lt w (e.E) e        (term mode)
            float s_k2_e[3] = {0.f, 0.f, 0.f};  // sum lt w k2 e           (term mode)
            float s_k2_a[3] = {0.f, 0.f, 0.f};  // sum lt w k2 (e x B)/c_s (term mode)
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                const float eu = edot<L>(a, ue);
                const float k2 = p.k2[a];
                const float Fr = p.w[a] * (p.A + p.Bp * eu + p.Cp * eu * eu + k2 * u2);  // F_a / rho
                const float heq = p.w[a] * (Adr + rho * (p.Bp * eu + p.Cp * eu * eu + k2 * u2));
                const float lw = lt[a] * p.w[a];
                gtau += lt[a] * (h[a] - heq);
                s_k2 += lw * k2;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const int ed = L::c(a, d);
                    if (ed != 0) {
                        s_e[d] += ed * lw;
                        s_eue[d] += ed * lw * eu;
                    }
                }
                if (FORCE == 0) {
                    rho_bar += lt[a] * Fr * inv_tau;
                } else {
                    const float eE = edot<L>(a, E);
                    float exb[3] = {0.f, 0.f, 0.f};
                    const float e3[3] = {(float)L::c(a, 0), (float)L::c(a, 1), (float)L::c(a, 2)};  // e_a
                    cross3(e3, p.B, exb);
                    const float ua = u[0] * E[0] + u[1] * E[1] + u[2] * E[2] +
                                     (u[0] * exb[0] + u[1] * exb[1] + u[2] * exb[2]) * p.cs_inv;
                    const float Sr = p.w[a] * (p.Bp * eE + 2.f * p.Cp * eu * eE + 2.f * k2 * ua);  // S_a / rho
                    rho_bar += lt[a] * (Fr * inv_tau + Sr);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int ed = L::c(a, d);
                        if (ed != 0) {
                            s_eE_e[d] += ed * lw * eE;
                            s_k2_e[d] += ed * lw * k2;
                        }
                        s_k2_a[d] += lw * k2 * exb[d] * p.cs_inv;
                    }
                }
            }
            gtau *= inv_tau * inv_tau;
            // dF/dv summed against lt w: rho [Bp s_e + 2 Cp s_eue + 2 s_k2 v]
            float dF[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) dF[d] = rho * (p.Bp * s_e[d] + 2.f * p.Cp * s_eue[d] + 2.f * s_k2 * ue[d]);
            float u_bar[3];
            float gEc[3], gBc[3];
            if (FORCE == 0) {
                float ue_bar[3] = {dF[0] * inv_tau, dF[1] * inv_tau, dF[2] * inv_tau};
                gtau += ue_bar[0] * acc_f[0] + ue_bar[1] * acc_f[1] + ue_bar[2] * acc_f[2];
                float t1[3], t2[3];
                cross3(ue_bar, u, t1);      // d(u x B)/dB transposed
                cross3(p.B, ue_bar, t2);    // d(u x B)/du transposed
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    gEc[d] = p.tau * ue_bar[d];
                    gBc[d] = p.tau * t1[d];
                    u_bar[d] = ue_bar[d] + p.tau * t2[d];
                }
            } else {
                // S_a depends on u through (e.u)(e.E) and u.a_a, and on E, B through a_a
                float bxk[3];
                // sum_a lt_a dS_a/du = rho [2 Cp s_eE_e + 2 (s_k2 E + s_k2_a)]
                // sum_a lt_a dS_a/da summed over a = dF (at v = u) -> dL/dE
                // dL/dB = sum_a (abar_a x e_a)/c_s with abar_a = lt w rho [Bp e + 2Cp (e.u) e + 2 k2 u]
                //       = (2 rho / c_s) u x (sum lt w k2 e)
                cross3(u, s_k2_e, bxk);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    u_bar[d] = dF[d] * inv_tau + rho * (2.f * p.Cp * s_eE_e[d] + 2.f * (s_k2 * E[d] + s_k2_a[d]));
                    gEc[d] = dF[d];
                    gBc[d] = 2.f * rho * p.cs_inv * bxk[d];
                }
            }
            rho_bar -= (u_bar[0] * u[0] + u_bar[1] * u[1] + u_bar[2] * u[2]) * inv_rho;
            float ub[3] = {u_bar[0] * inv_rho * p.cs_inv, u_bar[1] * inv_rho * p.cs_inv,
                           u_bar[2] * inv_rho * p.cs_inv};
            float wr = 0.f, wj[3] = {0.f, 0.f, 0.f};
            if (WIN) {
                wr = w_rho ? __ldg(w_rho + c.cell) : 0.f;
#pragma unroll
                for (int d = 0; d < L::D; ++d) wj[d] = w_j ? __ldg(w_j + (int64_t)d * p.N + c.cell) * p.cs_inv : 0.f;
                acc[4] = (double)wr * (double)rho + (double)wj[0] * (double)j[0] / p.cs_inv +
                         (double)wj[1] * (double)j[1] / p.cs_inv + (double)wj[2] * (double)j[2] / p.cs_inv;
            }
            const float omm = 1.0f - p.omega;
#pragma unroll
            for (int b = 0; b < L::Q; ++b) {
                float v = omm * lt[b] + rho_bar + edot<L>(b, ub);
                if (WIN) v += wr + edot<L>(b, wj);
                lam_out[(int64_t)b * p.N + c.cell] = v;
            }
            if (gE) {
#pragma unroll
                for (int d = 0; d < L::D; ++d) gE[(int64_t)d * p.N + c.cell] += (double)gEc[d];
            }
            acc[0] = gBc[0];
            acc[1] = gBc[1];
            acc[2] = gBc[2];
            acc[3] = gtau;
        }
    }
    block_accumulate(acc, slots);
}

Launch grid_of(const KParams& p) {
    Launch l;
    const int bx = p.nx >= kBlock ? kBlock : ((p.nx + 31) / 32) * 32;
    l.block = dim3(bx);
    l.grid = dim3((unsigned)(p.ny * p.nz), (unsigned)((p.nx + bx - 1) / bx));
    return l;
}

template <class F>
int dispatch_lattice(int vel, F&& f) {
    if (vel == LBM_D2V9) return f(LatD2V9{});
    return f(LatD3V19{});
}

template <class F>
int dispatch_storage(int storage, F&& f) {
    if (storage == LBM_F16_DEV) return f(StoreF16{});
    if (storage == LBM_BF16_DEV) return f(StoreBF16{});
    return f(StoreF32{});
}

}  // namespace

int64_t adjoint_slot_count(const KParams& p) {
    Launch l = grid_of(p);
    return (int64_t)l.grid.x * l.grid.y * kSlots;
}

int launch_adjoint_seed(int vel, int storage, const void* P, const uint32_t* nbr, const float* w_rho,
                        const float* w_j, float* lam, double* slots, bool in_window, const KParams& p,
                        cudaStream_t s) {
    Launch l = grid_of(p);
    return dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        return dispatch_storage(storage, [&](auto st) {
            using S = decltype(st);
            k_adjoint_seed<L, S><<<l.grid, l.block, 0, s>>>((const typename S::T*)P, nbr, w_rho, w_j, lam, slots,
                                                           in_window ? 1 : 0, p);
            return 1;
        });
    });
}

int launch_adjoint_step(int vel, int storage, int force, bool efield, bool in_window, const void* P,
                        const float* lam_in, float* lam_out, const uint32_t* nbr, const float* Ef,
                        const float* w_rho, const float* w_j, double* gE, double* slots, const KParams& p,
                        cudaStream_t s) {
    Launch l = grid_of(p);
    return dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        return dispatch_storage(storage, [&](auto st) {
            using S = decltype(st);
            const auto* Pt = (const typename S::T*)P;
#define LBM_ADJ(F, EFV, W) \
    k_adjoint_step<L, S, F, EFV, W><<<l.grid, l.block, 0, s>>>(Pt, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE, slots, p)
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
    });
}

}  // namespace lbm
