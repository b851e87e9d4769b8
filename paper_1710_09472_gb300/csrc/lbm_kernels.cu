// Device kernels of the semiclassical LBM step (Sec. 9.1 of arXiv 1710.09472):
// neighbour bitmask, equilibrium start state, the fused pull-stream + BGK
// collision + Lorentz forcing step, moments with FP64 reductions, and the
// population read-back.
//
// Layout: populations are structure-of-arrays, pop[a * N + cell] with
// cell = (z * ny + y) * nx + x.  The buffer holds the post-collision values of
// the previous step ("pull" scheme): the state f(x, t) of the method is
//   f_a(x, t) = P_a(x - e_a)   if x - e_a is fluid,
//             = P_abar(x)      otherwise (halfway bounce-back, Sec. 9.3-9.4),
// so one kernel per step reads f(x, t), collides it and writes P for t + 1.
//
// Every kernel is a plain grid over cells: blockIdx.x is the row (y, z),
// blockIdx.y the chunk of x, threads run along x for coalesced access.
#include <cstdio>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kBlock = 128;

struct Cell {
    int x, y, z;
    int64_t cell;
};

__device__ __forceinline__ bool cell_of_thread(const KParams& p, Cell& c) {
    c.x = blockIdx.y * blockDim.x + threadIdx.x;
    if (c.x >= p.nx) return false;
    const int row = blockIdx.x;
    c.y = row % p.ny;
    c.z = row / p.ny;
    c.cell = (int64_t)row * p.nx + c.x;
    return true;
}

// Index of x + s * e_a with periodic wrap (s = +1 or -1).
template <class L>
__device__ __forceinline__ int64_t shifted(const KParams& p, const Cell& c, int a, int s) {
    const int ex = s * L::c(a, 0), ey = s * L::c(a, 1), ez = s * L::c(a, 2);
    int xs = c.x, ys = c.y, zs = c.z;
    if (ex > 0) xs = (c.x == p.nx - 1) ? 0 : c.x + 1;
    if (ex < 0) xs = (c.x == 0) ? p.nx - 1 : c.x - 1;
    if (ey > 0) ys = (c.y == p.ny - 1) ? 0 : c.y + 1;
    if (ey < 0) ys = (c.y == 0) ? p.ny - 1 : c.y - 1;
    if (ez > 0) zs = (c.z == p.nz - 1) ? 0 : c.z + 1;
    if (ez < 0) zs = (c.z == 0) ? p.nz - 1 : c.z - 1;
    return ((int64_t)zs * p.ny + ys) * p.nx + xs;
}

// Pull the deviations h_a(x, t) of one fluid cell (stream + bounce-back).
template <class L, class S>
__device__ __forceinline__ void pull(const typename S::T* __restrict__ P, uint32_t m, const KParams& p,
                                     const Cell& c, float* h) {
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        int64_t idx;
        if (a == 0) {
            idx = c.cell;
        } else if ((m >> a) & 1u) {
            idx = (int64_t)opposite(a) * p.N + c.cell;
        } else {
            idx = (int64_t)a * p.N + shifted<L>(p, c, a, -1);
        }
        h[a] = S::load(P, idx, p.inv_scale);
    }
}

// Moments of the deviations: drho = sum h_a, j = sum h_a e_a / c_s (xi units).
template <class L>
__device__ __forceinline__ void moments_of(const float* h, const KParams& p, float& drho, float* j) {
    float s = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        s += h[a];
        if (L::c(a, 0) > 0) jx += h[a];
        if (L::c(a, 0) < 0) jx -= h[a];
        if (L::c(a, 1) > 0) jy += h[a];
        if (L::c(a, 1) < 0) jy -= h[a];
        if (L::c(a, 2) > 0) jz += h[a];
        if (L::c(a, 2) < 0) jz -= h[a];
    }
    drho = s;
    j[0] = jx * p.cs_inv;
    j[1] = jy * p.cs_inv;
    j[2] = (L::D == 3) ? jz * p.cs_inv : 0.f;
}

template <class L>
__device__ __forceinline__ float edot(int a, const float* v) {
    float r = 0.f;
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

template <class L>
__device__ __forceinline__ constexpr int esq(int a) {
    return L::c(a, 0) * L::c(a, 0) + L::c(a, 1) * L::c(a, 1) + L::c(a, 2) * L::c(a, 2);
}

// ---------------------------------------------------------------------------
// Neighbour bitmask: bit a set when x - e_a is solid; kSolidBit when x is.
// ---------------------------------------------------------------------------
template <class L>
__global__ void __launch_bounds__(kBlock) k_neighbors(const uint8_t* __restrict__ mask, uint32_t* __restrict__ nbr,
                                                      unsigned long long* __restrict__ fluid_count, KParams p) {
    Cell c;
    unsigned fluid = 0;
    if (cell_of_thread(p, c)) {
        uint32_t m = 0;
        if (mask[c.cell]) {
            m = kSolidBit;
        } else {
            fluid = 1;
#pragma unroll
            for (int a = 1; a < L::Q; ++a)
                if (mask[shifted<L>(p, c, a, -1)]) m |= (1u << a);
        }
        nbr[c.cell] = m;
    }
    // one atomic per warp
    const unsigned cnt = __popc(__ballot_sync(0xffffffffu, fluid));
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(fluid_count, (unsigned long long)cnt);
}

// ---------------------------------------------------------------------------
// Start state: P such that pulling it gives f^eq(rho(x), u(x)):
//   P_b(y) = f^eq_b(y + e_b) if y + e_b is fluid, else f^eq_bbar(y).
// ---------------------------------------------------------------------------
template <class L>
__device__ __forceinline__ float heq_at(const KParams& p, int a, float rho, const float* u) {
    // f^eq_a - f0_a = w_a [A (rho - rho0) + rho (Bp eu + Cp eu^2 + (Gp e^2 + H) u^2)]
    const float eu = edot<L>(a, u);
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return p.w[a] * (p.A * (rho - p.rho0) + rho * (p.Bp * eu + p.Cp * eu * eu + (p.Gp * esq<L>(a) + p.H) * u2));
}

template <class L, class S>
__global__ void __launch_bounds__(kBlock) k_init(typename S::T* __restrict__ P, const uint32_t* __restrict__ nbr,
                                                 const float* __restrict__ rho, const float* __restrict__ u,
                                                 KParams p) {
    Cell c;
    if (!cell_of_thread(p, c)) return;
    const uint32_t m = nbr[c.cell];
    if (m & kSolidBit) {
#pragma unroll
        for (int a = 0; a < L::Q; ++a) S::store(P, (int64_t)a * p.N + c.cell, 0.f, p.scale);
        return;
    }
    auto fields = [&](int64_t cell, float& r, float* uu) {
        r = rho ? rho[cell] : p.rho0;
        uu[0] = u ? u[cell] : 0.f;
        uu[1] = u ? u[p.N + cell] : 0.f;
        uu[2] = (u && L::D == 3) ? u[2 * p.N + cell] : 0.f;
    };
    float r0, u0[3];
    fields(c.cell, r0, u0);
#pragma unroll
    for (int b = 0; b < L::Q; ++b) {
        float v;
        if (b != 0 && ((m >> opposite(b)) & 1u)) {
            v = heq_at<L>(p, opposite(b), r0, u0);
        } else if (b == 0) {
            v = heq_at<L>(p, 0, r0, u0);
        } else {
            float r1, u1[3];
            fields(shifted<L>(p, c, b, +1), r1, u1);
            v = heq_at<L>(p, b, r1, u1);
        }
        S::store(P, (int64_t)b * p.N + c.cell, v, p.scale);
    }
}

// ---------------------------------------------------------------------------
// The fused step.  f(x, t) is pulled, its moments taken, the force applied,
// f^eq formed and the BGK relaxation written back (Sec. 9.1):
//   h*_a = (1 - 1/tau) h_a + heq_a / tau + S_a,
// where h = f - f0 are deviations from the rest equilibrium at rho0.
// FORCE 0: velocity shift u* = u + tau (E + u x B) (Sec. 7, Eq.
//          u-update-force-term-eq); S = 0.
// FORCE 1: S_a = a_a . grad_u f^eq_a with a_a = E + xi_a x B (Sec. 7, Eq.
//          forcing-term-integrals-eq):
//          S_a = rho w_a [Bp e.E + 2 Cp (e.u)(e.E) + 2 (Gp e^2 + H)(u.E + e.(B x u)/c_s)].
// ---------------------------------------------------------------------------
template <class L, class S, int FORCE, bool EF>
__global__ void __launch_bounds__(kBlock) k_step(const typename S::T* __restrict__ Pin, typename S::T* __restrict__ Pout,
                                                 const uint32_t* __restrict__ nbr, const float* __restrict__ Ef,
                                                 KParams p) {
    Cell c;
    if (!cell_of_thread(p, c)) return;
    const uint32_t m = __ldg(nbr + c.cell);
    if (m & kSolidBit) return;

    float h[L::Q];
    pull<L, S>(Pin, m, p, c, h);

    float drho, j[3];
    moments_of<L>(h, p, drho, j);
    const float rho = p.rho0 + drho;
    const float inv_rho = 1.0f / rho;
    float u[3] = {j[0] * inv_rho, j[1] * inv_rho, j[2] * inv_rho};

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

    float ue[3];
    if (FORCE == 0) {
        // a = E + u x B
        const float ax = E[0] + (u[1] * p.B[2] - u[2] * p.B[1]);
        const float ay = E[1] + (u[2] * p.B[0] - u[0] * p.B[2]);
        const float az = E[2] + (u[0] * p.B[1] - u[1] * p.B[0]);
        ue[0] = u[0] + p.tau * ax;
        ue[1] = u[1] + p.tau * ay;
        ue[2] = (L::D == 3) ? u[2] + p.tau * az : 0.f;
    } else {
        ue[0] = u[0];
        ue[1] = u[1];
        ue[2] = u[2];
    }
    const float u2 = ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2];
    const float Adr = p.A * drho;
    const float one_m_omega = 1.0f - p.omega;

    // force-term helpers (FORCE 1)
    float uE = 0.f, bu[3] = {0.f, 0.f, 0.f};
    if (FORCE == 1) {
        uE = u[0] * E[0] + u[1] * E[1] + u[2] * E[2];
        bu[0] = (p.B[1] * u[2] - p.B[2] * u[1]) * p.cs_inv;
        bu[1] = (p.B[2] * u[0] - p.B[0] * u[2]) * p.cs_inv;
        bu[2] = (p.B[0] * u[1] - p.B[1] * u[0]) * p.cs_inv;
    }

#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        const float eu = edot<L>(a, ue);
        const float k2 = p.Gp * (float)esq<L>(a) + p.H;
        const float heq = p.w[a] * (Adr + rho * (p.Bp * eu + p.Cp * eu * eu + k2 * u2));
        float hs = one_m_omega * h[a] + p.omega * heq;
        if (FORCE == 1) {
            const float eE = edot<L>(a, E);
            const float ua = uE + edot<L>(a, bu);
            hs += rho * p.w[a] * (p.Bp * eE + 2.f * p.Cp * eu * eE + 2.f * k2 * ua);
        }
        S::store(Pout, (int64_t)a * p.N + c.cell, hs, p.scale);
    }
}

// ---------------------------------------------------------------------------
// Moments of f(x, t) and FP64 block partials of the fluid totals.
// partials[block] = {sum rho, sum j_x, sum j_y, sum j_z} (warp shuffles, then
// one warp over the block's warps).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <class L, class S>
__global__ void __launch_bounds__(kBlock) k_moments(const typename S::T* __restrict__ P, const uint32_t* __restrict__ nbr,
                                                    float* __restrict__ rho_out, float* __restrict__ j_out,
                                                    double* __restrict__ partials, KParams p) {
    Cell c;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (cell_of_thread(p, c)) {
        const uint32_t m = nbr[c.cell];
        float r = 0.f, j[3] = {0.f, 0.f, 0.f};
        if (!(m & kSolidBit)) {
            float h[L::Q];
            pull<L, S>(P, m, p, c, h);
            float drho;
            moments_of<L>(h, p, drho, j);
            r = p.rho0 + drho;
            acc[0] = (double)r;
            acc[1] = (double)j[0];
            acc[2] = (double)j[1];
            acc[3] = (double)j[2];
        }
        if (rho_out) rho_out[c.cell] = r;
        if (j_out) {
#pragma unroll
            for (int d = 0; d < L::D; ++d) j_out[(int64_t)d * p.N + c.cell] = j[d];
        }
    }
    if (partials) {
        __shared__ double sh[kBlock / 32][4];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = warp_sum(acc[k]);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) sh[wid][k] = acc[k];
        }
        __syncthreads();
        if (wid == 0) {
            const int nw = (blockDim.x + 31) / 32;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                double v = lane < nw ? sh[lane][k] : 0.0;
                v = warp_sum(v);
                if (lane == 0) partials[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + k] = v;
            }
        }
    }
}

// One block sums the partials in a fixed order (deterministic).
constexpr int kReduceThreads = 512;
__global__ void __launch_bounds__(kReduceThreads) k_reduce_partials(const double* __restrict__ partials, int64_t n,
                                                                     double* __restrict__ out4) {
    __shared__ double sh[kReduceThreads / 32][4];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += partials[i * 4 + k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = warp_sum(acc[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[wid][k] = acc[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double v = lane < (int)(blockDim.x / 32) ? sh[lane][k] : 0.0;
            v = warp_sum(v);
            if (lane == 0) out4[k] = v;
        }
    }
}

// Full FP32 populations f_a(x, t) = f0_a + h_a.
template <class L, class S>
__global__ void __launch_bounds__(kBlock) k_populations(const typename S::T* __restrict__ P,
                                                        const uint32_t* __restrict__ nbr, float* __restrict__ f,
                                                        bool deviation, KParams p) {
    Cell c;
    if (!cell_of_thread(p, c)) return;
    const uint32_t m = nbr[c.cell];
    if (m & kSolidBit) {
#pragma unroll
        for (int a = 0; a < L::Q; ++a) f[(int64_t)a * p.N + c.cell] = 0.f;
        return;
    }
    float h[L::Q];
    pull<L, S>(P, m, p, c, h);
#pragma unroll
    for (int a = 0; a < L::Q; ++a) f[(int64_t)a * p.N + c.cell] = deviation ? h[a] : p.f0[a] + h[a];
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

int64_t moments_partial_count(const KParams& p) {
    Launch l = grid_of(p);
    return (int64_t)l.grid.x * l.grid.y;
}

int launch_build_neighbors(int vel, const uint8_t* mask, uint32_t* nbr, unsigned long long* fluid_count,
                           const KParams& p, cudaStream_t s) {
    Launch l = grid_of(p);
    return dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        k_neighbors<L><<<l.grid, l.block, 0, s>>>(mask, nbr, fluid_count, p);
        return 1;
    });
}

int launch_init(int vel, int storage, void* pop, const uint32_t* nbr, const float* rho, const float* u,
                const KParams& p, cudaStream_t s) {
    Launch l = grid_of(p);
    return dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        return dispatch_storage(storage, [&](auto st) {
            using S = decltype(st);
            k_init<L, S><<<l.grid, l.block, 0, s>>>((typename S::T*)pop, nbr, rho, u, p);
            return 1;
        });
    });
}

int launch_step(int vel, int storage, int force, bool efield, const void* fin, void* fout, const uint32_t* nbr,
                const float* Ef, const KParams& p, cudaStream_t s) {
    Launch l = grid_of(p);
    return dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        return dispatch_storage(storage, [&](auto st) {
            using S = decltype(st);
            using T = typename S::T;
            const T* in = (const T*)fin;
            T* out = (T*)fout;
            if (force == LBM_FORCE_SHIFT) {
                if (efield)
                    k_step<L, S, 0, true><<<l.grid, l.block, 0, s>>>(in, out, nbr, Ef, p);
                else
                    k_step<L, S, 0, false><<<l.grid, l.block, 0, s>>>(in, out, nbr, Ef, p);
            } else {
                if (efield)
                    k_step<L, S, 1, true><<<l.grid, l.block, 0, s>>>(in, out, nbr, Ef, p);
                else
                    k_step<L, S, 1, false><<<l.grid, l.block, 0, s>>>(in, out, nbr, Ef, p);
            }
            return 1;
        });
    });
}

int launch_moments(int vel, int storage, const void* pop, const uint32_t* nbr, float* rho, float* j,
                   double* partials, int64_t* n_partials, const KParams& p, cudaStream_t s) {
    Launch l = grid_of(p);
    if (n_partials) *n_partials = (int64_t)l.grid.x * l.grid.y;
    return dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        return dispatch_storage(storage, [&](auto st) {
            using S = decltype(st);
            k_moments<L, S><<<l.grid, l.block, 0, s>>>((const typename S::T*)pop, nbr, rho, j, partials, p);
            return 1;
        });
    });
}

int launch_reduce_partials(const double* partials, int64_t n_partials, double* out4, cudaStream_t s) {
    k_reduce_partials<<<1, kReduceThreads, 0, s>>>(partials, n_partials, out4);
    return 1;
}

int launch_populations(int vel, int storage, const void* pop, const uint32_t* nbr, float* f, bool deviation,
                       const KParams& p, cudaStream_t s) {
    Launch l = grid_of(p);
    return dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        return dispatch_storage(storage, [&](auto st) {
            using S = decltype(st);
            k_populations<L, S><<<l.grid, l.block, 0, s>>>((const typename S::T*)pop, nbr, f, deviation, p);
            return 1;
        });
    });
}

}  // namespace lbm
