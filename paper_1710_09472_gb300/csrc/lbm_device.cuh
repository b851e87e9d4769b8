// Device-side helpers shared by the step and adjoint kernels: thread-to-cell
// mapping, periodic neighbour indices, and lattice-vector dot products that
// unroll to adds and subtracts.
#pragma once

#include "lbm_internal.h"

namespace lbm {
namespace dev {

constexpr int kBlock = 128;

// One thread per cell: blockIdx.x is the row (y, z), blockIdx.y the chunk of
// x, threads run along x.  All cell indices fit in 32 bits (N < 2^31).
struct Cell {
    int x, y, z;
    uint32_t cell;
    int xm, xp;       // x - 1, x + 1 with periodic wrap
    uint32_t r[3][3]; // row base ((z + dz) * ny + (y + dy)) * nx for dy, dz in {-1, 0, 1}
};

__device__ __forceinline__ bool cell_of_thread(const KParams& p, Cell& c) {
    c.x = blockIdx.y * blockDim.x + threadIdx.x;
    const int row = blockIdx.x;
    c.y = row % p.ny;
    c.z = row / p.ny;
    c.cell = (uint32_t)row * (uint32_t)p.nx + (uint32_t)c.x;
    c.xm = c.x == 0 ? p.nx - 1 : c.x - 1;
    c.xp = c.x == p.nx - 1 ? 0 : c.x + 1;
    const int ys[3] = {c.y == 0 ? p.ny - 1 : c.y - 1, c.y, c.y == p.ny - 1 ? 0 : c.y + 1};
    const int zs[3] = {c.z == 0 ? p.nz - 1 : c.z - 1, c.z, c.z == p.nz - 1 ? 0 : c.z + 1};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) c.r[i][k] = ((uint32_t)zs[k] * (uint32_t)p.ny + (uint32_t)ys[i]) * (uint32_t)p.nx;
    return c.x < p.nx;
}

// Index of x + s e_a (s = +1 or -1) with periodic wrap.
template <class L>
__device__ __forceinline__ uint32_t shifted(const Cell& c, int a, int s) {
    const int ex = s * L::c(a, 0), ey = s * L::c(a, 1), ez = s * L::c(a, 2);
    const int xs = ex > 0 ? c.xp : (ex < 0 ? c.xm : c.x);
    return c.r[ey + 1][ez + 1] + (uint32_t)xs;
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

__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Pull the stored (scaled) deviations of f(x, t) from a state (populations P
// followed by the link buffer G): f_a(x) = P_a(x - e_a) when x - e_a is fluid;
// when it is solid (bit a of the link mask) the halfway bounce-back value
// f_a(x) = f*_abar(x), which the collision at x stored in the link slot of its
// outgoing direction abar.
template <class L, class S>
__device__ __forceinline__ void pull(const typename S::T* __restrict__ P, const KParams& p, uint32_t m, const Cell& c,
                                     float* h) {
    const typename S::T* __restrict__ G =
        reinterpret_cast<const typename S::T*>(reinterpret_cast<const char*>(P) + p.gofs);
    const uint32_t o = outgoing<L::Q>(m);
    const uint32_t base = m ? __ldg(p.lbase + c.cell) : 0u;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        if (a != 0 && ((m >> a) & 1u))
            h[a] = S::raw(G + link_slot(base, o, opposite(a)));
        else
            h[a] = S::raw(P + (int64_t)a * p.N + (a == 0 ? c.cell : shifted<L>(c, a, -1)));
    }
}

}  // namespace dev
}  // namespace lbm
