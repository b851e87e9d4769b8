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

// 16-byte asynchronous global -> shared copies (cp.async, L2 only).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// e_ay + 1 and e_az + 1 of every direction, 2 bits each, in two 64-bit words
// (19 directions need 38 bits per word); the unrolled loops fold to constants.
template <class L>
__device__ __forceinline__ unsigned long long packed_y() {
    unsigned long long v = 0;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) v |= (unsigned long long)(L::c(a, 1) + 1) << (2 * a);
    return v;
}
template <class L>
__device__ __forceinline__ unsigned long long packed_z() {
    unsigned long long v = 0;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) v |= (unsigned long long)(L::c(a, 2) + 1) << (2 * a);
    return v;
}

// Compacts the fluid cells of a staged row (link masks mrow[0..nx)) into
// flist: cells without solid neighbours (mask 0) from the front, cells with
// bounce-back links from the back (flist[nx - 1], flist[nx - 2], ...), so that
// a warp taking consecutive entries mostly sees one kind and skips the link
// code.  counts[0..1] must be zero on entry and receive the two numbers; the
// call ends with a block barrier and returns counts[0].  blockDim.x must be a
// multiple of 32.
__device__ __forceinline__ int compact_row(const uint32_t* mrow, int nx, uint32_t* flist, int* counts) {
    const unsigned lane = threadIdx.x & 31u, below = (1u << lane) - 1u;
    for (int x0 = 0; x0 < nx; x0 += blockDim.x) {
        const int x = x0 + (int)threadIdx.x;
        const uint32_t m = x < nx ? mrow[x] : kSolidBit;
        const bool inner = m == 0u;
        const bool bnd = m != 0u && !(m & kSolidBit);
        const unsigned bi = __ballot_sync(0xffffffffu, inner), bb = __ballot_sync(0xffffffffu, bnd);
        int base_i = 0, base_b = 0;
        if (lane == 0) {
            if (bi) base_i = atomicAdd(&counts[0], __popc(bi));
            if (bb) base_b = atomicAdd(&counts[1], __popc(bb));
        }
        base_i = __shfl_sync(0xffffffffu, base_i, 0);
        base_b = __shfl_sync(0xffffffffu, base_b, 0);
        if (inner) flist[base_i + __popc(bi & below)] = (uint32_t)x;
        if (bnd) flist[nx - 1 - (base_b + __popc(bb & below))] = (uint32_t)x;
    }
    __syncthreads();
    return counts[0];
}

}  // namespace dev
}  // namespace lbm
