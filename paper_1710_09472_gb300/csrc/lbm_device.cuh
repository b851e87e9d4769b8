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

// Storage index of direction a at the cell x + s e_a (s = -1, 0 or +1): slot
// pop_slot(a) of that cell's row (see pop_slot).
template <class L>
__device__ __forceinline__ int64_t pop_at(const KParams& p, const Cell& c, int a, int s) {
    const int ex = s * L::c(a, 0), ey = s * L::c(a, 1), ez = s * L::c(a, 2);
    const int xs = ex > 0 ? c.xp : (ex < 0 ? c.xm : c.x);
    return (int64_t)L::Q * c.r[ey + 1][ez + 1] + (int64_t)(pop_slot<L>(a) * p.nx + xs);
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

// Pull the stored (scaled) deviations of f(x, t) from a state (populations P,
// in the slot layout of pop_slot, followed by the link buffer G):
// f_a(x) = P_a(x - e_a) when x - e_a is fluid;
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
            h[a] = S::raw(P + pop_at<L>(p, c, a, -1));
    }
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

template <class L>
__device__ __forceinline__ unsigned long long packed_x() {
    unsigned long long v = 0;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) v |= (unsigned long long)(L::c(a, 0) + 1) << (2 * a);
    return v;
}

// Bounce-back patch of a staged row set.  Link k of the row is a fluid cell x
// with an outgoing direction b into a solid cell, descriptor x | b << 24.  The
// solid neighbour x + e_b is read by exactly one cell of the row for each
// direction: by x itself, in the pull of direction bbar (which reads
// x - e_bbar = x + e_b) and in the adjoint gather of direction b (which reads
// x + e_b).  So the halfway bounce-back value win[k - w0] is written into that
// staged slot, rows[slot(d) * rs + (x + e_bx mod nx)] (rows in slot order, rs
// the row stride) with d = bbar (PULL) or b (gather), and the cells then read
// their rows without any link logic.
// The descriptors come from the staged window desc (first element d0).
template <class L, bool PULL, class T>
__device__ __forceinline__ void patch_links(T* rows, int nx, int rs, const T* win, uint32_t w0, uint32_t g0,
                                            uint32_t g1, const uint32_t* desc, uint32_t d0) {
    const unsigned long long kPx = packed_x<L>();
    for (uint32_t k = g0 + threadIdx.x; k < g1; k += blockDim.x) {
        const uint32_t d = desc[k - d0];
        const int x = (int)(d & 0xFFFFFFu), b = (int)(d >> 24);
        int xs = x + (int)((kPx >> (2 * b)) & 3ull) - 1;
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        rows[slot_of<L>(PULL ? opposite(b) : b) * rs + xs] = win[k - w0];
    }
}

// Bytes reserved for a staged window of up to n elements of esize bytes.
__host__ __device__ __forceinline__ int window_cap(int n, int esize) {
    return (int)((((size_t)n * esize + 15) & ~(size_t)15) + 32);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (the non-tensor form of the Blackwell TMA engine)
// and mbarriers.  A stage is filled by one thread: mbarrier.arrive.expect_tx
// with the stage's byte count, then one cp.async.bulk per contiguous piece,
// each completing its bytes on the stage's mbarrier.  Output rows leave
// shared memory with cp.async.bulk stores (bulk groups).  Addresses and
// sizes are multiples of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// One potentially blocking test: the thread may be suspended in hardware
// until the phase completes or a system-dependent time limit passes.
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity to complete; gives up and returns
// false after `limit` SM clock cycles (default 2^31, about one second).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = 1ll << 31) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// Sleeps about n SM clock cycles.  After a wait has run out, a block pauses
// so that bulk copies it issued earlier land before it moves on or exits.
__device__ __forceinline__ void pause_cycles(long long n) {
    const long long t0 = clock64();
    while (clock64() - t0 < n) __nanosleep(1000);
}

// global -> shared, completing `bytes` on the mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// shared -> global, in the current bulk group
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// the sources of all committed bulk stores have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// all committed bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Bytes [b0, b1) of the 16-byte aligned window covering elements [g0, g1).
__device__ __forceinline__ void window_bytes(uint32_t g0, uint32_t g1, int esize, uint64_t& b0, uint64_t& b1) {
    b0 = ((uint64_t)g0 * esize) & ~15ull;
    b1 = ((uint64_t)g1 * esize + 15ull) & ~15ull;
}

}  // namespace dev
}  // namespace lbm
