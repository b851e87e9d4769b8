// Device kernels of the semiclassical LBM step (Sec. 9.1 of arXiv 1710.09472):
// link mask, equilibrium start state, the fused pull-stream + BGK collision +
// Lorentz forcing step, moments with FP64 reductions, and the population
// read-back.
//
// Layout: populations are structure-of-arrays, P[a * N + cell] with
// cell = (z * ny + y) * nx + x.  P holds post-collision values ("pull"
// scheme): the state f(x, t) of the method is f_a(x, t) = P_a(x - e_a) when
// x - e_a is fluid.
// Halfway bounce-back (Sec. 9.3, 9.4) uses a link buffer G stored after P in
// the same state buffer: every link from a fluid cell x into a solid cell
// (x + e_b solid) owns one slot, numbered in cell order (lbase[x] + rank of b
// among x's outgoing links), so the links of one row form a contiguous range
// rowG[r] .. rowG[r+1].  The collision stores f*_b(x) there, and the next
// step reads it back as f_bbar(x).
#include <algorithm>
#include <cstdio>

#include <cub/device/device_scan.cuh>

#include "lbm_device.cuh"

namespace lbm {
namespace {

using dev::Cell;
using dev::kBlock;

// ---------------------------------------------------------------------------
// Link mask: bit a set when x - e_a is solid (the link streaming into x along
// e_a bounces back); kSolidBit when x is solid.
// ---------------------------------------------------------------------------
template <class L>
__global__ void __launch_bounds__(kBlock) k_neighbors(const uint8_t* __restrict__ mask, uint32_t* __restrict__ nbr,
                                                      unsigned long long* __restrict__ fluid_count, KParams p) {
    Cell c;
    unsigned fluid = 0;
    if (dev::cell_of_thread(p, c)) {
        uint32_t m = 0;
        if (mask[c.cell]) {
            m = kSolidBit;
        } else {
            fluid = 1;
#pragma unroll
            for (int a = 1; a < L::Q; ++a)
                if (mask[dev::shifted<L>(c, a, -1)]) m |= (1u << a);
        }
        nbr[c.cell] = m;
    }
    const unsigned cnt = __popc(__ballot_sync(0xffffffffu, fluid));
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(fluid_count, (unsigned long long)cnt);
}

// ---------------------------------------------------------------------------
// Start state f(x, 0) = f^eq(rho(x), u(x)) for the pull with read-side
// bounce-back: slot P_b(y) of a fluid cell y is pulled by y + e_b when that
// cell is fluid (value f^eq_b(y + e_b)), and by y itself as its bounced
// population bbar when y + e_b is solid (value f^eq_bbar(y)); solid cells'
// slots are never read and hold 0.
// ---------------------------------------------------------------------------
template <class L>
__device__ __forceinline__ float heq_unscaled(const KParams& p, int a, float rho, const float* u) {
    const float eu = dev::edot<L>(a, u);
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return p.w[a] * (p.A * (rho - p.rho0) + rho * (p.Bp * eu + p.Cp * eu * eu + p.k2[a] * u2));
}

template <class L, class S>
__global__ void __launch_bounds__(kBlock) k_init(typename S::T* __restrict__ P, const uint32_t* __restrict__ nbr,
                                                 const float* __restrict__ rho, const float* __restrict__ u,
                                                 KParams p) {
    Cell c;
    if (!dev::cell_of_thread(p, c)) return;
    const uint32_t m = nbr[c.cell];
    typename S::T* G = reinterpret_cast<typename S::T*>(reinterpret_cast<char*>(P) + p.gofs);
    auto fields = [&](uint32_t cell, float& r, float* uu) {
        r = rho ? rho[cell] : p.rho0;
        uu[0] = u ? u[cell] : 0.f;
        uu[1] = (u && L::D >= 2) ? u[p.N + cell] : 0.f;
        uu[2] = (u && L::D == 3) ? u[2 * p.N + cell] : 0.f;
    };
    float r0, u0[3];
    fields(c.cell, r0, u0);
    const bool fluid = !(m & kSolidBit);
    const uint32_t o = fluid ? outgoing<L::Q>(m) : 0u;
    const uint32_t base = (fluid && o) ? p.lbase[c.cell] : 0u;
#pragma unroll
    for (int b = 0; b < L::Q; ++b) {
        float v = 0.f;
        if (fluid) {
            if (b != 0 && ((o >> b) & 1u)) {
                // link into a solid cell: next pull of bbar at this cell reads f^eq_bbar here
                S::put(G + link_slot(base, o, b), heq_unscaled<L>(p, opposite(b), r0, u0) * p.scale);
            } else {
                float r1 = r0, u1[3] = {u0[0], u0[1], u0[2]};
                if (b != 0) fields(dev::shifted<L>(c, b, +1), r1, u1);
                v = heq_unscaled<L>(p, b, r1, u1);
            }
        }
        S::put(P + dev::pop_at<L>(p, c, b, 0), v * p.scale);
    }
}

// Link layout: count outgoing links per fluid cell, exclusive scan, row starts.
template <class L>
__global__ void __launch_bounds__(kBlock) k_link_counts(const uint32_t* __restrict__ nbr, uint32_t* __restrict__ cnt,
                                                        KParams p) {
    Cell c;
    if (!dev::cell_of_thread(p, c)) return;
    const uint32_t m = nbr[c.cell];
    cnt[c.cell] = (m & kSolidBit) ? 0u : (uint32_t)__popc(outgoing<L::Q>(m));
}

// Descriptor of every link slot: the x coordinate of its fluid cell and its
// outgoing direction b, ldesc[slot] = x | b << 24.
template <class L>
__global__ void __launch_bounds__(kBlock) k_link_desc(const uint32_t* __restrict__ nbr,
                                                      const uint32_t* __restrict__ lbase,
                                                      uint32_t* __restrict__ ldesc, KParams p) {
    Cell c;
    if (!dev::cell_of_thread(p, c)) return;
    const uint32_t m = nbr[c.cell];
    if ((m & kSolidBit) || m == 0u) return;
    const uint32_t o = outgoing<L::Q>(m);
    const uint32_t base = lbase[c.cell];
#pragma unroll
    for (int b = 1; b < L::Q; ++b)
        if ((o >> b) & 1u) ldesc[link_slot(base, o, b)] = (uint32_t)c.x | ((uint32_t)b << 24);
}

// Cell order of each row for the row-staged kernels: entry 0 the number of
// fluid cells nf, entries 1..7 zero, entries 8 .. 8 + nf - 1 the fluid x
// ascending, then the solid x ascending, then zeros up to lorder.  One warp
// per row.
__global__ void __launch_bounds__(kBlock) k_row_order(const uint32_t* __restrict__ nbr, uint16_t* __restrict__ ord,
                                                      KParams p) {
    const int64_t R = (int64_t)p.ny * p.nz;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < R; r += nwarps) {
        const uint32_t* m = nbr + r * p.nx;
        uint16_t* o = ord + r * p.lorder;
        int nf = 0;
        for (int x0 = 0; x0 < p.nx; x0 += 32) {
            const int x = x0 + lane;
            nf += __popc(__ballot_sync(0xffffffffu, x < p.nx && !(m[x] & kSolidBit)));
        }
        int nfl = 0, nso = nf;  // entries written so far: fluid, and nf + solid
        for (int x0 = 0; x0 < p.nx; x0 += 32) {
            const int x = x0 + lane;
            const bool in = x < p.nx;
            const bool fluid = in && !(m[x] & kSolidBit);
            const unsigned bf = __ballot_sync(0xffffffffu, fluid), bs = __ballot_sync(0xffffffffu, in && !fluid);
            if (fluid) o[8 + nfl + __popc(bf & below)] = (uint16_t)x;
            if (in && !fluid) o[8 + nso + __popc(bs & below)] = (uint16_t)x;
            nfl += __popc(bf);
            nso += __popc(bs);
        }
        if (lane < 8) o[lane] = lane == 0 ? (uint16_t)nf : (uint16_t)0;
        for (int k = 8 + p.nx + lane; k < p.lorder; k += 32) o[k] = 0;
    }
}

template <class L>
__global__ void k_row_starts(const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ lbase,
                             uint32_t* __restrict__ rowG, KParams p) {
    const int64_t R = (int64_t)p.ny * p.nz;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= R; r += (int64_t)gridDim.x * blockDim.x) {
        if (r < R) {
            rowG[r] = lbase[r * p.nx];
        } else {
            const uint32_t m = nbr[p.N - 1];
            rowG[R] = lbase[p.N - 1] + ((m & kSolidBit) ? 0u : (uint32_t)__popc(outgoing<L::Q>(m)));
        }
    }
}

// ---------------------------------------------------------------------------
// Moments of f(x, t) and FP64 block partials of the fluid totals
// partials[block] = {sum rho, sum j_x, sum j_y, sum j_z}.
// ---------------------------------------------------------------------------
template <class L, class S>
__device__ __forceinline__ void cell_moments(const typename S::T* __restrict__ P, const uint32_t* __restrict__ nbr,
                                             const KParams& p, const Cell& c, float& rho, float* j) {
    float h[L::Q];
    dev::pull<L, S>(P, p, __ldg(nbr + c.cell), c, h);
    float drho = 0.f, jj[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        drho += h[a];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (L::c(a, d) > 0) jj[d] += h[a];
            if (L::c(a, d) < 0) jj[d] -= h[a];
        }
    }
    rho = p.rho0 + drho * p.inv_scale;
    const float k = p.inv_scale * p.cs_inv;
    j[0] = jj[0] * k;
    j[1] = jj[1] * k;
    j[2] = (L::D == 3) ? jj[2] * k : 0.f;
}

template <class L, class S>
__global__ void __launch_bounds__(kBlock) k_moments(const typename S::T* __restrict__ P, const uint32_t* __restrict__ nbr,
                                                    float* __restrict__ rho_out, float* __restrict__ j_out,
                                                    double* __restrict__ partials, KParams p) {
    Cell c;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (dev::cell_of_thread(p, c)) {
        const uint32_t m = nbr[c.cell];
        float r = 0.f, j[3] = {0.f, 0.f, 0.f};
        if (!(m & kSolidBit)) {
            cell_moments<L, S>(P, nbr, p, c, r, j);
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
        for (int k = 0; k < 4; ++k) acc[k] = dev::warp_sum(acc[k]);
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
                v = dev::warp_sum(v);
                if (lane == 0) partials[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + k] = v;
            }
        }
    }
}

// One block sums interleaved per-block slots in a fixed order (deterministic);
// with add != 0 the result is added to out (window sums stay on the device).
constexpr int kReduceThreads = 512;
constexpr int kMaxSlots = 8;
__global__ void __launch_bounds__(kReduceThreads) k_reduce_slots(const double* __restrict__ slots, int64_t nb,
                                                                 int ns, double* __restrict__ out, int add) {
    __shared__ double sh[kReduceThreads / 32][kMaxSlots];
    double acc[kMaxSlots];
#pragma unroll
    for (int k = 0; k < kMaxSlots; ++k) acc[k] = 0.0;
    for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < kMaxSlots; ++k)
            if (k < ns) acc[k] += slots[i * ns + k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kMaxSlots; ++k) acc[k] = dev::warp_sum(acc[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kMaxSlots; ++k) sh[wid][k] = acc[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < kMaxSlots; ++k) {
            double v = lane < (int)(blockDim.x / 32) ? sh[lane][k] : 0.0;
            v = dev::warp_sum(v);
            if (lane == 0 && k < ns) out[k] = add ? out[k] + v : v;
        }
    }
}

// FP32 populations f_a(x, t) = f0_a + h_a (or the deviations h_a).
template <class L, class S>
__global__ void __launch_bounds__(kBlock) k_populations(const typename S::T* __restrict__ P,
                                                        const uint32_t* __restrict__ nbr, float* __restrict__ f,
                                                        bool deviation, KParams p) {
    Cell c;
    if (!dev::cell_of_thread(p, c)) return;
    const uint32_t m = nbr[c.cell];
    if (m & kSolidBit) {
#pragma unroll
        for (int a = 0; a < L::Q; ++a) f[(int64_t)a * p.N + c.cell] = 0.f;
        return;
    }
    float h[L::Q];
    dev::pull<L, S>(P, p, m, c, h);
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        const float d = h[a] * p.inv_scale;
        f[(int64_t)a * p.N + c.cell] = deviation ? d : p.f0[a] + d;
    }
}

// Copies an FP32 field in the slot layout of the populations (see pop_slot)
// into direction-major order out[a * N + cell].
template <class L>
__global__ void __launch_bounds__(kBlock) k_unslot(const float* __restrict__ in, float* __restrict__ out, KParams p) {
    Cell c;
    if (!dev::cell_of_thread(p, c)) return;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) out[(int64_t)a * p.N + c.cell] = in[dev::pop_at<L>(p, c, a, 0)];
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
    if (vel == LBM_D3V27) return f(LatD3V27{});
    if (vel == LBM_D1V3) return f(LatD1V3{});
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

int launch_build_links(int vel, const uint32_t* nbr, uint32_t* lbase, uint32_t* rowG, void* temp,
                       size_t* temp_bytes, const KParams& p, cudaStream_t s) {
    const int n = (int)p.N;
    if (!temp) {
        // query the scan's temporary size
        return cub::DeviceScan::ExclusiveSum(nullptr, *temp_bytes, lbase, lbase, n, s) == cudaSuccess ? 0 : -1;
    }
    Launch l = grid_of(p);
    dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        k_link_counts<L><<<l.grid, l.block, 0, s>>>(nbr, lbase, p);
        return 1;
    });
    cub::DeviceScan::ExclusiveSum(temp, *temp_bytes, lbase, lbase, n, s);
    const int64_t R = (int64_t)p.ny * p.nz;
    const int blocks = (int)((R + 1 + 255) / 256 < 4096 ? (R + 1 + 255) / 256 : 4096);
    dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        k_row_starts<L><<<blocks, 256, 0, s>>>(nbr, lbase, rowG, p);
        return 1;
    });
    return 3;
}

// Failure-path probe: one block waits, with the staged kernels' bounded
// wait, on an mbarrier that nothing completes; the wait runs out after
// `limit` clocks and the block writes code 3 into the status word.
__global__ void k_wait_probe(int* status, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const bool done = dev::mbar_wait(&bar, 0u, limit);
    if (!done && threadIdx.x == 0 && status) atomicExch(status, 3);
}

int launch_wait_probe(int* status, long long limit, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(status, limit);
    return 1;
}

int launch_unslot(int vel, const float* in, float* out, const KParams& p, cudaStream_t s) {
    Launch l = grid_of(p);
    return dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        k_unslot<L><<<l.grid, l.block, 0, s>>>(in, out, p);
        return 1;
    });
}

int launch_build_row_order(const uint32_t* nbr, uint16_t* rorder, const KParams& p, cudaStream_t s) {
    const int64_t R = (int64_t)p.ny * p.nz;
    const int64_t blocks = std::min<int64_t>((R * 32 + kBlock - 1) / kBlock, 65535);
    k_row_order<<<(unsigned)blocks, kBlock, 0, s>>>(nbr, rorder, p);
    return 1;
}

int launch_build_link_desc(int vel, const uint32_t* nbr, const uint32_t* lbase, uint32_t* ldesc, const KParams& p,
                           cudaStream_t s) {
    Launch l = grid_of(p);
    return dispatch_lattice(vel, [&](auto lat) {
        using L = decltype(lat);
        k_link_desc<L><<<l.grid, l.block, 0, s>>>(nbr, lbase, ldesc, p);
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

int launch_step(int vel, int storage, int force, bool efield, bool sr, const void* fin, void* fout,
                const uint32_t* nbr, const float* Ef, const KParams& p, cudaStream_t s) {
    if (vel == LBM_D3V27 || vel == LBM_D1V3) {
        if (storage == LBM_F16_DEV) return launch_step_f16_x(vel, force, efield, sr, fin, fout, nbr, Ef, p, s);
        if (storage == LBM_BF16_DEV) return launch_step_bf16_x(vel, force, efield, sr, fin, fout, nbr, Ef, p, s);
        return launch_step_f32_x(vel, force, efield, false, fin, fout, nbr, Ef, p, s);
    }
    if (storage == LBM_F16_DEV) return launch_step_f16(vel, force, efield, sr, fin, fout, nbr, Ef, p, s);
    if (storage == LBM_BF16_DEV) return launch_step_bf16(vel, force, efield, sr, fin, fout, nbr, Ef, p, s);
    return launch_step_f32(vel, force, efield, false, fin, fout, nbr, Ef, p, s);
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
    k_reduce_slots<<<1, kReduceThreads, 0, s>>>(partials, n_partials, 4, out4, 0);
    return 1;
}

int launch_reduce_slots(const double* slots, int64_t n_blocks, int n_slots, double* out, cudaStream_t s) {
    if (n_slots > kMaxSlots) return 0;
    k_reduce_slots<<<1, kReduceThreads, 0, s>>>(slots, n_blocks, n_slots, out, 0);
    return 1;
}

int launch_accumulate_totals(const double* partials, int64_t n_partials, double* acc4, cudaStream_t s) {
    k_reduce_slots<<<1, kReduceThreads, 0, s>>>(partials, n_partials, 4, acc4, 1);
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
