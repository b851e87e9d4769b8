// Internal declarations of the GB300 semiclassical LBM library: context,
// lattice and storage traits, kernel parameter block and launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lbm.h"

namespace lbm {

constexpr int kMaxQ = 27;
// Per-cell link mask: bit a set when x - e_a is solid (a >= 1), i.e. the link
// that streams into x along e_a bounces back; kSolidBit when x itself is solid.
constexpr uint32_t kSolidBit = 0x80000000u;

// Outgoing-link mask from the incoming one: bit b set when x + e_b is solid,
// i.e. bit bbar of the incoming mask (opposite pairs are (a, a + 1), a odd).
template <int Q>
__host__ __device__ constexpr uint32_t odd_bits() {
    uint32_t v = 0;
    for (int b = 1; b < Q; b += 2) v |= 1u << b;
    return v;
}
template <int Q>
__host__ __device__ __forceinline__ uint32_t outgoing(uint32_t m) {
    constexpr uint32_t kOdd = odd_bits<Q>();
    constexpr uint32_t kEven = kOdd << 1;
    return ((m >> 1) & kOdd) | ((m << 1) & kEven);
}
// Link slot of outgoing direction b of a cell: base + number of its outgoing
// links below b.
__host__ __device__ __forceinline__ uint32_t link_slot(uint32_t base, uint32_t o, int b) {
#ifdef __CUDA_ARCH__
    return base + (uint32_t)__popc(o & ((1u << b) - 1u));
#else
    return base + (uint32_t)__builtin_popcount(o & ((1u << b) - 1u));
#endif
}

// ---------------------------------------------------------------------------
// Lattices (Sec. 8.1 D1V3, Sec. 8.2 D2V9, Table lattices-tab D3V19 and D3V27).
// Order: rest vector, then opposite pairs (a odd, a + 1 = -e_a), as
// documented in lbm.h.
// ---------------------------------------------------------------------------
struct LatD2V9 {
    static constexpr int D = 2;
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int c(int a, int d) {
        constexpr signed char t[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                         {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
        return t[a][d];
    }
};

struct LatD3V19 {
    static constexpr int D = 3;
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int c(int a, int d) {
        constexpr signed char t[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                          {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                          {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                          {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return t[a][d];
    }
};

struct LatD3V27 {
    static constexpr int D = 3;
    static constexpr int Q = 27;
    __host__ __device__ static constexpr int c(int a, int d) {
        constexpr signed char t[27][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},
                                          {0, 0, -1}, {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},
                                          {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},
                                          {0, -1, 1}, {1, 1, 1},   {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},
                                          {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
        return t[a][d];
    }
};

struct LatD1V3 {
    static constexpr int D = 1;
    static constexpr int Q = 3;
    __host__ __device__ static constexpr int c(int a, int d) { return d == 0 ? (a == 1 ? 1 : (a == 2 ? -1 : 0)) : 0; }
};

__host__ __device__ constexpr int opposite(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

// The moving directions fall into shells of equal |e|^2 (1: axes, 2: face
// diagonals, 3: corners), on which w_a and k2_a are constant.  shell_first(s)
// is the first direction of shell s, or -1 when the lattice has none.
template <class L>
__host__ __device__ constexpr int esq_of(int a) {
    return L::c(a, 0) * L::c(a, 0) + L::c(a, 1) * L::c(a, 1) + L::c(a, 2) * L::c(a, 2);
}
template <class L>
__host__ __device__ constexpr int shell_first(int s) {
    for (int a = 1; a < L::Q; ++a)
        if (esq_of<L>(a) == s) return a;
    return -1;
}

// ---------------------------------------------------------------------------
// Population storage.  Row r = z ny + y keeps its Q directions one after
// another, nx values each: direction a of cell (x, r) is element
// (r Q + slot(a)) nx + x.  The slots order the directions by (e_ay, e_az)
// (key 3 (e_ay + 1) + e_az + 1, ties by a), so the directions that a row
// pulls from one neighbouring row (y - e_ay, z - e_az) are consecutive slots
// of that row, and a row's Q directions are one contiguous block.
// ---------------------------------------------------------------------------
template <class L>
__host__ __device__ constexpr int pop_key(int a) {
    return (L::c(a, 1) + 1) * 3 + (L::c(a, 2) + 1);
}
template <class L>
__host__ __device__ constexpr int pop_slot_calc(int a) {
    int s = 0;
    for (int b = 0; b < L::Q; ++b)
        if (pop_key<L>(b) < pop_key<L>(a) || (pop_key<L>(b) == pop_key<L>(a) && b < a)) ++s;
    return s;
}
// the slots as a table built at compile time, so that a use with a known
// direction folds to a constant without re-running the count (for the
// 27-direction lattice, whose unrolled counts made compilation slow)
template <class L>
struct SlotTable {
    int s[L::Q];
    __host__ __device__ constexpr SlotTable() : s() {
        for (int a = 0; a < L::Q; ++a) s[a] = pop_slot_calc<L>(a);
    }
};
template <class L>
__host__ __device__ constexpr int pop_slot(int a) {
    if constexpr (L::Q > 19) {
        constexpr SlotTable<L> t{};
        return t.s[a];
    } else {
        return pop_slot_calc<L>(a);
    }
}
// first slot and number of directions with key k (0 .. 8), tabulated at compile time
template <class L>
struct KeyTable {
    int first[9], count[9];
    __host__ __device__ constexpr KeyTable() : first(), count() {
        for (int k = 0; k < 9; ++k)
            for (int b = 0; b < L::Q; ++b) {
                first[k] += pop_key<L>(b) < k ? 1 : 0;
                count[k] += pop_key<L>(b) == k ? 1 : 0;
            }
    }
};
template <class L>
__host__ __device__ constexpr int key_first(int k) {
    if constexpr (L::Q > 19) {
        constexpr KeyTable<L> t{};
        return t.first[k];
    } else {
        int s = 0;
        for (int b = 0; b < L::Q; ++b) s += pop_key<L>(b) < k ? 1 : 0;
        return s;
    }
}
template <class L>
__host__ __device__ constexpr int key_count(int k) {
    if constexpr (L::Q > 19) {
        constexpr KeyTable<L> t{};
        return t.count[k];
    } else {
        int s = 0;
        for (int b = 0; b < L::Q; ++b) s += pop_key<L>(b) == k ? 1 : 0;
        return s;
    }
}
// slot(a) for a direction known only at run time: 5 bits per direction,
// directions 12 k .. 12 k + 11 in word k
template <class L>
__host__ __device__ constexpr unsigned long long packed_slots(int word) {
    unsigned long long v = 0;
    for (int a = 12 * word; a < L::Q && a < 12 * (word + 1); ++a)
        v |= (unsigned long long)pop_slot_calc<L>(a) << (5 * (a - 12 * word));
    return v;
}
template <class L>
__host__ __device__ __forceinline__ int slot_of(int a) {
    constexpr unsigned long long w0 = packed_slots<L>(0), w1 = packed_slots<L>(1), w2 = packed_slots<L>(2);
    if constexpr (L::Q <= 24)
        return (int)((a < 12 ? (w0 >> (5 * a)) : (w1 >> (5 * (a - 12)))) & 31ull);
    else
        return (int)((a < 12 ? (w0 >> (5 * a)) : (a < 24 ? (w1 >> (5 * (a - 12))) : (w2 >> (5 * (a - 24))))) & 31ull);
}

// ---------------------------------------------------------------------------
// Storage of the deviation h_a = f_a - rho0 w_a / I_0.  The kernels work in
// the storage's scaled units h~ = scale * h (scale = 2^12 for FP16, 1
// otherwise): raw() decodes to FP32 without unscaling, put() rounds to
// nearest even.
// ---------------------------------------------------------------------------
// sr2() rounds two values stochastically: each is rounded up in magnitude
// with probability equal to the dropped fraction, so the expected stored
// value is the exact FP32 value (unbiased; no stagnation of increments
// smaller than half an ulp).  FP16 drops 13 mantissa bits of FP32, BF16 16.
struct StoreF32 {
    using T = float;
    static constexpr int kBytes = 4;
    __device__ __forceinline__ static float raw(const T* p) { return __ldg(p); }
    __device__ __forceinline__ static float cvt(T v) { return v; }
    __device__ __forceinline__ static void put(T* p, float v) { *p = v; }
    __device__ __forceinline__ static void sr2(float va, float vb, uint32_t, T& ta, T& tb) {
        ta = va;
        tb = vb;
    }
};

struct StoreF16 {
    using T = __half;
    static constexpr int kBytes = 2;
    __device__ __forceinline__ static float raw(const T* p) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static float cvt(T v) { return __half2float(v); }
    __device__ __forceinline__ static void put(T* p, float v) { *p = __float2half_rn(v); }
    // stochastic rounding of two values in one conversion (cvt.rs): the low
    // 13 bits of each 16-bit half of r are added below the kept mantissa of
    // va (low half) and vb (high half) before truncation
    __device__ __forceinline__ static void sr2(float va, float vb, uint32_t r, T& ta, T& tb) {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(vb), "f"(va), "r"(r));
        ta = __ushort_as_half((unsigned short)(d & 0xFFFFu));
        tb = __ushort_as_half((unsigned short)(d >> 16));
    }
};

struct StoreBF16 {
    using T = __nv_bfloat16;
    static constexpr int kBytes = 2;
    __device__ __forceinline__ static float raw(const T* p) { return __bfloat162float(__ldg(p)); }
    __device__ __forceinline__ static float cvt(T v) { return __bfloat162float(v); }
    __device__ __forceinline__ static void put(T* p, float v) { *p = __float2bfloat16_rn(v); }
    // as StoreF16::sr2, with all 16 bits of each half of r
    __device__ __forceinline__ static void sr2(float va, float vb, uint32_t r, T& ta, T& tb) {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(vb), "f"(va), "r"(r));
        ta = __ushort_as_bfloat16((unsigned short)(d & 0xFFFFu));
        tb = __ushort_as_bfloat16((unsigned short)(d >> 16));
    }
};

// ---------------------------------------------------------------------------
// Kernel parameter block (passed by value).  The equilibrium is the direct
// N = 2 form of Sec. 5.1 (Eq. feq-reduce-general-method-without-pol-eq) with
// xi_a = e_a / c_s folded into the constants:
//   f^eq_a = rho w_a [A + Bp (e_a.u) + Cp (e_a.u)^2 + k2_a u^2],
//   A = 1/I0, Bp = 1/(I2 c_s), Cp = 1/(2 I4 c_s^2),
//   k2_a = (Delta2^2 - 1) e_a^2 / (2 D I4 c_s^2) - I2 Delta2^2 / (2 I0 I4).
// The odd (momentum-carrying) coefficient W1_a = w_a Bp / c_s is kept as a
// double-float pair W1hi + W1lo so that sum_a W1_a e_a e_a = identity to
// ~1e-15: an FP32-rounded W1 would leak a fixed fraction ~1e-7 of the
// momentum in every collision, which compounds over thousands of steps.
// ---------------------------------------------------------------------------
struct KParams {
    int nx, ny, nz;
    int64_t N;
    float omega;  // 1 / tau
    float tau;
    float rho0;
    float A, Bp, Cp, Gp, H;
    float cs, cs_inv;
    float w[kMaxQ];
    float k2[kMaxQ];
    float W1hi[kMaxQ], W1lo[kMaxQ];
    float f0[kMaxQ];  // rho0 w_a A: the rest equilibrium at rho0 (unscaled)
    float E[3], B[3];
    float scale, inv_scale;
    uint32_t step;  // global step index of this launch (stochastic rounding stream)
    uint32_t seed;
    // Bounce-back link buffer G (see lbm_kernels.cu): byte offset of G inside
    // a state buffer, per-cell first link slot, per-row first link slot
    // (ny * nz + 1 entries) and the largest number of links in one row.
    uint64_t gofs;
    const uint32_t* lbase;
    const uint32_t* rowG;
    // per link slot k: x | b << 24, the x coordinate of its fluid cell and
    // its outgoing direction b (the row-staged kernels' link passes)
    const uint32_t* ldesc;
    int max_row_links;
    // per row, the cells in the order the row-staged kernels give them to
    // threads: entry 0 the number of fluid cells nf, entries 1..7 zero, then
    // the fluid x ascending and the solid x ascending (lorder entries per row,
    // a multiple of 8; null when nx > 65535)
    const uint16_t* rorder;
    int lorder;
    // byte offset of the link buffer inside an adjoint field (reverse sweep)
    uint64_t lgofs;
    // host-mapped status word: a kernel whose bounded wait ran out writes a
    // nonzero code here (read by the next synchronising API call)
    int* status;
    // Local chemical-potential model (lbm_set_local_mu; null table: off):
    // dth(r) = thetabar(r) - thetabar_w at r = rho / rho0 as a cubic Hermite
    // table of (dth, dth' dr) pairs on lmu_n uniform nodes; drho~ lmu_a is
    // (r - 1) / dr and lmu_b the index of the node r = 1 (the coordinate is
    // clamped to the table).  lmu_K[s] is
    // K_s = 1/2 (c2 + D cbar2) [(c2 + D cbar2) |e|^2 / c_s^2 + D c'2] of the
    // shell |e|^2 = s: the EDF gains rho w_a K_a dth.
    const float2* lmu_tab;
    float lmu_a, lmu_b;
    int lmu_n;
    float lmu_K[4];
};

struct Launch {
    dim3 grid, block;
};

// Launchers (lbm_kernels.cu).  Each returns the number of kernels launched.
int launch_build_neighbors(int vel, const uint8_t* mask, uint32_t* nbr, unsigned long long* fluid_count,
                           const KParams& p, cudaStream_t s);
// Link buffer layout: lbase[cell] (exclusive prefix of outgoing-link counts),
// rowG[0..ny*nz]; needs a temporary of *temp_bytes (queried with temp == NULL).
// Bounded-wait probe (writes code 3 into *status when its wait runs out).
int launch_wait_probe(int* status, long long limit, cudaStream_t s);
// Per-link descriptors ldesc[k] = x | b << 24 (needs lbase).
// FP32 field in the populations' slot layout -> direction-major out[a * N + cell].
int launch_unslot(int vel, const float* in, float* out, const KParams& p, cudaStream_t s);
// Per-row cell order (fluid cells first) for the row-staged kernels.
int launch_build_row_order(const uint32_t* nbr, uint16_t* rorder, const KParams& p, cudaStream_t s);
int launch_build_link_desc(int vel, const uint32_t* nbr, const uint32_t* lbase, uint32_t* ldesc, const KParams& p,
                           cudaStream_t s);
int launch_build_links(int vel, const uint32_t* nbr, uint32_t* lbase, uint32_t* rowG, void* temp,
                       size_t* temp_bytes, const KParams& p, cudaStream_t s);
int launch_init(int vel, int storage, void* pop, const uint32_t* nbr, const float* rho, const float* u,
                const KParams& p, cudaStream_t s);
int launch_step(int vel, int storage, int force, bool efield, bool sr, const void* fin, void* fout,
                const uint32_t* nbr, const float* Ef, const KParams& p, cudaStream_t s);
int launch_step_f32(int vel, int force, bool efield, bool sr, const void* fin, void* fout, const uint32_t* nbr,
                    const float* Ef, const KParams& p, cudaStream_t s);
int launch_step_f16(int vel, int force, bool efield, bool sr, const void* fin, void* fout, const uint32_t* nbr,
                    const float* Ef, const KParams& p, cudaStream_t s);
int launch_step_bf16(int vel, int force, bool efield, bool sr, const void* fin, void* fout, const uint32_t* nbr,
                     const float* Ef, const KParams& p, cudaStream_t s);
// the same for D3V27 and D1V3 (translation units lbm_step_*_x.cu)
int launch_step_f32_x(int vel, int force, bool efield, bool sr, const void* fin, void* fout, const uint32_t* nbr,
                      const float* Ef, const KParams& p, cudaStream_t s);
int launch_step_f16_x(int vel, int force, bool efield, bool sr, const void* fin, void* fout, const uint32_t* nbr,
                      const float* Ef, const KParams& p, cudaStream_t s);
int launch_step_bf16_x(int vel, int force, bool efield, bool sr, const void* fin, void* fout, const uint32_t* nbr,
                       const float* Ef, const KParams& p, cudaStream_t s);
int launch_moments(int vel, int storage, const void* pop, const uint32_t* nbr, float* rho, float* j,
                   double* partials, int64_t* n_partials, const KParams& p, cudaStream_t s);
int launch_reduce_partials(const double* partials, int64_t n_partials, double* out4, cudaStream_t s);
int launch_populations(int vel, int storage, const void* pop, const uint32_t* nbr, float* f, bool deviation,
                       const KParams& p, cudaStream_t s);
int64_t moments_partial_count(const KParams& p);

// Adjoint (lbm_adjoint.cu).
int64_t adjoint_slot_count(const KParams& p);
int launch_adjoint_seed(int vel, int storage, const void* P, const uint32_t* nbr, const float* w_rho,
                        const float* w_j, float* lam, double* slots, bool in_window, const KParams& p,
                        cudaStream_t s);
int launch_adjoint_step(int vel, int storage, int force, bool efield, bool in_window, const void* P,
                        const float* lam_in, float* lam_out, const uint32_t* nbr, const float* Ef,
                        const float* w_rho, const float* w_j, float* gE, double* slots, const KParams& p,
                        cudaStream_t s);
int launch_reduce_slots(const double* slots, int64_t n_blocks, int n_slots, double* out, cudaStream_t s);
// acc[i] += part[i] (FP64) and part[i] = 0 for i < n: folds the reverse
// steps' FP32 dL/dE partials into the caller's FP64 gradient.
int launch_fold_partials(float* part, double* acc, int64_t n, cudaStream_t s);
int launch_accumulate_totals(const double* partials, int64_t n_partials, double* acc4, cudaStream_t s);

// Local chemical-potential table (lbm_fd.cu): for the FD weight of dimension D
// at (theta, mu_w), node k of n at r_k = 1 + (k - k1) dr holds
// (thetabar(r_k) - thetabar(1), dthetabar/dr (r_k) dr), where thetabar(r) =
// I_2/I_0 at the mu with I_0(mu) = r I_0(mu_w).  Synchronises the stream.
lbm_status build_local_mu_table(int D, double theta, double mu_w, int n, int k1, double dr, float2* out,
                                cudaStream_t s);

}  // namespace lbm

namespace lbm {
// Kernel parameter block of a context (lbm_api.cu).
KParams make_params(const lbm_ctx* c);
}  // namespace lbm

// The context (opaque to C callers).
// Device buffers of lbm_adjoint, kept by the context between calls so that
// repeated calls allocate once (released by lbm_release_workspace,
// lbm_set_geometry and lbm_destroy).
struct AdjWorkspace {
    std::vector<void*> states;  // forward-state buffers of state_bytes each
    size_t state_bytes = 0;
    void* lam[2] = {nullptr, nullptr};
    size_t lam_bytes = 0;
    double* slots = nullptr;
    int64_t nslot = 0;
    double* red = nullptr;
    float* wstage = nullptr;  // loss weights staged from the host
    size_t wstage_bytes = 0;
    float* gpart = nullptr;   // FP32 dL/dE partials of the latest reverse steps (D N)
    size_t gpart_bytes = 0;
    size_t held() const {
        return states.size() * state_bytes + 2 * lam_bytes + sizeof(double) * (size_t)nslot + wstage_bytes +
               gpart_bytes;
    }
};

struct lbm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    lbm_lattice lat{};
    int D = 0, Q = 0;
    int64_t nx = 1, ny = 1, nz = 1, N = 0;
    int64_t n_fluid = 0;
    int storage = 0;
    bool stochastic = false;  // stochastic rounding of FP16/BF16 stores
    uint32_t rseed = 0;       // seed of the stochastic-rounding stream
    double tau = 1.0;
    double E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    // host-side constants (FP64)
    double I[5] = {0, 0, 0, 0, 0};
    double c0 = 0, c1 = 0, c2 = 0, cbar2 = 0, cprime2 = 0, thetabar = 0, J2 = 0, Delta2 = 0, cs = 0;
    double w[lbm::kMaxQ] = {};
    double A = 0, Bc = 0, Cc = 0, G = 0, H = 0;
    double scale = 1.0;
    // device buffers
    void* pop[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t* nbr = nullptr;
    uint32_t* lbase = nullptr;     // per-cell first slot in the link buffer
    uint32_t* rowG = nullptr;      // per-row first slot (ny * nz + 1)
    uint32_t* ldesc = nullptr;     // per link slot: x | b << 24
    uint16_t* rorder = nullptr;    // per row: fluid count, then fluid x, then solid x (lorder entries)
    int lorder = 0;
    int64_t n_links = 0;           // outgoing links into solid cells
    int max_row_links = 0;
    size_t state_bytes = 0;        // populations + link buffer
    size_t gofs = 0;               // byte offset of the link buffer in a state
    uint8_t* mask_dev = nullptr;
    float* Efield = nullptr;
    bool use_Efield = false;
    double* partials = nullptr;
    int64_t partials_cap = 0;
    double* totals_dev = nullptr;
    double* totals_host = nullptr;  // pinned, 4 doubles
    unsigned long long* count_dev = nullptr;
    AdjWorkspace ws;               // lbm_adjoint buffers kept between calls
    size_t mem_budget = 0;         // device bytes an lbm_adjoint call may allocate (0: free memory)
    int64_t adj_stats[4] = {0, 0, 0, 0};  // last lbm_adjoint: schedule, state buffers, forward steps, reverse steps
    float2* lmu_tab = nullptr;     // local-mu model table (null: off)
    int* status_host = nullptr;    // mapped pinned word written by kernels on a wait timeout
    int* status_dev = nullptr;     // its device address
    float* stage = nullptr;  // device staging for host-pointer arguments
    size_t stage_bytes = 0;
    bool geometry_counted = false;
    bool has_state = false;
    int64_t steps = 0;
    int64_t launches = 0;
    std::string err;
};
