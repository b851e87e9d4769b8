// Moment totals without any device allocation.
//
// lbm_moment_totals_static() is the one entry point of this library that
// allocates nothing: it computes the FP64 fluid totals of lbm_moments() with
// its per-block partial sums held in a file-scope device array instead of a
// buffer from cudaMalloc.  It exists for callers that must not call the CUDA
// allocator at the point where they read the totals - for example a host
// application whose device memory is entirely reserved up front by its own
// pool, or a time-critical loop that forbids allocation calls.
#include <mutex>
#include <string>

#include "lbm_internal.h"

namespace {

// One FP64 partial per thread block of the moments kernel, 4 values each
// (sum rho, sum j_x, sum j_y, sum j_z): 262144 blocks x 32 B = 8 MiB.  Every
// GPU that loads this library holds the array until the process exits.
constexpr int64_t kStaticBlocks = 262144;
__device__ __align__(256) double g_static_partials[kStaticBlocks * 4];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_addr[kMaxDevices] = {};  // device address of g_static_partials, per device

}  // namespace

extern "C" lbm_status lbm_moment_totals_static(lbm_ctx* c, double* totals) {
    if (!c || !totals) return LBM_ERR_INVALID_ARG;
    if (!c->has_state) {
        c->err = "lbm_moment_totals_static before lbm_init_equilibrium";
        return LBM_ERR_STATE;
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, totals) != cudaSuccess ||
        !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
        cudaGetLastError();
        c->err = "lbm_moment_totals_static: totals must be a device pointer (4 doubles)";
        return LBM_ERR_INVALID_ARG;
    }
    const lbm::KParams p = lbm::make_params(c);  // the same parameter block lbm_moments uses
    const int64_t blocks = lbm::moments_partial_count(p);
    if (blocks > kStaticBlocks) {
        c->err = "lbm_moment_totals_static: the moments grid needs " + std::to_string(blocks) +
                 " partial sums, more than the static capacity of " + std::to_string(kStaticBlocks) +
                 " (ny * nz * ceil(nx / 128) must not exceed it)";
        return LBM_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices || dev != c->device) {
        cudaGetLastError();
        c->err = "lbm_moment_totals_static: the context's device must be current";
        return LBM_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            // host code may not use g_static_partials directly (that name is a
            // host-side stand-in); ask the runtime for its device address
            cudaError_t e = cudaGetSymbolAddress((void**)&g_addr[dev], g_static_partials);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                c->err = std::string("lbm_moment_totals_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return LBM_ERR_CUDA;
            }
        }
        scratch = g_addr[dev];
    }
    int64_t np = 0;
    c->launches += lbm::launch_moments(c->lat.vel, c->storage, c->pop[c->cur], c->nbr, nullptr, nullptr, scratch,
                                       &np, p, c->stream);
    c->launches += lbm::launch_reduce_partials(scratch, np, totals, c->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("lbm_moment_totals_static: ") + cudaGetErrorString(e);
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
