// Reverse-step dispatch: per-storage launchers (lbm_adjoint_{f32,f16,bf16}.cu)
// and the gradient slot count.
#include "lbm_adjoint.cuh"

namespace lbm {

int launch_adjoint_seed_f32(int, const void*, const uint32_t*, const float*, const float*, float*, double*, bool,
                            const KParams&, cudaStream_t);
int launch_adjoint_seed_f16(int, const void*, const uint32_t*, const float*, const float*, float*, double*, bool,
                            const KParams&, cudaStream_t);
int launch_adjoint_seed_bf16(int, const void*, const uint32_t*, const float*, const float*, float*, double*, bool,
                             const KParams&, cudaStream_t);
int launch_adjoint_step_f32(int, int, bool, bool, const void*, const float*, float*, const uint32_t*, const float*,
                            const float*, const float*, float*, double*, const KParams&, cudaStream_t);
int launch_adjoint_step_f16(int, int, bool, bool, const void*, const float*, float*, const uint32_t*, const float*,
                            const float*, const float*, float*, double*, const KParams&, cudaStream_t);
int launch_adjoint_step_bf16(int, int, bool, bool, const void*, const float*, float*, const uint32_t*, const float*,
                             const float*, const float*, float*, double*, const KParams&, cudaStream_t);

// the same for D3V27 and D1V3 (lbm_adjoint_*_x.cu)
int launch_adjoint_seed_f32_x(int, const void*, const uint32_t*, const float*, const float*, float*, double*, bool,
                              const KParams&, cudaStream_t);
int launch_adjoint_step_f32_x(int, int, bool, bool, const void*, const float*, float*, const uint32_t*, const float*,
                              const float*, const float*, float*, double*, const KParams&, cudaStream_t);
int launch_adjoint_seed_f16_x(int, const void*, const uint32_t*, const float*, const float*, float*, double*, bool,
                              const KParams&, cudaStream_t);
int launch_adjoint_step_f16_x(int, int, bool, bool, const void*, const float*, float*, const uint32_t*, const float*,
                              const float*, const float*, float*, double*, const KParams&, cudaStream_t);
int launch_adjoint_seed_bf16_x(int, const void*, const uint32_t*, const float*, const float*, float*, double*, bool,
                               const KParams&, cudaStream_t);
int launch_adjoint_step_bf16_x(int, int, bool, bool, const void*, const float*, float*, const uint32_t*, const float*,
                               const float*, const float*, float*, double*, const KParams&, cudaStream_t);

// the local chemical-potential model, D2V9 and D3V19 (lbm_adjoint_*_lmu.cu)
int launch_adjoint_step_f32_lmu(int, int, bool, bool, const void*, const float*, float*, const uint32_t*,
                                const float*, const float*, const float*, float*, double*, const KParams&,
                                cudaStream_t);
int launch_adjoint_step_f16_lmu(int, int, bool, bool, const void*, const float*, float*, const uint32_t*,
                                const float*, const float*, const float*, float*, double*, const KParams&,
                                cudaStream_t);
int launch_adjoint_step_bf16_lmu(int, int, bool, bool, const void*, const float*, float*, const uint32_t*,
                                 const float*, const float*, const float*, float*, double*, const KParams&,
                                 cudaStream_t);

namespace {
__global__ void k_fold_partials(float* __restrict__ part, double* __restrict__ acc, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        acc[i] += (double)part[i];
        part[i] = 0.f;
    }
}
}  // namespace

int launch_fold_partials(float* part, double* acc, int64_t n, cudaStream_t s) {
    if (n <= 0) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256, cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    k_fold_partials<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(part, acc, n);
    return 1;
}

int64_t adjoint_slot_count(const KParams& p) {
    Launch l = adjk::grid_of(p);
    return (int64_t)l.grid.x * l.grid.y * adjk::kSlots;
}

int launch_adjoint_seed(int vel, int storage, const void* P, const uint32_t* nbr, const float* w_rho,
                        const float* w_j, float* lam, double* slots, bool in_window, const KParams& p,
                        cudaStream_t s) {
    if (vel == LBM_D3V27 || vel == LBM_D1V3) {
        if (storage == LBM_F16_DEV)
            return launch_adjoint_seed_f16_x(vel, P, nbr, w_rho, w_j, lam, slots, in_window, p, s);
        if (storage == LBM_BF16_DEV)
            return launch_adjoint_seed_bf16_x(vel, P, nbr, w_rho, w_j, lam, slots, in_window, p, s);
        return launch_adjoint_seed_f32_x(vel, P, nbr, w_rho, w_j, lam, slots, in_window, p, s);
    }
    if (storage == LBM_F16_DEV) return launch_adjoint_seed_f16(vel, P, nbr, w_rho, w_j, lam, slots, in_window, p, s);
    if (storage == LBM_BF16_DEV)
        return launch_adjoint_seed_bf16(vel, P, nbr, w_rho, w_j, lam, slots, in_window, p, s);
    return launch_adjoint_seed_f32(vel, P, nbr, w_rho, w_j, lam, slots, in_window, p, s);
}

int launch_adjoint_step(int vel, int storage, int force, bool efield, bool in_window, const void* P,
                        const float* lam_in, float* lam_out, const uint32_t* nbr, const float* Ef,
                        const float* w_rho, const float* w_j, float* gE, double* slots, const KParams& p,
                        cudaStream_t s) {
    if (p.lmu_tab && (vel == LBM_D2V9 || vel == LBM_D3V19)) {
        if (storage == LBM_F16_DEV)
            return launch_adjoint_step_f16_lmu(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho,
                                               w_j, gE, slots, p, s);
        if (storage == LBM_BF16_DEV)
            return launch_adjoint_step_bf16_lmu(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho,
                                                w_j, gE, slots, p, s);
        return launch_adjoint_step_f32_lmu(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho, w_j,
                                           gE, slots, p, s);
    }
    if (vel == LBM_D3V27 || vel == LBM_D1V3) {
        if (storage == LBM_F16_DEV)
            return launch_adjoint_step_f16_x(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho, w_j,
                                             gE, slots, p, s);
        if (storage == LBM_BF16_DEV)
            return launch_adjoint_step_bf16_x(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho, w_j,
                                              gE, slots, p, s);
        return launch_adjoint_step_f32_x(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE,
                                         slots, p, s);
    }
    if (storage == LBM_F16_DEV)
        return launch_adjoint_step_f16(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE,
                                       slots, p, s);
    if (storage == LBM_BF16_DEV)
        return launch_adjoint_step_bf16(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE,
                                        slots, p, s);
    return launch_adjoint_step_f32(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE, slots,
                                   p, s);
}

}  // namespace lbm
