// Reverse-step kernels instantiated for StoreF32 storage, D2V9 and D3V19 (see lbm_adjoint.cuh).
#include "lbm_adjoint.cuh"

namespace lbm {
int launch_adjoint_seed_f32(int vel, const void* P, const uint32_t* nbr, const float* w_rho, const float* w_j,
                        float* lam, double* slots, bool in_window, const KParams& p, cudaStream_t s) {
    return adjk::seed_storage<StoreF32, 0>(vel, P, nbr, w_rho, w_j, lam, slots, in_window, p, s);
}
int launch_adjoint_step_f32(int vel, int force, bool efield, bool in_window, const void* P, const float* lam_in,
                        float* lam_out, const uint32_t* nbr, const float* Ef, const float* w_rho,
                        const float* w_j, float* gE, double* slots, const KParams& p, cudaStream_t s) {
    return adjk::step_storage<StoreF32, 0>(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE,
                                    slots, p, s);
}
}  // namespace lbm
