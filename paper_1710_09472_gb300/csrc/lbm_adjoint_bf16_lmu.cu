// Reverse-step kernels of the local chemical-potential model (lbm_set_local_mu)
// for StoreBF16 storage, D2V9 and D3V19 (see lbm_adjoint.cuh).
#include "lbm_adjoint.cuh"

namespace lbm {
int launch_adjoint_step_bf16_lmu(int vel, int force, bool efield, bool in_window, const void* P, const float* lam_in,
                            float* lam_out, const uint32_t* nbr, const float* Ef, const float* w_rho,
                            const float* w_j, float* gE, double* slots, const KParams& p, cudaStream_t s) {
    return adjk::step_storage<StoreBF16, 2>(vel, force, efield, in_window, P, lam_in, lam_out, nbr, Ef, w_rho, w_j, gE,
                                        slots, p, s);
}
}  // namespace lbm
