// Step kernels instantiated for StoreF16 storage, D3V27 and D1V3 (see lbm_step.cuh).
#include "lbm_step.cuh"

namespace lbm {
int launch_step_f16_x(int vel, int force, bool efield, bool sr, const void* fin, void* fout, const uint32_t* nbr,
                      const float* Ef, const KParams& p, cudaStream_t s) {
    return stepk::launch_storage<StoreF16, true, 1>(vel, force, efield, sr, fin, fout, nbr, Ef, p, s);
}
}  // namespace lbm
