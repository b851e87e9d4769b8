// Step kernels instantiated for StoreF16 storage, D2V9 and D3V19 (see lbm_step.cuh).
#include "lbm_step.cuh"

namespace lbm {
int launch_step_f16(int vel, int force, bool efield, bool sr, const void* fin, void* fout, const uint32_t* nbr,
                      const float* Ef, const KParams& p, cudaStream_t s) {
    return stepk::launch_storage<StoreF16, true, 0>(vel, force, efield, sr, fin, fout, nbr, Ef, p, s);
}
}  // namespace lbm
