// Noise-site kernels: per-gate unraveling + sampling for every trajectory,
// and the standalone batched unraveling.  Compiled once (FP64).
#include <cuda_runtime.h>

#include "unravel_kernels.cuh"

namespace lemps {

void launch_unravel_gate(const GateState& s, const LayerDev& L, cudaStream_t st) {
  // FP64-bound per-thread work: small CTAs spread the batch over every SM.
  const unsigned grid = (unsigned)((s.B + 31) / 32);
  k_unravel_gate<<<grid, 32, 0, st>>>(s, L);
}

void launch_unravel_batch(const zd* rho, const zd* kraus, int r, int64_t batch, zd* kout, double* e_av, cudaStream_t st) {
  const unsigned grid = (unsigned)((batch + 31) / 32);
  k_unravel_batch<<<grid, 32, 0, st>>>(rho, kraus, r, batch, kout, e_av);
}

}  // namespace lemps
