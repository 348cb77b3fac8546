// Noise-site kernels: per-gate unraveling + sampling for every trajectory,
// and the standalone batched unraveling.  Compiled once (FP64).
#include <cuda_runtime.h>

#include "unravel_kernels.cuh"

namespace lemps {

namespace {
// One problem per thread, FP64-bound (a GB300 SM retires about two FP64 FMAs
// per cycle).  The batch is spread evenly over every SM: ceil(B / #SMs)
// threads per CTA (at most 32), so that no SM's FP64 pipe holds a whole warp
// of problems while others idle.
int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 1;
    cached[dev] = c;
  }
  return cached[dev];
}
void spread(int64_t n, unsigned* grid, unsigned* block) {
  const int64_t nsm = sm_count();
  int64_t tpb = (n + nsm - 1) / nsm;
  if (tpb < 1) tpb = 1;
  if (tpb > 32) tpb = 32;
  *block = (unsigned)tpb;
  *grid = (unsigned)((n + tpb - 1) / tpb);
}
}  // namespace

void launch_unravel_gate(const GateState& s, const LayerDev& L, cudaStream_t st) {
  unsigned grid, block;
  spread(s.B, &grid, &block);
  k_unravel_gate<<<grid, block, 0, st>>>(s, L);
}

void launch_unravel_batch(const zd* rho, const zd* kraus, int r, int64_t batch, zd* kout, double* e_av, cudaStream_t st) {
  unsigned grid, block;
  spread(batch, &grid, &block);
  k_unravel_batch<<<grid, block, 0, st>>>(rho, kraus, r, batch, kout, e_av);
}

}  // namespace lemps
