// Interface between the host orchestration and the noise-site kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace lemps {

// Operators of a Kraus set sampled as given (the optimal remix takes at most 4).
constexpr int kMaxKraus = 8;

struct LayerDev {
  const zd* gates;     // [n_gates][16]
  const zd* kraus;     // [r][4]
  int32_t r;
  double coin_p;
  int32_t mode;        // 0 optimal, 1 given (the Haar-optimal mode arrives here as given)
  uint64_t seed;
  int64_t traj_offset;
  int64_t gate_global;  // global index of this gate
  int32_t gate_local;
  int8_t* blog;         // branch log slot for this gate: [2][B] or null
};

// Per-trajectory state read and written by the noise-site kernel.
struct GateState {
  const zd* rho12;   // [B][16]
  zd* top;           // [B][16]
  int32_t* status;   // [B]
  int64_t B;
};

void launch_unravel_gate(const GateState& s, const LayerDev& L, cudaStream_t st);
void launch_unravel_batch(const zd* rho, const zd* kraus, int r, int64_t batch, zd* kout, double* e_av, cudaStream_t st);

}  // namespace lemps
