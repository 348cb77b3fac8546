// Per-gate noise-site unraveling and the standalone batch kernel.
#pragma once

#include "common.cuh"
#include "unravel.cuh"
#include "unravel_iface.h"

namespace lemps {

// ---- noise-site unraveling, sampling and the combined 4x4 operator ----------


// rho' = M rho M^dagger for a 4x4 M (row-major) and 4x4 rho.
__device__ inline void conj4(const zd* m, const zd* rho, zd* out) {
  zd tmp[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      zd acc = mk(0.0, 0.0);
      for (int k = 0; k < 4; ++k) cfma(acc, m[i * 4 + k], rho[k * 4 + j]);
      tmp[i * 4 + j] = acc;
    }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      zd acc = mk(0.0, 0.0);
      for (int k = 0; k < 4; ++k) cfma(acc, tmp[i * 4 + k], conj(m[j * 4 + k]));
      out[i * 4 + j] = acc;
    }
}

// One noise site: choose the Kraus set for the target's reduced state rho_t
// (trace 1), sample with u, return the applied single-qubit operator
// K_i / sqrt(p_i) in op.  Returns the branch index or -2 on numerical failure.
__device__ __noinline__ int noise_site(const zd* rho_t, const LayerDev& L, double u, zd* op, double* p_out) {
  zd kset[4 * kMaxKraus];
  int r = 4;
  if (L.mode == 0) {
    if (!unr::optimal_unraveling(rho_t, L.kraus, L.r, kset)) return -2;
  } else {
    r = L.r;
    for (int i = 0; i < 4 * r; ++i) kset[i] = L.kraus[i];
  }
  double p[kMaxKraus];
  unr::branch_weights(kset, r, rho_t, p);
  double cs[kMaxKraus], acc = 0.0;
  for (int k = 0; k < r; ++k) {
    if (!isfinite(p[k])) return -2;
    acc += p[k];
    cs[k] = acc;
  }
  double thr = u * cs[r - 1];
  int idx = r - 1;
  for (int k = 0; k < r; ++k)
    if (thr < cs[k]) { idx = k; break; }
  double pk = p[idx];
  if (!(pk > 0.0)) return -2;
  double sc = 1.0 / sqrt(pk);
  for (int i = 0; i < 4; ++i) op[i] = sc * kset[idx * 4 + i];
  *p_out = pk / cs[r - 1];
  return idx;
}



__global__ void k_unravel_gate(GateState s, LayerDev L) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.B) return;
  const zd* g = L.gates + 16 * L.gate_local;
  zd rho[16];
  double tr = 0.0;
  for (int i = 0; i < 16; ++i) rho[i] = s.rho12[t * 16 + i];
  tr = rho[0].re + rho[5].re + rho[10].re + rho[15].re;
  zd T[16];
  for (int i = 0; i < 16; ++i) T[i] = g[i];
  int8_t br0 = -1, br1 = -1;
  if (!(tr > 0.0) || !isfinite(tr)) {
    s.status[t] |= (tr == 0.0) ? TS_NORM : TS_NAN;
  } else {
    for (int i = 0; i < 16; ++i) rho[i] = (1.0 / tr) * rho[i];
    const uint64_t tg = (uint64_t)(L.traj_offset + t);
    bool active = true;
    if (L.coin_p < 1.0) active = philox_uniform(L.seed, tg, (uint64_t)L.gate_global, 2) < L.coin_p;
    if (active) {
      zd r1[16];
      conj4(g, rho, r1);  // after the gate
      // slot 0: target = first qubit, rho_A[s][t] = sum_x r1[(s x),(t x)]
      zd ra[4];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) ra[a * 2 + b] = r1[(2 * a) * 4 + 2 * b] + r1[(2 * a + 1) * 4 + 2 * b + 1];
      zd m1[4], m2[4];
      double p0, p1;
      int i0 = noise_site(ra, L, philox_uniform(L.seed, tg, (uint64_t)L.gate_global, 0), m1, &p0);
      if (i0 < 0) {
        s.status[t] |= TS_NAN;
      } else {
        zd mm[16];
        for (int a = 0; a < 2; ++a)
          for (int x = 0; x < 2; ++x)
            for (int b = 0; b < 2; ++b)
              for (int y = 0; y < 2; ++y) mm[(2 * a + x) * 4 + 2 * b + y] = (x == y) ? m1[a * 2 + b] : mk(0.0, 0.0);
        zd r2[16];
        conj4(mm, r1, r2);
        zd rb[4];
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) rb[a * 2 + b] = r2[a * 4 + b] + r2[(2 + a) * 4 + 2 + b];
        double trb = rb[0].re + rb[3].re;
        for (int i = 0; i < 4; ++i) rb[i] = (1.0 / trb) * rb[i];
        int i1 = noise_site(rb, L, philox_uniform(L.seed, tg, (uint64_t)L.gate_global, 1), m2, &p1);
        if (i1 < 0) {
          s.status[t] |= TS_NAN;
        } else {
          br0 = (int8_t)i0;
          br1 = (int8_t)i1;
          // T = (m1 (x) m2) G
          zd k12[16];
          for (int a = 0; a < 2; ++a)
            for (int x = 0; x < 2; ++x)
              for (int b = 0; b < 2; ++b)
                for (int y = 0; y < 2; ++y) k12[(2 * a + x) * 4 + 2 * b + y] = m1[a * 2 + b] * m2[x * 2 + y];
          for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
              zd acc = mk(0.0, 0.0);
              for (int k = 0; k < 4; ++k) cfma(acc, k12[i * 4 + k], g[k * 4 + j]);
              T[i * 4 + j] = acc;
            }
        }
      }
    }
    // keep the trajectory normalized: Theta has norm sqrt(tr)
    double sc = 1.0 / sqrt(tr);
    for (int i = 0; i < 16; ++i) T[i] = sc * T[i];
  }
  for (int i = 0; i < 16; ++i) s.top[t * 16 + i] = T[i];
  if (L.blog) {
    L.blog[t] = br0;
    L.blog[s.B + t] = br1;
  }
}

// ---- standalone unraveling ---------------------------------------------------------
__global__ void k_unravel_batch(const zd* rho, const zd* kraus, int r, int64_t batch, zd* kout, double* e_av) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  zd rh[4];
  for (int i = 0; i < 4; ++i) rh[i] = rho[b * 4 + i];
  double tr = rh[0].re + rh[3].re;
  for (int i = 0; i < 4; ++i) rh[i] = (1.0 / tr) * rh[i];
  zd ks[16];
  if (!unr::optimal_unraveling(rh, kraus, r, ks)) {
    for (int i = 0; i < 16; ++i) ks[i] = mk<double>(NAN, NAN);
  }
  double p[4];
  double e = unr::branch_weights(ks, 4, rh, p);
  for (int i = 0; i < 16; ++i) kout[b * 16 + i] = ks[i];
  if (e_av) e_av[b] = e;
}



}  // namespace lemps
