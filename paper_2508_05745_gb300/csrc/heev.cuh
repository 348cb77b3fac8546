// Batched Hermitian eigensolver for the truncating split (one CTA per
// trajectory): Householder tridiagonalization, bisection on Sturm counts for
// the kept eigenvalues, inverse iteration for their eigenvectors,
// Gram-Schmidt re-orthonormalization, and back-transformation.
//
// Only the top `keep` eigenpairs are formed, keep = min(chi_max, #{l >
// cutoff * trace}, n); the count comes from one Sturm sequence at
// cutoff * trace, so eigenvalues that will be discarded are never computed.
//
// Layout (buffers 16-byte aligned, n even): G (n x n row-major, Hermitian)
// in ws1, overwritten.  Householder vectors in ws3 (row j holds sqrt(2) v_j,
// v_j of unit norm, entries > j), in the back-transformation type.
// Eigenvectors are written column-major to ws2 in that type: U[k * n + i],
// k < keep.  Eigenvalues (double, descending) to
// evals[0..keep), keep and the trace to kept[] / trace[].
#pragma once

#include <type_traits>

#include "common.cuh"

namespace lemps {

template <class R>
struct HeevView {
  cpx<R>* ws1;      // Gram matrix, then the inverse-iteration vectors
  cpx<R>* ws2;      // eigenvectors (output)
  cpx<R>* ws3;      // Householder vectors
  int64_t ws_stride;
  double* evals;    // [B][2 chi]
  int32_t* kept;    // [B]
  double* trace;    // [B]
  int32_t* bond;    // [B][n+1]
  int32_t* status;  // [B] TrajStatus bits
  int32_t nq;       // qubits (bond row length n+1)
  int32_t chi;
  int64_t B;
};

// Number of eigenvalues of the real symmetric tridiagonal (d, e) that are
// strictly greater than x (Sturm sequence of T - x I with a pivot guard), in
// FP64 on range-normalized data (|d_i|, e_i^2 of order 1 or less,
// pivmin >= 1e-30): the quotient e^2 / q is e^2 r, where r is the FP32
// reciprocal of q refined by two Newton-Raphson steps r <- r + r (1 - q r)
// (each step doubles the correct bits, 24 -> 48 -> the full 53); the sign
// test and the pivot guard |q| < pivmin -> q = -pivmin read the bit pattern.
// On GB300 every FP64 instruction (add, compare, min/max as well as FMA)
// issues at 1/64 of the FP32 rate, so this count keeps to six of them per
// step.  Normalized |q| stays within [1e-30, 1e31], inside the FP32 range.
__device__ __forceinline__ int sturm_greater_f64(const double* d, const double* e2, int n, double x, double pivmin) {
  const long long pbits = __double_as_longlong(pivmin);
  const long long nbits = __double_as_longlong(-pivmin);
  int neg = 0;
  auto guard = [&](double v) {
    long long b = __double_as_longlong(v);
    if ((b & 0x7fffffffffffffffLL) < pbits) b = nbits;
    neg += (int)((unsigned long long)b >> 63);
    return __longlong_as_double(b);
  };
  double q = guard(d[0] - x);
  for (int i = 1; i < n; ++i) {
    double r = (double)__frcp_rn((float)q);
    r = fma(r, fma(-q, r, 1.0), r);
    r = fma(r, fma(-q, r, 1.0), r);
    q = guard(fma(-e2[i - 1], r, d[i] - x));
  }
  return n - neg;
}

// The Sturm count at x together with S = d/dx ln|det(T - x I)| =
// sum_i 1 / (x - lambda_i) (the Newton step for det(T - x I) is -1 / S):
// with q_i = (d_i - x) - e_{i-1}^2 / q_{i-1}, det = prod q_i and S = sum
// q_i' / q_i, q_i' = -1 + e_{i-1}^2 q_{i-1}' / q_{i-1}^2.  Same reciprocal
// and guards as sturm_greater_f64.
__device__ __forceinline__ int sturm_newton_f64(const double* d, const double* e2, int n, double x, double pivmin,
                                                double& S) {
  const long long pbits = __double_as_longlong(pivmin);
  const long long nbits = __double_as_longlong(-pivmin);
  int neg = 0;
  auto guard = [&](double v) {
    long long b = __double_as_longlong(v);
    if ((b & 0x7fffffffffffffffLL) < pbits) b = nbits;
    neg += (int)((unsigned long long)b >> 63);
    return __longlong_as_double(b);
  };
  auto rcp = [](double q) {
    double r = (double)__frcp_rn((float)q);
    r = fma(r, fma(-q, r, 1.0), r);
    return fma(r, fma(-q, r, 1.0), r);
  };
  double q = guard(d[0] - x), qp = -1.0, s = 0.0;
  for (int i = 1; i < n; ++i) {
    const double r = rcp(q);
    s = fma(qp, r, s);
    const double tq = e2[i - 1] * r;
    qp = fma(tq * r, qp, -1.0);
    q = guard((d[i] - x) - tq);
  }
  S = fma(qp, rcp(q), s);
  return n - neg;
}

// The same count and S in FP32, on FP32 copies of the range-normalized
// tridiagonal: 64 times cheaper per instruction than FP64 on this GPU, and
// accurate to about eps_32 ||T||, which is all it is used for (a starting
// point and a bracket that FP64 counts then confirm).
__device__ __forceinline__ int sturm_newton_f32(const float* d, const float* e2, int n, float x, float pivmin,
                                                float& S) {
  int neg = 0;
  auto guard = [&](float v) {
    if (fabsf(v) < pivmin) v = -pivmin;
    neg += v < 0.f;
    return v;
  };
  float q = guard(d[0] - x), qp = -1.f, s = 0.f;
  for (int i = 1; i < n; ++i) {
    const float r = __frcp_rn(q);
    s = fmaf(qp, r, s);
    const float tq = e2[i - 1] * r;
    qp = fmaf(tq * r, qp, -1.f);
    q = guard((d[i] - x) - tq);
  }
  S = fmaf(qp, __frcp_rn(q), s);
  return n - neg;
}

// The back-transformation stores each unit reflector v as u = sqrt(2) v, so that
// applying I - 2 v v^dagger = I - u u^dagger needs no scaling of the dots.
constexpr double kSqrt2 = 1.4142135623730950488;

// Deterministic start vector entries in [0.5, 1.5) (a hash of (k, i)).
__device__ __forceinline__ float start_entry(int k, int i) {
  uint32_t h = (uint32_t)k * 0x9E3779B1u ^ (uint32_t)(i + 1) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return 0.5f + (float)(h >> 8) * (1.0f / 16777216.0f);
}

// Shared-memory budget of k_heev (dynamic): a packed lower triangle of the
// trailing block once it fits, later the eigenvector block for Gram-Schmidt.
template <class R>
struct HeevSmem {
  static constexpr int kBytes = 196 * 1024;
  static constexpr int kCap = kBytes / (int)sizeof(cpx<R>);   // complex entries
};

__device__ __forceinline__ int pidx(int r, int c) { return r * (r + 1) / 2 + c; }

// Two adjacent complex entries from 16-byte aligned global memory.
__device__ __forceinline__ void load_pair(const cpx<float>* p, cpx<float>& a, cpx<float>& b) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  a = mk(t.x, t.y);
  b = mk(t.z, t.w);
}
__device__ __forceinline__ void load_pair(const cpx<double>* p, cpx<double>& a, cpx<double>& b) {
  const double2 t0 = reinterpret_cast<const double2*>(p)[0], t1 = reinterpret_cast<const double2*>(p)[1];
  a = mk(t0.x, t0.y);
  b = mk(t1.x, t1.y);
}

// Complex updates written as chains of fused multiply-adds: on GB300 each FP64
// instruction (FMA, multiply or add alike) takes one slot of the 1/64-rate FP64
// pipe, so x - a b as two multiplies and adds per component costs half as
// much again as the fused form.
// x - v1 conj(w1) - w2 conj(v2): one entry of a Hermitian rank-2 update.
template <class R>
__device__ __forceinline__ cpx<R> rank2_sub(cpx<R> x, cpx<R> v1, cpx<R> w1, cpx<R> w2, cpx<R> v2) {
  x.re = fma(-v1.re, w1.re, fma(-v1.im, w1.im, fma(-w2.re, v2.re, fma(-w2.im, v2.im, x.re))));
  x.im = fma(-v1.im, w1.re, fma(v1.re, w1.im, fma(-w2.im, v2.re, fma(w2.re, v2.im, x.im))));
  return x;
}
// acc -= a b
template <class R>
__device__ __forceinline__ void cfms(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(-a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(-a.re, b.im, fma(-a.im, b.re, acc.im));
}
// Sum over the block, returned to every thread: a warp butterfly, then each
// warp sums the per-warp totals by a second butterfly (cheaper on the FP64
// pipe than every thread adding them up).  `scratch` holds 32 values.
__device__ __forceinline__ double block_sum_f64(double v, double* scratch) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  return warp_sum(lane < nw ? scratch[lane] : 0.0);
}

// y_c <- (I - u u^dagger) y_c for a warp's NCOL columns (u = sqrt(2) v is the
// stored form of the unit reflector v) (PER entries per
// lane, row lane + 32 a).  Groups a < A0 are zero in v and are skipped at
// compile time; the NCOL complex dots are summed over the warp by one
// reduce-scatter / broadcast butterfly.
template <class R, int NCOL, int PER, int A0>
__device__ __forceinline__ void bt_reflector(cpx<R> (&y)[NCOL][PER], const cpx<R>* v, int lane, int nper) {
  constexpr int NV = 2 * NCOL;
  R d[NV];
#pragma unroll
  for (int e = 0; e < NV; ++e) d[e] = 0;
  cpx<R> vr[PER];
#pragma unroll
  for (int a = A0; a < PER; ++a) {
    vr[a] = (a < nper) ? v[lane + 32 * a] : mk<R>(0, 0);
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
      // d_c += conj(v_i) y_c[i]
      d[2 * c] = fma(vr[a].re, y[c][a].re, fma(vr[a].im, y[c][a].im, d[2 * c]));
      d[2 * c + 1] = fma(vr[a].re, y[c][a].im, fma(-vr[a].im, y[c][a].re, d[2 * c + 1]));
    }
  }
  const R tot = warp_reduce_scatter<NV>(d, lane);
  R dd[NV];
#pragma unroll
  for (int e = 0; e < NV; ++e) dd[e] = __shfl_sync(0xffffffffu, tot, Scatter<NV>::source(e));
#pragma unroll
  for (int a = A0; a < PER; ++a)
#pragma unroll
    for (int c = 0; c < NCOL; ++c) cfms(y[c][a], vr[a], mk<R>(dd[2 * c], dd[2 * c + 1]));
}

// mode / q select the matrix size as in gram_size(); want_vectors = 0 returns
// eigenvalues only (all n of them when cutoff = 0).  R is the arithmetic of
// the tridiagonalization, the eigenvalues and the tridiagonal eigenvectors;
// RB that of the back-transformation U = Q D z: the reflectors are stored
// and applied, and U is written, in cpx<RB> (each trajectory's slots of ws3
// and ws2, of ws_stride complex128 entries, viewed as cpx<RB> arrays).  Applying the reflectors is
// backward stable, so its rounding error (about n eps_RB relative) does not
// depend on the eigenvalue gaps, unlike the eigenpairs of a perturbed Gram.
template <class R, class RB = R>
__global__ void __launch_bounds__(512) k_heev(HeevView<R> s, int q, int mode, double cutoff, int keep_max,
                                               int want_vectors) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  const int32_t* bd = s.bond + t * (s.nq + 1);
  const int n = mode == 0 ? 2 * bd[q] : (mode == 1 ? 2 * bd[q + 2] : bd[q + 1]);
  cpx<R>* G = s.ws1 + t * s.ws_stride;
  // the cpx<RB> views start at this trajectory's own slot: the slot of the
  // next trajectories stays untouched whatever RB is (the phase-1 scratch of
  // another CTA may live there)
  cpx<RB>* Hv = reinterpret_cast<cpx<RB>*>(s.ws3 + t * s.ws_stride);
  cpx<RB>* U = reinterpret_cast<cpx<RB>*>(s.ws2 + t * s.ws_stride);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  extern __shared__ __align__(16) unsigned char heev_smem[];
  cpx<R>* Lp = reinterpret_cast<cpx<R>*>(heev_smem);   // packed lower triangle (trailing block)

  __shared__ R sd[256], se[256], se2[256];   // real tridiagonal: diagonal, |offdiag|, offdiag^2
  __shared__ cpx<R> sph[256];                // phases delta_i (T_real = D^dagger T_c D)
  __shared__ cpx<R> sv[256], sw[256];        // Householder vector and w of the current step
  __shared__ cpx<R> sec[256];                // complex off-diagonal e_j
  __shared__ R red[32];
  __shared__ double redd[32];
  __shared__ int s_keep;
  __shared__ double s_tr;
  __shared__ cpx<R> s_hh[3];                 // Householder scalars of a step

  // trace (FP64) for the cutoff and the discarded weight
  double trp = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) trp += (double)G[(int64_t)i * n + i].re;
  trp = block_sum_f64(trp, redd);
  if (threadIdx.x == 0) s_tr = trp;

  // ---- phase 1: tridiagonalization ------------------------------------------
  // The steps whose trailing block does not fit in shared memory run in
  // panels of 32 (blocked LATRD): G stays in global memory (L2), and the
  // rank-2 updates G_eff = G - sum_k (v_k w_k^dagger + w_k v_k^dagger) of the
  // panel's earlier steps are applied on the fly to the column and to the
  // matvec; between panels, and after the last one, a rank-2b update brings
  // the trailing block of G up to date.  The block G[j0:, j0:] left at the
  // end is packed into shared memory and the remaining steps stay on chip.
  // V and W (j0 x n each, row k = step k) live in shared memory when they
  // fit, else in ws2 (which receives the eigenvectors only at the end).
  int j0 = 0;
  while ((n - j0) * (n - j0 + 1) / 2 > HeevSmem<R>::kCap) ++j0;
  // V and W sit in shared memory (unused until the packing) when they fit
  const bool vw_sm = 2 * (size_t)j0 * n * sizeof(cpx<R>) <= (size_t)HeevSmem<R>::kBytes;
  cpx<R>* Vp = vw_sm ? Lp : s.ws2 + t * s.ws_stride;   // ws2 in R until U is written
  cpx<R>* Wp = Vp + (int64_t)j0 * n;
  // G[jt:, jt:] -= sum_{k in [kb0, kb1)} v_k w_k^dagger + w_k v_k^dagger, both
  // triangles (the panel matvec reads whole rows).  The lower triangle's
  // mt (mt + 1) / 2 entries are dealt out to the threads one at a time: an
  // FP64 instruction costs the pipe the same with any number of active lanes,
  // so tiles that straddle the diagonal or the edge would pay for the entries
  // they skip.  V and W are staged in shared memory in chunks of kch steps
  // (with V and W already in shared memory they are used in place).
  auto panel_update = [&](int kb0, int kb1, int jt) {
    const int mt = n - jt, nk = kb1 - kb0;
    if (nk <= 0 || mt <= 0) return;
    const int kch = vw_sm ? nk : min(nk, (int)(HeevSmem<R>::kBytes / (2 * (size_t)mt * sizeof(cpx<R>))));
    const int ldk = vw_sm ? n : mt;
    const int ne = mt * (mt + 1) / 2;
    for (int k0 = 0; k0 < nk; k0 += kch) {
      const int kc = min(kch, nk - k0);
      if (!vw_sm) {
        for (int e = threadIdx.x; e < kc * mt; e += blockDim.x) {
          const int kk = e / mt, i = e - kk * mt;
          Lp[e] = Vp[(int64_t)(kb0 + k0 + kk) * n + jt + i];
          Lp[(int64_t)kch * mt + e] = Wp[(int64_t)(kb0 + k0 + kk) * n + jt + i];
        }
      }
      __syncthreads();
      const cpx<R>* vs = vw_sm ? Vp + (int64_t)(kb0 + k0) * n + jt : Lp;
      const cpx<R>* ws = vw_sm ? Wp + (int64_t)(kb0 + k0) * n + jt : Lp + (int64_t)kch * mt;
      for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        // entry e = i (i + 1) / 2 + c of the packed lower triangle
        int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (i * (i + 1) / 2 > e) --i;
        while ((i + 1) * (i + 2) / 2 <= e) ++i;
        const int c = e - i * (i + 1) / 2;
        cpx<R> acc = mk<R>(0, 0);
#pragma unroll 4
        for (int kk = 0; kk < kc; ++kk) {
          cfmac(acc, ws[kk * ldk + c], vs[kk * ldk + i]);
          cfmac(acc, vs[kk * ldk + c], ws[kk * ldk + i]);
        }
        cpx<R>* g = G + (int64_t)(jt + i) * n + (jt + c);
        *g = *g - acc;
        if (c < i) {
          cpx<R>* gt = G + (int64_t)(jt + c) * n + (jt + i);
          *gt = *gt - conj(acc);
        }
      }
      __syncthreads();
    }
  };
  // Panels of kPanelWidth steps (blocked LATRD): the corrections of a column
  // and of a matvec only involve the steps of the current panel (their cost
  // grows with the panel width), and G is brought up to date between panels.
  constexpr int kPanelWidth = 32;
  int jp = 0;   // first step of the current panel
  for (int j = 0; j < j0 && j + 2 < n; ++j) {
    if (j - jp == kPanelWidth) {
      panel_update(jp, j, j);
      jp = j;
    }
    const int m = n - j - 1;
    // column j of G_eff below the diagonal, and its diagonal entry
    R part = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const int gi = j + 1 + i;
      cpx<R> x = G[(int64_t)gi * n + j];
      for (int k = jp; k < j; ++k)
        x = rank2_sub(x, Vp[(int64_t)k * n + gi], Wp[(int64_t)k * n + j], Wp[(int64_t)k * n + gi], Vp[(int64_t)k * n + j]);
      sv[i] = x;
      if (i > 0) part = fma(x.re, x.re, fma(x.im, x.im, part));
    }
    if (threadIdx.x == 0) {
      R dj = G[(int64_t)j * n + j].re;
      for (int k = jp; k < j; ++k) dj -= (R)2 * cdot(Wp[(int64_t)k * n + j], Vp[(int64_t)k * n + j]).re;
      sd[j] = dj;
    }
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    // the Householder scalars of the step, by one warp (FP64 instructions
    // cost the pipe the same with one lane or 32 active)
    if (warp == 0) {
      const R sig = warp_sum(lane < nwarp ? red[lane] : (R)0);
      if (lane == 0) {
        const cpx<R> x0 = sv[0];
        const R ax0 = sqrt(norm2(x0));
        const R nrm = sqrt(sig + ax0 * ax0);
        cpx<R> alpha = x0, v0 = mk<R>(0, 0);
        R inv = 0;
        if (sig > (R)0) {
          const cpx<R> ph = (ax0 > 0) ? mk<R>(x0.re / ax0, x0.im / ax0) : mk<R>(1, 0);
          alpha = mk<R>(-nrm * ph.re, -nrm * ph.im);
          inv = (R)1 / sqrt(sig + (ax0 + nrm) * (ax0 + nrm));
          v0 = (x0 - alpha) * inv;
        }
        s_hh[0] = alpha;
        s_hh[1] = v0;
        s_hh[2] = mk<R>(inv, sig > (R)0 ? (R)1 : (R)0);
      }
    }
    __syncthreads();
    const cpx<R> alpha = s_hh[0];
    const bool reflect = s_hh[2].im != (R)0;
    if (reflect) {
      const cpx<R> v0 = s_hh[1];
      const R inv = s_hh[2].re;
      for (int i = threadIdx.x; i < m; i += blockDim.x) sv[i] = (i == 0) ? v0 : sv[i] * inv;
    }
    __syncthreads();
    if (threadIdx.x == 0) sec[j] = alpha;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const cpx<R> vi = (i > j && reflect) ? sv[i - j - 1] : mk<R>(0, 0);
      Hv[(int64_t)j * n + i] = cast<RB>(kSqrt2 * vi);
      Vp[(int64_t)j * n + i] = vi;
    }
    if (!reflect) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) Wp[(int64_t)j * n + i] = mk<R>(0, 0);
      __syncthreads();
      continue;
    }
    // corrections c1_k = w_k^dagger v, c2_k = v_k^dagger v (jp <= k < j); sph
    // is free until the end of phase 1 and holds 2 (j - jp) <= 64 entries.
    // Eight dots per warp, four lanes per dot striding along i (an FP64
    // instruction costs the same with any number of active lanes, so the lane
    // mapping keeps the ragged last iteration small), summed over the four
    // lanes by two butterfly rounds.
    cpx<R>* cc = sph;
    const int np = j - jp;   // steps of the current panel before this one
    for (int kk0 = 8 * warp; kk0 < 2 * np; kk0 += 8 * nwarp) {
      const int kk = kk0 + (lane >> 2);
      const bool live = kk < 2 * np;
      const cpx<R>* src = live ? ((kk < np) ? (Wp + (int64_t)(jp + kk) * n) : (Vp + (int64_t)(jp + kk - np) * n)) + j + 1 : Wp;
      cpx<R> a0 = mk<R>(0, 0), a1 = mk<R>(0, 0);
      int i = lane & 3;
      for (; i + 4 < m; i += 8) {
        if (live) {
          cfmac(a0, src[i], sv[i]);
          cfmac(a1, src[i + 4], sv[i + 4]);
        }
      }
      if (i < m && live) cfmac(a0, src[i], sv[i]);
      a0 += a1;
#pragma unroll
      for (int o = 2; o > 0; o >>= 1) {
        a0.re += __shfl_xor_sync(0xffffffffu, a0.re, o);
        a0.im += __shfl_xor_sync(0xffffffffu, a0.im, o);
      }
      if (live && (lane & 3) == 0) cc[kk] = a0;
    }
    // y = G_sub v from the original (read-only) G, which is served from L2:
    // eight rows per warp, four lanes per row, each lane loading two adjacent
    // entries of its row at a time (16-byte aligned: the segment starts at
    // the even column c0 <= j + 1) into two independent accumulators; the
    // four lanes of a row are summed by two butterfly rounds.
    const int c0 = (j + 1) & ~1;
    const int off = j + 1 - c0;        // 1: column c0 = j lies left of the block (weight 0)
    const int npair = (n - c0) >> 1;
    for (int r0 = 8 * warp; r0 < m; r0 += 8 * nwarp) {
      const int r = r0 + (lane >> 2);
      const bool rin = r < m;
      const cpx<R>* row = G + (int64_t)(j + 1 + (rin ? r : 0)) * n + c0;
      cpx<R> acc0 = mk<R>(0, 0), acc1 = mk<R>(0, 0);
#pragma unroll 2
      for (int p2 = lane & 3; p2 < npair; p2 += 4) {
        const int c = 2 * p2 - off;    // local index of the first entry of the pair
        if (rin) {
          const cpx<R> x0 = (c >= 0) ? sv[c] : mk<R>(0, 0), x1 = sv[c + 1];
          cpx<R> e0, e1;
          load_pair(row + 2 * p2, e0, e1);
          cfma(acc0, e0, x0);
          cfma(acc1, e1, x1);
        }
      }
      acc0 += acc1;
#pragma unroll
      for (int o = 2; o > 0; o >>= 1) {
        acc0.re += __shfl_xor_sync(0xffffffffu, acc0.re, o);
        acc0.im += __shfl_xor_sync(0xffffffffu, acc0.im, o);
      }
      if (rin && (lane & 3) == 0) sw[r] = acc0;
    }
    __syncthreads();
    // y -= sum_k v_k (w_k^dagger v) + w_k (v_k^dagger v)
    R sp = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const int gi = j + 1 + i;
      cpx<R> y = sw[i];
      for (int k = 0; k < np; ++k) {
        cfms(y, Vp[(int64_t)(jp + k) * n + gi], cc[k]);
        cfms(y, Wp[(int64_t)(jp + k) * n + gi], cc[np + k]);
      }
      sw[i] = y;
      sp = fma(sv[i].re, y.re, fma(sv[i].im, y.im, sp));
    }
    R ss = block_sum_f64(sp, red);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const cpx<R> wi = (i > j) ? (R)2 * sw[i - j - 1] - ((R)2 * ss) * sv[i - j - 1] : mk<R>(0, 0);
      Wp[(int64_t)j * n + i] = wi;
    }
    __syncthreads();
  }
  if (j0 > 0) panel_update(jp, min(j0, n - 2), j0);
  // pack the lower triangle of the trailing block G[j0:, j0:]
  const int M0 = n - j0;
  for (int r = warp; r < M0; r += nwarp)
    for (int c = lane; c <= r; c += 32) Lp[pidx(r, c)] = G[(int64_t)(j0 + r) * n + (j0 + c)];
  __syncthreads();
  // The rank-2 update of each step is applied lazily: Lp holds the trailing
  // block without the update of the previous step, whose v and y (so that
  // w = 2 y - 2 (v^dagger y) v) sit in ping-pong buffers indexed by local row.
  // A step reads its column with that correction and forms v; then one pass
  // over the trailing triangle writes the corrected entries back and forms
  // y = A v (both halves); three barriers per step.
  // The warps add their partial sums of y in 64-bit fixed point, 2^-60 ||G||
  // at most per unit (the scale is a power of two with tr * scale < 2^60):
  // integer adds are exact and associative, so y does not depend on the
  // order in which the warps add (the run is deterministic) and its error is
  // the rounding of each partial sum to the unit.  Every partial sum of
  // (A v)_r over a subset of columns is at most ||A||_2 ||v|| <= tr (A is
  // similar to a block of the Gram matrix, v a unit vector), so the sums stay
  // below 2^61; the unit, 2^-60 tr <= 2^-60 n ||G||_2, is far below the FP64
  // rounding of the dot products themselves.  The y slots hold the integers
  // (re, im) in place of the complex value; zero has the same bits in both.
  __shared__ cpx<R> sy2[256];
  __shared__ R redn[32], reds[32];
  // scale and its inverse (powers of two) in shared memory: registers are
  // scarce at 512 threads
  __shared__ double s_ysc[2];
  if (threadIdx.x == 0) {
    int tr_exp = 0;
    (void)frexp(s_tr, &tr_exp);
    s_ysc[0] = (s_tr > 0.0 && isfinite(s_tr)) ? ldexp(1.0, 60 - tr_exp) : 1.0;
    s_ysc[1] = 1.0 / s_ysc[0];
  }
  auto yget = [&](const cpx<R>* y, int X) {
    const long long* yi = reinterpret_cast<const long long*>(y) + 2 * X;
    return mk<R>((R)(__ll2double_rn(yi[0]) * s_ysc[1]), (R)(__ll2double_rn(yi[1]) * s_ysc[1]));
  };
  auto yadd = [&](cpx<R>* y, int X, int comp, double v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(y) + 2 * X + comp,
              (unsigned long long)__double2ll_rn(v * s_ysc[0]));
  };
  for (int i = threadIdx.x; i < M0; i += blockDim.x) {
    sv[i] = mk<R>(0, 0); sw[i] = mk<R>(0, 0);
    sph[i] = mk<R>(0, 0); sy2[i] = mk<R>(0, 0);
  }
  __syncthreads();
  R ssP = 0;
  int pb = 0;   // buffers of the previous step
  for (int j = j0; j + 2 < n; ++j) {
    const int jl = j - j0;     // local index of column j
    const int m = n - j - 1;   // trailing size; local rows jl+1 .. M0-1
    const int qb = pb ^ 1;
    const cpx<R>* vP = pb ? sw : sv;
    const cpx<R>* yP = pb ? sy2 : sph;
    cpx<R>* vN = qb ? sw : sv;
    cpx<R>* yN = qb ? sy2 : sph;
    auto wprev = [&](int X) { return (R)2 * yget(yP, X) - ((R)2 * ssP) * vP[X]; };
    const cpx<R> vPj = vP[jl], wPj = wprev(jl);
    // column jl below the diagonal (one entry per thread; m < blockDim.x)
    const int i = threadIdx.x;
    cpx<R> x = mk<R>(0, 0), wi = mk<R>(0, 0);
    R part = 0;
    if (i < m) {
      const int Rr = jl + 1 + i;
      wi = wprev(Rr);
      x = rank2_sub(Lp[pidx(Rr, jl)], vP[Rr], wPj, wi, vPj);
      if (i > 0) part = fma(x.re, x.re, fma(x.im, x.im, part));
    }
    part = warp_sum(part);
    if (lane == 0) redn[warp] = part;
    __syncthreads();
    // the step's Householder scalars by one warp (an FP64 instruction costs
    // the pipe the same with one lane active as with 32)
    if (warp == 0) {
      const R sig = warp_sum(lane < nwarp ? redn[lane] : (R)0);
      if (lane == 0) {
        const cpx<R> x0 = rank2_sub(Lp[pidx(jl + 1, jl)], vP[jl + 1], wPj, wprev(jl + 1), vPj);
        const R ax0 = sqrt(norm2(x0));
        const R nrm = sqrt(sig + ax0 * ax0);
        cpx<R> alpha = x0, v0 = mk<R>(0, 0);
        R inv = 0;
        if (sig > (R)0) {
          const cpx<R> ph = (ax0 > 0) ? mk<R>(x0.re / ax0, x0.im / ax0) : mk<R>(1, 0);
          alpha = mk<R>(-nrm * ph.re, -nrm * ph.im);
          inv = (R)1 / sqrt(sig + (ax0 + nrm) * (ax0 + nrm));
          v0 = (x0 - alpha) * inv;
        }
        s_hh[1] = v0;
        s_hh[2] = mk<R>(inv, 0);
        sd[j] = Lp[pidx(jl, jl)].re - (R)2 * cdot(wPj, vPj).re;
        sec[j] = alpha;
      }
    }
    __syncthreads();
    const cpx<R> vi = (i == 0) ? s_hh[1] : x * s_hh[2].re;   // zero when sig = 0 (inv = 0, v0 = 0)
    // every thread has read y of the previous step: it now becomes w
    cpx<R>* wP = const_cast<cpx<R>*>(yP);
    if (i < m) {
      vN[jl + 1 + i] = vi;
      yN[jl + 1 + i] = mk<R>(0, 0);
      wP[jl + 1 + i] = wi;
      Hv[(int64_t)j * n + (j + 1 + i)] = cast<RB>(kSqrt2 * vi);
    }
    if (i <= j) Hv[(int64_t)j * n + i] = mk<RB>(0, 0);
    __syncthreads();
    // One pass over 32 x QW slices of the trailing triangle's 32 x 32 tiles
    // (aligned to multiples of 32 in local index), lane = row r.  It applies
    // the previous update to A[r][c], c <= r, writes it back, accumulates the
    // lower half y[r] += A[r][c] v[c] in a register and the strictly-upper half
    // conj(A[r][c]) v[r] per column in QW registers, which one reduce-scatter
    // butterfly sums over the rows.  A half-warp reads 16 rows starting at a
    // multiple of 16, whose triangular offsets r (r + 1) / 2 are distinct
    // mod 16: conflict-free.  QW = 16 (half-tiles): narrower slices balance the
    // warps better but cost more in per-slice butterflies and atomics, and
    // measured slower (QW = 8: 9.0 vs 8.5 ms per chi=128 launch).
    constexpr int QW = 16, NQ = 32 / QW, NVQ = 2 * QW;
    constexpr int LGQ = Scatter<NVQ>::LG;
    const int tb0 = (jl + 1) >> 5;
    const int ntb = ((M0 - 1) >> 5) - tb0 + 1;
    const int nun = ntb * (ntb + 1) / 2 * NQ;
    R ssp = 0;
    int I = 0;   // tile row of tile tl; a warp's tl only grow, so I carries over
    for (int u = warp; u < nun; u += nwarp) {
      const int tl = u / NQ, hf = u % NQ;
      while ((I + 1) * (I + 2) / 2 <= tl) ++I;
      const int J = tl - I * (I + 1) / 2;
      const int Rr = 32 * (tb0 + I) + lane;
      const bool rin = Rr > jl && Rr < M0;
      const int cb = 32 * (tb0 + J) + QW * hf;
      cpx<R> vr = mk<R>(0, 0), wr = mk<R>(0, 0), nr = mk<R>(0, 0);
      if (rin) {
        vr = vP[Rr];
        wr = wP[Rr];
        nr = vN[Rr];
      }
      cpx<R>* rowp = Lp + (rin ? pidx(Rr, 0) : 0);
      cpx<R> acc = mk<R>(0, 0);
      bool any = false;
      R d[NVQ];
#pragma unroll
      for (int cc = 0; cc < QW; ++cc) {
        const int C = cb + cc;
        cpx<R> qv = mk<R>(0, 0);
        if (C > jl && C < M0) {
          const cpx<R> cv = vP[C], cw = wP[C], cn = vN[C];
          if (rin && C <= Rr) {
            const cpx<R> aa = rank2_sub(rowp[C], vr, cw, wr, cv);
            rowp[C] = aa;
            cfma(acc, aa, cn);
            any = true;
            if (C < Rr) cfmac(qv, aa, nr);
          }
        }
        d[2 * cc] = qv.re;
        d[2 * cc + 1] = qv.im;
      }
      if (any) {
        yadd(yN, Rr, 0, acc.re);
        yadd(yN, Rr, 1, acc.im);
        ssp = fma(nr.re, acc.re, fma(nr.im, acc.im, ssp));
      }
      const R tot = warp_reduce_scatter<NVQ>(d, lane);
      const int e = Scatter<NVQ>::index(lane);   // value 2 c + {re, im} of column cb + c
      const int Cc = cb + (e >> 1);
      if ((lane & ((1 << (5 - LGQ)) - 1)) == 0 && Cc > jl && Cc < M0) {
        if (e & 1) {
          yadd(yN, Cc, 1, tot);
          ssp = fma(vN[Cc].im, tot, ssp);
        } else {
          yadd(yN, Cc, 0, tot);
          ssp = fma(vN[Cc].re, tot, ssp);
        }
      }
    }
    ssp = warp_sum(ssp);
    if (lane == 0) reds[warp] = ssp;
    __syncthreads();
    ssP = warp_sum(lane < nwarp ? reds[lane] : (R)0);
    pb = qb;
  }
  if (threadIdx.x == 0) {
    // the last two rows, with the pending update of the last step
    const cpx<R>* vP = pb ? sw : sv;
    const cpx<R>* yP = pb ? sy2 : sph;
    auto wprev = [&](int X) { return (R)2 * yget(yP, X) - ((R)2 * ssP) * vP[X]; };
    auto aeff = [&](int X, int Y) { return Lp[pidx(X, Y)] - vP[X] * conj(wprev(Y)) - wprev(X) * conj(vP[Y]); };
    const int a = n - 2 - j0, b = n - 1 - j0;   // local indices of the last two rows
    if (n >= 2) {
      sd[n - 2] = aeff(a, a).re;
      sec[n - 2] = aeff(b, a);
    }
    sd[n - 1] = aeff(b, b).re;
  }
  __syncthreads();
  // phase normalization delta_{j+1} = delta_j e_j / |e_j|: the moduli and unit
  // factors in parallel, their running product by one thread
  for (int j = threadIdx.x; j + 1 < n; j += blockDim.x) {
    const R aa = sqrt(norm2(sec[j]));
    se[j] = aa;
    se2[j] = aa * aa;
    sv[j] = (aa > 0) ? mk<R>(sec[j].re / aa, sec[j].im / aa) : mk<R>(1, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cpx<R> dl = mk<R>(1, 0);
    sph[0] = dl;
    for (int j = 0; j + 1 < n; ++j) {
      dl = dl * sv[j];
      sph[j + 1] = dl;
    }
  }
  __syncthreads();

  // ---- phase 2: how many to keep, and the kept eigenvalues by bisection ------
  // Gerschgorin bounds and the norm of T by a block reduction (every FP64
  // instruction counts on this pipe), then T scaled by 1 / tnorm into shared
  // memory (free once the packed triangle is done): the Sturm counts run on
  // data of order one.
  __shared__ double s_gl, s_gu, s_tn;
  {
    double lo = 1e300, hi = -1e300, tn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double rad = (i > 0 ? (double)se[i - 1] : 0.0) + (i + 1 < n ? (double)se[i] : 0.0);
      lo = fmin(lo, (double)sd[i] - rad);
      hi = fmax(hi, (double)sd[i] + rad);
      tn = fmax(tn, fabs((double)sd[i]) + rad);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    }
    double* rb = reinterpret_cast<double*>(heev_smem);
    if (lane == 0) { rb[warp] = lo; rb[32 + warp] = hi; rb[64 + warp] = tn; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w2 = 1; w2 < nwarp; ++w2) {
        lo = fmin(lo, rb[w2]);
        hi = fmax(hi, rb[32 + w2]);
        tn = fmax(tn, rb[64 + w2]);
      }
      s_gl = lo; s_gu = hi; s_tn = (tn > 0.0) ? tn : 1.0;
    }
    __syncthreads();
  }
  const double tnorm = s_tn, itn = 1.0 / tnorm;
  const double eps = 2.2e-16;
  const double pivmin = 1e-30;                     // normalized units
  const double pivmin_abs = pivmin * tnorm;
  const double gl = s_gl * itn - (2 * eps + pivmin), gu = s_gu * itn + (2 * eps + pivmin);
  double* tdn = reinterpret_cast<double*>(heev_smem) + 3 * blockDim.x;   // after the grid arrays
  double* te2n = tdn + 256;
  float* tdf = reinterpret_cast<float*>(te2n + 256);   // FP32 copies for the first Newton stage
  float* te2f = tdf + 256;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    tdn[i] = (double)sd[i] * itn;
    te2n[i] = (double)se2[i] * (itn * itn);
    tdf[i] = (float)tdn[i];
    te2f[i] = (float)te2n[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int cnt = (cutoff > 0.0) ? sturm_greater_f64(tdn, te2n, n, cutoff * s_tr * itn, pivmin) : n;
    // a two-site Gram matrix has rank <= min(2 d_l, 2 d_r)
    const int rank_bound = (mode == 2) ? n : min(2 * bd[q], 2 * bd[q + 2]);
    int kp = min(cnt, min(keep_max, min(n, rank_bound)));
    s_keep = max(kp, 1);
  }
  __syncthreads();
  const int keep = s_keep;
  double* ev = s.evals + t * (2 * s.chi);
  // Brackets: one Sturm count per thread on an increasing grid of blockDim.x
  // points.  When a cutoff is set, every kept eigenvalue lies above x_lo =
  // cutoff * trace and the grid is geometric from x_lo to gu (neighbouring
  // points about 5 % apart), so each eigenvalue starts from a narrow relative
  // interval instead of [gl, gu]; else it is uniform on [gl, gu].  Any
  // increasing grid is valid, so it is formed in single precision.
  double* gx = reinterpret_cast<double*>(heev_smem);
  int* gcnt = reinterpret_cast<int*>(gx + blockDim.x);
  __syncthreads();   // the reduction scratch above overlaps gx
  {
    const int ng = blockDim.x;
    const float xlo = (float)(cutoff * s_tr * itn), xhi = (float)gu;
    const bool geo = cutoff > 0.0 && xlo > 0.0f && xlo < xhi;
    const float f = (float)threadIdx.x / (float)(ng - 1);
    const double x = geo ? (double)(xlo * exp2f(log2f(xhi / xlo) * f))
                         : gl + (gu - gl) * (double)(threadIdx.x + 1) / (double)(ng + 1);
    gx[threadIdx.x] = x;
    gcnt[threadIdx.x] = sturm_greater_f64(tdn, te2n, n, x, pivmin);
  }
  __syncthreads();
  {
    // One lane per kept eigenvalue k, on warps 0..3 only (an FP64
    // instruction costs its SMSP 64 cycles whatever the number of active
    // lanes, so more lanes per eigenvalue or more warps only add cost).
    // Safeguarded Newton on det(T - x I) inside the bracket [lo, hi] from the
    // grid: each round evaluates the Sturm count and S = d/dx ln|det| at the
    // iterate x_n, moves one end of the bracket to x_n, and steps to x_n -
    // 1 / S, or to the bracket midpoint when that leaves the bracket or does
    // not at least halve the previous step (at a repeated eigenvalue Newton
    // converges only linearly, from one side, and the far end of the bracket
    // would never move).  A
    // Newton step below tol / 4 only says that x_n is near some eigenvalue,
    // possibly a neighbour just outside the bracket, so the next point is then
    // x_n +/- tol / 2 on the side where the count puts eigenvalue k: when it
    // lands beyond the eigenvalue the bracket closes to that width.  The
    // eigenvalue is done when its bracket is tol = 4 eps ||T|| wide
    // (normalized: 4 eps): as accurate as the backward-stable reduction from
    // G allows (a few eps ||G|| absolute), which is all that the shifts of the
    // inverse iteration and the entropies need.  From the 5 % grid brackets
    // this takes about nine rounds (at most twelve for a warp of 32); a
    // multiplicity of 32 takes about seventy.
    // Most of those rounds now run in FP32 first (64 times cheaper per
    // instruction): the same safeguarded Newton on the FP32 copies down to a
    // bracket of tol32 = 4e-6.  FP64 then evaluates at its midpoint, which
    // fixes one end of the FP64 bracket from an FP64 count, and confirms the
    // other end at tol32-plus-rounding away with one more FP64 count (else the
    // grid bracket stays); the FP64 rounds below start from there.  Where FP32
    // cannot resolve eigenvalue k (below eps_32 ||T||, or inside a cluster),
    // the confirmation fails or the bracket is wide, and FP64 does the work as
    // before.
    const double tol = 4.0 * eps + pivmin;
    const float tol32 = 4e-6f;
    constexpr int kNewtonWarps = 4;
    if (warp < kNewtonWarps) {
      for (int kb = 0; kb < keep; kb += 32 * kNewtonWarps) {
        const int k = kb + warp * 32 + lane;
        double lo = gl, hi = gu;
        if (k < keep) {
          // grid counts do not increase along the grid: a = last point below
          // eigenvalue k (count > k), b = a + 1 the first at or above it
          int a = -1, b = (int)blockDim.x;
          while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (gcnt[mid] > k) a = mid;
            else b = mid;
          }
          if (a >= 0) lo = gx[a];
          if (b < (int)blockDim.x) hi = gx[b];
        }
        bool done = k >= keep;
        double xn = 0.5 * (lo + hi), prev = INFINITY;   // prev: the last accepted Newton step
        {
          // FP32 stage
          float l32 = __double2float_rd(lo), h32 = __double2float_ru(hi);
          float x32 = 0.5f * (l32 + h32), p32 = INFINITY;
          bool d32 = done;
          for (int it = 0; it < 120; ++it) {
            if (h32 - l32 <= tol32) d32 = true;
            if (__all_sync(0xffffffffu, d32)) break;
            if (d32) continue;
            float S32 = 0.f;
            const bool up = sturm_newton_f32(tdf, te2f, n, x32, 1e-30f, S32) > k;
            if (up) l32 = x32;
            else h32 = x32;
            const float st = (S32 != 0.f) ? -1.f / S32 : 0.f;
            const float xnew = x32 + st;
            if (S32 != 0.f && xnew > l32 && xnew < h32 && fabsf(st) <= 0.5f * p32) {
              x32 = xnew;
              p32 = fabsf(st);
            } else {
              x32 = 0.5f * (l32 + h32);
              p32 = INFINITY;
            }
          }
          // FP64 evaluation at the FP32 midpoint, and confirmation of the far end
          if (!done) {
            const double xs = 0.5 * ((double)l32 + (double)h32);
            if (xs > lo && xs < hi) {
              const double w = 2.0 * (double)tol32 + 8.0 * eps;
              double S = 0.0;
              const bool up = sturm_newton_f64(tdn, te2n, n, xs, pivmin, S) > k;
              double cand;
              if (up) {
                lo = xs;
                cand = xs + w;
              } else {
                hi = xs;
                cand = xs - w;
              }
              if (cand > lo && cand < hi) {
                const bool cup = sturm_greater_f64(tdn, te2n, n, cand, pivmin) > k;
                if (up && !cup) hi = cand;   // eigenvalue k in (xs, cand]
                if (!up && cup) lo = cand;   // eigenvalue k in (cand, xs]
              }
              const double st = (S != 0.0) ? -1.0 / S : 0.0;
              xn = (S != 0.0 && xs + st > lo && xs + st < hi) ? xs + st : 0.5 * (lo + hi);
            }
          }
        }
        for (int it = 0; it < 300; ++it) {
          if (hi - lo <= tol) done = true;
          if (__all_sync(0xffffffffu, done)) break;
          if (done) continue;
          double S = 0.0;
          const bool up = sturm_newton_f64(tdn, te2n, n, xn, pivmin, S) > k;   // eigenvalue k above x_n
          if (up) lo = xn;
          else hi = xn;
          const double step = (S != 0.0) ? -1.0 / S : 0.0;
          double xnew = xn + step;
          if (S != 0.0 && fabs(step) <= 0.25 * tol) {
            xnew = xn + (up ? 0.5 * tol : -0.5 * tol);
            prev = INFINITY;
            if (!(xnew > lo && xnew < hi)) xnew = 0.5 * (lo + hi);
          } else if (S != 0.0 && xnew > lo && xnew < hi && fabs(step) <= 0.5 * prev) {
            prev = fabs(step);
          } else {
            // Newton left the bracket or did not halve its step (a repeated
            // eigenvalue, where it converges only linearly from one side): bisect
            xnew = 0.5 * (lo + hi);
            prev = INFINITY;
          }
          xn = xnew;
        }
        const double val = 0.5 * (lo + hi);
        if (k < keep) ev[k] = val * tnorm;
      }
    }
  }
  if (threadIdx.x == 0) {
    s.kept[t] = keep;
    s.trace[t] = s_tr;
  }
  if (!want_vectors) return;
  __syncthreads();

  // ---- phase 3: inverse iteration (LDL^T of T - l I, two solves) ------------
  // Each thread owns one kept eigenvalue.  The LDL^T factors and the iterate
  // of a chunk of vectors live in shared memory (the packed triangle is no
  // longer needed): per vector k the arrays dd[i], ll[i], z[i] at
  // ((i * 3 + a) * kc + k); a chunk holds at least 32 vectors for n <= 256.
  // Results go to the global scratch (the Gram matrix is no longer needed)
  // as Zg[k n + i], one contiguous vector per eigenvalue.
  R* Zg = reinterpret_cast<R*>(G);
  {
    const int chunk_cap = HeevSmem<R>::kBytes / (3 * n * (int)sizeof(R));
    if (chunk_cap < 32) {   // cannot happen for n <= 256
      if (threadIdx.x == 0) atomicOr(s.status + t, (int32_t)TS_SHAPE);
      return;
    }
    const int kc_max = min(chunk_cap, (int)blockDim.x);
    R* wsp = reinterpret_cast<R*>(heev_smem);
    for (int k0 = 0; k0 < keep; k0 += kc_max) {
      const int kc = min(kc_max, keep - k0);
      const int ld = kc;      // row stride of the work arrays
      for (int kk = threadIdx.x; kk < kc; kk += blockDim.x) {
        const int k = k0 + kk;
        R* w3 = wsp + kk;
        const R lam = (R)ev[k];
        // w3[i][0] holds 1 / d_i (the solves multiply), w3[i][1] l_i, w3[i][2]
        // the iterate.  Stores to w3 would keep the compiler from hoisting the
        // next step's loads (the strides are runtime values), so the loops run
        // in blocks of four steps whose loads all precede their stores; the
        // chains then wait on arithmetic only.  The start vector enters the
        // first forward solve directly, the rescaling of the first iterate the
        // second one, and that of the second the copy-out.
        auto recip = [](R x) { return sizeof(R) == 4 ? (R)__fdividef(1.0f, (float)x) : (R)1 / x; };
        auto Dr = [&](int i) -> R& { return w3[(i * 3 + 0) * ld]; };
        auto Lw = [&](int i) -> R& { return w3[(i * 3 + 1) * ld]; };
        auto Zw = [&](int i) -> R& { return w3[(i * 3 + 2) * ld]; };
        R dprev = sd[0] - lam;
        if (fabs(dprev) < pivmin_abs) dprev = pivmin_abs;
        R rprev = recip(dprev);
        Dr(0) = rprev;
        {
          auto step = [&](R si, R di) {   // returns l_i, advances rprev to 1 / d_{i+1}
            const R li = si * rprev;
            R dn = di - li * si;
            if (fabs(dn) < pivmin_abs) dn = pivmin_abs;
            rprev = recip(dn);
            return li;
          };
          int i = 0;
          for (; i + 4 < n; i += 4) {
            R s4[4], d4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              s4[q] = se[i + q];
              d4[q] = sd[i + q + 1] - lam;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              Lw(i + q) = step(s4[q], d4[q]);
              Dr(i + q + 1) = rprev;
            }
          }
          for (; i + 1 < n; ++i) {
            Lw(i) = step(se[i], sd[i + 1] - lam);
            Dr(i + 1) = rprev;
          }
        }
        R sc = 1;
        for (int iter = 0; iter < 2; ++iter) {
          auto zin = [&](int i) { return iter == 0 ? (R)start_entry(k, i) : sc * Zw(i); };
          R y = zin(0);
          Zw(0) = y;
          int i = 1;
          for (; i + 3 < n; i += 4) {
            R z4[4], l4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              z4[q] = zin(i + q);
              l4[q] = Lw(i + q - 1);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              y = z4[q] - l4[q] * y;
              Zw(i + q) = y;
            }
          }
          for (; i < n; ++i) {
            y = zin(i) - Lw(i - 1) * y;
            Zw(i) = y;
          }
          R zn = Zw(n - 1) * Dr(n - 1);
          Zw(n - 1) = zn;
          R amax = fabs(zn);
          i = n - 2;
          for (; i >= 3; i -= 4) {
            R z4[4], d4[4], l4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              z4[q] = Zw(i - q);
              d4[q] = Dr(i - q);
              l4[q] = Lw(i - q);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              zn = z4[q] * d4[q] - l4[q] * zn;
              Zw(i - q) = zn;
              amax = fmax(amax, fabs(zn));
            }
          }
          for (; i >= 0; --i) {
            zn = Zw(i) * Dr(i) - Lw(i) * zn;
            Zw(i) = zn;
            amax = fmax(amax, fabs(zn));
          }
          sc = (amax > 0) ? (R)1 / amax : (R)1;
        }
        Dr(0) = sc;   // the factors are done with: slot 0 keeps the final scale
      }
      __syncthreads();
      // copy-out with the scale, coalesced along each vector
      for (int kk = warp; kk < kc; kk += nwarp) {
        const R* w3 = wsp + kk;
        const R sc = w3[0];
        for (int i = lane; i < n; i += 32) Zg[(size_t)(k0 + kk) * n + i] = sc * w3[(i * 3 + 2) * ld];
      }
      __syncthreads();
    }
  }
  // ---- phase 4: Gram-Schmidt in descending eigenvalue order -----------------
  // In the back-transformation type RG = RB: in FP64 mode in place on Zg; in
  // mixed mode on an FP32 copy of the vectors (placed after the first n^2
  // doubles of this trajectory's Gram slot), since the vectors go on to the
  // complex64 back-transformation and the split (orthonormal to ~eps_32
  // either way) while the eigenvalues and the inverse iteration, which depend
  // on the gaps, stay FP64.
  using RG = RB;
  RG* Zs;
  if constexpr (std::is_same<RG, R>::value) {
    Zs = reinterpret_cast<RG*>(Zg);
  } else {
    Zs = reinterpret_cast<RG*>(Zg + (size_t)n * n);
    for (int e = threadIdx.x; e < keep * n; e += blockDim.x) Zs[e] = (RG)Zg[e];
    __syncthreads();
  }
  // Blocks of NB = 16 vectors are orthonormalized in turn (block classical
  // Gram-Schmidt).  The block is staged in shared memory; the earlier vectors
  // stay in Zs (L2-resident, 256 KB per trajectory at n = 256, keep = 128).
  // Projection: the coefficients <z_a, z_b> by one warp per earlier vector a
  // (lanes along i, 16 sums per lane, one reduce-scatter butterfly), then
  // z_b -= sum_a c_ab z_a with the z_a streamed from L2, coalesced.  Then
  // Cholesky QR of the block's 16 x 16 Gram matrix.  A second pass follows
  // only where the first may have left more than a few ulps of
  // non-orthogonality (Daniel-Gragg-Kaufman-Stewart: the projection removed
  // more than half of some vector's squared norm, or a Cholesky pivot fell
  // below half of its diagonal entry); inverse-iteration vectors of
  // well-separated eigenvalues pass with one.  A block whose pivots show
  // near-dependence (pivot < 1e-8 (FP64) or 1e-4 (FP32) of the squared norm)
  // is redone vector by vector, each projected twice against everything
  // before it.
  {
    constexpr int NB = 16;
    const int ldb = n + 2;                       // row stride of the staged block
    RG* Zb = reinterpret_cast<RG*>(heev_smem);     // [NB][ldb]
    RG* cb = Zb + NB * ldb;                       // [128][NB] projection coefficients
    RG* gq = cb + 128 * NB;                       // [NB][NB] block Gram matrix
    RG* lq = gq + NB * NB;                        // [NB][NB] its Cholesky factor
    __shared__ int s_fail, s_redo;
    __shared__ RG s_n0[NB];                       // squared norms before the projection
    const RG tol = (RG)(sizeof(RG) == 4 ? 1e-4 : 1e-8);   // near-dependence of a block
    const int nper = (n + 31) >> 5;
    // c[a][b] = <z_a, Zb_b> for a in [a0, a1): warp per a
    auto coeffs = [&](int a0, int a1, int nbk) {
      for (int a = a0 + warp; a < a1; a += nwarp) {
        RG za[8];
#pragma unroll
        for (int t2 = 0; t2 < 8; ++t2) {
          const int i = lane + 32 * t2;
          za[t2] = (t2 < nper && i < n) ? Zs[(size_t)a * n + i] : (RG)0;
        }
        RG d[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          RG acc = 0;
#pragma unroll
          for (int t2 = 0; t2 < 8; ++t2) {
            const int i = lane + 32 * t2;
            if (t2 < nper && i < n && b < nbk) acc = fma(za[t2], Zb[b * ldb + i], acc);
          }
          d[b] = acc;
        }
        const RG tot = warp_reduce_scatter<NB>(d, lane);
        if ((lane & 1) == 0) cb[(a - a0) * NB + Scatter<NB>::index(lane)] = tot;
      }
    };
    // Zb_b -= sum_{a in [a0, a1)} c[a][b] z_a: thread (row i, half h of the block)
    auto subtract = [&](int a0, int a1, int nbk) {
      const int i = threadIdx.x & 255, h = threadIdx.x >> 8;
      if (i < n && h < 2) {
        RG y[NB / 2];
#pragma unroll
        for (int q2 = 0; q2 < NB / 2; ++q2) y[q2] = (h * NB / 2 + q2 < nbk) ? Zb[(h * NB / 2 + q2) * ldb + i] : (RG)0;
#pragma unroll 2
        for (int a = a0; a < a1; ++a) {
          const RG za = Zs[(size_t)a * n + i];
          const RG* c = cb + (a - a0) * NB + h * NB / 2;
#pragma unroll
          for (int q2 = 0; q2 < NB / 2; ++q2) y[q2] = fma(-c[q2], za, y[q2]);
        }
#pragma unroll
        for (int q2 = 0; q2 < NB / 2; ++q2)
          if (h * NB / 2 + q2 < nbk) Zb[(h * NB / 2 + q2) * ldb + i] = y[q2];
      }
    };
    for (int kb = 0; kb < keep; kb += NB) {
      const int nbk = min(NB, keep - kb);
      for (int e = threadIdx.x; e < NB * n; e += blockDim.x) {
        const int b = e / n, i = e - b * n;
        Zb[b * ldb + i] = (b < nbk) ? Zs[(size_t)(kb + b) * n + i] : (RG)0;
      }
      __syncthreads();
      for (int rep = 0; rep < 2; ++rep) {
        if (kb > 0) {
          if (rep == 0 && warp < nbk) {
            RG acc = 0;
            for (int i = lane; i < n; i += 32) acc = fma(Zb[warp * ldb + i], Zb[warp * ldb + i], acc);
            acc = warp_sum(acc);
            if (lane == 0) s_n0[warp] = acc;
          }
          // earlier vectors in chunks of 128 coefficient rows
          for (int a0 = 0; a0 < kb; a0 += 128) {
            const int a1 = min(kb, a0 + 128);
            coeffs(a0, a1, nbk);
            __syncthreads();
            subtract(a0, a1, nbk);
            __syncthreads();
          }
        }
        // Gram matrix of the block: thread pair (b, c), halves of the row
        {
          const int ent = threadIdx.x >> 1, h = threadIdx.x & 1;
          const int bb = ent / NB, cc2 = ent % NB;
          RG acc = 0;
          if (bb < nbk && cc2 < nbk)
            for (int i = h; i < n; i += 2) acc = fma(Zb[bb * ldb + i], Zb[cc2 * ldb + i], acc);
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          if (h == 0 && ent < NB * NB) gq[ent] = acc;
        }
        __syncthreads();
        // Cholesky G = L L^T by warp 0 (lane i owns row i)
        if (warp == 0) {
          RG li[NB];
#pragma unroll
          for (int c = 0; c < NB; ++c) li[c] = 0;
          int fail = 0, redo = 0;
          const RG gii = (lane < nbk) ? gq[lane * NB + lane] : (RG)1;
#pragma unroll
          for (int j = 0; j < NB; ++j) {
            if (j < nbk) {
              RG sj = (lane < nbk) ? gq[lane * NB + j] : (RG)0;
#pragma unroll
              for (int c = 0; c < j; ++c) sj -= li[c] * __shfl_sync(0xffffffffu, li[c], j);
              const RG piv = __shfl_sync(0xffffffffu, sj, j);
              const RG gjj = __shfl_sync(0xffffffffu, gii, j);
              if (!(piv > tol * gjj) || !(gjj > (RG)0)) fail = 1;
              if (!(piv >= (RG)0.5 * gjj) || (kb > 0 && !(gjj >= (RG)0.5 * s_n0[j]))) redo = 1;
              const RG ljj = sqrt(fmax(piv, (RG)0));
              if (lane == j) li[j] = ljj;
              else if (lane > j) li[j] = (ljj > 0) ? sj / ljj : (RG)0;
            }
          }
          if (lane < NB)
#pragma unroll
            for (int c = 0; c < NB; ++c) lq[lane * NB + c] = li[c];
          if (lane == 0) {
            s_fail = fail;
            s_redo = redo;
          }
        }
        __syncthreads();
        if (s_fail) {
          // vector by vector: project twice against all earlier vectors and
          // the block's earlier members, then normalize
          RG* cv = cb;   // coefficients, [kb + NB]
          for (int b = 0; b < nbk; ++b) {
            for (int pass = 0; pass < 2; ++pass) {
              for (int a = warp; a < kb + b; a += nwarp) {
                const RG* za = (a < kb) ? Zs + (size_t)a * n : Zb + (a - kb) * ldb;
                RG acc = 0;
                for (int i = lane; i < n; i += 32) acc = fma(za[i], Zb[b * ldb + i], acc);
                acc = warp_sum(acc);
                if (lane == 0) cv[a] = acc;
              }
              __syncthreads();
              for (int i = threadIdx.x; i < n; i += blockDim.x) {
                RG v = Zb[b * ldb + i];
                for (int a = 0; a < kb + b; ++a) v = fma(-cv[a], (a < kb) ? Zs[(size_t)a * n + i] : Zb[(a - kb) * ldb + i], v);
                Zb[b * ldb + i] = v;
              }
              __syncthreads();
            }
            RG part = 0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) part = fma(Zb[b * ldb + i], Zb[b * ldb + i], part);
            const RG nn = block_sum(part, reinterpret_cast<RG*>(red));
            const RG inv = nn > 0 ? (RG)1 / sqrt(nn) : (RG)0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) Zb[b * ldb + i] *= inv;
            __syncthreads();
          }
        } else {
          // Zb <- L^{-1} Zb, one row entry i per thread
          for (int i = threadIdx.x; i < n; i += blockDim.x) {
            RG x[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) x[b] = (b < nbk) ? Zb[b * ldb + i] : (RG)0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              if (b < nbk) {
                RG v = x[b];
#pragma unroll
                for (int c = 0; c < b; ++c) v = fma(-lq[b * NB + c], x[c], v);
                x[b] = v / lq[b * NB + b];
              }
            }
#pragma unroll
            for (int b = 0; b < NB; ++b)
              if (b < nbk) Zb[b * ldb + i] = x[b];
          }
          __syncthreads();
        }
        if (rep == 0 && !s_fail && !s_redo) break;   // uniform: set before the barriers above
      }
      for (int e = threadIdx.x; e < nbk * n; e += blockDim.x) {
        const int b = e / n, i = e - b * n;
        Zs[(size_t)(kb + b) * n + i] = Zb[b * ldb + i];
      }
      __syncthreads();
    }
  }
  // ---- phase 5: back-transformation U = Q D z --------------------------------
  // Each warp owns NCOL columns held in registers (PER entries per lane each).
  // The reflectors stream through two shared-memory buffers of rc rows (row
  // stride ldv = 32 * nper, zero-padded), placed after the shared-memory copy
  // of z and filled by bulk copies on one mbarrier each: the copy of chunk
  // g + 1 runs while chunk g is applied, and a buffer is refilled (chunk g +
  // 2) once every warp has passed the barrier that ends chunk g.  Chunks run
  // from the last reflector down and repeat for each pass over the columns.
  // Reflector j is zero in rows <= j, so the 32-row groups above it are
  // skipped (bt_reflector, specialized on the first live group).
  constexpr int PER = 8;  // n <= 256 -> 8 elements per lane
  constexpr int NCOL = sizeof(RB) == 4 ? 4 : 2;
  const int nper = (n + 31) >> 5;
  const int ldv = 32 * nper;
  const size_t zbytes = 0;   // the vectors are read from Zs
  const int rc = min(32, (int)((HeevSmem<R>::kBytes - zbytes) / (2 * (size_t)ldv * sizeof(cpx<RB>))));
  if (rc < 1) {   // cannot happen for n <= 256 (the z copy leaves >= 8 n entries)
    if (threadIdx.x == 0) atomicOr(s.status + t, (int32_t)TS_SHAPE);
    return;
  }
  cpx<RB>* vbuf[2];
  vbuf[0] = reinterpret_cast<cpx<RB>*>(heev_smem + zbytes);
  vbuf[1] = vbuf[0] + (size_t)rc * ldv;
  __shared__ __align__(8) uint64_t s_bar[2];
  const int nch = (n >= 3) ? (n - 3) / rc + 1 : 0;   // chunks per pass
  const int ngroups = (keep + NCOL - 1) / NCOL;
  const int passes = (ngroups + nwarp - 1) / nwarp;
  const int nchunk = nch * passes;
  auto issue = [&](int g) {   // one thread: copy chunk g into buffer g & 1
    const int c = g % nch;
    const int jtop = n - 3 - c * rc, jlo = max(0, jtop - rc + 1), rows = jtop - jlo + 1;
    uint64_t* bar = &s_bar[g & 1];
    mbar_expect_tx(bar, (uint32_t)(rows * n * sizeof(cpx<RB>)));
    if (ldv == n) {
      bulk_g2s(vbuf[g & 1], Hv + (int64_t)jlo * n, (uint32_t)(rows * n * sizeof(cpx<RB>)), bar);
    } else {
      for (int rr = 0; rr < rows; ++rr)
        bulk_g2s(vbuf[g & 1] + (size_t)rr * ldv, Hv + (int64_t)(jlo + rr) * n, (uint32_t)(n * sizeof(cpx<RB>)), bar);
    }
  };
  if (ldv != n)   // padding columns n .. ldv-1 of both buffers, never copied over
    for (int e = threadIdx.x; e < 2 * rc * (ldv - n); e += blockDim.x) {
      const int r = e / (ldv - n), i = n + e % (ldv - n);
      vbuf[0][(size_t)r * ldv + i] = mk<RB>(0, 0);
    }
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
  }
  // Hv was written with ordinary stores and the buffers last held other data
  fence_for_bulk_copies();
  __syncthreads();
  if (threadIdx.x == 0)
    for (int g = 0; g < min(2, nchunk); ++g) issue(g);
  cpx<RB> y[NCOL][PER];
  for (int pass = 0; pass < passes; ++pass) {
    const int k0 = NCOL * (warp + pass * nwarp);
    const bool act = k0 < keep;
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
      for (int a = 0; a < PER; ++a) {
        const int i = lane + 32 * a;
        y[c][a] = (i < n && k0 + c < keep) ? cast<RB>(sph[i]) * Zs[(size_t)(k0 + c) * n + i] : mk<RB>(0, 0);
      }
    for (int c = 0; c < nch; ++c) {
      const int g = pass * nch + c;
      const int jtop = n - 3 - c * rc, jlo = max(0, jtop - rc + 1);
      const cpx<RB>* vst = vbuf[g & 1];
      const bool ready = mbar_wait(&s_bar[g & 1], (uint32_t)((g >> 1) & 1));
      if (act && ready) {
        for (int j = jtop; j >= jlo; --j) {
          const cpx<RB>* v = vst + (j - jlo) * ldv;
          switch ((j + 1) >> 5) {   // groups a < (j + 1) / 32 hold rows <= j only
            case 0: bt_reflector<RB, NCOL, PER, 0>(y, v, lane, nper); break;
            case 1: bt_reflector<RB, NCOL, PER, 1>(y, v, lane, nper); break;
            case 2: bt_reflector<RB, NCOL, PER, 2>(y, v, lane, nper); break;
            case 3: bt_reflector<RB, NCOL, PER, 3>(y, v, lane, nper); break;
            case 4: bt_reflector<RB, NCOL, PER, 4>(y, v, lane, nper); break;
            case 5: bt_reflector<RB, NCOL, PER, 5>(y, v, lane, nper); break;
            case 6: bt_reflector<RB, NCOL, PER, 6>(y, v, lane, nper); break;
            default: bt_reflector<RB, NCOL, PER, 7>(y, v, lane, nper); break;
          }
        }
      }
      if (__syncthreads_or(!ready)) {
        // a copy missed its time limit: flag the trajectory, give the copies
        // still in flight (chunks g and g + 1) a bounded wait, and stop
        if (threadIdx.x == 0) {
          atomicOr(s.status + t, (int32_t)TS_COPY);
          for (int h = g; h < min(g + 2, nchunk); ++h) mbar_wait(&s_bar[h & 1], (uint32_t)((h >> 1) & 1));
        }
        return;
      }
      if (threadIdx.x == 0 && g + 2 < nchunk) issue(g + 2);
    }
#pragma unroll
    for (int a = 0; a < PER; ++a) {
      const int i = lane + 32 * a;
      if (i < n) {
#pragma unroll
        for (int c2 = 0; c2 < NCOL; ++c2)
          if (k0 + c2 < keep) U[(int64_t)(k0 + c2) * n + i] = y[c2][a];
      }
    }
  }
}

}  // namespace lemps
