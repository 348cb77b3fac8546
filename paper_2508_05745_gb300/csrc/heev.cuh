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
// in ws1, overwritten.  Householder vectors in ws3 (row j holds v_j, unit
// norm, entries > j).  Eigenvectors are written column-major to ws2:
// U[k * n + i], k < keep.  Eigenvalues (double, descending) to
// evals[0..keep), keep and the trace to kept[] / trace[].
#pragma once

#include <type_traits>

#include "common.cuh"

namespace lemps {

template <class R>
struct HeevView {
  cpx<R>* ws1;      // Gram matrix, then LDL^T scratch of the inverse iteration
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
// strictly greater than x (Sturm sequence of T - x I with a pivot guard).
template <class R>
__device__ __forceinline__ int sturm_greater(const R* d, const R* e2, int n, R x, R pivmin) {
  int neg = 0;
  R q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  neg += (q < 0);
  for (int i = 1; i < n; ++i) {
    // c64: fast reciprocal-based divide (|q| >= pivmin keeps it in range)
    q = (d[i] - x) - (sizeof(R) == 4 ? (R)__fdividef((float)e2[i - 1], (float)q) : e2[i - 1] / q);
    if (fabs(q) < pivmin) q = -pivmin;
    neg += (q < 0);
  }
  return n - neg;
}

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

// y_c <- (I - 2 v v^dagger) y_c for a warp's NCOL columns (PER entries per
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
  for (int e = 0; e < NV; ++e) dd[e] = (R)2 * __shfl_sync(0xffffffffu, tot, Scatter<NV>::source(e));
#pragma unroll
  for (int a = A0; a < PER; ++a)
#pragma unroll
    for (int c = 0; c < NCOL; ++c) y[c][a] -= vr[a] * mk<R>(dd[2 * c], dd[2 * c + 1]);
}

// mode / q select the matrix size as in gram_size(); want_vectors = 0 returns
// eigenvalues only (all n of them when cutoff = 0).
template <class R>
__global__ void __launch_bounds__(512) k_heev(HeevView<R> s, int q, int mode, double cutoff, int keep_max,
                                               int want_vectors) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  const int32_t* bd = s.bond + t * (s.nq + 1);
  const int n = mode == 0 ? 2 * bd[q] : (mode == 1 ? 2 * bd[q + 2] : bd[q + 1]);
  cpx<R>* G = s.ws1 + t * s.ws_stride;
  cpx<R>* Hv = s.ws3 + t * s.ws_stride;
  cpx<R>* U = s.ws2 + t * s.ws_stride;
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

  // trace (FP64) for the cutoff and the discarded weight
  double trp = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) trp += (double)G[(int64_t)i * n + i].re;
  trp = block_sum(trp, redd);
  if (threadIdx.x == 0) s_tr = trp;

  // ---- phase 1: tridiagonalization ------------------------------------------
  // Steps whose trailing block does not fit in shared memory form one panel
  // (LATRD style): G stays read-only in global memory, and the rank-2 updates
  // G_eff = G - sum_k (v_k w_k^dagger + w_k v_k^dagger) of earlier panel steps
  // are applied on the fly to the column and to the matvec.  After the panel,
  // one tiled rank-2 j0 update brings the trailing block G[j0:, j0:] up to
  // date; its lower triangle is then packed into shared memory and the
  // remaining steps stay on chip.  V and W (j0 x n each, row k = step k) live
  // in shared memory when they fit, else in ws2 (which receives the
  // eigenvectors only at the end).
  int j0 = 0;
  while ((n - j0) * (n - j0 + 1) / 2 > HeevSmem<R>::kCap) ++j0;
  // V and W sit in shared memory (unused until the packing) when they fit
  const bool vw_sm = 2 * (size_t)j0 * n * sizeof(cpx<R>) <= (size_t)HeevSmem<R>::kBytes;
  cpx<R>* Vp = vw_sm ? Lp : U;
  cpx<R>* Wp = Vp + (int64_t)j0 * n;
  for (int j = 0; j < j0 && j + 2 < n; ++j) {
    const int m = n - j - 1;
    // column j of G_eff below the diagonal, and its diagonal entry
    R part = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const int gi = j + 1 + i;
      cpx<R> x = G[(int64_t)gi * n + j];
      for (int k = 0; k < j; ++k)
        x -= Vp[(int64_t)k * n + gi] * conj(Wp[(int64_t)k * n + j]) + Wp[(int64_t)k * n + gi] * conj(Vp[(int64_t)k * n + j]);
      sv[i] = x;
      if (i > 0) part += norm2(x);
    }
    if (threadIdx.x == 0) {
      R dj = G[(int64_t)j * n + j].re;
      for (int k = 0; k < j; ++k) dj -= (R)2 * cdot(Wp[(int64_t)k * n + j], Vp[(int64_t)k * n + j]).re;
      sd[j] = dj;
    }
    R sig = block_sum(part, red);
    cpx<R> x0 = sv[0];
    R ax0 = sqrt(norm2(x0));
    R nrm = sqrt(sig + ax0 * ax0);
    const bool reflect = sig > (R)0;
    cpx<R> alpha = x0;
    if (reflect) {
      cpx<R> ph = (ax0 > 0) ? mk<R>(x0.re / ax0, x0.im / ax0) : mk<R>(1, 0);
      alpha = mk<R>(-nrm * ph.re, -nrm * ph.im);
      R inv = (R)1 / sqrt(sig + (ax0 + nrm) * (ax0 + nrm));
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += blockDim.x) sv[i] = (i == 0) ? (x0 - alpha) * inv : sv[i] * inv;
    }
    __syncthreads();
    if (threadIdx.x == 0) sec[j] = alpha;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const cpx<R> vi = (i > j && reflect) ? sv[i - j - 1] : mk<R>(0, 0);
      Hv[(int64_t)j * n + i] = vi;
      Vp[(int64_t)j * n + i] = vi;
    }
    if (!reflect) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) Wp[(int64_t)j * n + i] = mk<R>(0, 0);
      __syncthreads();
      continue;
    }
    // corrections c1_k = w_k^dagger v, c2_k = v_k^dagger v (k < j); sph is
    // free until the end of phase 1 and holds 2 j < 2 j0 <= 256 entries
    cpx<R>* cc = sph;
    for (int kk = warp; kk < 2 * j; kk += nwarp) {
      const cpx<R>* src = (kk < j) ? (Wp + (int64_t)kk * n) : (Vp + (int64_t)(kk - j) * n);
      cpx<R> acc = mk<R>(0, 0);
      for (int i = lane; i < m; i += 32) cfmac(acc, src[j + 1 + i], sv[i]);
      acc.re = warp_sum(acc.re);
      acc.im = warp_sum(acc.im);
      if (lane == 0) cc[kk] = acc;
    }
    // y = G_sub v from the original (read-only) G, which is served from L2:
    // four rows per warp, each lane loading two adjacent entries of a row at
    // a time (16-byte aligned: the segment starts at the even column c0 <= j +
    // 1) with two such loads per row in flight; the eight partial sums of the
    // four rows are reduced by one butterfly.
    const int c0 = (j + 1) & ~1;
    const int off = j + 1 - c0;        // 1: column c0 = j lies left of the block (weight 0)
    const int npair = (n - c0) >> 1;
    for (int r0 = 4 * warp; r0 < m; r0 += 4 * nwarp) {
      const int nq = min(4, m - r0);
      const cpx<R>* row = G + (int64_t)(j + 1 + r0) * n + c0;
      cpx<R> acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = mk<R>(0, 0);
#pragma unroll 2
      for (int p2 = lane; p2 < npair; p2 += 32) {
        const int c = 2 * p2 - off;    // local index of the first entry of the pair
        const cpx<R> x0 = (c >= 0) ? sv[c] : mk<R>(0, 0), x1 = sv[c + 1];
        cpx<R> a0[4], a1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nq) load_pair(row + (int64_t)q * n + 2 * p2, a0[q], a1[q]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nq) {
            cfma(acc[q], a0[q], x0);
            cfma(acc[q], a1[q], x1);
          }
      }
      R d[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        d[2 * q] = acc[q].re;
        d[2 * q + 1] = acc[q].im;
      }
      const R tot = warp_reduce_scatter<8>(d, lane);
      if ((lane & 3) == 0) {
        const int e = Scatter<8>::index(lane);
        const int r = r0 + (e >> 1);
        if (r < m) {
          if (e & 1) sw[r].im = tot;
          else sw[r].re = tot;
        }
      }
    }
    __syncthreads();
    // y -= sum_k v_k (w_k^dagger v) + w_k (v_k^dagger v)
    R sp = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const int gi = j + 1 + i;
      cpx<R> y = sw[i];
      for (int k = 0; k < j; ++k) y -= Vp[(int64_t)k * n + gi] * cc[k] + Wp[(int64_t)k * n + gi] * cc[j + k];
      sw[i] = y;
      sp += cdot(sv[i], y).re;
    }
    R ss = block_sum(sp, red);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const cpx<R> wi = (i > j) ? (R)2 * sw[i - j - 1] - ((R)2 * ss) * sv[i - j - 1] : mk<R>(0, 0);
      Wp[(int64_t)j * n + i] = wi;
    }
    __syncthreads();
  }
  if (j0 > 0) {
    // G[j0:, j0:] -= sum_k v_k w_k^dagger + w_k v_k^dagger over the panel
    // (lower triangle only).  V and W are staged in shared memory in chunks
    // of kch steps; 64 x 64 output tiles, each of the 512 threads (32 x 16)
    // owns rows ty + 16 r and columns tx + 32 c of a tile.
    // (With V and W already in shared memory they are used in place.)
    const int mt = n - j0;
    const int kch = vw_sm ? j0 : min(j0, (int)(HeevSmem<R>::kBytes / (2 * (size_t)mt * sizeof(cpx<R>))));
    const int ldk = vw_sm ? n : mt;
    const cpx<R>* Vs = vw_sm ? Vp + j0 : Lp;
    const cpx<R>* Ws = vw_sm ? Wp + j0 : Lp + (int64_t)kch * mt;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int ntile = (mt + 63) / 64;
    for (int k0 = 0; k0 < j0; k0 += kch) {
      const int kc = min(kch, j0 - k0);
      if (!vw_sm) {
        for (int e = threadIdx.x; e < kc * mt; e += blockDim.x) {
          const int kk = e / mt, i = e - kk * mt;
          Lp[e] = Vp[(int64_t)(k0 + kk) * n + j0 + i];
          Lp[(int64_t)kch * mt + e] = Wp[(int64_t)(k0 + kk) * n + j0 + i];
        }
      }
      __syncthreads();
      for (int ti = 0; ti < ntile; ++ti)
        for (int tc = 0; tc <= ti; ++tc) {
          cpx<R> acc[4][2];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) acc[r][c] = mk<R>(0, 0);
          for (int kk = 0; kk < kc; ++kk) {
            cpx<R> va[4], wa[4], vb[2], wb[2];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int i = ti * 64 + ty + 16 * r;
              va[r] = i < mt ? Vs[kk * ldk + i] : mk<R>(0, 0);
              wa[r] = i < mt ? Ws[kk * ldk + i] : mk<R>(0, 0);
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const int i = tc * 64 + tx + 32 * c;
              vb[c] = i < mt ? Vs[kk * ldk + i] : mk<R>(0, 0);
              wb[c] = i < mt ? Ws[kk * ldk + i] : mk<R>(0, 0);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
              for (int c = 0; c < 2; ++c) {
                cfmac(acc[r][c], wb[c], va[r]);
                cfmac(acc[r][c], vb[c], wa[r]);
              }
          }
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const int i = ti * 64 + ty + 16 * r, cc = tc * 64 + tx + 32 * c;
              if (i < mt && cc <= i) {
                cpx<R>* g = G + (int64_t)(j0 + i) * n + (j0 + cc);
                *g = *g - acc[r][c];
              }
            }
        }
      __syncthreads();
    }
  }
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
  __shared__ cpx<R> sy2[256];
  __shared__ R redn[32], reds[32];
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
    auto wprev = [&](int X) { return (R)2 * yP[X] - ((R)2 * ssP) * vP[X]; };
    const cpx<R> vPj = vP[jl], wPj = wprev(jl);
    // column jl below the diagonal (one entry per thread; m < blockDim.x)
    const int i = threadIdx.x;
    cpx<R> x = mk<R>(0, 0), wi = mk<R>(0, 0);
    R part = 0;
    if (i < m) {
      const int Rr = jl + 1 + i;
      wi = wprev(Rr);
      x = Lp[pidx(Rr, jl)] - vP[Rr] * conj(wPj) - wi * conj(vPj);
      if (i > 0) part = norm2(x);
    }
    const cpx<R> x0 = Lp[pidx(jl + 1, jl)] - vP[jl + 1] * conj(wPj) - wprev(jl + 1) * conj(vPj);
    part = warp_sum(part);
    if (lane == 0) redn[warp] = part;
    __syncthreads();
    R sig = 0;
    for (int w2 = 0; w2 < nwarp; ++w2) sig += redn[w2];
    const R ax0 = sqrt(norm2(x0));
    const R nrm = sqrt(sig + ax0 * ax0);
    cpx<R> alpha = x0, vi = mk<R>(0, 0);
    if (sig > (R)0) {
      cpx<R> ph = (ax0 > 0) ? mk<R>(x0.re / ax0, x0.im / ax0) : mk<R>(1, 0);
      alpha = mk<R>(-nrm * ph.re, -nrm * ph.im);
      const R inv = (R)1 / sqrt(sig + (ax0 + nrm) * (ax0 + nrm));
      vi = (i == 0) ? (x0 - alpha) * inv : x * inv;
    }
    // every thread has read y of the previous step: it now becomes w
    cpx<R>* wP = const_cast<cpx<R>*>(yP);
    if (i < m) {
      vN[jl + 1 + i] = vi;
      yN[jl + 1 + i] = mk<R>(0, 0);
      wP[jl + 1 + i] = wi;
      Hv[(int64_t)j * n + (j + 1 + i)] = vi;
    }
    if (i <= j) Hv[(int64_t)j * n + i] = mk<R>(0, 0);
    if (threadIdx.x == 0) {
      sd[j] = Lp[pidx(jl, jl)].re - (R)2 * cdot(wPj, vPj).re;
      sec[j] = alpha;
    }
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
            const cpx<R> aa = rowp[C] - vr * conj(cw) - wr * conj(cv);
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
        atomicAdd(&yN[Rr].re, acc.re);
        atomicAdd(&yN[Rr].im, acc.im);
        ssp += cdot(nr, acc).re;
      }
      const R tot = warp_reduce_scatter<NVQ>(d, lane);
      const int e = Scatter<NVQ>::index(lane);   // value 2 c + {re, im} of column cb + c
      const int Cc = cb + (e >> 1);
      if ((lane & ((1 << (5 - LGQ)) - 1)) == 0 && Cc > jl && Cc < M0) {
        if (e & 1) {
          atomicAdd(&yN[Cc].im, tot);
          ssp += vN[Cc].im * tot;
        } else {
          atomicAdd(&yN[Cc].re, tot);
          ssp += vN[Cc].re * tot;
        }
      }
    }
    ssp = warp_sum(ssp);
    if (lane == 0) reds[warp] = ssp;
    __syncthreads();
    R ss = 0;
    for (int w2 = 0; w2 < nwarp; ++w2) ss += reds[w2];
    ssP = ss;
    pb = qb;
  }
  if (threadIdx.x == 0) {
    // the last two rows, with the pending update of the last step
    const cpx<R>* vP = pb ? sw : sv;
    const cpx<R>* yP = pb ? sy2 : sph;
    auto wprev = [&](int X) { return (R)2 * yP[X] - ((R)2 * ssP) * vP[X]; };
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
  R gl = sd[0], gu = sd[0], tnorm = 0;
  for (int i = 0; i < n; ++i) {
    R rad = (i > 0 ? se[i - 1] : (R)0) + (i + 1 < n ? se[i] : (R)0);
    gl = fmin(gl, sd[i] - rad);
    gu = fmax(gu, sd[i] + rad);
    tnorm = fmax(tnorm, fabs(sd[i]) + rad);
  }
  const R eps = (sizeof(R) == 8) ? (R)2.2e-16 : (R)1.2e-7;
  const R pivmin = fmax((R)1e-30 * tnorm, (sizeof(R) == 8) ? (R)1e-290 : (R)1e-35);
  gl -= 2 * eps * tnorm + pivmin;
  gu += 2 * eps * tnorm + pivmin;
  if (threadIdx.x == 0) {
    int cnt = (cutoff > 0.0) ? sturm_greater<R>(sd, se2, n, (R)(cutoff * s_tr), pivmin) : n;
    // a two-site Gram matrix has rank <= min(2 d_l, 2 d_r)
    const int rank_bound = (mode == 2) ? n : min(2 * bd[q], 2 * bd[q + 2]);
    int kp = min(cnt, min(keep_max, min(n, rank_bound)));
    s_keep = max(kp, 1);
  }
  __syncthreads();
  const int keep = s_keep;
  double* ev = s.evals + t * (2 * s.chi);
  // Brackets: one Sturm count per thread on an increasing grid of blockDim.x
  // points (the packed triangle's shared memory is free by now).  When a
  // cutoff is set, every kept eigenvalue lies above x_lo = cutoff * trace and
  // the grid is geometric from x_lo to gu (neighbouring points about 5 %
  // apart), so each eigenvalue starts from a narrow relative interval instead
  // of [gl, gu]; else it is uniform on [gl, gu].  Any increasing grid is
  // valid, so it is formed in single precision.
  R* gx = reinterpret_cast<R*>(heev_smem);
  int* gcnt = reinterpret_cast<int*>(gx + blockDim.x);
  {
    const int ng = blockDim.x;
    const float xlo = (float)(cutoff * s_tr), xhi = (float)gu;
    const bool geo = cutoff > 0.0 && xlo > 0.0f && xlo < xhi;
    const float f = (float)threadIdx.x / (float)(ng - 1);
    const R x = geo ? (R)(xlo * exp2f(log2f(xhi / xlo) * f)) : gl + (gu - gl) * (R)(threadIdx.x + 1) / (R)(ng + 1);
    gx[threadIdx.x] = x;
    gcnt[threadIdx.x] = sturm_greater<R>(sd, se2, n, x, pivmin);
  }
  __syncthreads();
  {
    // Multisection: G lanes of a warp share eigenvalue k and evaluate the
    // Sturm count at G interior points of its interval, which shrinks by
    // G + 1 per round (G = 4 when 128 eigenvalues are kept on 512 threads).
    int G = 1;
    while (G < 32 && keep * (2 * G) <= (int)blockDim.x) G *= 2;
    const int per_warp = 32 / G;
    const int gi = lane & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
    for (int kb = 0; kb < keep; kb += nwarp * per_warp) {
      const int k = kb + warp * per_warp + lane / G;
      R lo = gl, hi = gu;
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
      for (int it = 0; it < 200; ++it) {
        const R h = (hi - lo) / (R)(G + 1);
        if (hi - lo <= eps * (fabs(lo) + fabs(hi)) + (R)1e-3 * eps * tnorm + pivmin || !(lo + h > lo) ||
            !(hi - h < hi))
          done = true;
        if (__all_sync(0xffffffffu, done)) break;
        const R x = lo + h * (R)(gi + 1);
        const bool above = !done && sturm_greater<R>(sd, se2, n, x, pivmin) > k;
        const unsigned grp = (__ballot_sync(0xffffffffu, above) >> (lane & ~(G - 1))) & gmask;
        const int pcount = __popc(grp);   // interior points below eigenvalue k
        if (!done) {
          const R nlo = (pcount > 0) ? lo + h * (R)pcount : lo;
          const R nhi = (pcount < G) ? lo + h * (R)(pcount + 1) : hi;
          lo = nlo;
          hi = nhi;
        }
      }
      if (k < keep && gi == 0) ev[k] = (double)((R)0.5 * (lo + hi));
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
  // live in shared memory (the packed triangle is no longer needed) when a
  // chunk of vectors fits, else in the global scratch (ws1): per vector k the
  // arrays dd[i], ll[i], z[i] at ((i * 3 + a) * kc + k).  Results go to the
  // global scratch z[i][k] = scr[(i * 3 + 2) * keep + k].
  R* scr = reinterpret_cast<R*>(G);
  {
    const int chunk_cap = HeevSmem<R>::kBytes / (3 * n * (int)sizeof(R));
    const bool in_smem = chunk_cap >= 32;
    const int kc_max = in_smem ? min(chunk_cap, (int)blockDim.x) : keep;
    R* wsp = in_smem ? reinterpret_cast<R*>(heev_smem) : scr;
    for (int k0 = 0; k0 < keep; k0 += kc_max) {
      const int kc = min(kc_max, keep - k0);
      const int ld = in_smem ? kc : keep;      // row stride of the work arrays
      const int koff = in_smem ? 0 : k0;
      for (int kk = threadIdx.x; kk < kc; kk += blockDim.x) {
        const int k = k0 + kk;
        R* w3 = wsp + koff + kk;
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
        if (fabs(dprev) < pivmin) dprev = pivmin;
        R rprev = recip(dprev);
        Dr(0) = rprev;
        {
          auto step = [&](R si, R di) {   // returns l_i, advances rprev to 1 / d_{i+1}
            const R li = si * rprev;
            R dn = di - li * si;
            if (fabs(dn) < pivmin) dn = pivmin;
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
        if (in_smem) {
          for (int i = 0; i < n; ++i) scr[(i * 3 + 2) * keep + k] = sc * Zw(i);
        } else {
          for (int i = 0; i < n; ++i) Zw(i) *= sc;
        }
      }
      __syncthreads();
    }
  }
  // ---- phase 4: Gram-Schmidt in descending eigenvalue order -----------------
  // When the vectors fit in shared memory (Z[k * ldz + i], rows padded so
  // that 16-byte loads of consecutive rows hit distinct banks) they are
  // orthonormalized in blocks of 16 (block classical Gram-Schmidt): project
  // the block against all earlier vectors, then orthonormalize it by
  // Cholesky QR of its 16 x 16 Gram matrix.  A second pass follows only when
  // the first may have left an orthogonality error above a few ulps (the
  // Daniel-Gragg-Kaufman-Stewart criterion): the projection removed more than
  // half of some vector's squared norm, or a Cholesky pivot fell below half
  // of its diagonal entry (an ill-conditioned block).  Inverse-iteration
  // vectors of well-separated eigenvalues pass with one.  A block whose
  // pivots show near-dependence (pivot < tol * squared norm) is redone by
  // per-vector classical Gram-Schmidt (twice).  When the vectors do not fit,
  // they stay in the global scratch and the per-vector scheme runs for all.
  constexpr int NB = 16;
  constexpr int E = 16 / (int)sizeof(R);             // elements per 16-byte load
  constexpr int ROWQ = 128 / (int)sizeof(R);         // elements per 128 bytes
  const int ldz = ((n + ROWQ - 1) / ROWQ) * ROWQ + E;
  const size_t zs_bytes = (size_t)keep * ldz * sizeof(R);
  const size_t cb_bytes = (size_t)128 * NB * sizeof(R);
  const bool zsm = keep <= 128 && zs_bytes + cb_bytes + 8 * (size_t)n * sizeof(cpx<R>) <= (size_t)HeevSmem<R>::kBytes;
  R* Zs = reinterpret_cast<R*>(heev_smem);
  if (zsm)
    for (int e = threadIdx.x; e < keep * ldz; e += blockDim.x) {
      const int k = e / ldz, i = e - k * ldz;
      Zs[e] = (i < n) ? scr[(i * 3 + 2) * keep + k] : (R)0;
    }
  __syncthreads();
  auto Z = [&](int k, int i) -> R& { return zsm ? Zs[k * ldz + i] : scr[(i * 3 + 2) * keep + k]; };
  R* cbuf = reinterpret_cast<R*>(sw);
  // per-vector CGS2 + normalization of vectors k in [k_from, k_to), against
  // all vectors in [p_from, k)
  auto cgs_vectors = [&](int p_from, int k_from, int k_to) {
    for (int k = k_from; k < k_to; ++k) {
      for (int pass = 0; pass < 2; ++pass) {
        for (int jj = p_from + warp; jj < k; jj += nwarp) {
          R acc = 0;
          for (int i = lane; i < n; i += 32) acc += Z(jj, i) * Z(k, i);
          acc = warp_sum(acc);
          if (lane == 0) cbuf[jj - p_from] = acc;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          R v = Z(k, i);
          for (int jj = p_from; jj < k; ++jj) v -= cbuf[jj - p_from] * Z(jj, i);
          Z(k, i) = v;
        }
        __syncthreads();
      }
      R part = 0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) part += Z(k, i) * Z(k, i);
      R nn = block_sum(part, red);
      R inv = nn > 0 ? (R)1 / sqrt(nn) : (R)0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) Z(k, i) *= inv;
      __syncthreads();
    }
  };
  if (!zsm) {
    cgs_vectors(0, 0, keep);
  } else {
    using V16 = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
    R* cb = Zs + (size_t)keep * ldz;                   // [128][NB] projection coefficients
    R* gq = reinterpret_cast<R*>(sv);                  // [NB][NB] block Gram matrix
    R* lq = gq + NB * NB;                              // [NB][NB] its Cholesky factor
    __shared__ int s_fail, s_redo;
    __shared__ R s_n0[NB];   // squared norms of the block before its projection
    const int nvec = (n + E - 1) / E;
    const R tol = (sizeof(R) == 8) ? (R)1e-8 : (R)1e-3;
    for (int kb = 0; kb < keep; kb += NB) {
      const int nbk = min(NB, keep - kb);
      for (int rep = 0; rep < 2; ++rep) {
        if (rep == 0 && kb > 0 && warp < nbk) {   // read after the Gram barrier below
          R acc = 0;
          for (int i = lane; i < n; i += 32) acc = fma(Zs[(size_t)(kb + warp) * ldz + i], Zs[(size_t)(kb + warp) * ldz + i], acc);
          acc = warp_sum(acc);
          if (lane == 0) s_n0[warp] = acc;
        }
        if (kb > 0) {
          // cb[a][b] = <z_a, z_{kb+b}>, a < kb: thread (a, 4 consecutive b)
          {
            const int b0 = (threadIdx.x >> 7) * 4;
            for (int aa = threadIdx.x & 127; aa < kb; aa += 128) {
              R acc[4] = {0, 0, 0, 0};
              const V16* za = reinterpret_cast<const V16*>(Zs + (size_t)aa * ldz);
              const V16* zb[4];
#pragma unroll
              for (int c = 0; c < 4; ++c)
                zb[c] = reinterpret_cast<const V16*>(Zs + (size_t)min(kb + b0 + c, keep - 1) * ldz);
              for (int v = 0; v < nvec; ++v) {
                const V16 x = za[v];
                const R* xr = reinterpret_cast<const R*>(&x);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  const V16 y = zb[c][v];
                  const R* yr = reinterpret_cast<const R*>(&y);
#pragma unroll
                  for (int e = 0; e < E; ++e) acc[c] = fma(xr[e], yr[e], acc[c]);
                }
              }
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (b0 + c < nbk) cb[aa * NB + b0 + c] = acc[c];
            }
          }
          __syncthreads();
          // z_{kb+b} -= sum_a cb[a][b] z_a: thread (16-byte column slice, 2 b)
          {
            const int b0 = (threadIdx.x >> 6) * 2;
            if (b0 < nbk)
              for (int v = threadIdx.x & 63; v < nvec; v += 64) {
                V16* y0p = reinterpret_cast<V16*>(Zs + (size_t)(kb + b0) * ldz) + v;
                V16* y1p = reinterpret_cast<V16*>(Zs + (size_t)(kb + min(b0 + 1, nbk - 1)) * ldz) + v;
                V16 y0 = *y0p, y1 = *y1p;
                R* r0 = reinterpret_cast<R*>(&y0);
                R* r1 = reinterpret_cast<R*>(&y1);
                for (int aa = 0; aa < kb; ++aa) {
                  const V16 x = reinterpret_cast<const V16*>(Zs + (size_t)aa * ldz)[v];
                  const R* xr = reinterpret_cast<const R*>(&x);
                  const R c0 = cb[aa * NB + b0], c1 = cb[aa * NB + b0 + 1];
#pragma unroll
                  for (int e = 0; e < E; ++e) {
                    r0[e] = fma(-c0, xr[e], r0[e]);
                    r1[e] = fma(-c1, xr[e], r1[e]);
                  }
                }
                *y0p = y0;
                if (b0 + 1 < nbk) *y1p = y1;
              }
          }
          __syncthreads();
        }
        // Gram matrix of the block: thread pair (b, c), halves of the row
        {
          const int ent = threadIdx.x >> 1, h = threadIdx.x & 1;
          const int bb = ent / NB, cc2 = ent % NB;
          R acc = 0;
          if (bb < nbk && cc2 < nbk) {
            const V16* zb = reinterpret_cast<const V16*>(Zs + (size_t)(kb + bb) * ldz);
            const V16* zc = reinterpret_cast<const V16*>(Zs + (size_t)(kb + cc2) * ldz);
            for (int v = h; v < nvec; v += 2) {
              const V16 x = zb[v], y = zc[v];
              const R* xr = reinterpret_cast<const R*>(&x);
              const R* yr = reinterpret_cast<const R*>(&y);
#pragma unroll
              for (int e = 0; e < E; ++e) acc = fma(xr[e], yr[e], acc);
            }
          }
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          if (h == 0 && ent < NB * NB) gq[ent] = acc;
        }
        __syncthreads();
        // Cholesky G = L L^T by warp 0 (lane i owns row i)
        if (warp == 0) {
          R li[NB];
#pragma unroll
          for (int c = 0; c < NB; ++c) li[c] = 0;
          int fail = 0, redo = 0;
          const R gii = (lane < nbk) ? gq[lane * NB + lane] : (R)1;
#pragma unroll
          for (int j = 0; j < NB; ++j) {
            if (j < nbk) {
              R sj = (lane < nbk) ? gq[lane * NB + j] : (R)0;
#pragma unroll
              for (int c = 0; c < j; ++c) sj -= li[c] * __shfl_sync(0xffffffffu, li[c], j);
              const R piv = __shfl_sync(0xffffffffu, sj, j);
              const R gjj = __shfl_sync(0xffffffffu, gii, j);
              if (!(piv > tol * gjj) || !(gjj > (R)0)) fail = 1;
              if (!(piv >= (R)0.5 * gjj) || (kb > 0 && !(gjj >= (R)0.5 * s_n0[j]))) redo = 1;
              const R ljj = sqrt(fmax(piv, (R)0));
              if (lane == j) li[j] = ljj;
              else if (lane > j) li[j] = (ljj > 0) ? sj / ljj : (R)0;
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
          cgs_vectors(kb, kb, kb + nbk);
        } else {
          // Z_blk <- L^{-1} Z_blk, one column entry i per thread
          for (int i = threadIdx.x; i < n; i += blockDim.x) {
            R x[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) x[b] = (b < nbk) ? Zs[(size_t)(kb + b) * ldz + i] : (R)0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              if (b < nbk) {
                R v = x[b];
#pragma unroll
                for (int c = 0; c < b; ++c) v -= lq[b * NB + c] * x[c];
                x[b] = v / lq[b * NB + b];
              }
            }
#pragma unroll
            for (int b = 0; b < NB; ++b)
              if (b < nbk) Zs[(size_t)(kb + b) * ldz + i] = x[b];
          }
          __syncthreads();
        }
        if (rep == 0 && !s_fail && !s_redo) break;   // uniform: set before the barriers above
      }
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
  constexpr int NCOL = sizeof(R) == 4 ? 4 : 2;
  const int nper = (n + 31) >> 5;
  const int ldv = 32 * nper;
  const size_t zbytes = zsm ? zs_bytes + cb_bytes : 0;
  const int rc = min(32, (int)((HeevSmem<R>::kBytes - zbytes) / (2 * (size_t)ldv * sizeof(cpx<R>))));
  if (rc < 1) {   // cannot happen for n <= 256 (the z copy leaves >= 8 n entries)
    if (threadIdx.x == 0) atomicOr(s.status + t, (int32_t)TS_SHAPE);
    return;
  }
  cpx<R>* vbuf[2];
  vbuf[0] = reinterpret_cast<cpx<R>*>(heev_smem + zbytes);
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
    mbar_expect_tx(bar, (uint32_t)(rows * n * sizeof(cpx<R>)));
    if (ldv == n) {
      bulk_g2s(vbuf[g & 1], Hv + (int64_t)jlo * n, (uint32_t)(rows * n * sizeof(cpx<R>)), bar);
    } else {
      for (int rr = 0; rr < rows; ++rr)
        bulk_g2s(vbuf[g & 1] + (size_t)rr * ldv, Hv + (int64_t)(jlo + rr) * n, (uint32_t)(n * sizeof(cpx<R>)), bar);
    }
  };
  if (ldv != n)   // padding columns n .. ldv-1 of both buffers, never copied over
    for (int e = threadIdx.x; e < 2 * rc * (ldv - n); e += blockDim.x) {
      const int r = e / (ldv - n), i = n + e % (ldv - n);
      vbuf[0][(size_t)r * ldv + i] = mk<R>(0, 0);
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
  cpx<R> y[NCOL][PER];
  for (int pass = 0; pass < passes; ++pass) {
    const int k0 = NCOL * (warp + pass * nwarp);
    const bool act = k0 < keep;
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
      for (int a = 0; a < PER; ++a) {
        const int i = lane + 32 * a;
        y[c][a] = (i < n && k0 + c < keep) ? sph[i] * Z(k0 + c, i) : mk<R>(0, 0);
      }
    for (int c = 0; c < nch; ++c) {
      const int g = pass * nch + c;
      const int jtop = n - 3 - c * rc, jlo = max(0, jtop - rc + 1);
      const cpx<R>* vst = vbuf[g & 1];
      const bool ready = mbar_wait(&s_bar[g & 1], (uint32_t)((g >> 1) & 1));
      if (act && ready) {
        for (int j = jtop; j >= jlo; --j) {
          const cpx<R>* v = vst + (j - jlo) * ldv;
          switch ((j + 1) >> 5) {   // groups a < (j + 1) / 32 hold rows <= j only
            case 0: bt_reflector<R, NCOL, PER, 0>(y, v, lane, nper); break;
            case 1: bt_reflector<R, NCOL, PER, 1>(y, v, lane, nper); break;
            case 2: bt_reflector<R, NCOL, PER, 2>(y, v, lane, nper); break;
            case 3: bt_reflector<R, NCOL, PER, 3>(y, v, lane, nper); break;
            case 4: bt_reflector<R, NCOL, PER, 4>(y, v, lane, nper); break;
            case 5: bt_reflector<R, NCOL, PER, 5>(y, v, lane, nper); break;
            case 6: bt_reflector<R, NCOL, PER, 6>(y, v, lane, nper); break;
            default: bt_reflector<R, NCOL, PER, 7>(y, v, lane, nper); break;
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
