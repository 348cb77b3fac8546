// Batched MPS-trajectory kernels.  One CTA per trajectory; every kernel is
// templated on the real type R of the MPS storage (double: LEMPS_FP64,
// float: LEMPS_MIXED).  Reduced densities, the unraveling, branch weights,
// discarded weights and entropies are FP64 in both modes.
//
// Storage: site k of trajectory t is a slot of cap[k] x 2 x cap[k+1] complex
// numbers at mps + site_off[k] + t * slot(k); element (a, s, b) sits at
// (2a + s) * cap[k+1] + b.  Actual bond dimensions bond[t * (n+1) + k] <= cap[k].
// The orthogonality centre is the same site for every trajectory.
#pragma once

#include "common.cuh"
#include "heev.cuh"
#include "gemm.cuh"
#include "tc_contract.cuh"

namespace lemps {

template <class R>
struct SimView {
  cpx<R>* mps;
  const int64_t* site_off;   // [n]
  const int32_t* cap;        // [n+1]
  int32_t* bond;             // [B][n+1]
  int32_t n;
  int64_t B;
  int32_t chi;
  cpx<R>* ws0;               // [B][ws_stride] two-site tensor / QR matrix
  cpx<R>* ws1;               // [B][ws_stride] Gram matrix / reflectors
  cpx<R>* ws2;               // [B][ws_stride] eigenvectors / Q factor
  cpx<R>* ws3;               // [B][ws_stride] scratch
  // complex128 views of ws1..ws3 (allocated at 16 bytes per entry in both
  // precisions): the Gram matrix and the eigensolver's tridiagonalization
  // are FP64 in both modes; the reflectors and the kept eigenvectors are
  // complex128 when u_fp64 is set, else cpx<R> at the start of each
  // trajectory's complex128 slot
  zd* g64;
  zd* u64;
  zd* h64;
  int32_t u_fp64;
  int64_t ws_stride;         // (2 chi)^2
  double* evals;             // [B][2 chi]
  zd* rho12;                 // [B][16]
  zd* top;                   // [B][16] operator applied to the two-site tensor
  double* eps_layer;         // [B]
  double* eps_tot;           // [B]
  double* disc_last;         // [B] discarded weight of the last split
  int32_t* status;           // [B]
  int32_t* kept;             // [B] eigenpairs kept by the last eigensolve
  double* trace;             // [B] trace of the last Gram matrix (FP64)
};

template <class R>
__device__ __forceinline__ cpx<R>* site_ptr(const SimView<R>& s, int k, int64_t t) {
  return s.mps + s.site_off[k] + t * (int64_t)s.cap[k] * 2 * s.cap[k + 1];
}

// ---- initial state |0...0> -----------------------------------------------------
template <class R>
__global__ void k_init_state(SimView<R> s) {
  int64_t t = blockIdx.x;
  if (t >= s.B) return;
  for (int k = threadIdx.x; k <= s.n; k += blockDim.x) s.bond[t * (s.n + 1) + k] = 1;
  for (int k = threadIdx.x; k < s.n; k += blockDim.x) site_ptr(s, k, t)[0] = mk<R>(1, 0);
  if (threadIdx.x == 0) {
    s.eps_layer[t] = 0.0;
    s.eps_tot[t] = 0.0;
    s.status[t] = TS_OK;
  }
}

// ---- blocked Householder QR of a column-major m x n matrix X (ld = m) --------
// Panels of NB columns are factored in shared memory (one warp per column,
// reflectors H = I - 2 v v^dagger with unit v); each panel's compact WY form
// H_0 ... H_{pb-1} = I - V T V^dagger updates the trailing columns and, in a
// backward pass, forms Q = H_0 ... H_{kmin-1} [I; 0] (m x kq) with tiled GEMMs.
// On exit the upper triangle of X holds R; V (m x kmin) keeps the reflectors.
template <class R>
struct QrSmem {
  static constexpr int NB = (sizeof(R) == 8) ? 8 : 16;
  static constexpr int MMAX = 256;
  cpx<R> vs[NB * MMAX];   // panel reflectors, column-major (pm rows)
  cpx<R> p[NB * MMAX];    // panel being factored
  cpx<R> w[NB * 128];     // W = V^dagger X_trail (NB x nt)
  cpx<R> tm[NB * NB];     // T (upper triangular), row-major
  GemmSmem<R> g;
  R red[32];
};

template <class R>
__device__ void qr_build_t(QrSmem<R>& sm, int pm, int pb) {
  constexpr int NB = QrSmem<R>::NB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // D[a][b] = v_a^dagger v_b for a < b, into w (reused).  Warp w takes the
  // columns b = w and NB - 1 - w (NB - 1 pairs together), eight a at a time
  // with lanes over rows; one reduce-scatter butterfly sums the eight dots.
  auto dots = [&](int bcol) {
    if (bcol >= pb) return;
    for (int a0 = 0; a0 < bcol; a0 += 8) {
      R d[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) d[e] = 0;
#pragma unroll 2
      for (int i = lane; i < pm; i += 32) {
        const cpx<R> vb = sm.vs[bcol * pm + i];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (a0 + q < bcol) {
            const cpx<R> va = sm.vs[(a0 + q) * pm + i];
            d[2 * q] = fma(va.re, vb.re, fma(va.im, vb.im, d[2 * q]));
            d[2 * q + 1] = fma(va.re, vb.im, fma(-va.im, vb.re, d[2 * q + 1]));
          }
        }
      }
      const R tot = warp_reduce_scatter<16>(d, lane);
      const int e = Scatter<16>::index(lane), a = a0 + (e >> 1);
      if ((lane & 1) == 0 && a < bcol) {
        if (e & 1) sm.w[a * NB + bcol].im = tot;
        else sm.w[a * NB + bcol].re = tot;
      }
    }
  };
  for (int bq = warp; bq < NB / 2; bq += nwarp) {
    dots(bq);
    dots(NB - 1 - bq);
  }
  __syncthreads();
  // T recurrence T[0:i, i] = -2 T[0:i, 0:i] D[0:i, i], T[i][i] = 2, by one
  // warp: lane r keeps row r of T in registers
  if (warp == 0) {
    cpx<R> trow[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) trow[c] = mk<R>(0, 0);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      if (i < pb) {
        // four partial sums: the chain over c is a quarter as deep
        cpx<R> acc[4] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
#pragma unroll
        for (int c = 0; c < i; ++c)
          if (c >= lane) cfma(acc[c & 3], trow[c], sm.w[c * NB + i]);
        const cpx<R> sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        trow[i] = (lane < i) ? (R)-2 * sum : mk<R>(lane == i ? 2 : 0, 0);
      }
    }
    if (lane < NB)
#pragma unroll
      for (int c = 0; c < NB; ++c) sm.tm[lane * NB + c] = trow[c];
  }
  __syncthreads();
}

// W[a][c] = sum_i conj(V[a][i]) Y[row0 + i][colbase + c] for a < pb, c < ncc
// (<= 128): V is the panel in shared memory, Y column-major in global memory.
// A skinny product (pb <= 16 rows), so instead of 64 x 64 GEMM tiles: slabs
// of SL rows of Y are staged in the panel buffer sm.p (free once the panel is
// factored; SL = 32 in c64, 16 in c128), XOR-swizzled so that both the
// column-wise store and the row-wise read are conflict-free, and thread (c, h)
// accumulates rows a in [h NB / 2, (h + 1) NB / 2) of column c.
template <class R>
__device__ void qr_vdag_y(QrSmem<R>& sm, const cpx<R>* Y, int ldy, int row0, int colbase, int pm, int pb,
                          int ncc) {
  constexpr int NB = QrSmem<R>::NB;
  constexpr int HA = NB / 2;
  constexpr int SL = NB * QrSmem<R>::MMAX / 128;   // staged rows per slab
  static_assert(SL == 16 || SL == 32, "slab height");
  constexpr int PF = SL * 128 / 256;                // staged entries per thread
  cpx<R>* ys = sm.p;
  const int c = threadIdx.x & 127, h = threadIdx.x >> 7;   // 256 threads
  cpx<R> acc[HA];
#pragma unroll
  for (int a = 0; a < HA; ++a) acc[a] = mk<R>(0, 0);
  // the next slab's entries are loaded into registers while this one is used
  cpx<R> pre[PF];
  auto fetch = [&](int i0) {
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      const int e = threadIdx.x + 256 * k, ii = e & (SL - 1), cc = e / SL;
      pre[k] = (i0 + ii < pm && cc < ncc) ? Y[(int64_t)(colbase + cc) * ldy + row0 + i0 + ii] : mk<R>(0, 0);
    }
  };
  fetch(0);
  for (int i0 = 0; i0 < pm; i0 += SL) {
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      const int e = threadIdx.x + 256 * k, ii = e & (SL - 1), cc = e / SL;
      ys[ii * 128 + (cc ^ ii)] = pre[k];
    }
    __syncthreads();
    if (i0 + SL < pm) fetch(i0 + SL);
    const int ni = min(SL, pm - i0);
    for (int ii = 0; ii < ni; ++ii) {
      const cpx<R> y = ys[ii * 128 + (c ^ ii)];
      const cpx<R>* vrow = sm.vs + (h * HA) * pm + i0 + ii;
#pragma unroll
      for (int a = 0; a < HA; ++a) cfmac(acc[a], vrow[a * pm], y);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < HA; ++a)
    if (h * HA + a < pb && c < ncc) sm.w[(h * HA + a) * 128 + c] = acc[a];
}

// Y[row0 + i][colbase + c] -= sum_a V[a][i] W[a][c] for i < pm, c < ncc (<=
// 128): V (the panel) and W in shared memory, Y column-major in global
// memory.  A warp owns 64 rows x 8 columns: lane l holds rows l and l + 32 of
// the 8 columns in registers, so every global load and store covers 32
// consecutive rows of one column; V is read conflict-free, W by broadcast.
template <class R>
__device__ void qr_update_y(QrSmem<R>& sm, cpx<R>* Y, int ldy, int row0, int colbase, int pm, int pb, int ncc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int nrb = (pm + 63) >> 6, ncb = (ncc + 7) >> 3;
  for (int u = warp; u < nrb * ncb; u += nwarp) {
    const int rb = u % nrb, c0 = (u / nrb) * 8;
    const int i0 = rb * 64 + lane, i1 = i0 + 32;
    const bool in0 = i0 < pm, in1 = i1 < pm;
    cpx<R> y0[8], y1[8];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const bool cin = c0 + cc < ncc;
      cpx<R>* col = Y + (int64_t)(colbase + c0 + cc) * ldy + row0;
      y0[cc] = (cin && in0) ? col[i0] : mk<R>(0, 0);
      y1[cc] = (cin && in1) ? col[i1] : mk<R>(0, 0);
    }
#pragma unroll 4
    for (int a = 0; a < pb; ++a) {
      const cpx<R> v0 = in0 ? sm.vs[a * pm + i0] : mk<R>(0, 0);
      const cpx<R> v1 = in1 ? sm.vs[a * pm + i1] : mk<R>(0, 0);
      const cpx<R>* wr = sm.w + a * 128 + c0;
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        const cpx<R> w = wr[cc];
        y0[cc] -= v0 * w;
        y1[cc] -= v1 * w;
      }
    }
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      if (c0 + cc < ncc) {
        cpx<R>* col = Y + (int64_t)(colbase + c0 + cc) * ldy + row0;
        if (in0) col[i0] = y0[cc];
        if (in1) col[i1] = y1[cc];
      }
    }
  }
}

// Q_sub (rows p0.., kq columns) <- (I - V T V^dagger) Q_sub, or with T^dagger
// when adjoint (the factorization's trailing update on X).
template <class R>
__device__ void qr_apply_block(QrSmem<R>& sm, cpx<R>* Y, int ldy, int row0, int col0, int pm, int pb, int nc,
                               bool adjoint) {
  constexpr int NB = QrSmem<R>::NB;
  for (int c0 = 0; c0 < nc; c0 += 128) {
    const int ncc = min(128, nc - c0);
    // W = V^dagger Y  (pb x ncc)
    qr_vdag_y(sm, Y, ldy, row0, col0 + c0, pm, pb, ncc);
    __syncthreads();
    // W <- T W  or  T^dagger W: thread (e, h) reads column e of W into
    // registers and, after a barrier, writes its rows [h NB/2, (h+1) NB/2)
    {
      const int e = threadIdx.x & 127, h = threadIdx.x >> 7;   // 256 threads
      cpx<R> col[NB];
#pragma unroll
      for (int bb = 0; bb < NB; ++bb) col[bb] = (bb < pb && e < ncc) ? sm.w[bb * 128 + e] : mk<R>(0, 0);
      __syncthreads();
      if (e < ncc) {
#pragma unroll
        for (int q = 0; q < NB / 2; ++q) {
          const int a = h * (NB / 2) + q;
          if (a < pb) {
            cpx<R> acc = mk<R>(0, 0);
#pragma unroll
            for (int bb = 0; bb < NB; ++bb)
              if (bb < pb) cfma(acc, adjoint ? conj(sm.tm[bb * NB + a]) : sm.tm[a * NB + bb], col[bb]);
            sm.w[a * 128 + e] = acc;
          }
        }
      }
    }
    __syncthreads();
    // Y -= V W
    qr_update_y(sm, Y, ldy, row0, col0 + c0, pm, pb, ncc);
    __syncthreads();
  }
}

template <class R>
__device__ void householder_qr(cpx<R>* X, cpx<R>* V, cpx<R>* Qm, int m, int n, int kq, QrSmem<R>& sm) {
  constexpr int NB = QrSmem<R>::NB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int kmin = min(m, n);
  for (int p0 = 0; p0 < kmin; p0 += NB) {
    const int pb = min(NB, kmin - p0), pm = m - p0;
    for (int jj = warp; jj < pb; jj += nwarp)
      for (int i = lane; i < pm; i += 32) sm.p[jj * pm + i] = X[(int64_t)(p0 + jj) * m + p0 + i];
    __syncthreads();
    // tail norm of column 0 by a block reduction; the norm of each later
    // column is formed by the warp that applies the previous reflector to it
    __shared__ R s_nrm[2];
    {
      R part = 0;
      for (int i = threadIdx.x; i < pm; i += blockDim.x) part += norm2(sm.p[i]);
      part = block_sum(part, sm.red);
      if (threadIdx.x == 0) s_nrm[0] = part;
      __syncthreads();
    }
    for (int jj = 0; jj < pb; ++jj) {
      const R nrm2 = s_nrm[jj & 1];
      R nrm = sqrt(nrm2);
      cpx<R> x0 = sm.p[jj * pm + jj];
      R ax0 = sqrt(norm2(x0));
      cpx<R> ph = (ax0 > 0) ? mk<R>(x0.re / ax0, x0.im / ax0) : mk<R>(1, 0);
      cpx<R> alpha = mk<R>(-nrm * ph.re, -nrm * ph.im);
      R vn2 = nrm2 + nrm2 + 2 * nrm * ax0;
      R inv = (vn2 > 0) ? (R)1 / sqrt(vn2) : (R)0;
      for (int i = threadIdx.x; i < pm; i += blockDim.x) {
        cpx<R> vi = mk<R>(0, 0);
        if (i > jj) vi = sm.p[jj * pm + i] * inv;
        else if (i == jj) vi = (x0 - alpha) * inv;
        sm.vs[jj * pm + i] = vi;
      }
      __syncthreads();
      for (int c = jj + warp; c < pb; c += nwarp) {
        cpx<R> d = mk<R>(0, 0);
#pragma unroll 4
        for (int i = jj + lane; i < pm; i += 32) cfmac(d, sm.vs[jj * pm + i], sm.p[c * pm + i]);
        d.re = warp_sum(d.re);
        d.im = warp_sum(d.im);
        d = (R)2 * d;
        R nn = 0;
        // unrolled so that the loads of several rows precede their stores
#pragma unroll 4
        for (int i = jj + lane; i < pm; i += 32) {
          const cpx<R> y = sm.p[c * pm + i] - sm.vs[jj * pm + i] * d;
          sm.p[c * pm + i] = y;
          if (i > jj) nn += norm2(y);
        }
        if (c == jj + 1) {
          nn = warp_sum(nn);
          if (lane == 0) s_nrm[(jj + 1) & 1] = nn;
        }
      }
      __syncthreads();
    }
    for (int jj = warp; jj < pb; jj += nwarp) {
      for (int i = lane; i < pm; i += 32) X[(int64_t)(p0 + jj) * m + p0 + i] = sm.p[jj * pm + i];
      for (int i = lane; i < m; i += 32)
        V[(int64_t)(p0 + jj) * m + i] = (i >= p0) ? sm.vs[jj * pm + (i - p0)] : mk<R>(0, 0);
    }
    __syncthreads();
    if (p0 + pb < n) {
      qr_build_t(sm, pm, pb);
      qr_apply_block(sm, X, m, p0, p0 + pb, pm, pb, n - p0 - pb, true);
    }
  }
  // Q = H_0 ... H_{kmin-1} [I; 0]
  for (int c = warp; c < kq; c += nwarp)
    for (int i = lane; i < m; i += 32) Qm[(int64_t)c * m + i] = mk<R>(i == c ? 1 : 0, 0);
  __syncthreads();
  const int npanel = (kmin + NB - 1) / NB;
  for (int pi = npanel - 1; pi >= 0; --pi) {
    const int p0 = pi * NB, pb = min(NB, kmin - p0), pm = m - p0;
    for (int jj = warp; jj < pb; jj += nwarp)
      for (int i = lane; i < pm; i += 32) sm.vs[jj * pm + i] = V[(int64_t)(p0 + jj) * m + p0 + i];
    __syncthreads();
    qr_build_t(sm, pm, pb);
    // columns j < p0 are still e_j here (the later reflectors touch rows >= p0
    // only), so this block changes columns p0.. alone
    qr_apply_block(sm, Qm, m, p0, p0, pm, pb, kq - p0, false);
  }
}

// dst[q * ldd + p] = src[p * lds + q] for p < P, q < Q: a transposing copy
// through shared memory (TP x TQ tiles, rows padded by one entry), with
// coalesced global loads and stores; a tile's loads are all issued before
// its stores.  `tile` holds TP * (TQ + 1) entries; 256 threads.
template <class R>
__device__ void transpose_copy(cpx<R>* dst, int64_t ldd, const cpx<R>* src, int64_t lds, int P, int Q, cpx<R>* tile) {
  constexpr int TP = 32, TQ = sizeof(R) == 4 ? 128 : 64, LDT = TQ + 1;
  constexpr int PT = TP * TQ / kGemmThreads;
  for (int p0 = 0; p0 < P; p0 += TP)
    for (int q0 = 0; q0 < Q; q0 += TQ) {
      cpx<R> r[PT];
#pragma unroll
      for (int k = 0; k < PT; ++k) {
        const int e = threadIdx.x + kGemmThreads * k, pp = e / TQ, qq = e % TQ;
        r[k] = (p0 + pp < P && q0 + qq < Q) ? src[(int64_t)(p0 + pp) * lds + q0 + qq] : mk<R>(0, 0);
      }
#pragma unroll
      for (int k = 0; k < PT; ++k) {
        const int e = threadIdx.x + kGemmThreads * k, pp = e / TQ, qq = e % TQ;
        tile[pp * LDT + qq] = r[k];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < PT; ++k) {
        const int e = threadIdx.x + kGemmThreads * k, pp = e % TP, qq = e / TP;
        if (p0 + pp < P && q0 + qq < Q) dst[(int64_t)(q0 + qq) * ldd + p0 + pp] = tile[pp * LDT + qq];
      }
      __syncthreads();
    }
}

// Move the centre from site k to k+1 (dir = +1, QR of A_k as (2 dl) x dr) or
// to k-1 (dir = -1, LQ of A_k as dl x (2 dr)).
template <class R>
__global__ void __launch_bounds__(kGemmThreads, sizeof(R) == 4 ? 2 : 1) k_move_center(SimView<R> s, int k, int dir) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  extern __shared__ __align__(16) unsigned char move_smem[];
  QrSmem<R>& qs = *reinterpret_cast<QrSmem<R>*>(move_smem);
  GemmSmem<R>& sm = qs.g;
  int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[k], dr = bd[k + 1];
  const int capr = s.cap[k + 1];
  cpx<R>* A = site_ptr(s, k, t);
  cpx<R>* X = s.ws0 + t * s.ws_stride;
  cpx<R>* V = s.ws1 + t * s.ws_stride;
  cpx<R>* Qm = s.ws2 + t * s.ws_stride;
  cpx<R>* Tm = s.ws3 + t * s.ws_stride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // element copies run as (warp, lane) loops, lanes along the site tensor's
  // contiguous index, with no per-element division; the transposing copies
  // of the QR direction go through shared-memory tiles
  cpx<R>* tile = reinterpret_cast<cpx<R>*>(move_smem);
  static_assert(sizeof(QrSmem<R>) >= 32 * ((sizeof(R) == 4 ? 128 : 64) + 1) * sizeof(cpx<R>),
                "the transpose tile fits in the QR shared memory");
  if (dir > 0) {
    const int m = 2 * dl, n = dr, r = min(m, n);
    transpose_copy(X, m, A, capr, m, n, tile);
    householder_qr(X, V, Qm, m, n, r, qs);
    // A_{k+1} <- R A_{k+1}: A_{k+1} is dr x (2 d2), R is r x dr (upper part of X)
    const int d2 = bd[k + 2], cap2 = s.cap[k + 2];
    cpx<R>* B = site_ptr(s, k + 1, t);
    cta_gemm<R, false, false>(
        r, 2 * d2, dr, [&](int i, int l) { return l >= i ? X[(int64_t)l * m + i] : mk<R>(0, 0); },
        [&](int l, int cc) {
          const int ss = cc >= d2, b = cc - ss * d2;   // cc < 2 d2
          return B[(int64_t)(l * 2 + ss) * cap2 + b];
        },
        [&](int i, int cc, cpx<R> v) { Tm[(int64_t)i * 2 * d2 + cc] = v; }, sm);
    __syncthreads();
    for (int i = warp; i < r; i += nwarp)
      for (int cc = lane; cc < 2 * d2; cc += 32) {
        const int ss = cc >= d2, b = cc - ss * d2;
        B[(int64_t)(i * 2 + ss) * cap2 + b] = Tm[(int64_t)i * 2 * d2 + cc];
      }
    // A_k <- Q (m x r) reshaped (dl, 2, r)
    transpose_copy(A, capr, Qm, m, r, m, tile);
    if (threadIdx.x == 0) bd[k + 1] = r;
  } else {
    // X = A_k^dagger: (2 dr) x dl, column-major, X[c][i] = conj(A[i][c])
    const int m = 2 * dr, n = dl, r = min(m, n);
    for (int c = warp; c < n; c += nwarp)   // row c of A, column i of A (= (s, b))
      for (int i = lane; i < m; i += 32) {
        const int ss = i >= dr, b = i - ss * dr;
        X[(int64_t)c * m + i] = conj(A[(int64_t)(c * 2 + ss) * capr + b]);
      }
    __syncthreads();
    householder_qr(X, V, Qm, m, n, r, qs);
    // A_k = L Q with L = R'^dagger (dl x r), Q = Q'^dagger (r x 2dr).
    // A_{k-1} <- A_{k-1} L: A_{k-1} is (2 d0) x dl, result (2 d0) x r.
    const int d0 = bd[k - 1], cap1 = s.cap[k];
    cpx<R>* P = site_ptr(s, k - 1, t);
    cta_gemm<R, true, false>(
        2 * d0, r, dl, [&](int row, int l) { return P[(int64_t)row * cap1 + l]; },
        [&](int l, int j) { return l >= j ? conj(X[(int64_t)l * m + j]) : mk<R>(0, 0); },
        [&](int row, int j, cpx<R> v) { Tm[(int64_t)row * r + j] = v; }, sm);
    __syncthreads();
    for (int row = warp; row < 2 * d0; row += nwarp)
      for (int j = lane; j < r; j += 32) P[(int64_t)row * cap1 + j] = Tm[(int64_t)row * r + j];
    // A_k <- Q'^dagger: A[j][ss][b] = conj(Q'[(ss, b)][j])
    for (int j = warp; j < r; j += nwarp)
      for (int i = lane; i < m; i += 32) {
        const int ss = i >= dr, b = i - ss * dr;
        A[(int64_t)(j * 2 + ss) * capr + b] = conj(Qm[(int64_t)j * m + i]);
      }
    if (threadIdx.x == 0) bd[k] = r;
  }
}

// ---- two-site contraction and the 4x4 reduced density ------------------------
// Theta[a][s1][s2][b] = sum_m A_q[a][s1][m] A_{q+1}[m][s2][b] into ws0 as a
// (2 dl) x (2 dr) row-major matrix; rho12[(s1 s2), (t1 t2)] =
// sum_{a,b} Theta[a,s1,s2,b] conj(Theta[a,t1,t2,b]) in FP64.
// rho12[(s1 s2), (t1 t2)] = sum_{a,b} Theta[a,s1,s2,b] conj(Theta[a,t1,t2,b]) in
// FP64 from the two-site tensor in ws0 (row-major, ld = 2 dr).
// Compensated FP32 sum (s, c): TwoSum (Knuth) keeps each addition's rounding
// error in c, so s + c carries about twice FP32's precision.
__device__ __forceinline__ void comp_add(float& s, float& c, float x) {
  const float t = s + x, bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

template <class R>
__device__ __forceinline__ void contract_rho12(const SimView<R>& s, int64_t t, const cpx<R>* th, int dl, int dr,
                                               double* red, double* scratch) {
  const int64_t ld = 2 * dr;
  const int nel = dl * dr;
  if constexpr (sizeof(R) == 4) {
    // rho12 is Hermitian: the 10 entries i <= j are formed.  Products in
    // complex64, each thread's sums in compensated FP32 (an FP64 instruction
    // costs the FP64 pipe 64 cycles per warp here), combined over the warp with
    // FP32 shuffles; only the per-warp partials are added in FP64.  scratch:
    // 20 x (warps) doubles of shared memory.
    float sum[20], cmp[20];
#pragma unroll
    for (int p = 0; p < 20; ++p) sum[p] = cmp[p] = 0.f;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      const int a = e / dr, b = e - a * dr;
      cpx<R> v[4];
      v[0] = th[(int64_t)(2 * a) * ld + b];
      v[1] = th[(int64_t)(2 * a) * ld + dr + b];
      v[2] = th[(int64_t)(2 * a + 1) * ld + b];
      v[3] = th[(int64_t)(2 * a + 1) * ld + dr + b];
      int p = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j, ++p) {
          comp_add(sum[2 * p], cmp[2 * p], v[i].re * v[j].re + v[i].im * v[j].im);
          comp_add(sum[2 * p + 1], cmp[2 * p + 1], v[i].im * v[j].re - v[i].re * v[j].im);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    // butterfly: every lane ends with the warp's totals; lane p keeps value p
    float ms = 0.f, mc = 0.f;
#pragma unroll
    for (int p = 0; p < 20; ++p) {
      float sv = sum[p], cv = cmp[p];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, sv, o), c2 = __shfl_xor_sync(0xffffffffu, cv, o);
        cv += c2;
        comp_add(sv, cv, s2);
      }
      if (lane == p) {
        ms = sv;
        mc = cv;
      }
    }
    if (lane < 20) scratch[lane * nw + warp] = (double)ms + (double)mc;
    __syncthreads();
    if (threadIdx.x < 10) {
      const int p = threadIdx.x;
      double re = 0.0, im = 0.0;
      for (int w = 0; w < nw; ++w) {
        re += scratch[(2 * p) * nw + w];
        im += scratch[(2 * p + 1) * nw + w];
      }
      int i = 0, j = p;   // p-th pair i <= j in row order
      while (j >= 4 - i) {
        j -= 4 - i;
        ++i;
      }
      j += i;
      s.rho12[t * 16 + i * 4 + j] = mk(re, im);
      if (j != i) s.rho12[t * 16 + j * 4 + i] = mk(re, -im);
    }
    return;
  } else {
    (void)scratch;
    // rho12 is Hermitian: the 10 entries i <= j are formed, in FP64.
    double acc[10][2];
#pragma unroll
    for (int p = 0; p < 10; ++p) acc[p][0] = acc[p][1] = 0.0;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      const int a = e / dr, b = e - a * dr;
      cpx<R> v[4];
      v[0] = th[(int64_t)(2 * a) * ld + b];
      v[1] = th[(int64_t)(2 * a) * ld + dr + b];
      v[2] = th[(int64_t)(2 * a + 1) * ld + b];
      v[3] = th[(int64_t)(2 * a + 1) * ld + dr + b];
      int p = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j, ++p) {
          acc[p][0] += v[i].re * v[j].re + v[i].im * v[j].im;
          acc[p][1] += v[i].im * v[j].re - v[i].re * v[j].im;
        }
    }
    int p = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = i; j < 4; ++j, ++p) {
        double re = block_sum(acc[p][0], red);
        double im = block_sum(acc[p][1], red);
        if (threadIdx.x == 0) {
          s.rho12[t * 16 + i * 4 + j] = mk(re, im);
          if (j != i) s.rho12[t * 16 + j * 4 + i] = mk(re, -im);
        }
      }
  }
}

// TILE selects the GEMM tile shape (GemmTileShape<R, TILE>); every shape
// gives the same result bit for bit.
template <class R, int TILE = 0>
__global__ void __launch_bounds__(kGemmThreads) k_contract(SimView<R> s, int q) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  __shared__ double red[32];
  __shared__ GemmSmem<R, GemmTileShape<R, TILE>::BM, GemmTileShape<R, TILE>::BN> sm;
  const int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[q], dm = bd[q + 1], dr = bd[q + 2];
  const int capm = s.cap[q + 1], capr = s.cap[q + 2];
  const cpx<R>* A = site_ptr(s, q, t);
  const cpx<R>* B = site_ptr(s, q + 1, t);
  cpx<R>* th = s.ws0 + t * s.ws_stride;
  const int64_t ld = 2 * dr;
  cta_gemm<R, true, false>(
      2 * dl, 2 * dr, dm, [&](int i, int k) { return A[(int64_t)i * capm + k]; },
      [&](int k, int j) {
        const int s2 = j >= dr, b = j - s2 * dr;   // j < 2 dr
        return B[(int64_t)(2 * k + s2) * capr + b];
      },
      [&](int i, int j, cpx<R> v) { th[(int64_t)i * ld + j] = v; }, sm);
  __syncthreads();
  contract_rho12(s, t, th, dl, dr, red, reinterpret_cast<double*>(&sm));
}

// The same contraction on the tensor cores (mixed precision; 3xTF32 complex
// GEMM, tc_contract.cuh) for gates whose three site capacities lie in [64,
// 128]: mapA views site q as [2 cap_q][cap_{q+1}] complex64 rows, mapB site q
// + 1 as [2 cap_{q+1}][cap_{q+2}], both over all trajectories.  One CTA per
// trajectory holding all 512 tensor-memory columns (at most one CTA per SM).
__global__ void __launch_bounds__(tc::kThreads, 1) k_contract_tc(const __grid_constant__ CUtensorMap mapA,
                                                                 const __grid_constant__ CUtensorMap mapB,
                                                                 SimView<float> s, int q) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bars[tc::kNumBars];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ double red[32];
  const int warp = threadIdx.x >> 5;
  const int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[q], dm = bd[q + 1], dr = bd[q + 2];
  const int capr = s.cap[q + 2];
  cpx<float>* th = s.ws0 + t * s.ws_stride;
  if (threadIdx.x == 0) {
    tc::init_bars(bars);
    s_err = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(&s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_for_bulk_copies();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const bool ok = tc::gemm(&mapA, &mapB, (int)t, 2 * dl, dm, dr, capr, site_ptr(s, q, t), s.cap[q + 1],
                           site_ptr(s, q + 1, t), sm, bars, tmem, th, 2 * dr, &s_err);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(s.status + t, (int32_t)TS_COPY);
    return;
  }
  // the stages of the GEMM are free: scratch for the epilogue's partial sums
  contract_rho12(s, t, th, dl, dr, red, reinterpret_cast<double*>(sm));
}

// ---- apply T to Theta and build the Gram matrix ------------------------------
// side = 0: left Gram  G = Theta Theta^dagger (2dl x 2dl)
// side = 1: right Gram G = Theta^dagger Theta (2dr x 2dr)
// TILE selects the GEMM tile shape of the Gram product, as in k_contract.
template <class R, int TILE = 0>
__global__ void __launch_bounds__(kGemmThreads) k_apply_gram(SimView<R> s, int q, int side) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  __shared__ GemmSmem<R, GemmTileShape<R, TILE>::BM, GemmTileShape<R, TILE>::BN> sm;
  const int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[q], dr = bd[q + 2];
  cpx<R>* th = s.ws0 + t * s.ws_stride;
  zd* G = s.g64 + t * s.ws_stride;   // FP64 input of the eigensolver
  // T (FP64 from the unraveling) is applied in the storage precision
  __shared__ cpx<R> T[16];
  if (threadIdx.x < 16) T[threadIdx.x] = cast<R>(s.top[t * 16 + threadIdx.x]);
  __syncthreads();
  const int64_t ld = 2 * dr;
  for (int e = threadIdx.x; e < dl * dr; e += blockDim.x) {
    const int a = e / dr, b = e - a * dr;
    cpx<R> v[4];
    v[0] = th[(int64_t)(2 * a) * ld + b];
    v[1] = th[(int64_t)(2 * a) * ld + dr + b];
    v[2] = th[(int64_t)(2 * a + 1) * ld + b];
    v[3] = th[(int64_t)(2 * a + 1) * ld + dr + b];
    cpx<R> w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      cpx<R> acc = mk<R>(0, 0);
#pragma unroll
      for (int k = 0; k < 4; ++k) cfma(acc, T[i * 4 + k], v[k]);
      w[i] = acc;
    }
    th[(int64_t)(2 * a) * ld + b] = w[0];
    th[(int64_t)(2 * a) * ld + dr + b] = w[1];
    th[(int64_t)(2 * a + 1) * ld + b] = w[2];
    th[(int64_t)(2 * a + 1) * ld + dr + b] = w[3];
  }
  __syncthreads();
  const int ng = side == 0 ? 2 * dl : 2 * dr;
  auto st = [&](int i, int j, cpx<R> v) {
    if (j >= i) {
      const zd d = cast<double>(v);
      G[(int64_t)i * ng + j] = d;
      G[(int64_t)j * ng + i] = conj(d);
    }
  };
  if (side == 0) {
    cta_gemm<R, true, true>(
        ng, ng, 2 * dr, [&](int i, int k) { return th[(int64_t)i * ld + k]; },
        [&](int k, int j) { return conj(th[(int64_t)j * ld + k]); }, st, sm, true);
  } else {
    cta_gemm<R, false, false>(
        ng, ng, 2 * dl, [&](int i, int k) { return conj(th[(int64_t)k * ld + i]); },
        [&](int k, int j) { return th[(int64_t)k * ld + j]; }, st, sm, true);
  }
}

// Size of the Gram matrix: mode 0: 2 bond[k] (left Gram of the pair at k),
// mode 1: 2 bond[k+2] (right Gram), mode 2: bond[k+1] (site Gram of A_k).
__device__ __forceinline__ int gram_size(const int32_t* bd, int k, int mode) {
  return mode == 0 ? 2 * bd[k] : (mode == 1 ? 2 * bd[k + 2] : bd[k + 1]);
}

template <class R>
HeevView<double> heev_view(const SimView<R>& s) {
  HeevView<double> h;
  h.ws1 = s.g64; h.ws2 = s.u64; h.ws3 = s.h64; h.ws_stride = s.ws_stride;
  h.evals = s.evals; h.kept = s.kept; h.trace = s.trace; h.bond = s.bond; h.status = s.status;
  h.nq = s.n; h.chi = s.chi; h.B = s.B;
  return h;
}

// ---- split and truncate ------------------------------------------------------
// U (ws2, column-major, ng x keep; complex128 or the storage precision, as
// the eigensolver back-transformed it) holds the kept eigenvectors of the
// Gram matrix; they enter the products in the storage precision.  side 0 (left Gram, centre -> q+1):
//   A_q = U (left-orthonormal), B = U^dagger Theta, R = Theta - U B,
//   A_{q+1} = B / ||B||.
// side 1 (right Gram, centre -> q):
//   A_{q+1} = U^dagger (right-orthonormal), B = Theta U, R = Theta - B U^dagger,
//   A_q = B / ||B||.
// The discarded weight is eps = ||R||_F^2 / ||Theta||_F^2, accumulated in FP64
// from the residual itself, which keeps it accurate in complex64 (a sum of
// discarded eigenvalues would carry an error of ~ n eps_32).  The split keeps
// the default GEMM tile: its norms are summed per thread inside the GEMM
// epilogues, so another tile shape would change their rounding (and the
// normalization of the new site tensor with it).
template <class R>
__global__ void __launch_bounds__(kGemmThreads) k_split(SimView<R> s, int q, int side) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  __shared__ double redd[32];
  __shared__ GemmSmem<R> sm;
  int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[q], dr = bd[q + 2];
  const int ng = side == 0 ? 2 * dl : 2 * dr;
  const int keep = s.kept[t];
  const double tot = s.trace[t];
  const cpx<R>* th = s.ws0 + t * s.ws_stride;
  // the eigensolver writes U in complex128 (u_fp64) or in the storage
  // precision, at the start of this trajectory's complex128 slot of ws2
  const zd* U64 = s.u64 + t * s.ws_stride;
  const cpx<R>* Us = reinterpret_cast<const cpx<R>*>(U64);
  const bool u64 = s.u_fp64 != 0;
  auto U = [&](int64_t e) { return u64 ? cast<R>(U64[e]) : Us[e]; };
  const int64_t ld = 2 * dr;
  cpx<R>* A = site_ptr(s, q, t);
  cpx<R>* B = site_ptr(s, q + 1, t);
  const int capm = s.cap[q + 1], capr = s.cap[q + 2];
  auto bslot = [&](int k, int j) -> cpx<R>& {
    const int s2 = j >= dr, b = j - s2 * dr;   // j < 2 dr
    return B[(int64_t)(k * 2 + s2) * capr + b];
  };
  double bn = 0.0, rn = 0.0;
  // The projection B and the residual are formed one block of Theta at a time
  // (kBlk = 64 columns for side 0, 64 rows for side 1): the block is read by
  // both products while it is still in L2, and so is U, instead of re-reading
  // Theta once per output tile row of a whole-matrix product (measured at
  // chi = 128: 1.54 MB of DRAM traffic per trajectory against 1.28 MB of
  // operands and outputs; 1.85 MB with blocks of 128, 2.78 MB unblocked).
  constexpr int kBlk = kGemmBN;
  if (side == 0) {
    // A_q = U: U is column-major (ng rows), A_q row-major; 32 x 32 tiles
    // through shared memory keep both sides of the copy contiguous
    static_assert(sizeof(GemmSmem<R>) >= 32 * 33 * sizeof(cpx<R>), "transpose tile");
    cpx<R>* tile = reinterpret_cast<cpx<R>*>(&sm);   // 32 x 33
    for (int r0 = 0; r0 < 2 * dl; r0 += 32)
      for (int k0 = 0; k0 < keep; k0 += 32) {
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
          const int kk = e >> 5, rr = e & 31;
          if (r0 + rr < 2 * dl && k0 + kk < keep) tile[kk * 33 + rr] = U((int64_t)(k0 + kk) * ng + r0 + rr);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
          const int rr = e >> 5, kk = e & 31;
          if (r0 + rr < 2 * dl && k0 + kk < keep) A[(int64_t)(r0 + rr) * capm + k0 + kk] = tile[kk * 33 + rr];
        }
        __syncthreads();
      }
    for (int j0 = 0; j0 < 2 * dr; j0 += kBlk) {
      const int nb = min(kBlk, 2 * dr - j0);
      // B[:, block] = U^dagger Theta[:, block]  (keep x nb)
      cta_gemm<R, true, false>(
          keep, nb, 2 * dl, [&](int i, int k) { return conj(U((int64_t)i * ng + k)); },
          [&](int k, int j) { return th[(int64_t)k * ld + j0 + j]; },
          [&](int i, int j, cpx<R> v) {
            bslot(i, j0 + j) = v;
            bn += (double)norm2(v);
          },
          sm);
      __syncthreads();
      // residual Theta[:, block] - U B[:, block]
      cta_gemm<R, false, false>(
          2 * dl, nb, keep, [&](int i, int k) { return U((int64_t)k * ng + i); },
          [&](int k, int j) { return bslot(k, j0 + j); },
          [&](int i, int j, cpx<R> v) { rn += (double)norm2(th[(int64_t)i * ld + j0 + j] - v); }, sm);
      __syncthreads();
    }
  } else {
    for (int e = threadIdx.x; e < keep * 2 * dr; e += blockDim.x) {
      const int k = e / (2 * dr), c = e % (2 * dr);
      bslot(k, c) = conj(U((int64_t)k * ng + c));
    }
    for (int i0 = 0; i0 < 2 * dl; i0 += kBlk) {
      const int mb = min(kBlk, 2 * dl - i0);
      // B[block, :] = Theta[block, :] U  (mb x keep) into A_q
      cta_gemm<R, true, true>(
          mb, keep, 2 * dr, [&](int i, int k) { return th[(int64_t)(i0 + i) * ld + k]; },
          [&](int k, int j) { return U((int64_t)j * ng + k); },
          [&](int i, int j, cpx<R> v) {
            A[(int64_t)(i0 + i) * capm + j] = v;
            bn += (double)norm2(v);
          },
          sm);
      __syncthreads();
      // residual Theta[block, :] - B[block, :] U^dagger
      cta_gemm<R, true, false>(
          mb, 2 * dr, keep, [&](int i, int k) { return A[(int64_t)(i0 + i) * capm + k]; },
          [&](int k, int j) { return conj(U((int64_t)k * ng + j)); },
          [&](int i, int j, cpx<R> v) { rn += (double)norm2(th[(int64_t)(i0 + i) * ld + j] - v); }, sm);
      __syncthreads();
    }
  }
  rn = block_sum(rn, redd);
  bn = block_sum(bn, redd);
  const double nrm = bn > 0.0 ? 1.0 / sqrt(bn) : 0.0;
  if (side == 0) {
    for (int e = threadIdx.x; e < keep * 2 * dr; e += blockDim.x) {
      cpx<R>& p = bslot(e / (2 * dr), e % (2 * dr));
      p = (R)nrm * p;
    }
  } else {
    for (int e = threadIdx.x; e < 2 * dl * keep; e += blockDim.x) {
      cpx<R>* p = A + (int64_t)(e / keep) * capm + (e % keep);
      *p = (R)nrm * *p;
    }
  }
  if (threadIdx.x == 0) {
    // keeping the full rank min(2 dl, 2 dr) discards nothing: eps = 0 exactly
    const bool full = keep >= min(2 * dl, 2 * dr);
    const double disc = (tot > 0.0 && !full) ? fmin(fmax(rn / tot, 0.0), 1.0) : 0.0;
    if (!(tot > 0.0) || !isfinite(tot) || !isfinite(rn) || !(bn > 0.0)) atomicOr(s.status + t, (int32_t)TS_NORM);
    s.disc_last[t] = disc;
    s.eps_layer[t] += disc;
    bd[q + 1] = keep;
  }
}

// ---- layer bookkeeping: eps_tot += 4 sqrt(2 sum_k eps_k) (App. B) -------------
template <class R>
__global__ void k_layer_end(SimView<R> s, double* hist, int hist_stride, int layer) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.B) return;
  const double e = 4.0 * sqrt(2.0 * s.eps_layer[t]);
  s.eps_tot[t] += e;
  s.eps_layer[t] = 0.0;
  if (hist) hist[t * hist_stride + layer] = e;   // per-layer history (concentration bound)
}

// Concentration-improved bound (Sec. III.C; appendix on concentration):
// out[t] = sum_l w(L - 1 - l) hist[t][l] over the L layers, w(k) = alpha^k
// (kind 0, param alpha) or min(sqrt(8 n) (1 - p)^k, 1) (kind 1, param p),
// capped like the plain bound (kept when <= eps_max - 2, else eps_max).
__global__ void k_eps_weighted(const double* hist, int hist_stride, int64_t B, int L, int kind, double param,
                               int n, double eps_max, double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B) return;
  const double c = sqrt(8.0 * (double)n);
  double e = 0.0;
  for (int l = 0; l < L; ++l) {
    const int k = L - 1 - l;
    const double w = (kind == 0) ? pow(param, (double)k) : fmin(c * pow(1.0 - param, (double)k), 1.0);
    e += w * hist[t * hist_stride + l];
  }
  out[t] = (e <= eps_max - 2.0) ? e : eps_max;
}

// Output-distribution sampling (Lemma sampling_reduction): with the centre on
// site 0 (sites 1.. right-orthonormal), bit k of a shot is drawn from the
// conditional weights p_s = ||v A_k[:, s, :]||^2 of the running row vector v
// (v = [1] before site 0, then v <- v A_k[:, b, :] / sqrt(p_b)): bit 0 when
// u (p0 + p1) < p0, u = Philox(seed; trajectory id, 2^62 + shot, k), a counter
// domain the noise sites never use.  One CTA per (trajectory, shot); v and the
// products in FP64.
template <class R>
__global__ void __launch_bounds__(256) k_sample_bits(SimView<R> s, int n_shots, uint64_t seed, int64_t traj_offset,
                                                     uint8_t* out) {
  const int64_t t = blockIdx.x;
  const int shot = blockIdx.y;
  if (t >= s.B) return;
  __shared__ zd v[256], w0s[256], w1s[256];
  __shared__ double red[32];
  const int32_t* bd = s.bond + t * (s.n + 1);
  if (threadIdx.x == 0) v[0] = mk(1.0, 0.0);
  __syncthreads();
  for (int k = 0; k < s.n; ++k) {
    const int dl = bd[k], dr = bd[k + 1], capr = s.cap[k + 1];
    const cpx<R>* A = site_ptr(s, k, t);
    double part0 = 0.0, part1 = 0.0;
    for (int b = threadIdx.x; b < dr; b += blockDim.x) {
      zd w0 = mk(0.0, 0.0), w1 = mk(0.0, 0.0);
      for (int a = 0; a < dl; ++a) {
        const zd va = v[a];
        cfma(w0, va, cast<double>(A[(int64_t)(a * 2) * capr + b]));
        cfma(w1, va, cast<double>(A[(int64_t)(a * 2 + 1) * capr + b]));
      }
      w0s[b] = w0;
      w1s[b] = w1;
      part0 += norm2(w0);
      part1 += norm2(w1);
    }
    const double p0 = block_sum(part0, red);
    const double p1 = block_sum(part1, red);
    const double u = philox_uniform(seed, (uint64_t)(traj_offset + t), (1ull << 62) + (uint64_t)shot, (uint64_t)k);
    const int bit = (u * (p0 + p1) < p0) ? 0 : 1;
    const double pb = bit ? p1 : p0;
    const double sc = pb > 0.0 ? 1.0 / sqrt(pb) : 0.0;
    for (int b = threadIdx.x; b < dr; b += blockDim.x) v[b] = sc * (bit ? w1s[b] : w0s[b]);
    if (threadIdx.x == 0) out[(t * n_shots + shot) * (int64_t)s.n + k] = (uint8_t)bit;
    __syncthreads();
  }
}

// ---- measure helpers ------------------------------------------------------------
// With the centre at q, rho12 of the pair (q, q+1) gives <Z_q>, <Z_{q+1}>,
// <Z_q Z_{q+1}> from its diagonal.
__global__ void k_obs_from_rho12(const zd* rho12, int64_t B, int n, int q, double* z, double* zz) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B) return;
  const zd* r = rho12 + t * 16;
  double p00 = r[0].re, p01 = r[5].re, p10 = r[10].re, p11 = r[15].re;
  double tr = p00 + p01 + p10 + p11;
  double inv = tr > 0.0 ? 1.0 / tr : 0.0;
  z[t * n + q] = (p00 + p01 - p10 - p11) * inv;
  if (q + 1 == n - 1) z[t * n + q + 1] = (p00 - p01 + p10 - p11) * inv;
  zz[t * (n - 1) + q] = (p00 - p01 - p10 + p11) * inv;
}

// Gram of the centre site A_k as (2 dl) x dr: G = M^dagger M (dr x dr) into
// the FP64 Gram buffer, accumulated in FP64 (the half-chain entropy is an
// FP64 quantity in both precisions).
template <class R>
__global__ void k_site_gram(SimView<R> s, int k) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  const int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[k], dr = bd[k + 1], capr = s.cap[k + 1];
  const cpx<R>* A = site_ptr(s, k, t);
  zd* G = s.g64 + t * s.ws_stride;
  for (int e = threadIdx.x; e < dr * dr; e += blockDim.x) {
    int i = e / dr, j = e % dr;
    zd acc = mk(0.0, 0.0);
    for (int r = 0; r < 2 * dl; ++r)
      cfmac(acc, cast<double>(A[(int64_t)r * capr + i]), cast<double>(A[(int64_t)r * capr + j]));
    G[e] = acc;
  }
}

// Entropy (nats) of the eigenvalues of a Gram matrix of size ng stored in evals.
__global__ void k_entropy_from_evals(const double* evals, int stride, const int32_t* bond, int np1, int kb,
                                     int64_t B, double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B) return;
  const int ng = bond[t * np1 + kb];
  const double* ev = evals + t * stride;
  double tot = 0.0;
  for (int k = 0; k < ng; ++k) tot += fmax(ev[k], 0.0);
  double e = 0.0;
  for (int k = 0; k < ng; ++k) {
    double l = fmax(ev[k], 0.0) / tot;
    if (l > 0.0) e -= l * log(l);
  }
  out[t] = e;
}

}  // namespace lemps
