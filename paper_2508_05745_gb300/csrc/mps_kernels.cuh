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
  int64_t ws_stride;         // (2 chi)^2
  double* evals;             // [B][2 chi]
  zd* rho12;                 // [B][16]
  zd* top;                   // [B][16] operator applied to the two-site tensor
  double* eps_layer;         // [B]
  double* eps_tot;           // [B]
  double* disc_last;         // [B] discarded weight of the last split
  int32_t* status;           // [B]
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

// ---- Householder QR of a column-major m x n matrix X (ld = m) --------------
// Reflectors v_j (length m, zero above j) are stored column-major in V.
// On exit the upper triangle of X holds R.  Then Q (m x kq) is formed in Qm.
template <class R>
__device__ void householder_qr(cpx<R>* X, cpx<R>* V, cpx<R>* Qm, int m, int n, int kq, R* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int kmin = min(m, n);
  for (int j = 0; j < kmin; ++j) {
    // norm of X[j:m, j]
    R part = 0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) part += norm2(X[(int64_t)j * m + i]);
    R nrm2 = block_sum(part, red);
    R nrm = sqrt(nrm2);
    cpx<R> x0 = X[(int64_t)j * m + j];
    R ax0 = sqrt(norm2(x0));
    cpx<R> ph = (ax0 > 0) ? mk<R>(x0.re / ax0, x0.im / ax0) : mk<R>(1, 0);
    cpx<R> alpha = mk<R>(-nrm * ph.re, -nrm * ph.im);
    // v = x - alpha e_j ; ||v||^2 = nrm2 - 2 Re(conj(alpha) x0) + |alpha|^2
    R vn2 = nrm2 + nrm2 + 2 * nrm * ax0;
    R inv = (vn2 > 0) ? (R)1 / sqrt(vn2) : (R)0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      cpx<R> vi = mk<R>(0, 0);
      if (i > j) vi = X[(int64_t)j * m + i] * inv;
      else if (i == j) vi = (x0 - alpha) * inv;
      V[(int64_t)j * m + i] = vi;
    }
    __syncthreads();
    // apply H = I - 2 v v^dagger to columns j..n-1 (one warp per column)
    for (int c = j + warp; c < n; c += nwarp) {
      cpx<R> d = mk<R>(0, 0);
      for (int i = j + lane; i < m; i += 32) cfmac(d, V[(int64_t)j * m + i], X[(int64_t)c * m + i]);
      d.re = warp_sum(d.re);
      d.im = warp_sum(d.im);
      d = (R)2 * d;
      for (int i = j + lane; i < m; i += 32) X[(int64_t)c * m + i] -= V[(int64_t)j * m + i] * d;
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{kmin-1} [I; 0] (m x kq)
  for (int64_t e = threadIdx.x; e < (int64_t)m * kq; e += blockDim.x) {
    int c = (int)(e / m), i = (int)(e % m);
    Qm[e] = mk<R>(i == c ? 1 : 0, 0);
  }
  __syncthreads();
  for (int j = kmin - 1; j >= 0; --j) {
    for (int c = warp; c < kq; c += nwarp) {
      cpx<R> d = mk<R>(0, 0);
      for (int i = j + lane; i < m; i += 32) cfmac(d, V[(int64_t)j * m + i], Qm[(int64_t)c * m + i]);
      d.re = warp_sum(d.re);
      d.im = warp_sum(d.im);
      d = (R)2 * d;
      for (int i = j + lane; i < m; i += 32) Qm[(int64_t)c * m + i] -= V[(int64_t)j * m + i] * d;
    }
    __syncthreads();
  }
}

// Move the centre from site k to k+1 (dir = +1, QR of A_k as (2 dl) x dr) or
// to k-1 (dir = -1, LQ of A_k as dl x (2 dr)).
template <class R>
__global__ void k_move_center(SimView<R> s, int k, int dir) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  __shared__ R red[32];
  int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[k], dr = bd[k + 1];
  const int capr = s.cap[k + 1];
  cpx<R>* A = site_ptr(s, k, t);
  cpx<R>* X = s.ws0 + t * s.ws_stride;
  cpx<R>* V = s.ws1 + t * s.ws_stride;
  cpx<R>* Qm = s.ws2 + t * s.ws_stride;
  cpx<R>* Tm = s.ws3 + t * s.ws_stride;
  if (dir > 0) {
    const int m = 2 * dl, n = dr, r = min(m, n);
    for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) {
      int c = (int)(e / m), i = (int)(e % m);
      X[e] = A[(int64_t)i * capr + c];
    }
    __syncthreads();
    householder_qr(X, V, Qm, m, n, r, red);
    // A_{k+1} <- R A_{k+1}: A_{k+1} is dr x (2 d2), R is r x dr (upper part of X)
    const int d2 = bd[k + 2], cap2 = s.cap[k + 2];
    cpx<R>* B = site_ptr(s, k + 1, t);
    for (int64_t e = threadIdx.x; e < (int64_t)r * 2 * d2; e += blockDim.x) {
      int i = (int)(e / (2 * d2)), cc = (int)(e % (2 * d2));
      int ss = cc / d2, b = cc % d2;
      cpx<R> acc = mk<R>(0, 0);
      for (int l = i; l < dr; ++l) cfma(acc, X[(int64_t)l * m + i], B[(int64_t)(l * 2 + ss) * cap2 + b]);
      Tm[e] = acc;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)r * 2 * d2; e += blockDim.x) {
      int i = (int)(e / (2 * d2)), cc = (int)(e % (2 * d2));
      int ss = cc / d2, b = cc % d2;
      B[(int64_t)(i * 2 + ss) * cap2 + b] = Tm[e];
    }
    // A_k <- Q (m x r) reshaped (dl, 2, r)
    for (int64_t e = threadIdx.x; e < (int64_t)m * r; e += blockDim.x) {
      int c = (int)(e / m), i = (int)(e % m);
      A[(int64_t)i * capr + c] = Qm[e];
    }
    if (threadIdx.x == 0) bd[k + 1] = r;
  } else {
    // X = A_k^dagger: (2 dr) x dl, column-major, X[c][i] = conj(A[i][c])
    const int m = 2 * dr, n = dl, r = min(m, n);
    for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) {
      int c = (int)(e / m), i = (int)(e % m);  // row c of A, column i of A (= (s, b))
      int ss = i / dr, b = i % dr;
      X[e] = conj(A[(int64_t)(c * 2 + ss) * capr + b]);
    }
    __syncthreads();
    householder_qr(X, V, Qm, m, n, r, red);
    // A_k = L Q with L = R'^dagger (dl x r), Q = Q'^dagger (r x 2dr).
    // A_{k-1} <- A_{k-1} L: A_{k-1} is (2 d0) x dl, result (2 d0) x r.
    const int d0 = bd[k - 1], cap1 = s.cap[k];
    cpx<R>* P = site_ptr(s, k - 1, t);
    for (int64_t e = threadIdx.x; e < (int64_t)2 * d0 * r; e += blockDim.x) {
      int row = (int)(e / r), j = (int)(e % r);
      cpx<R> acc = mk<R>(0, 0);
      for (int l = j; l < dl; ++l) cfma(acc, P[(int64_t)row * cap1 + l], conj(X[(int64_t)l * m + j]));
      Tm[e] = acc;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)2 * d0 * r; e += blockDim.x) {
      int row = (int)(e / r), j = (int)(e % r);
      P[(int64_t)row * cap1 + j] = Tm[e];
    }
    // A_k <- Q'^dagger: A[j][ss][b] = conj(Q'[(ss, b)][j])
    for (int64_t e = threadIdx.x; e < (int64_t)m * r; e += blockDim.x) {
      int j = (int)(e / m), i = (int)(e % m);
      int ss = i / dr, b = i % dr;
      A[(int64_t)(j * 2 + ss) * capr + b] = conj(Qm[e]);
    }
    if (threadIdx.x == 0) bd[k] = r;
  }
}

// ---- two-site contraction and the 4x4 reduced density ------------------------
// Theta[a][s1][s2][b] = sum_m A_q[a][s1][m] A_{q+1}[m][s2][b] into ws0 as a
// (2 dl) x (2 dr) row-major matrix; rho12[(s1 s2), (t1 t2)] =
// sum_{a,b} Theta[a,s1,s2,b] conj(Theta[a,t1,t2,b]) in FP64.
template <class R>
__global__ void k_contract(SimView<R> s, int q) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  __shared__ double red[32];
  const int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[q], dm = bd[q + 1], dr = bd[q + 2];
  const int capm = s.cap[q + 1], capr = s.cap[q + 2];
  const cpx<R>* A = site_ptr(s, q, t);
  const cpx<R>* B = site_ptr(s, q + 1, t);
  cpx<R>* th = s.ws0 + t * s.ws_stride;
  double acc[16][2];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i][0] = acc[i][1] = 0.0;
  for (int e = threadIdx.x; e < dl * dr; e += blockDim.x) {
    const int a = e / dr, b = e % dr;
    cpx<R> v[4] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
    for (int m = 0; m < dm; ++m) {
      cpx<R> a0 = A[(int64_t)(2 * a) * capm + m], a1 = A[(int64_t)(2 * a + 1) * capm + m];
      cpx<R> b0 = B[(int64_t)(2 * m) * capr + b], b1 = B[(int64_t)(2 * m + 1) * capr + b];
      cfma(v[0], a0, b0); cfma(v[1], a0, b1); cfma(v[2], a1, b0); cfma(v[3], a1, b1);
    }
    const int64_t ld = 2 * dr;
    th[(int64_t)(2 * a) * ld + b] = v[0];
    th[(int64_t)(2 * a) * ld + dr + b] = v[1];
    th[(int64_t)(2 * a + 1) * ld + b] = v[2];
    th[(int64_t)(2 * a + 1) * ld + dr + b] = v[3];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        zd vi = cast<double>(v[i]), vj = cast<double>(v[j]);
        acc[i * 4 + j][0] += vi.re * vj.re + vi.im * vj.im;
        acc[i * 4 + j][1] += vi.im * vj.re - vi.re * vj.im;
      }
  }
  for (int i = 0; i < 16; ++i) {
    double re = block_sum(acc[i][0], red);
    double im = block_sum(acc[i][1], red);
    if (threadIdx.x == 0) s.rho12[t * 16 + i] = mk(re, im);
  }
}

// ---- apply T to Theta and build the Gram matrix ------------------------------
// side = 0: left Gram  G = Theta Theta^dagger (2dl x 2dl)
// side = 1: right Gram G = Theta^dagger Theta (2dr x 2dr)
template <class R>
__global__ void k_apply_gram(SimView<R> s, int q, int side) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  const int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[q], dr = bd[q + 2];
  cpx<R>* th = s.ws0 + t * s.ws_stride;
  cpx<R>* G = s.ws1 + t * s.ws_stride;
  __shared__ zd T[16];
  if (threadIdx.x < 16) T[threadIdx.x] = s.top[t * 16 + threadIdx.x];
  __syncthreads();
  const int64_t ld = 2 * dr;
  for (int e = threadIdx.x; e < dl * dr; e += blockDim.x) {
    const int a = e / dr, b = e % dr;
    zd v[4];
    v[0] = cast<double>(th[(int64_t)(2 * a) * ld + b]);
    v[1] = cast<double>(th[(int64_t)(2 * a) * ld + dr + b]);
    v[2] = cast<double>(th[(int64_t)(2 * a + 1) * ld + b]);
    v[3] = cast<double>(th[(int64_t)(2 * a + 1) * ld + dr + b]);
    zd w[4];
    for (int i = 0; i < 4; ++i) {
      zd acc = mk(0.0, 0.0);
      for (int k = 0; k < 4; ++k) cfma(acc, T[i * 4 + k], v[k]);
      w[i] = acc;
    }
    th[(int64_t)(2 * a) * ld + b] = cast<R>(w[0]);
    th[(int64_t)(2 * a) * ld + dr + b] = cast<R>(w[1]);
    th[(int64_t)(2 * a + 1) * ld + b] = cast<R>(w[2]);
    th[(int64_t)(2 * a + 1) * ld + dr + b] = cast<R>(w[3]);
  }
  __syncthreads();
  const int nr = 2 * dl, nc = 2 * dr;
  const int ng = side == 0 ? nr : nc;
  for (int e = threadIdx.x; e < ng * ng; e += blockDim.x) {
    const int i = e / ng, j = e % ng;
    if (j < i) continue;
    cpx<R> acc = mk<R>(0, 0);
    if (side == 0) {
      for (int c = 0; c < nc; ++c) cfma(acc, th[(int64_t)i * ld + c], conj(th[(int64_t)j * ld + c]));
    } else {
      for (int r = 0; r < nr; ++r) cfmac(acc, th[(int64_t)r * ld + i], th[(int64_t)r * ld + j]);
    }
    G[(int64_t)i * ng + j] = acc;
    G[(int64_t)j * ng + i] = conj(acc);
  }
}

// ---- Hermitian eigensolver: cyclic parallel two-sided Jacobi ----------------
// Diagonalizes G (ng x ng row-major, in ws1) in place; eigenvectors
// accumulate as columns of V (ws2, row-major).  Pairs follow a round-robin
// tournament so each round's ng/2 rotations are disjoint; every round applies
// all rotations to G through 2x2 blocks, so G and V make one pass per round.
// Eigenvalues are written to evals sorted descending together with a
// permutation perm (int stored in ws3 reinterpret).
// Size of the Gram matrix: mode 0: 2 bond[k] (left Gram of the pair at k),
// mode 1: 2 bond[k+2] (right Gram), mode 2: bond[k+1] (site Gram of A_k).
__device__ __forceinline__ int gram_size(const int32_t* bd, int k, int mode) {
  return mode == 0 ? 2 * bd[k] : (mode == 1 ? 2 * bd[k + 2] : bd[k + 1]);
}

template <class R>
__global__ void k_jacobi(SimView<R> s, int q, int mode, int max_sweeps, R tol) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  const int32_t* bd = s.bond + t * (s.n + 1);
  const int ng = gram_size(bd, q, mode);
  cpx<R>* G = s.ws1 + t * s.ws_stride;
  cpx<R>* V = s.ws2 + t * s.ws_stride;
  __shared__ int pos[256];
  __shared__ R rc[128], rs[128];
  __shared__ cpx<R> rph[128];   // e^{-i phi} of each pair
  __shared__ R red[32];
  for (int e = threadIdx.x; e < ng * ng; e += blockDim.x) {
    int i = e / ng, j = e % ng;
    V[e] = mk<R>(i == j ? 1 : 0, 0);
  }
  R fro = 0;
  for (int e = threadIdx.x; e < ng * ng; e += blockDim.x) fro += norm2(G[e]);
  fro = block_sum(fro, red);
  // Round robin needs an even count: an odd size gets a dummy index ng that
  // never rotates.
  const int np2 = ng + (ng & 1);
  const int half = np2 / 2;
  bool converged = (ng <= 1);
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    for (int i = threadIdx.x; i < np2; i += blockDim.x) pos[i] = i;
    __syncthreads();
    for (int round = 0; round < np2 - 1; ++round) {
      // rotation parameters for pair k: (pos[k], pos[np2-1-k])
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int p = pos[k], qq = pos[np2 - 1 - k];
        if (p > qq) { int tmp = p; p = qq; qq = tmp; }
        R c = 1, sn = 0;
        cpx<R> e = mk<R>(1, 0);
        if (qq < ng) {
          cpx<R> g = G[(int64_t)p * ng + qq];
          R gn = sqrt(norm2(g));
          R app = G[(int64_t)p * ng + p].re, aqq = G[(int64_t)qq * ng + qq].re;
          if (gn > tol * sqrt(fabs(app * aqq)) && gn > (R)1e-300) {
            R zeta = (aqq - app) / (2 * gn);
            R tt = (zeta >= 0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt((R)1 + zeta * zeta));
            c = (R)1 / sqrt((R)1 + tt * tt);
            sn = c * tt;
            e = mk<R>(g.re / gn, -g.im / gn);
          }
        }
        rc[k] = c; rs[k] = sn; rph[k] = e;
      }
      __syncthreads();
      // 2x2 block update of G: rows (p_i, q_i) x cols (p_j, q_j); the dummy
      // index only ever pairs with an identity rotation and is skipped.
      for (int e = threadIdx.x; e < half * half; e += blockDim.x) {
        const int bi = e / half, bj = e % half;
        int pi = pos[bi], qi = pos[np2 - 1 - bi];
        if (pi > qi) { int tmp = pi; pi = qi; qi = tmp; }
        int pj = pos[bj], qj = pos[np2 - 1 - bj];
        if (pj > qj) { int tmp = pj; pj = qj; qj = tmp; }
        const bool vi = qi < ng, vj = qj < ng;
        cpx<R> g00 = G[(int64_t)pi * ng + pj];
        cpx<R> g01 = vj ? G[(int64_t)pi * ng + qj] : mk<R>(0, 0);
        cpx<R> g10 = vi ? G[(int64_t)qi * ng + pj] : mk<R>(0, 0);
        cpx<R> g11 = (vi && vj) ? G[(int64_t)qi * ng + qj] : mk<R>(0, 0);
        // columns: [g_p, g_q] J_j, J = [[c, s], [-s e, c e]]
        R cj = rc[bj], sj = rs[bj];
        cpx<R> ej = rph[bj];
        cpx<R> h00 = cj * g00 - sj * (ej * g01), h01 = sj * g00 + cj * (ej * g01);
        cpx<R> h10 = cj * g10 - sj * (ej * g11), h11 = sj * g10 + cj * (ej * g11);
        // rows: J_i^dagger [h_p; h_q], J^dagger = [[c, -s e*], [s, c e*]]
        R ci = rc[bi], si = rs[bi];
        cpx<R> eci = conj(rph[bi]);
        G[(int64_t)pi * ng + pj] = ci * h00 - si * (eci * h10);
        if (vj) G[(int64_t)pi * ng + qj] = ci * h01 - si * (eci * h11);
        if (vi) G[(int64_t)qi * ng + pj] = si * h00 + ci * (eci * h10);
        if (vi && vj) G[(int64_t)qi * ng + qj] = si * h01 + ci * (eci * h11);
      }
      // V <- V J (columns p, q of every row)
      for (int e = threadIdx.x; e < ng * half; e += blockDim.x) {
        const int row = e / half, k = e % half;
        int p = pos[k], qq = pos[np2 - 1 - k];
        if (p > qq) { int tmp = p; p = qq; qq = tmp; }
        if (qq >= ng) continue;
        cpx<R> vp = V[(int64_t)row * ng + p], vq = rph[k] * V[(int64_t)row * ng + qq];
        V[(int64_t)row * ng + p] = rc[k] * vp - rs[k] * vq;
        V[(int64_t)row * ng + qq] = rs[k] * vp + rc[k] * vq;
      }
      __syncthreads();
      // rotate positions 1..np2-1 (round robin)
      if (threadIdx.x == 0) {
        int last = pos[np2 - 1];
        for (int i = np2 - 1; i > 1; --i) pos[i] = pos[i - 1];
        pos[1] = last;
      }
      __syncthreads();
    }
    R off = 0;
    for (int e = threadIdx.x; e < ng * ng; e += blockDim.x) {
      int i = e / ng, j = e % ng;
      if (i != j) off += norm2(G[e]);
    }
    off = block_sum(off, red);
    converged = (off <= tol * tol * fro);
  }
  if (!converged && threadIdx.x == 0 && ng > 1) atomicOr(s.status + t, (int32_t)TS_JACOBI);
  // sort eigenvalues descending: rank of each
  double* ev = s.evals + t * (2 * s.chi);
  int* perm = reinterpret_cast<int*>(s.ws3 + t * s.ws_stride);
  for (int i = threadIdx.x; i < ng; i += blockDim.x) {
    R li = G[(int64_t)i * ng + i].re;
    int rank = 0;
    for (int j = 0; j < ng; ++j) {
      R lj = G[(int64_t)j * ng + j].re;
      if (lj > li || (lj == li && j < i)) ++rank;
    }
    ev[rank] = (double)li;
    perm[rank] = i;
  }
}

// ---- split and truncate ------------------------------------------------------
// Keeps chi' = min(chi_max, #{l_k > cutoff * sum l}) eigenpairs.  side 0:
// A_q <- U' (left-orthonormal), A_{q+1} <- U'^dagger Theta / sqrt(kept),
// centre at q+1.  side 1: A_{q+1} <- V'^dagger, A_q <- Theta V' / sqrt(kept),
// centre at q.
template <class R>
__global__ void k_split(SimView<R> s, int q, int side, double cutoff) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  __shared__ int s_keep;
  __shared__ double s_norm;
  int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[q], dr = bd[q + 2];
  const int ng = side == 0 ? 2 * dl : 2 * dr;
  const double* ev = s.evals + t * (2 * s.chi);
  const int* perm = reinterpret_cast<const int*>(s.ws3 + t * s.ws_stride);
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < ng; ++k) tot += fmax(ev[k], 0.0);
    int keep = 0;
    for (int k = 0; k < ng; ++k)
      if (ev[k] > cutoff * tot) ++keep;
    keep = min(keep, s.chi);
    keep = min(keep, min(2 * dl, 2 * dr));
    keep = max(keep, 1);
    double kept = 0.0;
    for (int k = 0; k < keep; ++k) kept += fmax(ev[k], 0.0);
    double disc = (tot > 0.0) ? fmax(tot - kept, 0.0) / tot : 0.0;
    if (!(tot > 0.0) || !isfinite(tot)) atomicOr(s.status + t, (int32_t)TS_NORM);
    s.disc_last[t] = disc;
    s.eps_layer[t] += disc;
    s_keep = keep;
    s_norm = (kept > 0.0) ? 1.0 / sqrt(kept) : 0.0;
  }
  __syncthreads();
  const int keep = s_keep;
  const R nrm = (R)s_norm;
  const cpx<R>* th = s.ws0 + t * s.ws_stride;
  const cpx<R>* V = s.ws2 + t * s.ws_stride;
  const int64_t ld = 2 * dr;
  cpx<R>* A = site_ptr(s, q, t);
  cpx<R>* B = site_ptr(s, q + 1, t);
  const int capm = s.cap[q + 1], capr = s.cap[q + 2];
  if (side == 0) {
    // A_q[a][s1][k] = U[2a+s1][perm[k]]
    for (int e = threadIdx.x; e < 2 * dl * keep; e += blockDim.x) {
      int row = e / keep, k = e % keep;
      A[(int64_t)row * capm + k] = V[(int64_t)row * ng + perm[k]];
    }
    // A_{q+1}[k][s2][b] = nrm * sum_r conj(U[r][perm k]) Theta[r][s2 dr + b]
    for (int e = threadIdx.x; e < keep * 2 * dr; e += blockDim.x) {
      int k = e / (2 * dr), c = e % (2 * dr);
      int col = perm[k];
      cpx<R> acc = mk<R>(0, 0);
      for (int r = 0; r < 2 * dl; ++r) cfmac(acc, V[(int64_t)r * ng + col], th[(int64_t)r * ld + c]);
      int s2 = c / dr, b = c % dr;
      B[(int64_t)(k * 2 + s2) * capr + b] = nrm * acc;
    }
  } else {
    // A_{q+1}[k][s2][b] = conj(V[s2 dr + b][perm k])
    for (int e = threadIdx.x; e < keep * 2 * dr; e += blockDim.x) {
      int k = e / (2 * dr), c = e % (2 * dr);
      int s2 = c / dr, b = c % dr;
      B[(int64_t)(k * 2 + s2) * capr + b] = conj(V[(int64_t)c * ng + perm[k]]);
    }
    // A_q[a][s1][k] = nrm * sum_c Theta[2a+s1][c] V[c][perm k]
    for (int e = threadIdx.x; e < 2 * dl * keep; e += blockDim.x) {
      int row = e / keep, k = e % keep;
      int col = perm[k];
      cpx<R> acc = mk<R>(0, 0);
      for (int c = 0; c < 2 * dr; ++c) cfma(acc, th[(int64_t)row * ld + c], V[(int64_t)c * ng + col]);
      A[(int64_t)row * capm + k] = nrm * acc;
    }
  }
  if (threadIdx.x == 0) bd[q + 1] = keep;
}

// ---- layer bookkeeping: eps_tot += 4 sqrt(2 sum_k eps_k) (App. B) -------------
template <class R>
__global__ void k_layer_end(SimView<R> s) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= s.B) return;
  s.eps_tot[t] += 4.0 * sqrt(2.0 * s.eps_layer[t]);
  s.eps_layer[t] = 0.0;
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

// Gram of the centre site A_k as (2 dl) x dr: G = M^dagger M (dr x dr) into ws1.
template <class R>
__global__ void k_site_gram(SimView<R> s, int k) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  const int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[k], dr = bd[k + 1], capr = s.cap[k + 1];
  const cpx<R>* A = site_ptr(s, k, t);
  cpx<R>* G = s.ws1 + t * s.ws_stride;
  for (int e = threadIdx.x; e < dr * dr; e += blockDim.x) {
    int i = e / dr, j = e % dr;
    cpx<R> acc = mk<R>(0, 0);
    for (int r = 0; r < 2 * dl; ++r) cfmac(acc, A[(int64_t)r * capr + i], A[(int64_t)r * capr + j]);
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
