// Kernels for bond dimensions above 128 (chi_max up to 512): the Hermitian
// eigensolver of the split for Gram matrices of size n <= 1024, and the
// centre move with a Householder QR of up to 1024 rows.  The kernels of
// heev.cuh and the blocked QR of mps_kernels.cuh keep their working sets on
// chip and stop at n = 256 and 256 rows; these keep the matrices in global
// memory (L2) and are simple and unblocked: O(n^3) like the others, but
// without the on-chip staging.  The host uses them only where a site capacity
// exceeds 128.
#pragma once

#include "heev.cuh"
#include "mps_kernels.cuh"

namespace lemps {

constexpr int kBigN = 1024;        // largest Gram matrix / QR row count (2 chi_max)
constexpr int kBigHeevThreads = 512;

struct BigHeevSmem {
  zd v[kBigN];      // Householder vector of the step; later a reflector in RB
  zd y[kBigN];      // A v; later the unit factors of the off-diagonal
  zd w[kBigN];      // w = 2 (y - (v^dagger y) v)
  zd ec[kBigN];     // complex off-diagonal e_j = T[j+1][j]
  zd ph[kBigN];     // phases delta_j with T_real = D^dagger T D
  double d[kBigN], e[kBigN], e2[kBigN];   // real tridiagonal: diagonal, |e_j|, |e_j|^2
  double dn[kBigN], e2n[kBigN];           // the same scaled by 1 / ||T|| (Sturm counts)
  double c[kBigN];                        // Gram-Schmidt coefficients
  double red[96];
};

// Hermitian eigensolver of a Gram matrix (complex128, n x n row-major in ws1,
// n <= kBigN; n from the bonds as in k_heev: mode 0 2 d_q, mode 1 2 d_{q+2},
// mode 2 d_{q+1}).  Same outputs as k_heev: the top keep = max(1, min(#{l >
// cutoff tr}, keep_max, n, rank bound)) eigenvalues (descending) in evals,
// keep and the trace in kept / trace, and with want_vectors the eigenvectors
// U (column-major n x keep, cpx<RB>) at the start of the trajectory's ws2
// slot; the reflectors (sqrt(2) v_j in row j, in cpx<RB>) go to ws3.
//  1. Householder tridiagonalization in FP64, one column per step: v from the
//     column below the diagonal, y = A v by one warp per row (the lower
//     triangle read along the row, the upper part as the conjugate of the
//     lower triangle's column), w = 2 (y - (v^H y) v), A <- A - v w^H - w v^H
//     on the lower triangle of the trailing block only.
//  2. Phases D with T_real = D^H T D real (|e_j| off the diagonal).
//  3. Each kept eigenvalue by bisection on Sturm counts of T_real / ||T||
//     (one thread per eigenvalue) to 4 eps ||T||.
//  4. Inverse iteration (two LDL^T solves of T_real - l I, one thread per
//     vector, factors in the Gram slot), then classical Gram-Schmidt twice
//     over the kept vectors in RB, normalized.
//  5. U = Q D z: the phases, then the reflectors from the last to the first,
//     one warp per column, in RB.
template <class RB>
__global__ void __launch_bounds__(kBigHeevThreads) k_heev_big(HeevView<double> s, int q, int mode, double cutoff,
                                                                int keep_max, int want_vectors) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  extern __shared__ __align__(16) unsigned char big_heev_smem[];
  BigHeevSmem& sm = *reinterpret_cast<BigHeevSmem*>(big_heev_smem);
  __shared__ double s_tr, s_sc[4], s_gl, s_gu, s_tn;
  __shared__ int s_keep;
  const int32_t* bd = s.bond + t * (s.nq + 1);
  const int n = mode == 0 ? 2 * bd[q] : (mode == 1 ? 2 * bd[q + 2] : bd[q + 1]);
  if (n < 1 || n > kBigN) {
    if (threadIdx.x == 0) atomicOr(s.status + t, (int32_t)TS_SHAPE);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  zd* G = s.ws1 + t * s.ws_stride;
  cpx<RB>* Hv = reinterpret_cast<cpx<RB>*>(s.ws3 + t * s.ws_stride);
  cpx<RB>* U = reinterpret_cast<cpx<RB>*>(s.ws2 + t * s.ws_stride);

  double trp = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) trp += G[(int64_t)i * n + i].re;
  trp = block_sum_f64(trp, sm.red);
  if (threadIdx.x == 0) s_tr = trp;

  // ---- 1: tridiagonalization ---------------------------------------------------
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    double part = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const zd x = G[(int64_t)(j + 1 + i) * n + j];
      sm.v[i] = x;
      if (i > 0) part = fma(x.re, x.re, fma(x.im, x.im, part));
    }
    const double sig = block_sum_f64(part, sm.red);
    if (threadIdx.x == 0) {
      const zd x0 = sm.v[0];
      const double ax0 = sqrt(norm2(x0));
      const double nrm = sqrt(sig + ax0 * ax0);
      zd alpha = x0, v0 = mk(0.0, 0.0);
      double inv = 0.0;
      if (sig > 0.0) {
        const zd ph = (ax0 > 0.0) ? mk(x0.re / ax0, x0.im / ax0) : mk(1.0, 0.0);
        alpha = mk(-nrm * ph.re, -nrm * ph.im);
        inv = 1.0 / sqrt(sig + (ax0 + nrm) * (ax0 + nrm));
        v0 = (x0 - alpha) * inv;
      }
      sm.d[j] = G[(int64_t)j * n + j].re;
      sm.ec[j] = alpha;
      s_sc[0] = v0.re;
      s_sc[1] = v0.im;
      s_sc[2] = inv;
      s_sc[3] = (sig > 0.0) ? 1.0 : 0.0;
    }
    __syncthreads();
    const bool reflect = s_sc[3] != 0.0;
    {
      const zd v0 = mk(s_sc[0], s_sc[1]);
      const double inv = s_sc[2];
      for (int i = threadIdx.x; i < m; i += blockDim.x)
        sm.v[i] = reflect ? ((i == 0) ? v0 : sm.v[i] * inv) : mk(0.0, 0.0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      Hv[(int64_t)j * n + i] = cast<RB>((i > j) ? kSqrt2 * sm.v[i - j - 1] : mk(0.0, 0.0));
    if (!reflect) {
      __syncthreads();
      continue;
    }
    // y = A v over the trailing block (rows and columns j+1 .. n-1); only the
    // lower triangle is current: A[r][c] for c <= r along row r, conj(A[c][r])
    // for c > r down column r
    for (int r = warp; r < m; r += nwarp) {
      const zd* row = G + (int64_t)(j + 1 + r) * n + (j + 1);
      const zd* colr = G + (int64_t)(j + 1) * n + (j + 1 + r);   // A[c][r] at colr[c * n]
      zd acc = mk(0.0, 0.0);
      for (int c = lane; c <= r; c += 32) cfma(acc, row[c], sm.v[c]);
      for (int c = r + 1 + lane; c < m; c += 32) cfmac(acc, colr[(int64_t)c * n], sm.v[c]);
      acc.re = warp_sum(acc.re);
      acc.im = warp_sum(acc.im);
      if (lane == 0) sm.y[r] = acc;
    }
    __syncthreads();
    double kp = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      kp = fma(sm.v[i].re, sm.y[i].re, fma(sm.v[i].im, sm.y[i].im, kp));
    const double K = block_sum_f64(kp, sm.red);   // v^H y (real: A is Hermitian)
    for (int i = threadIdx.x; i < m; i += blockDim.x) sm.w[i] = 2.0 * (sm.y[i] - K * sm.v[i]);
    __syncthreads();
    for (int r = warp; r < m; r += nwarp) {
      zd* row = G + (int64_t)(j + 1 + r) * n + (j + 1);
      const zd vr = sm.v[r], wr = sm.w[r];
      for (int c = lane; c <= r; c += 32) row[c] = rank2_sub(row[c], vr, sm.w[c], wr, sm.v[c]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (n >= 2) {
      sm.d[n - 2] = G[(int64_t)(n - 2) * n + (n - 2)].re;
      sm.ec[n - 2] = G[(int64_t)(n - 1) * n + (n - 2)];
    }
    sm.d[n - 1] = G[(int64_t)(n - 1) * n + (n - 1)].re;
  }
  __syncthreads();

  // ---- 2: phases of the off-diagonal ---------------------------------------------
  for (int j = threadIdx.x; j + 1 < n; j += blockDim.x) {
    const double a = sqrt(norm2(sm.ec[j]));
    sm.e[j] = a;
    sm.e2[j] = a * a;
    sm.y[j] = (a > 0.0) ? mk(sm.ec[j].re / a, sm.ec[j].im / a) : mk(1.0, 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    zd dl = mk(1.0, 0.0);
    sm.ph[0] = dl;
    for (int j = 0; j + 1 < n; ++j) {
      dl = dl * sm.y[j];
      sm.ph[j + 1] = dl;
    }
  }
  __syncthreads();

  // ---- 3: Gerschgorin bounds, how many to keep, bisection --------------------
  {
    double lo = 1e300, hi = -1e300, tn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double rad = (i > 0 ? sm.e[i - 1] : 0.0) + (i + 1 < n ? sm.e[i] : 0.0);
      lo = fmin(lo, sm.d[i] - rad);
      hi = fmax(hi, sm.d[i] + rad);
      tn = fmax(tn, fabs(sm.d[i]) + rad);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    }
    if (lane == 0) {
      sm.red[warp] = lo;
      sm.red[32 + warp] = hi;
      sm.red[64 + warp] = tn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w2 = 1; w2 < nwarp; ++w2) {
        lo = fmin(lo, sm.red[w2]);
        hi = fmax(hi, sm.red[32 + w2]);
        tn = fmax(tn, sm.red[64 + w2]);
      }
      s_gl = lo;
      s_gu = hi;
      s_tn = (tn > 0.0) ? tn : 1.0;
    }
    __syncthreads();
  }
  const double tnorm = s_tn, itn = 1.0 / tnorm;
  const double eps = 2.2e-16;
  const double pivmin = 1e-30;                 // normalized units
  const double pivmin_abs = pivmin * tnorm;
  const double gl = s_gl * itn - (2 * eps + pivmin), gu = s_gu * itn + (2 * eps + pivmin);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sm.dn[i] = sm.d[i] * itn;
    sm.e2n[i] = sm.e2[i] * (itn * itn);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int cnt = (cutoff > 0.0) ? sturm_greater_f64(sm.dn, sm.e2n, n, cutoff * s_tr * itn, pivmin) : n;
    const int rank_bound = (mode == 2) ? n : min(2 * bd[q], 2 * bd[q + 2]);
    s_keep = max(min(cnt, min(keep_max, min(n, rank_bound))), 1);
  }
  __syncthreads();
  const int keep = s_keep;
  double* ev = s.evals + t * (2 * s.chi);
  {
    // eigenvalue k (descending, 0-based) lies in (a, b] while
    // count(a) > k >= count(b); halve until b - a <= 4 eps (normalized)
    const double tol = 4.0 * eps + pivmin;
    for (int k = threadIdx.x; k < keep; k += blockDim.x) {
      double a = gl, b = gu;
      for (int it = 0; it < 200 && b - a > tol; ++it) {
        const double mid = 0.5 * (a + b);
        if (sturm_greater_f64(sm.dn, sm.e2n, n, mid, pivmin) > k) a = mid;
        else b = mid;
      }
      ev[k] = 0.5 * (a + b) * tnorm;
    }
  }
  if (threadIdx.x == 0) {
    s.kept[t] = keep;
    s.trace[t] = s_tr;
  }
  if (!want_vectors) return;
  __syncthreads();

  // ---- 4: inverse iteration, then Gram-Schmidt -------------------------------
  // The real vectors z_k (RB, column-major n x keep) are kept after U in the
  // ws2 slot (n keep complex entries + n keep reals fit in ws_stride complex128
  // entries, since keep <= the bond capacity and n <= twice it).  The LDL^T
  // factors of a chunk of vectors sit in the Gram slot, entry (i, a) of vector
  // kk at (i * 3 + a) * kc + kk (coalesced over the threads of a warp).
  RB* Z = reinterpret_cast<RB*>(U + (size_t)n * keep);
  {
    double* wsp = reinterpret_cast<double*>(G);
    const int64_t cap = 2 * s.ws_stride;   // doubles in the Gram slot
    const int kc_max = (int)min((int64_t)blockDim.x, max((int64_t)1, cap / (3 * (int64_t)n)));
    for (int k0 = 0; k0 < keep; k0 += kc_max) {
      const int kc = min(kc_max, keep - k0);
      const int kk = threadIdx.x;
      if (kk < kc) {
        const int k = k0 + kk;
        double* w3 = wsp + kk;
        auto Dr = [&](int i) -> double& { return w3[(int64_t)(i * 3 + 0) * kc]; };
        auto Lw = [&](int i) -> double& { return w3[(int64_t)(i * 3 + 1) * kc]; };
        auto Zw = [&](int i) -> double& { return w3[(int64_t)(i * 3 + 2) * kc]; };
        const double lam = ev[k];
        double dp = sm.d[0] - lam;
        if (fabs(dp) < pivmin_abs) dp = pivmin_abs;
        Dr(0) = 1.0 / dp;
        for (int i = 0; i + 1 < n; ++i) {
          const double li = sm.e[i] * Dr(i);
          double dn = (sm.d[i + 1] - lam) - li * sm.e[i];
          if (fabs(dn) < pivmin_abs) dn = pivmin_abs;
          Lw(i) = li;
          Dr(i + 1) = 1.0 / dn;
        }
        double sc = 1.0;
        for (int iter = 0; iter < 2; ++iter) {
          double y = (iter == 0) ? (double)start_entry(k, 0) : sc * Zw(0);
          Zw(0) = y;
          for (int i = 1; i < n; ++i) {
            y = ((iter == 0) ? (double)start_entry(k, i) : sc * Zw(i)) - Lw(i - 1) * y;
            Zw(i) = y;
          }
          double zn = Zw(n - 1) * Dr(n - 1);
          Zw(n - 1) = zn;
          double amax = fabs(zn);
          for (int i = n - 2; i >= 0; --i) {
            zn = Zw(i) * Dr(i) - Lw(i) * zn;
            Zw(i) = zn;
            amax = fmax(amax, fabs(zn));
          }
          sc = (amax > 0.0) ? 1.0 / amax : 1.0;
        }
        Dr(0) = sc;   // the factors are done with: slot 0 keeps the final scale
      }
      __syncthreads();
      for (int v = warp; v < kc; v += nwarp) {
        const double* w3 = wsp + v;
        const double sc = w3[0];
        for (int i = lane; i < n; i += 32) Z[(size_t)(k0 + v) * n + i] = (RB)(sc * w3[(int64_t)(i * 3 + 2) * kc]);
      }
      __syncthreads();
    }
  }
  // classical Gram-Schmidt, two passes per vector, in descending eigenvalue order
  for (int k = 0; k < keep; ++k) {
    RB* zk = Z + (size_t)k * n;
    for (int pass = 0; pass < 2 && k > 0; ++pass) {
      for (int j = warp; j < k; j += nwarp) {
        const RB* zj = Z + (size_t)j * n;
        RB c = 0;
        for (int i = lane; i < n; i += 32) c = fma(zj[i], zk[i], c);
        c = warp_sum(c);
        if (lane == 0) sm.c[j] = (double)c;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        RB acc = 0;
        for (int j = 0; j < k; ++j) acc = fma((RB)sm.c[j], Z[(size_t)j * n + i], acc);
        zk[i] -= acc;
      }
      __syncthreads();
    }
    double nn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) nn += (double)zk[i] * (double)zk[i];
    nn = block_sum_f64(nn, sm.red);
    const RB inv = (nn > 0.0) ? (RB)(1.0 / sqrt(nn)) : (RB)0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) zk[i] *= inv;
    __syncthreads();
  }

  // ---- 5: U = Q D z ---------------------------------------------------------------
  for (int e = threadIdx.x; e < keep * n; e += blockDim.x) {
    const int i = e % n;
    U[e] = cast<RB>(sm.ph[i]) * Z[e];
  }
  __syncthreads();
  cpx<RB>* su = reinterpret_cast<cpx<RB>*>(sm.v);
  for (int j = n - 3; j >= 0; --j) {
    const int m = n - j - 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) su[i] = Hv[(int64_t)j * n + j + 1 + i];
    __syncthreads();
    for (int k = warp; k < keep; k += nwarp) {
      cpx<RB>* uk = U + (size_t)k * n + j + 1;
      cpx<RB> d = mk<RB>(0, 0);
      for (int i = lane; i < m; i += 32) cfmac(d, su[i], uk[i]);
      d.re = warp_sum(d.re);
      d.im = warp_sum(d.im);
      for (int i = lane; i < m; i += 32) uk[i] = uk[i] - su[i] * d;
    }
    __syncthreads();
  }
}

// ---- centre move with an unblocked Householder QR in global memory ------------
// QR of the column-major m x n matrix X (ld = m, m <= kBigN) as in
// householder_qr: reflector c (H = I - 2 v v^dagger, unit v) in column c of V
// (zero above row c), R in the upper triangle of X, and Q = H_0 ... H_{kq-1}
// [I; 0] (m x kq) in Qm.  One warp per column applies a reflector; sv (m
// entries of shared memory) holds the current one.  256 threads.
template <class R>
__device__ void householder_qr_big(cpx<R>* X, cpx<R>* V, cpx<R>* Qm, int m, int n, int kq, cpx<R>* sv, R* red,
                                   R* sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int kmin = min(m, n);
  for (int c = 0; c < kmin; ++c) {
    const int pm = m - c;
    const cpx<R>* col = X + (int64_t)c * m + c;
    R part = 0;
    for (int i = threadIdx.x; i < pm; i += blockDim.x) {
      const cpx<R> x = col[i];
      sv[i] = x;
      part += norm2(x);
    }
    const R nrm2 = block_sum(part, red);
    if (threadIdx.x == 0) {
      const cpx<R> x0 = sv[0];
      const R nrm = sqrt(nrm2);
      const R ax0 = sqrt(norm2(x0));
      const cpx<R> ph = (ax0 > 0) ? mk<R>(x0.re / ax0, x0.im / ax0) : mk<R>(1, 0);
      const cpx<R> alpha = mk<R>(-nrm * ph.re, -nrm * ph.im);
      const R vn2 = nrm2 + nrm2 + 2 * nrm * ax0;
      const R inv = (vn2 > 0) ? (R)1 / sqrt(vn2) : (R)0;
      const cpx<R> v0 = (x0 - alpha) * inv;
      sc[0] = v0.re;
      sc[1] = v0.im;
      sc[2] = inv;
    }
    __syncthreads();
    {
      const cpx<R> v0 = mk<R>(sc[0], sc[1]);
      const R inv = sc[2];
      for (int i = threadIdx.x; i < pm; i += blockDim.x) sv[i] = (i == 0) ? v0 : sv[i] * inv;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) V[(int64_t)c * m + i] = (i >= c) ? sv[i - c] : mk<R>(0, 0);
    for (int cc = c + warp; cc < n; cc += nwarp) {
      cpx<R>* y = X + (int64_t)cc * m + c;
      cpx<R> d = mk<R>(0, 0);
      for (int i = lane; i < pm; i += 32) cfmac(d, sv[i], y[i]);
      d.re = warp_sum(d.re);
      d.im = warp_sum(d.im);
      d = (R)2 * d;
      for (int i = lane; i < pm; i += 32) y[i] = y[i] - sv[i] * d;
    }
    __syncthreads();
  }
  for (int c = warp; c < kq; c += nwarp)
    for (int i = lane; i < m; i += 32) Qm[(int64_t)c * m + i] = mk<R>(i == c ? 1 : 0, 0);
  __syncthreads();
  for (int c = kmin - 1; c >= 0; --c) {
    const int pm = m - c;
    for (int i = threadIdx.x; i < pm; i += blockDim.x) sv[i] = V[(int64_t)c * m + c + i];
    __syncthreads();
    // columns q < c are still e_q: the reflectors applied so far touch rows > c
    for (int qq = c + warp; qq < kq; qq += nwarp) {
      cpx<R>* y = Qm + (int64_t)qq * m + c;
      cpx<R> d = mk<R>(0, 0);
      for (int i = lane; i < pm; i += 32) cfmac(d, sv[i], y[i]);
      d.re = warp_sum(d.re);
      d.im = warp_sum(d.im);
      d = (R)2 * d;
      for (int i = lane; i < pm; i += 32) y[i] = y[i] - sv[i] * d;
    }
    __syncthreads();
  }
}

// Dynamic shared memory of k_move_center_big: the GEMM tiles of the merge,
// the transpose tile and the reflector of the QR share one region (used one
// after another), then the reduction scratch.
template <class R>
struct BigMoveSmem {
  static constexpr size_t kTile = 32 * ((sizeof(R) == 4 ? 128 : 64) + 1) * sizeof(cpx<R>);
  static constexpr size_t kVec = kBigN * sizeof(cpx<R>);
  static constexpr size_t kGemm = sizeof(GemmSmem<R>);
  static constexpr size_t kShared = (kTile > kVec ? (kTile > kGemm ? kTile : kGemm) : (kVec > kGemm ? kVec : kGemm));
  static constexpr size_t kBytes = ((kShared + 15) / 16) * 16 + 40 * sizeof(R);
};

// The centre move of k_move_center (dir = +1: QR of A_k as (2 dl) x dr, R merged
// into A_{k+1}; dir = -1: LQ of A_k as dl x (2 dr), L merged into A_{k-1})
// for site capacities above 128, with householder_qr_big.
template <class R>
__global__ void __launch_bounds__(kGemmThreads) k_move_center_big(SimView<R> s, int k, int dir) {
  const int64_t t = blockIdx.x;
  if (t >= s.B) return;
  extern __shared__ __align__(16) unsigned char big_move_smem[];
  GemmSmem<R>& sm = *reinterpret_cast<GemmSmem<R>*>(big_move_smem);
  cpx<R>* tile = reinterpret_cast<cpx<R>*>(big_move_smem);
  cpx<R>* sv = reinterpret_cast<cpx<R>*>(big_move_smem);
  R* red = reinterpret_cast<R*>(big_move_smem + ((BigMoveSmem<R>::kShared + 15) / 16) * 16);
  R* sc = red + 32;
  int32_t* bd = s.bond + t * (s.n + 1);
  const int dl = bd[k], dr = bd[k + 1];
  const int capr = s.cap[k + 1];
  cpx<R>* A = site_ptr(s, k, t);
  cpx<R>* X = s.ws0 + t * s.ws_stride;
  cpx<R>* V = s.ws1 + t * s.ws_stride;
  cpx<R>* Qm = s.ws2 + t * s.ws_stride;
  cpx<R>* Tm = s.ws3 + t * s.ws_stride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (2 * max(dl, dr) > kBigN) {
    if (threadIdx.x == 0) atomicOr(s.status + t, (int32_t)TS_SHAPE);
    return;
  }
  if (dir > 0) {
    const int m = 2 * dl, n = dr, r = min(m, n);
    transpose_copy(X, m, A, capr, m, n, tile);
    householder_qr_big(X, V, Qm, m, n, r, sv, red, sc);
    const int d2 = bd[k + 2], cap2 = s.cap[k + 2];
    cpx<R>* B = site_ptr(s, k + 1, t);
    cta_gemm<R, false, false>(
        r, 2 * d2, dr, [&](int i, int l) { return l >= i ? X[(int64_t)l * m + i] : mk<R>(0, 0); },
        [&](int l, int cc) {
          const int ss = cc >= d2, b = cc - ss * d2;
          return B[(int64_t)(l * 2 + ss) * cap2 + b];
        },
        [&](int i, int cc, cpx<R> v) { Tm[(int64_t)i * 2 * d2 + cc] = v; }, sm);
    __syncthreads();
    for (int i = warp; i < r; i += nwarp)
      for (int cc = lane; cc < 2 * d2; cc += 32) {
        const int ss = cc >= d2, b = cc - ss * d2;
        B[(int64_t)(i * 2 + ss) * cap2 + b] = Tm[(int64_t)i * 2 * d2 + cc];
      }
    __syncthreads();
    transpose_copy(A, capr, Qm, m, r, m, tile);
    if (threadIdx.x == 0) bd[k + 1] = r;
  } else {
    const int m = 2 * dr, n = dl, r = min(m, n);
    for (int c = warp; c < n; c += nwarp)
      for (int i = lane; i < m; i += 32) {
        const int ss = i >= dr, b = i - ss * dr;
        X[(int64_t)c * m + i] = conj(A[(int64_t)(c * 2 + ss) * capr + b]);
      }
    __syncthreads();
    householder_qr_big(X, V, Qm, m, n, r, sv, red, sc);
    const int d0 = bd[k - 1], cap1 = s.cap[k];
    cpx<R>* P = site_ptr(s, k - 1, t);
    cta_gemm<R, true, false>(
        2 * d0, r, dl, [&](int row, int l) { return P[(int64_t)row * cap1 + l]; },
        [&](int l, int j) { return l >= j ? conj(X[(int64_t)l * m + j]) : mk<R>(0, 0); },
        [&](int row, int j, cpx<R> v) { Tm[(int64_t)row * r + j] = v; }, sm);
    __syncthreads();
    for (int row = warp; row < 2 * d0; row += nwarp)
      for (int j = lane; j < r; j += 32) P[(int64_t)row * cap1 + j] = Tm[(int64_t)row * r + j];
    for (int j = warp; j < r; j += nwarp)
      for (int i = lane; i < m; i += 32) {
        const int ss = i >= dr, b = i - ss * dr;
        A[(int64_t)(j * 2 + ss) * capr + b] = conj(Qm[(int64_t)j * m + i]);
      }
    if (threadIdx.x == 0) bd[k] = r;
  }
}

}  // namespace lemps
