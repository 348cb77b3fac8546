// Locally entanglement-optimal unraveling of a single-qubit channel (Sec. IV.B,
// App. F.2), FP64, one thread per noise site.
//
// Input: the target qubit's reduced state rho_A (2x2, trace 1) and a Kraus
// set {K_j} (r <= 4).  Steps:
//   1. eigenpairs of rho_A -> effective two-qubit state
//      psi_eff = sqrt(l0)|u0>|0> + sqrt(l1)|u1>|1>    (Sec. IV.B.2)
//   2. induced decomposition phi_j = (K_j (x) I) psi_eff (Eq. Kraus_to_ensemble)
//   3. SVD of phi by one-sided (Hestenes) Jacobi: v = phi V_phi   (Eq. v_to_phi)
//   4. tau = v^dagger (Y(x)Y) v^*, Takagi factorization tau = U diag(s) U^T via
//      the real symmetric embedding [[Re tau, Im tau], [Im tau, -Re tau]]
//      (eigenvalues +-s_k, eigenvector [a; b] <-> Takagi vector a + i b);
//      x = v U                                             (App. F.2, Step 1)
//   5. C = s1 - s2 - s3 - s4; entangled: y = x diag(1,i,i,i) (Step 2),
//      M = y^dagger tilde y - C y^dagger y, Re M = Q D Q^T, z = y Q H_4 (Step 3);
//      separable: z = x diag(e^{i theta}) H_4 with the trapezoid angles
//   6. W = V_phi T with z = v T; K'_k = sum_j W[j][k] K_j   (Sec. IV.B.4)
// Canonical rules (identical, written independently, in the CPU oracle):
//   R1 rho_A eigenvector phases make <REF2|u_k> real positive; degenerate
//      rho_A uses the computational basis.
//   R2/R3 reference Gram-Schmidt of blocks with a real-orthogonal (equal
//      Takagi values, equal eigenvalues of Re M) or unitary (zero Takagi
//      values) freedom, against the fixed vectors REF4.
//   R4 rank / zero / degeneracy tolerances RANK_TOL, ZERO_TOL, DEG_TOL.
//   R5 separability test C > 0.
//   R6 a pure target (l1 <= PURE_TOL) keeps the given Kraus set.
#pragma once

#include "common.cuh"

namespace lemps {
namespace unr {

constexpr double RANK_TOL = 1e-12;
constexpr double PURE_TOL = 1e-12;
constexpr double DEG_TOL = 1e-9;
constexpr double ZERO_TOL = 1e-10;
constexpr double kPi = 3.14159265358979323846;

// REF2 and REF4 as (re, im) pairs.
__device__ __constant__ double kRef2[4] = {0.8, 0.0, 0.36, 0.48};
__device__ __constant__ double kRef4[8][8] = {
    {0.47, 0.0, 0.31, 0.22, -0.18, 0.53, 0.26, -0.52},
    {0.12, 0.44, 0.58, 0.0, -0.37, -0.21, -0.33, 0.38},
    {-0.29, 0.35, 0.14, -0.41, 0.62, 0.0, 0.23, 0.41},
    {0.36, -0.27, -0.45, 0.16, 0.28, 0.33, 0.61, 0.0},
    {0.5, 0.0, 0.0, -0.5, 0.5, 0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5, 0.0, -0.5, 0.0, 0.5, 0.0},
    {1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0}};

__device__ __forceinline__ zd ref4(int r, int i) { return mk(kRef4[r][2 * i], kRef4[r][2 * i + 1]); }

// (Y (x) Y) is real: it maps e0 -> -e3, e1 -> e2, e2 -> e1, e3 -> -e0.
// tilde w = (Y(x)Y) w^*.
__device__ __forceinline__ void spin_flip(const zd* w, zd* out) {
  out[0] = -conj(w[3]);
  out[1] = conj(w[2]);
  out[2] = conj(w[1]);
  out[3] = -conj(w[0]);
}

// Cyclic Jacobi for a real symmetric N x N matrix (row-major, N <= 8).
// Returns eigenvalues in w (descending) and eigenvectors as columns of v.
// The size is a template parameter so that the row/column updates unroll
// into independent loads and FMAs (the matrices live in local memory).
template <int N>
__device__ inline void jacobi_sym_n(double* a, double* v, double* w) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) v[i * N + j] = (i == j) ? 1.0 : 0.0;
  double tot = 0.0;
#pragma unroll
  for (int i = 0; i < N * N; ++i) tot += a[i] * a[i];
  // rotate only |a_pq| above eps_64 ||A||_F, the accuracy of a backward-stable
  // eigensolver; smaller entries are rounding noise of the earlier rotations
  const double thresh = 2.2e-16 * sqrt(tot);
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < N - 1; ++p)
      for (int q = p + 1; q < N; ++q) {
        double apq = a[p * N + q];
        if (fabs(apq) <= thresh) continue;
        rotated = true;
        // t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (a_qq - a_pp) / (2 a_pq),
        // written with one square root and one divide (each a sequence of FP64
        // operations), and c = 1 / sqrt(1 + t^2) by the reciprocal square root
        const double diff = a[q * N + q] - a[p * N + p], ta = 2.0 * apq;
        const double sz = (diff == 0.0 || ((diff > 0.0) == (apq > 0.0))) ? 1.0 : -1.0;
        const double t = sz * fabs(ta) / (fabs(diff) + sqrt(diff * diff + ta * ta));
        const double c = rsqrt(1.0 + t * t), s = c * t;
        // A <- J^T A J, J = [[c, s], [-s, c]] on (p, q).  A stays symmetric, so
        // rows p, q are rotated once and mirrored into the columns, and the
        // pivot block takes its closed form (a_pq -> 0, a_pp -= t a_pq, a_qq
        // += t a_pq): about 0.6 of the FP64 operations of two full passes,
        // which is what a rotation costs at the FP64 rate.
        const double app = a[p * N + p], aqq = a[q * N + q];
#pragma unroll
        for (int k = 0; k < N; ++k) {
          if (k == p || k == q) continue;
          const double akp = a[k * N + p], akq = a[k * N + q];
          const double nkp = c * akp - s * akq, nkq = s * akp + c * akq;
          a[k * N + p] = nkp;
          a[p * N + k] = nkp;
          a[k * N + q] = nkq;
          a[q * N + k] = nkq;
        }
        a[p * N + p] = app - t * apq;
        a[q * N + q] = aqq + t * apq;
        a[p * N + q] = 0.0;
        a[q * N + p] = 0.0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          double vkp = v[k * N + p], vkq = v[k * N + q];
          v[k * N + p] = c * vkp - s * vkq;
          v[k * N + q] = s * vkp + c * vkq;
        }
      }
    if (!rotated) break;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) w[i] = a[i * N + i];
  for (int i = 0; i < N - 1; ++i) {  // selection sort, descending
    int best = i;
    for (int j = i + 1; j < N; ++j)
      if (w[j] > w[best]) best = j;
    if (best != i) {
      double t = w[i]; w[i] = w[best]; w[best] = t;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        double u = v[k * N + i]; v[k * N + i] = v[k * N + best]; v[k * N + best] = u;
      }
    }
  }
}

// n = 2 rank (2, 4, 6, 8) for the Takagi embedding, 4 for M_R.
__device__ inline void jacobi_sym(double* a, double* v, double* w, int n) {
  switch (n) {
    case 1: jacobi_sym_n<1>(a, v, w); break;
    case 2: jacobi_sym_n<2>(a, v, w); break;
    case 3: jacobi_sym_n<3>(a, v, w); break;
    case 4: jacobi_sym_n<4>(a, v, w); break;
    case 5: jacobi_sym_n<5>(a, v, w); break;
    case 6: jacobi_sym_n<6>(a, v, w); break;
    case 7: jacobi_sym_n<7>(a, v, w); break;
    default: jacobi_sym_n<8>(a, v, w); break;
  }
}

// Reference Gram-Schmidt (rules R2/R3).  A: 4 x m complex, column-major
// (a[c*4 + i]).  Writes B (m x m, column-major) such that A B is canonical.
// complex_freedom = false restricts B to real orthogonal.
__device__ inline void reference_basis(const zd* a, int m, bool complex_freedom, zd* b) {
  double scale = 0.0;
  for (int i = 0; i < 4 * m; ++i) scale += norm2(a[i]);
  scale = sqrt(scale);
  if (scale < 1e-300) scale = 1e-300;
  int nb = 0;
  for (int r = 0; r < 8 && nb < m; ++r) {
    zd g[4];
    double rn = 0.0;
    for (int i = 0; i < 4; ++i) rn += norm2(ref4(r, i));
    rn = sqrt(rn);
    for (int c = 0; c < m; ++c) {
      zd s = mk(0.0, 0.0);
      for (int i = 0; i < 4; ++i) cfmac(s, a[c * 4 + i], ref4(r, i));  // (A^dagger r)_c
      g[c] = complex_freedom ? s : mk(s.re, 0.0);
    }
    for (int k = 0; k < nb; ++k) {
      zd d = mk(0.0, 0.0);
      for (int c = 0; c < m; ++c) cfmac(d, b[k * m + c], g[c]);
      for (int c = 0; c < m; ++c) g[c] -= d * b[k * m + c];
    }
    double nrm = 0.0;
    for (int c = 0; c < m; ++c) nrm += norm2(g[c]);
    nrm = sqrt(nrm);
    if (nrm > 1e-8 * scale * rn) {
      for (int c = 0; c < m; ++c) b[nb * m + c] = (1.0 / nrm) * g[c];
      ++nb;
    }
  }
  for (int e = 0; e < m && nb < m; ++e) {  // rank-deficient block: complete
    zd g[4];
    for (int c = 0; c < m; ++c) g[c] = mk(c == e ? 1.0 : 0.0, 0.0);
    for (int k = 0; k < nb; ++k) {
      zd d = mk(0.0, 0.0);
      for (int c = 0; c < m; ++c) cfmac(d, b[k * m + c], g[c]);
      for (int c = 0; c < m; ++c) g[c] -= d * b[k * m + c];
    }
    double nrm = 0.0;
    for (int c = 0; c < m; ++c) nrm += norm2(g[c]);
    nrm = sqrt(nrm);
    if (nrm > 1e-6) {
      for (int c = 0; c < m; ++c) b[nb * m + c] = (1.0 / nrm) * g[c];
      ++nb;
    }
  }
}

// Apply the canonical basis to columns idx[0..m) of x (4 x 4 column-major)
// and of ut (4 x 4 column-major).
__device__ inline void canonicalize_block(zd* x, zd* ut, const int* idx, int m, bool complex_freedom) {
  zd a[16], b[16], tmpx[16], tmpu[16];
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < 4; ++i) a[c * 4 + i] = x[idx[c] * 4 + i];
  reference_basis(a, m, complex_freedom, b);
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < 4; ++i) {
      zd sx = mk(0.0, 0.0), su = mk(0.0, 0.0);
      for (int k = 0; k < m; ++k) {
        cfma(sx, x[idx[k] * 4 + i], b[c * m + k]);
        cfma(su, ut[idx[k] * 4 + i], b[c * m + k]);
      }
      tmpx[c * 4 + i] = sx;
      tmpu[c * 4 + i] = su;
    }
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < 4; ++i) {
      x[idx[c] * 4 + i] = tmpx[c * 4 + i];
      ut[idx[c] * 4 + i] = tmpu[c * 4 + i];
    }
}

// Trapezoid angles of the separable case (Eq. separating_angles_condition).
__device__ inline void separable_angles(const double* l, double* th) {
  double l1 = l[0], l2 = l[1], l3 = l[2], l4 = l[3];
  if (l1 - l4 <= DEG_TOL * fmax(l1, 1e-300)) {
    th[0] = 0.0; th[1] = kPi / 4; th[2] = kPi / 2; th[3] = 3 * kPi / 4;
    return;
  }
  double d = l1 - l4;
  double s0 = d, s1 = l2, s2 = l3, t;  // sort descending (Kahan's Heron)
  if (s0 < s1) { t = s0; s0 = s1; s1 = t; }
  if (s1 < s2) { t = s1; s1 = s2; s2 = t; }
  if (s0 < s1) { t = s0; s0 = s1; s1 = t; }
  double prod = (s0 + (s1 + s2)) * (s2 - (s0 - s1)) * (s2 + (s0 - s1)) * (s0 + (s1 - s2));
  double area = 0.25 * sqrt(fmax(0.0, prod));
  double h = 2.0 * area / d;
  double a2 = (l2 > 0.0) ? kPi - asin(fmin(1.0, h / l2)) : 0.0;
  double a3 = 0.0;
  if (l3 > 0.0) {
    double b3 = asin(fmin(1.0, h / l3));
    a3 = (l2 * cos(a2) + d > 0.0) ? kPi + b3 : -b3;
  }
  th[0] = 0.0; th[1] = 0.5 * a2; th[2] = 0.5 * a3; th[3] = 0.5 * kPi;
}

// 2x2 Hermitian [[a, b], [b*, d]]: eigenvalues l0 >= l1.
__device__ __forceinline__ void eig2_values(double a, double d, zd b, double* l0, double* l1) {
  double m = 0.5 * (a + d), r = sqrt(0.25 * (a - d) * (a - d) + norm2(b));
  *l0 = m + r;
  *l1 = m - r;
}

__device__ __forceinline__ double xlogx(double x) { return x > 0.0 ? x * log(x) : 0.0; }

// von Neumann entropy (nats) of a 2x2 Hermitian PSD matrix divided by its trace.
__device__ inline double entropy2(const zd* s) {
  double tr = s[0].re + s[3].re;
  if (!(tr > 0.0)) return 0.0;
  double l0, l1;
  eig2_values(s[0].re / tr, s[3].re / tr, (1.0 / tr) * s[1], &l0, &l1);
  return -(xlogx(fmax(l0, 0.0)) + xlogx(fmax(l1, 0.0)));
}

// p_k = Tr(K_k rho K_k^dagger) and E_av = sum_k p_k S(K_k rho K_k^dagger / p_k).
__device__ inline double branch_weights(const zd* kr, int r, const zd* rho, double* p) {
  double e = 0.0;
  for (int k = 0; k < r; ++k) {
    const zd* K = kr + 4 * k;
    zd kr_[4], s[4];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        zd acc = mk(0.0, 0.0);
        for (int l = 0; l < 2; ++l) cfma(acc, K[i * 2 + l], rho[l * 2 + j]);
        kr_[i * 2 + j] = acc;
      }
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        zd acc = mk(0.0, 0.0);
        for (int l = 0; l < 2; ++l) cfma(acc, kr_[i * 2 + l], conj(K[j * 2 + l]));
        s[i * 2 + j] = acc;
      }
    p[k] = s[0].re + s[3].re;
    e += p[k] * entropy2(s);
  }
  return e;
}

// Main routine.  rho: 2x2 row-major, trace 1.  kin: r operators, row-major
// 2x2.  kout: 4 operators.  Returns false when the input was not finite.
__device__ __noinline__ bool optimal_unraveling(const zd* rho, const zd* kin, int r, zd* kout) {
  zd kpad[16];
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i < 4; ++i) kpad[k * 4 + i] = (k < r) ? kin[k * 4 + i] : mk(0.0, 0.0);
  double a = rho[0].re, d = rho[3].re;
  zd b = rho[1];
  if (!isfinite(a) || !isfinite(d) || !isfinite(b.re) || !isfinite(b.im)) return false;
  double l0, l1;
  eig2_values(a, d, b, &l0, &l1);
  if (l1 <= PURE_TOL * fmax(l0 + l1, 1e-300)) {  // R6
    for (int i = 0; i < 16; ++i) kout[i] = kpad[i];
    return true;
  }
  // R1: eigenvectors of rho_A
  zd u[2][2];  // u[k][component]
  if (l0 - l1 <= DEG_TOL * l0) {
    u[0][0] = mk(1.0, 0.0); u[0][1] = mk(0.0, 0.0);
    u[1][0] = mk(0.0, 0.0); u[1][1] = mk(1.0, 0.0);
  } else {
    zd e0, e1;
    if (a >= d) { e0 = mk(l0 - d, 0.0); e1 = conj(b); }
    else { e0 = b; e1 = mk(l0 - a, 0.0); }
    double nn = sqrt(norm2(e0) + norm2(e1));
    e0 = (1.0 / nn) * e0; e1 = (1.0 / nn) * e1;
    u[0][0] = e0; u[0][1] = e1;
    u[1][0] = -conj(e1); u[1][1] = conj(e0);
    for (int k = 0; k < 2; ++k) {
      zd ov = mk(0.0, 0.0);
      cfmac(ov, mk(kRef2[0], kRef2[1]), u[k][0]);
      cfmac(ov, mk(kRef2[2], kRef2[3]), u[k][1]);
      double on = sqrt(norm2(ov));
      zd ph = (1.0 / on) * conj(ov);
      u[k][0] = u[k][0] * ph; u[k][1] = u[k][1] * ph;
    }
  }
  // psi_eff[2t + k] = sqrt(l_k) u_k[t]
  zd psi[4];
  double sl[2] = {sqrt(fmax(l0, 0.0)), sqrt(fmax(l1, 0.0))};
  for (int t = 0; t < 2; ++t)
    for (int k = 0; k < 2; ++k) psi[2 * t + k] = sl[k] * u[k][t];
  // phi (column-major 4 x 4): phi[j*4 + 2t + k] = sum_s K_j[t][s] psi[2s + k]
  zd f[16];
  for (int j = 0; j < 4; ++j)
    for (int t = 0; t < 2; ++t)
      for (int k = 0; k < 2; ++k) {
        zd acc = mk(0.0, 0.0);
        for (int s = 0; s < 2; ++s) cfma(acc, kpad[j * 4 + t * 2 + s], psi[2 * s + k]);
        f[j * 4 + 2 * t + k] = acc;
      }
  // One-sided Jacobi: f <- f V_phi with orthogonal columns.
  zd vphi[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) vphi[j * 4 + i] = mk(i == j ? 1.0 : 0.0, 0.0);
  double fnorm2 = 0.0;
  for (int i = 0; i < 16; ++i) fnorm2 += norm2(f[i]);
  for (int sweep = 0; sweep < 40; ++sweep) {
    bool rotated = false;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = p + 1; q < 4; ++q) {
        double al = 0.0, be = 0.0;
        zd g = mk(0.0, 0.0);
        for (int i = 0; i < 4; ++i) {
          al += norm2(f[p * 4 + i]);
          be += norm2(f[q * 4 + i]);
          cfmac(g, f[p * 4 + i], f[q * 4 + i]);
        }
        const double gn2 = norm2(g);
        if (gn2 <= 1e-32 * (al * be) || gn2 <= 1e-60 * (fnorm2 * fnorm2)) continue;
        rotated = true;
        // as in the symmetric case: zeta = (be - al) / (2 |g|) > -0 picks the sign
        const double ign = rsqrt(gn2), gn = gn2 * ign, diff = be - al;
        const double t = (diff >= 0.0 ? 1.0 : -1.0) * (2.0 * gn) / (fabs(diff) + sqrt(diff * diff + 4.0 * gn2));
        const double c = rsqrt(1.0 + t * t), s = c * t;
        const zd eph = mk(g.re * ign, -g.im * ign);  // e^{-i phi}
        for (int i = 0; i < 4; ++i) {
          zd fp = f[p * 4 + i], fq = f[q * 4 + i] * eph;
          f[p * 4 + i] = c * fp - s * fq;
          f[q * 4 + i] = s * fp + c * fq;
          zd vp = vphi[p * 4 + i], vq = vphi[q * 4 + i] * eph;
          vphi[p * 4 + i] = c * vp - s * vq;
          vphi[q * 4 + i] = s * vp + c * vq;
        }
      }
    if (!rotated) break;
  }
  double sv[4];
  for (int j = 0; j < 4; ++j) {
    double s = 0.0;
    for (int i = 0; i < 4; ++i) s += norm2(f[j * 4 + i]);
    sv[j] = sqrt(s);
  }
  for (int i = 0; i < 3; ++i) {  // sort columns by descending norm
    int best = i;
    for (int j = i + 1; j < 4; ++j)
      if (sv[j] > sv[best]) best = j;
    if (best != i) {
      double t = sv[i]; sv[i] = sv[best]; sv[best] = t;
      for (int k = 0; k < 4; ++k) {
        zd x = f[i * 4 + k]; f[i * 4 + k] = f[best * 4 + k]; f[best * 4 + k] = x;
        zd y = vphi[i * 4 + k]; vphi[i * 4 + k] = vphi[best * 4 + k]; vphi[best * 4 + k] = y;
      }
    }
  }
  int rank = 0;
  for (int j = 0; j < 4; ++j)
    if (sv[j] > RANK_TOL * sv[0]) ++rank;
  zd v[16];
  for (int j = 0; j < 4; ++j)
    for (int i = 0; i < 4; ++i) v[j * 4 + i] = (j < rank) ? f[j * 4 + i] : mk(0.0, 0.0);
  // tau = v^dagger tilde v on the leading rank block
  zd vt[16];
  for (int j = 0; j < 4; ++j) spin_flip(v + 4 * j, vt + 4 * j);
  zd ut[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) ut[j * 4 + i] = mk(i == j ? 1.0 : 0.0, 0.0);
  double sig[4] = {0.0, 0.0, 0.0, 0.0};
  if (rank > 0) {
    const int n2 = 2 * rank;
    double e[64], ev[64], w[8];
    for (int i = 0; i < rank; ++i)
      for (int j = 0; j < rank; ++j) {
        zd tij = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) cfmac(tij, v[i * 4 + k], vt[j * 4 + k]);
        e[i * n2 + j] = tij.re;
        e[i * n2 + rank + j] = tij.im;
        e[(rank + i) * n2 + j] = tij.im;
        e[(rank + i) * n2 + rank + j] = -tij.re;
      }
    // symmetrize (tau is symmetric up to rounding)
    for (int i = 0; i < n2; ++i)
      for (int j = i + 1; j < n2; ++j) {
        double m = 0.5 * (e[i * n2 + j] + e[j * n2 + i]);
        e[i * n2 + j] = m; e[j * n2 + i] = m;
      }
    jacobi_sym(e, ev, w, n2);
    int nz = 0;
    for (int k = 0; k < rank; ++k)
      if (w[k] > ZERO_TOL * w[0]) ++nz;
    zd ur[16];  // columns of the Takagi factor of the rank block (rank x rank, column-major)
    for (int k = 0; k < nz; ++k) {
      for (int i = 0; i < rank; ++i) ur[k * rank + i] = mk(ev[i * n2 + k], ev[(rank + i) * n2 + k]);
      sig[k] = w[k];
    }
    int got = nz;
    for (int k = nz; k < n2 - nz && got < rank; ++k) {  // zero Takagi values: complex GS
      zd g[4];
      for (int i = 0; i < rank; ++i) g[i] = mk(ev[i * n2 + k], ev[(rank + i) * n2 + k]);
      for (int c = 0; c < got; ++c) {
        zd dd = mk(0.0, 0.0);
        for (int i = 0; i < rank; ++i) cfmac(dd, ur[c * rank + i], g[i]);
        for (int i = 0; i < rank; ++i) g[i] -= dd * ur[c * rank + i];
      }
      double nn = 0.0;
      for (int i = 0; i < rank; ++i) nn += norm2(g[i]);
      nn = sqrt(nn);
      if (nn > 1e-6) {
        for (int i = 0; i < rank; ++i) ur[got * rank + i] = (1.0 / nn) * g[i];
        ++got;
      }
    }
    for (int c = 0; c < rank; ++c)
      for (int i = 0; i < rank; ++i) ut[c * 4 + i] = ur[c * rank + i];
  }
  // x = v ut
  zd x[16];
  for (int c = 0; c < 4; ++c)
    for (int i = 0; i < 4; ++i) {
      zd acc = mk(0.0, 0.0);
      for (int k = 0; k < 4; ++k) cfma(acc, v[k * 4 + i], ut[c * 4 + k]);
      x[c * 4 + i] = acc;
    }
  // R2/R3 on the Takagi vectors
  if (rank > 0) {
    double s1 = sig[0];
    int nzi[4], zi[4], nnz = 0, nzero = 0;
    for (int k = 0; k < rank; ++k) {
      if (sig[k] <= ZERO_TOL * s1) zi[nzero++] = k;
      else nzi[nnz++] = k;
    }
    int start = 0;
    while (start < nnz) {
      int end = start + 1;
      double scale = fmax(fabs(sig[nzi[0]]), 1e-300);
      while (end < nnz && sig[nzi[end - 1]] - sig[nzi[end]] <= DEG_TOL * scale) ++end;
      canonicalize_block(x, ut, nzi + start, end - start, false);
      start = end;
    }
    if (nzero > 0) {
      canonicalize_block(x, ut, zi, nzero, true);
      for (int k = 0; k < nzero; ++k) sig[zi[k]] = 0.0;
    }
  }
  double cc = sig[0] - sig[1] - sig[2] - sig[3];
  zd tmat[16];  // T (column-major) with z = v T
  const double h4[16] = {0.5, 0.5, 0.5, 0.5, 0.5, 0.5, -0.5, -0.5,
                         0.5, -0.5, 0.5, -0.5, 0.5, -0.5, -0.5, 0.5};  // symmetric
  if (cc > 0.0) {
    zd y[16], yt[16];
    for (int c = 0; c < 4; ++c)
      for (int i = 0; i < 4; ++i) y[c * 4 + i] = (c == 0) ? x[c * 4 + i] : mk(-x[c * 4 + i].im, x[c * 4 + i].re);
    for (int c = 0; c < 4; ++c) spin_flip(y + 4 * c, yt + 4 * c);
    double mr[16], q[16], dq[4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        zd a1 = mk(0.0, 0.0), a2 = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) {
          cfmac(a1, y[i * 4 + k], yt[j * 4 + k]);
          cfmac(a2, y[i * 4 + k], y[j * 4 + k]);
        }
        mr[i * 4 + j] = a1.re - cc * a2.re;
      }
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j) {
        double m = 0.5 * (mr[i * 4 + j] + mr[j * 4 + i]);
        mr[i * 4 + j] = m; mr[j * 4 + i] = m;
      }
    jacobi_sym(mr, q, dq, 4);
    // a = y Q, canonicalize per eigenvalue cluster
    zd qc[16], aq[16], qdummy[16];
    for (int c = 0; c < 4; ++c)
      for (int i = 0; i < 4; ++i) qc[c * 4 + i] = mk(q[i * 4 + c], 0.0);
    for (int c = 0; c < 4; ++c)
      for (int i = 0; i < 4; ++i) {
        zd acc = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) cfma(acc, y[k * 4 + i], qc[c * 4 + k]);
        aq[c * 4 + i] = acc;
      }
    double scale = 0.0;
    for (int k = 0; k < 4; ++k) scale = fmax(scale, fabs(dq[k]));
    scale = fmax(scale, 1e-300);
    int start = 0;
    while (start < 4) {
      int end = start + 1;
      while (end < 4 && dq[end - 1] - dq[end] <= DEG_TOL * scale) ++end;
      int idx[4];
      for (int k = start; k < end; ++k) idx[k - start] = k;
      for (int i = 0; i < 16; ++i) qdummy[i] = mk(0.0, 0.0);
      // canonicalize_block rotates aq's columns and qc's columns together
      canonicalize_block(aq, qc, idx, end - start, false);
      start = end;
    }
    // T = ut diag(1,i,i,i) Q H4
    zd m1[16];
    for (int c = 0; c < 4; ++c)
      for (int i = 0; i < 4; ++i) {
        zd acc = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) {
          zd uk = ut[k * 4 + i];
          if (k > 0) uk = mk(-uk.im, uk.re);
          cfma(acc, uk, qc[c * 4 + k]);
        }
        m1[c * 4 + i] = acc;
      }
    for (int c = 0; c < 4; ++c)
      for (int i = 0; i < 4; ++i) {
        zd acc = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) acc += h4[k * 4 + c] * m1[k * 4 + i];
        tmat[c * 4 + i] = acc;
      }
  } else {
    double th[4];
    separable_angles(sig, th);
    zd m1[16];
    for (int c = 0; c < 4; ++c) {
      double sn, cs;
      sincos(th[c], &sn, &cs);
      zd ph = mk(cs, sn);
      for (int i = 0; i < 4; ++i) m1[c * 4 + i] = ut[c * 4 + i] * ph;
    }
    for (int c = 0; c < 4; ++c)
      for (int i = 0; i < 4; ++i) {
        zd acc = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) acc += h4[k * 4 + c] * m1[k * 4 + i];
        tmat[c * 4 + i] = acc;
      }
  }
  // W = V_phi T ; K'_k = sum_j W[j][k] K_j
  for (int k = 0; k < 4; ++k) {
    zd wk[4];
    for (int j = 0; j < 4; ++j) {
      zd acc = mk(0.0, 0.0);
      for (int l = 0; l < 4; ++l) cfma(acc, vphi[l * 4 + j], tmat[k * 4 + l]);
      wk[j] = acc;
    }
    for (int e = 0; e < 4; ++e) {
      zd acc = mk(0.0, 0.0);
      for (int j = 0; j < 4; ++j) cfma(acc, wk[j], kpad[j * 4 + e]);
      kout[k * 4 + e] = acc;
    }
  }
  return true;
}

}  // namespace unr
}  // namespace lemps
