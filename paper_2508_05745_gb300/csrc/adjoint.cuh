// Expected branch entanglement of a remixed Kraus set and its adjoint
// (the cost of Eq. target_optimal_unitary as a function of the mixing unitary
// U = exp(iH), remix K'_k = sum_j U[j][k] K_j, Eq. unitarity_kraus).
//
//   E(H) = sum_k p_k S(sigma_k / p_k),   sigma_k = K'_k rho K'_k^dagger
//
// Gradient, with dE = Re Tr(Gamma^dagger dH) on Hermitian dH:
//   dE/dsigma_k  = -ln(sigma_k / p_k)                       (G_k, Hermitian)
//   dE/dK'_k     = 2 G_k K'_k rho                            (Gbar_k)
//   dE/dU[j][k]  = Tr(K_j^dagger Gbar_k)                     (Omega)
//   exp at A = iH = V diag(i h) V^dagger: the Frechet derivative's adjoint is
//   Y = V (conj(F) o (V^dagger Omega V)) V^dagger with the divided differences
//   F_jk = e^{i (h_j + h_k)/2} sin(d/2)/(d/2), d = h_j - h_k (equal-eigenvalue
//   limit e^{i h_j}, so degenerate spectra need no special case);
//   Gamma = Herm(-i Y).
// Zero eigenvalues of sigma_k are clamped to 1e-300 inside the logarithm.
#pragma once

#include "common.cuh"

namespace lemps {
namespace adj {

// Two-sided cyclic Jacobi for a 4x4 complex Hermitian matrix (row-major).
// Eigenvectors are the columns of v; eigenvalues in w (unsorted).
__device__ inline void jacobi_herm4(zd* a, zd* v, double* w) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) v[i * 4 + j] = mk(i == j ? 1.0 : 0.0, 0.0);
  double tot = 0.0;
  for (int i = 0; i < 16; ++i) tot += norm2(a[i]);
  const double thresh = 1e-17 * sqrt(tot);
  for (int sweep = 0; sweep < 40; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < 3; ++p)
      for (int q = p + 1; q < 4; ++q) {
        zd g = a[p * 4 + q];
        double gn = sqrt(norm2(g));
        if (gn <= thresh) continue;
        rotated = true;
        double zeta = (a[q * 4 + q].re - a[p * 4 + p].re) / (2.0 * gn);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        zd e = mk(g.re / gn, -g.im / gn);
        for (int k = 0; k < 4; ++k) {  // columns
          zd xp = a[k * 4 + p], xq = e * a[k * 4 + q];
          a[k * 4 + p] = c * xp - s * xq;
          a[k * 4 + q] = s * xp + c * xq;
          zd vp = v[k * 4 + p], vq = e * v[k * 4 + q];
          v[k * 4 + p] = c * vp - s * vq;
          v[k * 4 + q] = s * vp + c * vq;
        }
        zd ec = conj(e);
        for (int k = 0; k < 4; ++k) {  // rows
          zd xp = a[p * 4 + k], xq = ec * a[q * 4 + k];
          a[p * 4 + k] = c * xp - s * xq;
          a[q * 4 + k] = s * xp + c * xq;
        }
      }
    if (!rotated) break;
  }
  for (int i = 0; i < 4; ++i) w[i] = a[i * 4 + i].re;
}

__device__ inline void depolarizing_set(double p, zd* k) {
  const double a = sqrt(1.0 - 0.75 * p), b = 0.5 * sqrt(p);
  for (int i = 0; i < 16; ++i) k[i] = mk(0.0, 0.0);
  k[0] = mk(a, 0.0); k[3] = mk(a, 0.0);                // I
  k[4 + 1] = mk(b, 0.0); k[4 + 2] = mk(b, 0.0);        // X
  k[8 + 1] = mk(0.0, -b); k[8 + 2] = mk(0.0, b);       // Y
  k[12 + 0] = mk(b, 0.0); k[12 + 3] = mk(-b, 0.0);     // Z
}

// 2x2 Hermitian eigendecomposition: values l[0] >= l[1], vectors columns of e.
__device__ inline void eig2(const zd* s, double* l, zd* e) {
  double a = s[0].re, d = s[3].re;
  zd b = s[1];
  double m = 0.5 * (a + d), r = sqrt(0.25 * (a - d) * (a - d) + norm2(b));
  l[0] = m + r;
  l[1] = m - r;
  zd e0, e1;
  if (norm2(b) == 0.0) {
    if (a >= d) { e0 = mk(1.0, 0.0); e1 = mk(0.0, 0.0); }
    else { e0 = mk(0.0, 0.0); e1 = mk(1.0, 0.0); }
  } else if (a >= d) {
    e0 = mk(l[0] - d, 0.0); e1 = conj(b);
  } else {
    e0 = b; e1 = mk(l[0] - a, 0.0);
  }
  double nn = sqrt(norm2(e0) + norm2(e1));
  e0 = (1.0 / nn) * e0; e1 = (1.0 / nn) * e1;
  e[0] = e0; e[2] = e1;                 // column 0
  e[1] = -conj(e1); e[3] = conj(e0);    // column 1
}

// Cost and (optionally) gradient for one problem.
__device__ inline double cost_grad(const zd* rho, double p, const zd* h_in, zd* grad) {
  zd kr[16];
  depolarizing_set(p, kr);
  zd a[16], v[16];
  double hw[4];
  for (int i = 0; i < 16; ++i) a[i] = h_in[i];
  for (int i = 0; i < 4; ++i)  // Hermitian part of the input
    for (int j = 0; j < 4; ++j) a[i * 4 + j] = 0.5 * (h_in[i * 4 + j] + conj(h_in[j * 4 + i]));
  jacobi_herm4(a, v, hw);
  zd u[16];  // U = V diag(e^{i h}) V^dagger
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      zd acc = mk(0.0, 0.0);
      for (int k = 0; k < 4; ++k) {
        double sn, cs;
        sincos(hw[k], &sn, &cs);
        cfma(acc, v[i * 4 + k] * mk(cs, sn), conj(v[j * 4 + k]));
      }
      u[i * 4 + j] = acc;
    }
  zd kp[16];
  for (int k = 0; k < 4; ++k)
    for (int e = 0; e < 4; ++e) {
      zd acc = mk(0.0, 0.0);
      for (int j = 0; j < 4; ++j) cfma(acc, u[j * 4 + k], kr[j * 4 + e]);
      kp[k * 4 + e] = acc;
    }
  double cost = 0.0;
  zd gbar[16];
  for (int k = 0; k < 4; ++k) {
    const zd* K = kp + 4 * k;
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
    double pk = s[0].re + s[3].re;
    double lam[2];
    zd ev[4];
    eig2(s, lam, ev);
    double lnp = log(fmax(pk, 1e-300));
    for (int i = 0; i < 2; ++i) {
      double li = fmax(lam[i], 0.0);
      if (li > 0.0) cost -= li * log(li);
    }
    if (pk > 0.0) cost += pk * lnp;
    if (grad) {
      // G_k = -sum_i (ln l_i - ln p) e_i e_i^dagger
      zd gk[4];
      for (int i = 0; i < 4; ++i) gk[i] = mk(0.0, 0.0);
      for (int m = 0; m < 2; ++m) {
        double f = -(log(fmax(lam[m], 1e-300)) - lnp);
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) gk[i * 2 + j] += f * (ev[i * 2 + m] * conj(ev[j * 2 + m]));
      }
      // Gbar_k = 2 G_k K'_k rho = 2 G_k kr_
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          zd acc = mk(0.0, 0.0);
          for (int l = 0; l < 2; ++l) cfma(acc, gk[i * 2 + l], kr_[l * 2 + j]);
          gbar[k * 4 + i * 2 + j] = 2.0 * acc;
        }
    }
  }
  if (grad) {
    zd om[16];  // Omega[j][k] = Tr(K_j^dagger Gbar_k)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) {
        zd acc = mk(0.0, 0.0);
        for (int e = 0; e < 4; ++e) cfmac(acc, kr[j * 4 + e], gbar[k * 4 + e]);
        om[j * 4 + k] = acc;
      }
    zd t1[16], op[16];  // op = V^dagger Omega V
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        zd acc = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) cfma(acc, om[i * 4 + k], v[k * 4 + j]);
        t1[i * 4 + j] = acc;
      }
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        zd acc = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) cfmac(acc, v[k * 4 + i], t1[k * 4 + j]);
        op[i * 4 + j] = acc;
      }
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        double m = 0.5 * (hw[i] + hw[j]), dd = 0.5 * (hw[i] - hw[j]);
        double sc = (fabs(dd) < 1e-8) ? 1.0 - dd * dd / 6.0 : sin(dd) / dd;
        double sn, cs;
        sincos(m, &sn, &cs);
        zd f = mk(cs * sc, sn * sc);
        op[i * 4 + j] = conj(f) * op[i * 4 + j];
      }
    zd y[16];  // Y = V op V^dagger
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        zd acc = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) cfma(acc, v[i * 4 + k], op[k * 4 + j]);
        t1[i * 4 + j] = acc;
      }
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        zd acc = mk(0.0, 0.0);
        for (int k = 0; k < 4; ++k) cfma(acc, t1[i * 4 + k], conj(v[j * 4 + k]));
        y[i * 4 + j] = acc;
      }
    // Gamma = Herm(-i Y)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        zd a1 = mk(y[i * 4 + j].im, -y[i * 4 + j].re);        // -i Y_ij
        zd a2 = mk(y[j * 4 + i].im, -y[j * 4 + i].re);        // -i Y_ji
        grad[i * 4 + j] = 0.5 * (a1 + conj(a2));
      }
  }
  return cost;
}

// rho[b] = sum Theta[a][s][x][c] conj(Theta[a][t][x][c]) / trace; one CTA per problem.
template <class R>
__global__ void k_rho_target(const cpx<R>* theta, int64_t batch, int chi, zd* rho) {
  const int64_t b = blockIdx.x;
  if (b >= batch) return;
  __shared__ double red[32];
  const cpx<R>* th = theta + b * (int64_t)chi * 4 * chi;
  const int64_t npair = (int64_t)chi * 2 * chi;  // (a, x, c)
  double r00 = 0.0, r11 = 0.0, r01r = 0.0, r01i = 0.0;
  for (int64_t u = threadIdx.x; u < npair; u += blockDim.x) {
    const int64_t a = u / (2 * chi), rem = u % (2 * chi);  // rem = x * chi + c
    const int64_t e0 = a * 4 * chi + rem, e1 = e0 + 2 * chi;
    zd x0 = cast<double>(th[e0]), x1 = cast<double>(th[e1]);
    r00 += norm2(x0);
    r11 += norm2(x1);
    r01r += x0.re * x1.re + x0.im * x1.im;   // x0 conj(x1)
    r01i += x0.im * x1.re - x0.re * x1.im;
  }
  r00 = block_sum(r00, red);
  r11 = block_sum(r11, red);
  r01r = block_sum(r01r, red);
  r01i = block_sum(r01i, red);
  if (threadIdx.x == 0) {
    double tr = r00 + r11;
    double inv = tr > 0.0 ? 1.0 / tr : 0.0;
    rho[b * 4 + 0] = mk(r00 * inv, 0.0);
    rho[b * 4 + 1] = mk(r01r * inv, r01i * inv);
    rho[b * 4 + 2] = mk(r01r * inv, -r01i * inv);
    rho[b * 4 + 3] = mk(r11 * inv, 0.0);
  }
}

__global__ void k_cost_grad(const zd* rho, const double* p, const zd* h, int64_t batch, double* cost, zd* grad) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  zd g[16];
  double c = cost_grad(rho + 4 * b, p[b], h + 16 * b, grad ? g : nullptr);
  cost[b] = c;
  if (grad)
    for (int i = 0; i < 16; ++i) grad[b * 16 + i] = g[i];
}

// Gradient steps H <- H - alpha Gamma with a backtracking step size: each
// step tries alpha (lr at the first step, then twice the previous step's
// accepted or last tried value, at most kMaxStep), halving it until the
// sufficient-decrease (Armijo) condition E(H - alpha Gamma) <= E(H) -
// kArmijo alpha ||Gamma||_F^2 holds; below kMinStep the step is skipped.
// trace[s][b] = cost after step s.
constexpr double kArmijo = 1e-4, kMinStep = 1e-12, kMaxStep = 1e4;

__global__ void k_descend(const zd* rho, const double* p, int64_t batch, int steps, double lr, zd* h, double* trace) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  zd hh[16], g[16], hn[16], r[4];
  for (int i = 0; i < 16; ++i) hh[i] = h[b * 16 + i];
  for (int i = 0; i < 4; ++i) r[i] = rho[b * 4 + i];
  const double pb = p[b];
  double e = cost_grad(r, pb, hh, g);
  double alpha = lr;
  for (int s = 0; s < steps; ++s) {
    double gg = 0.0;
    for (int i = 0; i < 16; ++i) gg += norm2(g[i]);
    bool moved = false;
    for (;;) {
      for (int i = 0; i < 16; ++i) hn[i] = hh[i] - alpha * g[i];
      const double en = cost_grad(r, pb, hn, nullptr);
      if (en <= e - kArmijo * alpha * gg) {
        moved = true;
        break;
      }
      alpha *= 0.5;
      if (alpha < kMinStep) break;
    }
    if (moved) {
      for (int i = 0; i < 16; ++i) hh[i] = hn[i];
      e = cost_grad(r, pb, hh, g);
    }
    if (trace) trace[(int64_t)s * batch + b] = e;
    alpha = fmin(2.0 * alpha, kMaxStep);
  }
  for (int i = 0; i < 16; ++i) h[b * 16 + i] = hh[i];
}

}  // namespace adj
}  // namespace lemps
