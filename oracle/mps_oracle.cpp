// Oracle (test infrastructure: only the tests, the smoke check and the
// benchmark's CPU-baseline leg load it; the GPU library shares no code with
// it).  Plain C++17, FP64: Monte-Carlo MPS trajectories of a noisy circuit
// with the locally entanglement-optimal unraveling, one trajectory per OpenMP
// task.
//
// It restates, step by step, the Python oracle (oracle/trajectories.py,
// oracle/unravel.py, oracle/philox.py), with its own small dense linear
// algebra:
//  - cyclic complex Jacobi for the Hermitian (and real symmetric) eigenproblems
//    of size <= 8;
//  - one-sided (Hestenes) Jacobi for every SVD: the induced decomposition of
//    Sec. IV.B, the two-site split of Sec. II (Eq. MPS_truncation_error) and
//    the half-chain Schmidt values.  It resolves a singular value to about
//    eps * sigma_max, as a bidiagonal SVD does, so squared values far below
//    eps * sigma_max^2 are not mistaken for kept weight;
//  - Householder QR for the centre moves;
//  - the Takagi factorization of App. F.2 Step 1 from the real symmetric
//    embedding [[Re tau, Im tau], [Im tau, -Re tau]], whose eigenpairs for the
//    positive eigenvalues s are [Re u; Im u] with tau conj(u) = s u; zero
//    Takagi values get an orthonormal completion (their unitary freedom is
//    fixed by rule R3 below in any case).
// The canonical rules R1-R6 of the unraveling (effective-state phases,
// reference Gram-Schmidt per block of equal Takagi values or Re M
// eigenvalues, rank and zero tolerances, the separability test, the pure
// target) are those of the Python oracle, so both give the same branch
// sequences and agree to rounding.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// ---- Philox4x64-10 (Salmon et al., SC'11; the published multipliers and
// Weyl increments), counter (trajectory, global gate, slot, 0), key (seed,
// "LEMPSTRA"); u = top 53 bits of the first word x 2^-53 (Alg. 1, "sample").
constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ULL, kM1 = 0xCA5A826395121157ULL;
constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ULL, kW1 = 0xBB67AE8584CAA73BULL;
constexpr uint64_t kDomain = 0x4C454D5053545241ULL;

void philox(uint64_t c[4], uint64_t k0, uint64_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kW0;
      k1 += kW1;
    }
    const unsigned __int128 p0 = (unsigned __int128)kM0 * c[0];
    const unsigned __int128 p1 = (unsigned __int128)kM1 * c[2];
    const uint64_t n0 = (uint64_t)(p1 >> 64) ^ c[1] ^ k0, n1 = (uint64_t)p1;
    const uint64_t n2 = (uint64_t)(p0 >> 64) ^ c[3] ^ k1, n3 = (uint64_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
}

double uniform(uint64_t seed, uint64_t traj, uint64_t gate, uint64_t slot) {
  uint64_t c[4] = {traj, gate, slot, 0};
  philox(c, seed, kDomain);
  return (double)(c[0] >> 11) * (1.0 / 9007199254740992.0);
}

// ---- dense complex matrices, column-major ------------------------------------
struct Mat {
  int r = 0, c = 0;
  std::vector<cd> a;
  Mat() = default;
  Mat(int rows, int cols) : r(rows), c(cols), a((size_t)rows * cols) {}
  cd& operator()(int i, int j) { return a[(size_t)j * r + i]; }
  cd operator()(int i, int j) const { return a[(size_t)j * r + i]; }
  static Mat eye(int n) {
    Mat m(n, n);
    for (int i = 0; i < n; ++i) m(i, i) = 1.0;
    return m;
  }
};

Mat mul(const Mat& x, const Mat& y) {
  Mat z(x.r, y.c);
  for (int j = 0; j < y.c; ++j)
    for (int k = 0; k < x.c; ++k) {
      const cd b = y(k, j);
      if (b == 0.0) continue;
      for (int i = 0; i < x.r; ++i) z(i, j) += x(i, k) * b;
    }
  return z;
}

Mat adj(const Mat& x) {
  Mat z(x.c, x.r);
  for (int i = 0; i < x.r; ++i)
    for (int j = 0; j < x.c; ++j) z(j, i) = std::conj(x(i, j));
  return z;
}

Mat cols(const Mat& x, const std::vector<int>& idx) {
  Mat z(x.r, (int)idx.size());
  for (size_t j = 0; j < idx.size(); ++j)
    for (int i = 0; i < x.r; ++i) z(i, (int)j) = x(i, idx[j]);
  return z;
}

void set_cols(Mat& x, const std::vector<int>& idx, const Mat& v) {
  for (size_t j = 0; j < idx.size(); ++j)
    for (int i = 0; i < x.r; ++i) x(i, idx[j]) = v(i, (int)j);
}

// Hermitian eigenproblem by cyclic Jacobi: each rotation first makes a_pq
// real by a phase on index q, then zeroes it with the real rotation whose
// tangent t is the smaller root of t^2 + 2 theta t - 1 = 0, theta = (a_qq -
// a_pp) / (2 |a_pq|).  Eigenvalues descending, eigenvectors in V's columns.
void heev_jacobi(Mat A, std::vector<double>& w, Mat& V) {
  const int n = A.r;
  V = Mat::eye(n);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) (i == j ? diag : off) += std::norm(A(i, j));
    if (off == 0.0 || off <= 1e-34 * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double b = std::abs(A(p, q));
        if (b == 0.0 || b <= 1e-300) continue;
        const cd ph = std::conj(A(p, q)) / b;   // e^{-i arg a_pq}
        for (int k = 0; k < n; ++k) {
          A(k, q) *= ph;
          A(q, k) *= std::conj(ph);
          V(k, q) *= ph;
        }
        const double app = A(p, p).real(), aqq = A(q, q).real();
        const double th = (aqq - app) / (2.0 * b);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const cd x = A(k, p), y = A(k, q);
          A(k, p) = c * x - s * y;
          A(k, q) = s * x + c * y;
        }
        for (int k = 0; k < n; ++k) {
          const cd x = A(p, k), y = A(q, k);
          A(p, k) = c * x - s * y;
          A(q, k) = s * x + c * y;
        }
        A(p, q) = A(q, p) = 0.0;
        A(p, p) = A(p, p).real();
        A(q, q) = A(q, q).real();
        for (int k = 0; k < n; ++k) {
          const cd x = V(k, p), y = V(k, q);
          V(k, p) = c * x - s * y;
          V(k, q) = s * x + c * y;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return A(x, x).real() > A(y, y).real(); });
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A(ord[i], ord[i]).real();
  V = cols(V, ord);
}

// One-sided Jacobi SVD of W (m x nc): rotates column pairs until all are
// mutually orthogonal; on return W = A V has orthogonal columns of norms s
// (descending, columns permuted to match) and V (nc x nc) is unitary.  Each
// rotation makes w_p^H w_q real by a phase on column q, then applies the real
// rotation with tangent the smaller root of t^2 + 2 zeta t - 1 = 0, zeta =
// (|w_q|^2 - |w_p|^2) / (2 |w_p^H w_q|).
void svd_jacobi(Mat& W, Mat* V, std::vector<double>& s) {
  const int m = W.r, nc = W.c;
  if (V) *V = Mat::eye(nc);
  std::vector<double> nrm(nc);
  for (int sweep = 0; sweep < 80; ++sweep) {
    for (int j = 0; j < nc; ++j) {
      double t = 0.0;
      const cd* w = &W.a[(size_t)j * m];
      for (int i = 0; i < m; ++i) t += std::norm(w[i]);
      nrm[j] = t;
    }
    bool rotated = false;
    for (int p = 0; p < nc - 1; ++p)
      for (int q = p + 1; q < nc; ++q) {
        const double al = nrm[p], be = nrm[q];
        if (!(al > 0.0) || !(be > 0.0)) continue;   // a column at rounding level
        cd* wp = &W.a[(size_t)p * m];
        cd* wq = &W.a[(size_t)q * m];
        cd g = 0.0;
        for (int i = 0; i < m; ++i) g += std::conj(wp[i]) * wq[i];
        const double ga = std::abs(g);
        if (ga == 0.0 || ga <= 1e-15 * std::sqrt(al * be)) continue;
        rotated = true;
        const cd ph = std::conj(g) / ga;
        const double ze = (be - al) / (2.0 * ga);
        const double t = (ze >= 0.0 ? 1.0 : -1.0) / (std::fabs(ze) + std::sqrt(1.0 + ze * ze));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < m; ++i) {
          const cd x = wp[i], y = wq[i] * ph;
          wp[i] = c * x - sn * y;
          wq[i] = sn * x + c * y;
        }
        // running squared norms (recomputed each sweep); a rank-deficient pair
        // leaves one at rounding level, kept non-negative
        nrm[p] = std::max(0.0, al - t * ga);
        nrm[q] = std::max(0.0, be + t * ga);
        if (V) {
          cd* vp = &V->a[(size_t)p * nc];
          cd* vq = &V->a[(size_t)q * nc];
          for (int i = 0; i < nc; ++i) {
            const cd x = vp[i], y = vq[i] * ph;
            vp[i] = c * x - sn * y;
            vq[i] = sn * x + c * y;
          }
        }
      }
    if (!rotated) break;
  }
  s.resize(nc);
  for (int j = 0; j < nc; ++j) {
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += std::norm(W(i, j));
    s[j] = std::sqrt(t);
  }
  std::vector<int> ord(nc);
  for (int i = 0; i < nc; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return s[x] > s[y]; });
  std::vector<double> so(nc);
  for (int i = 0; i < nc; ++i) so[i] = s[ord[i]];
  s = so;
  W = cols(W, ord);
  if (V) *V = cols(*V, ord);
}

// Householder QR of A (m x n): Q (m x k) with orthonormal columns, R (k x n)
// upper triangular, k = min(m, n).
void qr_householder(Mat A, Mat& Q, Mat& R) {
  const int m = A.r, n = A.c, k = std::min(m, n);
  std::vector<std::vector<cd>> vs(k);
  std::vector<double> vn(k, 0.0);
  for (int j = 0; j < k; ++j) {
    double nx = 0.0;
    for (int i = j; i < m; ++i) nx += std::norm(A(i, j));
    nx = std::sqrt(nx);
    std::vector<cd> v(m - j);
    if (nx == 0.0) {
      vs[j] = v;
      continue;
    }
    const cd x0 = A(j, j);
    const cd alpha = (std::abs(x0) > 0.0 ? -(x0 / std::abs(x0)) : cd(-1.0)) * nx;
    for (int i = j; i < m; ++i) v[i - j] = A(i, j);
    v[0] -= alpha;
    double vv = 0.0;
    for (const cd& x : v) vv += std::norm(x);
    for (int c = j; c < n; ++c) {
      cd d = 0.0;
      for (int i = j; i < m; ++i) d += std::conj(v[i - j]) * A(i, c);
      d *= 2.0 / vv;
      for (int i = j; i < m; ++i) A(i, c) -= d * v[i - j];
    }
    vs[j] = v;
    vn[j] = vv;
  }
  R = Mat(k, n);
  for (int c = 0; c < n; ++c)
    for (int i = 0; i <= std::min(c, k - 1); ++i) R(i, c) = A(i, c);
  Q = Mat(m, k);
  for (int i = 0; i < k; ++i) Q(i, i) = 1.0;
  for (int j = k - 1; j >= 0; --j) {
    if (vn[j] == 0.0) continue;
    const std::vector<cd>& v = vs[j];
    for (int c = 0; c < k; ++c) {
      cd d = 0.0;
      for (int i = j; i < m; ++i) d += std::conj(v[i - j]) * Q(i, c);
      d *= 2.0 / vn[j];
      for (int i = j; i < m; ++i) Q(i, c) -= d * v[i - j];
    }
  }
}

// ---- the locally entanglement-optimal unraveling (Sec. IV.B, App. E-F) -------
constexpr double kRankTol = 1e-12, kPureTol = 1e-12, kDegTol = 1e-9, kZeroTol = 1e-10;
const cd kI(0.0, 1.0);
const cd kRef2[2] = {cd(0.8, 0.0), cd(0.36, 0.48)};
const cd kRef4[8][4] = {{cd(0.47, 0), cd(0.31, 0.22), cd(-0.18, 0.53), cd(0.26, -0.52)},
                        {cd(0.12, 0.44), cd(0.58, 0), cd(-0.37, -0.21), cd(-0.33, 0.38)},
                        {cd(-0.29, 0.35), cd(0.14, -0.41), cd(0.62, 0), cd(0.23, 0.41)},
                        {cd(0.36, -0.27), cd(-0.45, 0.16), cd(0.28, 0.33), cd(0.61, 0)},
                        {cd(0.5, 0), cd(0, -0.5), cd(0.5, 0), cd(0, 0.5)},
                        {cd(0, 0.5), cd(0.5, 0), cd(-0.5, 0), cd(0.5, 0)},
                        {cd(1, 0), cd(0, 0), cd(0, 0), cd(0, 0)},
                        {cd(0, 0), cd(0, 0), cd(0, 0), cd(1, 0)}};

// (Y (x) Y) conj(v), column by column (Eq. spin-flip-vector); Y (x) Y is the
// real anti-diagonal (-1, 1, 1, -1).
Mat spin_flip(const Mat& v) {
  Mat z(4, v.c);
  for (int j = 0; j < v.c; ++j) {
    z(0, j) = -std::conj(v(3, j));
    z(1, j) = std::conj(v(2, j));
    z(2, j) = std::conj(v(1, j));
    z(3, j) = -std::conj(v(0, j));
  }
  return z;
}

// Groups of consecutive indices of a descending array whose neighbours differ
// by at most tol * max|vals|.
std::vector<std::vector<int>> clusters(const std::vector<double>& vals, double tol) {
  double scale = 1e-300;
  for (double v : vals) scale = std::max(scale, std::fabs(v));
  std::vector<std::vector<int>> g;
  for (int i = 0; i < (int)vals.size(); ++i) {
    if (!g.empty() && vals[g.back().back()] - vals[i] <= tol * scale) g.back().push_back(i);
    else g.push_back({i});
  }
  return g;
}

// Rule R2: B (m x m; real orthogonal, or unitary when complex_freedom) such
// that members B is the canonical basis of the block: Gram-Schmidt on the
// gradients Re(A^dagger r) (or A^dagger r) of the reference vectors r, then a
// deterministic completion for members of rank < m.
Mat reference_basis(const Mat& members, bool complex_freedom) {
  const int m = members.c;
  double scale = 0.0;
  for (const cd& x : members.a) scale += std::norm(x);
  scale = std::max(std::sqrt(scale), 1e-300);
  std::vector<std::vector<cd>> basis;
  auto orth = [&](std::vector<cd>& g) {
    for (const auto& b : basis) {
      cd d = 0.0;
      for (int i = 0; i < m; ++i) d += std::conj(b[i]) * g[i];
      for (int i = 0; i < m; ++i) g[i] -= d * b[i];
    }
    double nr = 0.0;
    for (int i = 0; i < m; ++i) nr += std::norm(g[i]);
    return std::sqrt(nr);
  };
  for (int r = 0; r < 8 && (int)basis.size() < m; ++r) {
    double rn = 0.0;
    for (int i = 0; i < 4; ++i) rn += std::norm(kRef4[r][i]);
    rn = std::sqrt(rn);
    std::vector<cd> g(m);
    for (int j = 0; j < m; ++j) {
      cd d = 0.0;
      for (int i = 0; i < 4; ++i) d += std::conj(members(i, j)) * kRef4[r][i];
      g[j] = complex_freedom ? d : cd(d.real(), 0.0);
    }
    const double nr = orth(g);
    if (nr > 1e-8 * scale * rn) {
      for (auto& x : g) x /= nr;
      basis.push_back(g);
    }
  }
  for (int k = 0; k < m && (int)basis.size() < m; ++k) {
    std::vector<cd> g(m);
    g[k] = 1.0;
    const double nr = orth(g);
    if (nr > 1e-6) {
      for (auto& x : g) x /= nr;
      basis.push_back(g);
    }
  }
  Mat out(m, m);
  for (int j = 0; j < (int)basis.size(); ++j)
    for (int i = 0; i < m; ++i) out(i, j) = complex_freedom ? basis[j][i] : cd(basis[j][i].real(), 0.0);
  return out;
}

// Takagi factorization tau = U diag(s) U^T of a complex symmetric r x r
// matrix (App. F.2, Step 1), s descending; see the file header.
void takagi(const Mat& tau, Mat& U, std::vector<double>& s) {
  const int r = tau.r;
  Mat M(2 * r, 2 * r);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) {
      const double x = tau(i, j).real(), y = tau(i, j).imag();
      M(i, j) = x;
      M(i, r + j) = y;
      M(r + i, j) = y;
      M(r + i, r + j) = -x;
    }
  std::vector<double> w;
  Mat Vm;
  heev_jacobi(M, w, Vm);
  const double smax = std::max(w[0], 0.0);
  U = Mat(r, r);
  s.assign(r, 0.0);
  int nz = 0;
  for (int k = 0; k < r; ++k) {
    if (!(w[k] > kZeroTol * smax) || smax <= 0.0) break;
    double nr = 0.0;
    for (int i = 0; i < r; ++i) {
      U(i, nz) = cd(Vm(i, k).real(), Vm(r + i, k).real());
      nr += std::norm(U(i, nz));
    }
    nr = std::sqrt(nr);
    for (int i = 0; i < r; ++i) U(i, nz) /= nr;
    s[nz++] = w[k];
  }
  // zero Takagi values: an orthonormal completion of the columns found
  for (int e = 0; e < r && nz < r; ++e) {
    std::vector<cd> g(r);
    g[e] = 1.0;
    for (int j = 0; j < nz; ++j) {
      cd d = 0.0;
      for (int i = 0; i < r; ++i) d += std::conj(U(i, j)) * g[i];
      for (int i = 0; i < r; ++i) g[i] -= d * U(i, j);
    }
    double nr = 0.0;
    for (int i = 0; i < r; ++i) nr += std::norm(g[i]);
    nr = std::sqrt(nr);
    if (nr > 1e-6) {
      for (int i = 0; i < r; ++i) U(i, nz) = g[i] / nr;
      ++nz;
    }
  }
}

// Phases theta with sum_j exp(2 i theta_j) lam_j = 0 for a separable state
// (Eq. separating_angles_condition), from the trapezoid of App. F.2 with
// Heron's area in Kahan's arrangement; equal values use the square.
void separable_angles(const double lam[4], double th[4]) {
  const double l1 = lam[0], l2 = lam[1], l3 = lam[2], l4 = lam[3];
  if (l1 - l4 <= kDegTol * std::max(l1, 1e-300)) {
    th[0] = 0.0; th[1] = kPi / 4; th[2] = kPi / 2; th[3] = 3 * kPi / 4;
    return;
  }
  const double d = l1 - l4;
  double v[3] = {d, l2, l3};
  std::sort(v, v + 3, [](double x, double y) { return x > y; });
  const double a = v[0], b = v[1], c = v[2];
  const double prod = (a + (b + c)) * (c - (a - b)) * (c + (a - b)) * (a + (b - c));
  const double area = 0.25 * std::sqrt(std::max(0.0, prod));
  const double h = 2.0 * area / d;
  const double a2 = l2 > 0.0 ? kPi - std::asin(std::min(1.0, h / l2)) : 0.0;
  double a3 = 0.0;
  if (l3 > 0.0) {
    const double b3 = std::asin(std::min(1.0, h / l3));
    a3 = (l2 * std::cos(a2) + d > 0.0) ? kPi + b3 : -b3;
  }
  th[0] = 0.0; th[1] = 0.5 * a2; th[2] = 0.5 * a3; th[3] = 0.5 * kPi;
}

Mat h4() {
  static const double s[4][4] = {{1, 1, 1, 1}, {1, 1, -1, -1}, {1, -1, 1, -1}, {1, -1, -1, 1}};
  Mat m(4, 4);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) m(i, j) = 0.5 * s[i][j];
  return m;
}

// Wootters' optimal decomposition z = v T of rho = v v^dagger (App. F.2);
// columns of v beyond rank are zero.  Returns T.
Mat wootters(const Mat& v, int rank) {
  const Mat vt = spin_flip(v);
  const Mat tau = mul(adj(v), vt);
  Mat ut = Mat::eye(4);
  double sig[4] = {0, 0, 0, 0};
  if (rank > 0) {
    Mat tr(rank, rank);
    for (int i = 0; i < rank; ++i)
      for (int j = 0; j < rank; ++j) tr(i, j) = tau(i, j);
    Mat ur;
    std::vector<double> sr;
    takagi(tr, ur, sr);
    for (int i = 0; i < rank; ++i) {
      sig[i] = sr[i];
      for (int j = 0; j < rank; ++j) ut(i, j) = ur(i, j);
    }
  }
  Mat x = mul(v, ut);
  if (rank > 0) {   // rule R3 on the Takagi vectors
    const double s1 = sig[0];
    std::vector<int> zero, nonzero;
    for (int k = 0; k < rank; ++k) (sig[k] <= kZeroTol * s1 ? zero : nonzero).push_back(k);
    if (!nonzero.empty()) {
      std::vector<double> sv;
      for (int k : nonzero) sv.push_back(sig[k]);
      for (const auto& g : clusters(sv, kDegTol)) {
        std::vector<int> idx;
        for (int i : g) idx.push_back(nonzero[i]);
        const Mat rot = reference_basis(cols(x, idx), false);
        set_cols(x, idx, mul(cols(x, idx), rot));
        set_cols(ut, idx, mul(cols(ut, idx), rot));
      }
    }
    if (!zero.empty()) {
      const Mat rot = reference_basis(cols(x, zero), true);
      set_cols(x, zero, mul(cols(x, zero), rot));
      set_cols(ut, zero, mul(cols(ut, zero), rot));
      for (int k : zero) sig[k] = 0.0;
    }
  }
  const double c = sig[0] - sig[1] - sig[2] - sig[3];
  Mat U2 = Mat::eye(4);
  U2(1, 1) = U2(2, 2) = U2(3, 3) = kI;
  if (c > 0.0) {   // entangled: Steps 2 and 3
    const Mat y = mul(x, U2);
    const Mat yt = spin_flip(y);
    const Mat m1 = mul(adj(y), yt), m2 = mul(adj(y), y);
    Mat mr(4, 4);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const double a = (m1(i, j) - c * m2(i, j)).real(), b = (m1(j, i) - c * m2(j, i)).real();
        mr(i, j) = 0.5 * (a + b);
      }
    std::vector<double> d;
    Mat q;
    heev_jacobi(mr, d, q);
    for (auto& e : q.a) e = cd(e.real(), 0.0);
    for (const auto& g : clusters(d, kDegTol)) {
      const Mat qg = cols(q, g);
      set_cols(q, g, mul(qg, reference_basis(mul(y, qg), false)));
    }
    return mul(mul(mul(ut, U2), q), h4());
  }
  double th[4];
  separable_angles(sig, th);
  Mat ph(4, 4);
  for (int k = 0; k < 4; ++k) ph(k, k) = std::exp(kI * th[k]);
  return mul(mul(ut, ph), h4());
}

// Locally entanglement-optimal Kraus set for a target with reduced state
// rho_a (Thm. 2, Sec. IV.B.4): kout[k] = sum_j W[j, k] kraus[j] with W =
// V_phi (T (+) I), over max(r, 4) operators (zero operators pad r < 4).
// Kraus operators are 2x2 column-major Mats.
std::vector<Mat> optimal_unraveling(const Mat& rho_a, const std::vector<Mat>& kraus, Mat* Wout = nullptr) {
  const int r = (int)kraus.size(), rp = std::max(r, 4);
  std::vector<Mat> kpad(rp, Mat(2, 2));
  for (int j = 0; j < r; ++j) kpad[j] = kraus[j];
  Mat h(2, 2);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) h(i, j) = 0.5 * (rho_a(i, j) + std::conj(rho_a(j, i)));
  std::vector<double> wr;
  Mat ur;
  heev_jacobi(h, wr, ur);
  // rule R6: a pure target leaves the Kraus set unchanged
  if (wr[1] <= kPureTol * std::max(wr[0] + wr[1], 1e-300)) {
    if (Wout) *Wout = Mat::eye(rp);
    return kpad;
  }
  // effective state (Eqs. schmidt_1_n-1, effective_two_qubit_state), rule R1
  const double tr = rho_a(0, 0).real() + rho_a(1, 1).real();
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) h(i, j) /= tr;
  heev_jacobi(h, wr, ur);
  for (double& x : wr) x = std::max(x, 0.0);
  if (wr[0] - wr[1] <= kDegTol * std::max(wr[0], 1e-300)) {
    ur = Mat::eye(2);
  } else {
    for (int k = 0; k < 2; ++k) {
      const cd ov = std::conj(kRef2[0]) * ur(0, k) + std::conj(kRef2[1]) * ur(1, k);
      const cd f = std::conj(ov) / std::abs(ov);
      ur(0, k) *= f;
      ur(1, k) *= f;
    }
  }
  cd psi[4] = {0, 0, 0, 0};   // index 2 t + k: target t, effective partner k
  for (int k = 0; k < 2; ++k)
    for (int t = 0; t < 2; ++t) psi[2 * t + k] += std::sqrt(wr[k]) * ur(t, k);
  // induced decomposition phi = sum_j (K_j (x) I)|psi><j| (Eq. Kraus_to_ensemble)
  Mat phi(4, rp);
  for (int j = 0; j < rp; ++j)
    for (int a = 0; a < 2; ++a)
      for (int k = 0; k < 2; ++k) {
        cd acc = 0.0;
        for (int t = 0; t < 2; ++t) acc += kpad[j](a, t) * psi[2 * t + k];
        phi(2 * a + k, j) = acc;
      }
  // v = phi V_phi (Eq. v_to_phi) from its SVD; rule R4 for the rank
  Mat W = phi, Vphi;
  std::vector<double> s;
  svd_jacobi(W, &Vphi, s);
  int rank = 0;
  for (int k = 0; k < std::min(4, rp); ++k)
    if (s[k] > kRankTol * s[0]) ++rank;
  Mat v(4, 4);
  for (int j = 0; j < rank; ++j)
    for (int i = 0; i < 4; ++i) v(i, j) = W(i, j);
  const Mat t = wootters(v, rank);
  Mat tt = Mat::eye(rp);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) tt(i, j) = t(i, j);
  const Mat Wm = mul(Vphi, tt);
  std::vector<Mat> kout(rp, Mat(2, 2));
  for (int k = 0; k < rp; ++k)
    for (int j = 0; j < rp; ++j) {
      const cd w = Wm(j, k);
      if (w == 0.0) continue;
      for (int e = 0; e < 4; ++e) kout[k].a[e] += w * kpad[j].a[e];
    }
  if (Wout) *Wout = Wm;
  return kout;
}

// ---- MPS in mixed-canonical form (Sec. II, Eq. def_MPS) ------------------------
// Site k: a row-major (d_k, 2, d_{k+1}) block, entry (a, s, b) at (2a + s) d_{k+1} + b.
struct Site {
  int dl = 1, dr = 1;
  std::vector<cd> t;
};

struct Circuit {
  int n = 0;
  std::vector<int> gate_begin;           // [layers + 1]
  std::vector<int> left;                 // [gates]
  std::vector<cd> gates;                 // [gates][4][4] row-major
  std::vector<int> kraus_begin;          // [layers + 1] operator index
  std::vector<std::vector<Mat>> kraus;   // per layer
  std::vector<std::vector<Mat>> haar;    // per layer: the Bell state's optimal set
  std::vector<double> coin_p;            // [layers]
  int layers() const { return (int)coin_p.size(); }
};

enum Mode { kOptimal = 0, kGiven = 1, kHaarOptimal = 2 };

struct Trajectory {
  std::vector<Site> a;
  int center = 0;
  int64_t gglob = 0;
  double eps_tot = 0.0;
  int layer = 0;
  std::vector<int32_t> branch;
  // smallest relative gap (w_keep - w_keep+1) / w_1 of the squared Schmidt
  // values at a truncating cut (1 when no cut truncated)
  double min_gap = 1.0;
  // outputs
  std::vector<double> z, zz;
  double s_half = 0.0, eps_bound = 0.0;
};

void init_state(Trajectory& T, int n) {
  T.a.assign(n, Site());
  for (auto& s : T.a) s.t = {cd(1.0), cd(0.0)};
  T.center = 0;
}

// Row-major (rows x cols) block <-> Mat.
Mat from_rows(const std::vector<cd>& t, int rows, int c) {
  Mat m(rows, c);
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < c; ++j) m(i, j) = t[(size_t)i * c + j];
  return m;
}
std::vector<cd> to_rows(const Mat& m) {
  std::vector<cd> t((size_t)m.r * m.c);
  for (int i = 0; i < m.r; ++i)
    for (int j = 0; j < m.c; ++j) t[(size_t)i * m.c + j] = m(i, j);
  return t;
}

void move_center(Trajectory& T, int target) {
  while (T.center < target) {   // A_k = Q R as (2 d_l) x d_r; R into A_{k+1}
    const int k = T.center;
    Site& A = T.a[k];
    Site& B = T.a[k + 1];
    Mat Q, R;
    qr_householder(from_rows(A.t, 2 * A.dl, A.dr), Q, R);
    A.t = to_rows(Q);
    A.dr = Q.c;
    const Mat nb = mul(R, from_rows(B.t, B.dl, 2 * B.dr));
    B.t = to_rows(nb);
    B.dl = nb.r;
    ++T.center;
  }
  while (T.center > target) {   // A_k^T = Q R as (2 d_r) x d_l; A_k = Q^T, R^T into A_{k-1}
    const int k = T.center;
    Site& A = T.a[k];
    Site& P = T.a[k - 1];
    const Mat Ak = from_rows(A.t, A.dl, 2 * A.dr);
    Mat At(Ak.c, Ak.r);
    for (int i = 0; i < Ak.r; ++i)
      for (int j = 0; j < Ak.c; ++j) At(j, i) = Ak(i, j);
    Mat Q, R;
    qr_householder(At, Q, R);
    Mat Qt(Q.c, Q.r);
    for (int i = 0; i < Q.r; ++i)
      for (int j = 0; j < Q.c; ++j) Qt(j, i) = Q(i, j);
    A.t = to_rows(Qt);
    A.dl = Qt.r;
    Mat Rt(R.c, R.r);
    for (int i = 0; i < R.r; ++i)
      for (int j = 0; j < R.c; ++j) Rt(j, i) = R(i, j);
    const Mat np = mul(from_rows(P.t, 2 * P.dl, P.dr), Rt);
    P.t = to_rows(np);
    P.dr = np.c;
    --T.center;
  }
}

// Two-site tensor of (q, q+1) as a (2 d_l) x (2 d_r) row-major block, entry
// (2a + s, t d_r + b), after moving the centre onto the pair; the gate (4x4
// on index 2s + t) applied when given.
std::vector<cd> pair_tensor(Trajectory& T, int q, const cd* gate, int& dl, int& dr) {
  if (T.center < q) move_center(T, q);
  else if (T.center > q + 1) move_center(T, q + 1);
  const Site& A = T.a[q];
  const Site& B = T.a[q + 1];
  dl = A.dl;
  dr = B.dr;
  const int dm = A.dr, m = 2 * dl, nn = 2 * dr;
  std::vector<cd> th((size_t)m * nn);
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < dm; ++k) {
      const cd x = A.t[(size_t)i * dm + k];
      if (x == 0.0) continue;
      const cd* b = &B.t[(size_t)k * nn];
      cd* o = &th[(size_t)i * nn];
      for (int j = 0; j < nn; ++j) o[j] += x * b[j];
    }
  if (gate) {
    for (int a = 0; a < dl; ++a)
      for (int b = 0; b < dr; ++b) {
        cd v[4], w[4];
        for (int s = 0; s < 2; ++s)
          for (int t = 0; t < 2; ++t) v[2 * s + t] = th[(size_t)(2 * a + s) * nn + t * dr + b];
        for (int u = 0; u < 4; ++u) {
          w[u] = 0.0;
          for (int e = 0; e < 4; ++e) w[u] += gate[u * 4 + e] * v[e];
        }
        for (int s = 0; s < 2; ++s)
          for (int t = 0; t < 2; ++t) th[(size_t)(2 * a + s) * nn + t * dr + b] = w[2 * s + t];
      }
  }
  return th;
}

// SVD split of the pair (Eq. MPS_truncation_error): keep chi' = max(1,
// min(cap, #{s_k^2 > cutoff * sum s^2})) values, renormalize, centre on q+1;
// returns the discarded weight.
double split(Trajectory& T, int q, const std::vector<cd>& th, int dl, int dr, int cap, double cutoff) {
  const int m = 2 * dl, nn = 2 * dr;
  const Mat Th = from_rows(th, m, nn);
  std::vector<double> s;
  Mat Ul, Bk;   // kept left vectors (m x keep), kept rows s_k v_k^H (keep x nn)
  int keep = 0;
  double tot = 0.0, kept = 0.0;
  auto decide = [&]() {
    for (double x : s) tot += x * x;
    int cnt = 0;
    for (double x : s)
      if (x * x > cutoff * tot) ++cnt;
    keep = std::max(1, std::min(cap, cnt));
    for (int k = 0; k < keep; ++k) kept += s[k] * s[k];
  };
  if (nn <= m) {   // Jacobi on the columns of Theta: W = Theta V = U S
    Mat W = Th, V;
    svd_jacobi(W, &V, s);
    decide();
    Ul = Mat(m, keep);
    Bk = Mat(keep, nn);
    for (int k = 0; k < keep; ++k) {
      for (int i = 0; i < m; ++i) Ul(i, k) = W(i, k) / s[k];
      for (int j = 0; j < nn; ++j) Bk(k, j) = s[k] * std::conj(V(j, k));
    }
  } else {         // Jacobi on the columns of Theta^H: W = Theta^H U = V S
    Mat W = adj(Th), U;
    svd_jacobi(W, &U, s);
    decide();
    Ul = Mat(m, keep);
    Bk = Mat(keep, nn);
    for (int k = 0; k < keep; ++k) {
      for (int i = 0; i < m; ++i) Ul(i, k) = U(i, k);
      for (int j = 0; j < nn; ++j) Bk(k, j) = std::conj(W(j, k));
    }
  }
  double disc = 0.0;
  for (int k = keep; k < (int)s.size(); ++k) disc += s[k] * s[k];
  if (keep < (int)s.size())   // a truncating cut: its conditioning
    T.min_gap = std::min(T.min_gap, (s[keep - 1] * s[keep - 1] - s[keep] * s[keep]) / (s[0] * s[0]));
  const double eps = disc / tot;
  const double nrm = 1.0 / std::sqrt(kept);
  Site& A = T.a[q];
  Site& B = T.a[q + 1];
  A.dl = dl;
  A.dr = keep;
  A.t = to_rows(Ul);
  for (auto& x : Bk.a) x *= nrm;
  B.dl = keep;
  B.dr = dr;
  B.t = to_rows(Bk);
  T.center = q + 1;
  return eps;
}

int sample_index(const std::vector<double>& p, double u) {
  std::vector<double> cs(p.size());
  double acc = 0.0;
  for (size_t i = 0; i < p.size(); ++i) cs[i] = (acc += p[i]);
  const double thr = u * cs.back();
  for (size_t i = 0; i < cs.size(); ++i)
    if (thr < cs[i]) return (int)i;
  return (int)p.size() - 1;
}

// The noise on slot 0 (qubit q) or 1 (q+1) of a two-site tensor: reduced
// state, Kraus set, branch weights p_i = Tr(K_i rho K_i^dagger), sampled
// branch, and the renormalized operator applied (the channel unraveling
// subprocedure of Alg. 1).
int noise_site(std::vector<cd>& th, int dl, int dr, int slot, const Circuit& C, int layer, int mode, double u) {
  const int nn = 2 * dr;
  auto at = [&](int a, int s, int t, int b) -> cd& { return th[(size_t)(2 * a + s) * nn + t * dr + b]; };
  Mat rho(2, 2);
  for (int a = 0; a < dl; ++a)
    for (int x = 0; x < 2; ++x)
      for (int b = 0; b < dr; ++b) {
        cd v[2];
        for (int s = 0; s < 2; ++s) v[s] = slot == 0 ? at(a, s, x, b) : at(a, x, s, b);
        for (int s = 0; s < 2; ++s)
          for (int t = 0; t < 2; ++t) rho(s, t) += v[s] * std::conj(v[t]);
      }
  std::vector<Mat> kp;
  if (mode == kGiven) kp = C.kraus[layer];
  else if (mode == kHaarOptimal) kp = C.haar[layer];
  else kp = optimal_unraveling(rho, C.kraus[layer]);
  std::vector<double> p(kp.size());
  for (size_t i = 0; i < kp.size(); ++i) p[i] = mul(mul(kp[i], rho), adj(kp[i]))(0, 0).real() +
                                                 mul(mul(kp[i], rho), adj(kp[i]))(1, 1).real();
  const int i = sample_index(p, u);
  const double f = 1.0 / std::sqrt(p[i]);
  const Mat& op = kp[i];
  for (int a = 0; a < dl; ++a)
    for (int x = 0; x < 2; ++x)
      for (int b = 0; b < dr; ++b) {
        cd v[2], w[2];
        for (int s = 0; s < 2; ++s) v[s] = slot == 0 ? at(a, s, x, b) : at(a, x, s, b);
        for (int uu = 0; uu < 2; ++uu) w[uu] = f * (op(uu, 0) * v[0] + op(uu, 1) * v[1]);
        for (int s = 0; s < 2; ++s) (slot == 0 ? at(a, s, x, b) : at(a, x, s, b)) = w[s];
      }
  return i;
}

struct Batch {
  Circuit C;
  int64_t traj0 = 0;
  uint64_t seed = 0;
  int chi = 1, mode = kOptimal, layering = 0;
  double cutoff = 1e-20, eps_max = 4.0;
  std::vector<Trajectory> T;
};

// One layer of one trajectory (Sec. IV.A, layering "local": Trunc o
// N(x)N o U per gate; "global": all gates split without the cap, the noise on
// every gated pair, then a left-to-right truncating sweep).  The per-layer
// bound is 4 sqrt(2 sum eps) (Thm. 1, App. B).
void run_layer(const Batch& b, Trajectory& T, int64_t tid) {
  const Circuit& C = b.C;
  const int l = T.layer;
  const int uncapped = 1 << 30;
  double eps_layer = 0.0;
  const bool local = b.layering == 0;
  int dl, dr;
  if (!local)
    for (int g = C.gate_begin[l]; g < C.gate_begin[l + 1]; ++g) {
      const int q = C.left[g];
      std::vector<cd> th = pair_tensor(T, q, &C.gates[(size_t)g * 16], dl, dr);
      eps_layer += split(T, q, th, dl, dr, uncapped, b.cutoff);
    }
  for (int g = C.gate_begin[l]; g < C.gate_begin[l + 1]; ++g) {
    const int q = C.left[g];
    std::vector<cd> th = pair_tensor(T, q, local ? &C.gates[(size_t)g * 16] : nullptr, dl, dr);
    bool active = true;
    if (C.coin_p[l] < 1.0) active = uniform(b.seed, (uint64_t)tid, (uint64_t)T.gglob, 2) < C.coin_p[l];
    for (int slot = 0; slot < 2; ++slot) {
      if (!active) {
        T.branch.push_back(-1);
        continue;
      }
      const double u = uniform(b.seed, (uint64_t)tid, (uint64_t)T.gglob, (uint64_t)slot);
      T.branch.push_back(noise_site(th, dl, dr, slot, C, l, b.mode, u));
    }
    eps_layer += split(T, q, th, dl, dr, local ? b.chi : uncapped, b.cutoff);
    ++T.gglob;
  }
  if (!local)
    for (int k = 0; k + 1 < C.n; ++k) {
      std::vector<cd> th = pair_tensor(T, k, nullptr, dl, dr);
      eps_layer += split(T, k, th, dl, dr, b.chi, b.cutoff);
    }
  T.eps_tot += 4.0 * std::sqrt(2.0 * eps_layer);
  ++T.layer;
}

// <Z_i>, <Z_i Z_{i+1}> and the entropy of bond n/2 (nats) from the centre
// site as it sweeps left to right.
void observables(Trajectory& T, int n) {
  T.z.assign(n, 0.0);
  T.zz.assign(n - 1, 0.0);
  move_center(T, 0);
  for (int k = 0; k < n; ++k) {
    move_center(T, k);
    const Site& A = T.a[k];
    double z = 0.0;
    for (int a = 0; a < A.dl; ++a)
      for (int b = 0; b < A.dr; ++b)
        z += std::norm(A.t[(size_t)(2 * a) * A.dr + b]) - std::norm(A.t[(size_t)(2 * a + 1) * A.dr + b]);
    T.z[k] = z;
    if (k + 1 < n) {
      int dl, dr;
      const std::vector<cd> th = pair_tensor(T, k, nullptr, dl, dr);
      double w[2][2] = {{0, 0}, {0, 0}};
      for (int a = 0; a < dl; ++a)
        for (int s = 0; s < 2; ++s)
          for (int t = 0; t < 2; ++t)
            for (int b = 0; b < dr; ++b) w[s][t] += std::norm(th[(size_t)(2 * a + s) * 2 * dr + t * dr + b]);
      T.zz[k] = w[0][0] - w[0][1] - w[1][0] + w[1][1];
    }
    if (k == n / 2 - 1) {
      Mat W = from_rows(A.t, 2 * A.dl, A.dr);
      if (W.c > W.r) W = adj(W);
      std::vector<double> s;
      svd_jacobi(W, nullptr, s);
      double tot = 0.0;
      for (double x : s) tot += x * x;
      double S = 0.0;
      for (double x : s) {
        const double lam = x * x / tot;
        if (lam > 0.0) S -= lam * std::log(lam);
      }
      T.s_half = S;
    }
  }
}

std::vector<Mat> read_kraus(const double* p, int r) {
  std::vector<Mat> k(r, Mat(2, 2));
  for (int j = 0; j < r; ++j)
    for (int a = 0; a < 2; ++a)
      for (int c = 0; c < 2; ++c) k[j](a, c) = cd(p[((j * 2 + a) * 2 + c) * 2], p[((j * 2 + a) * 2 + c) * 2 + 1]);
  return k;
}

}  // namespace

// ---- C interface (for the Python test harness) --------------------------------
extern "C" {

// Counter-based uniform of the trajectory sampler (oracle/philox.py).
double oracle_uniform(uint64_t seed, uint64_t traj, uint64_t gate, uint64_t slot) {
  return uniform(seed, traj, gate, slot);
}

// Locally entanglement-optimal Kraus set (Thm. 2): rho [2][2] complex
// (interleaved re, im), kraus [r][2][2] complex; writes max(r, 4) operators
// to out and W [rp][rp] (row j, column k) to w_out.  Returns rp.
int oracle_optimal_unraveling(const double* rho, const double* kraus, int r, double* out, double* w_out) {
  Mat rh(2, 2);
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < 2; ++c) rh(a, c) = cd(rho[(a * 2 + c) * 2], rho[(a * 2 + c) * 2 + 1]);
  Mat W;
  const std::vector<Mat> k = optimal_unraveling(rh, read_kraus(kraus, r), &W);
  const int rp = (int)k.size();
  for (int j = 0; j < rp; ++j)
    for (int a = 0; a < 2; ++a)
      for (int c = 0; c < 2; ++c) {
        out[((j * 2 + a) * 2 + c) * 2] = k[j](a, c).real();
        out[((j * 2 + a) * 2 + c) * 2 + 1] = k[j](a, c).imag();
      }
  if (w_out)
    for (int j = 0; j < rp; ++j)
      for (int c = 0; c < rp; ++c) {
        w_out[(j * rp + c) * 2] = W(j, c).real();
        w_out[(j * rp + c) * 2 + 1] = W(j, c).imag();
      }
  return rp;
}

// A batch of trajectories traj0 .. traj0 + n_traj - 1 of one circuit.
// Circuit arrays: gate_begin [layers + 1] (gates of layer l are gate_begin[l]
// .. gate_begin[l+1]-1), left [gates], gates [gates][4][4] complex,
// kraus_begin [layers + 1] (operators of layer l), kraus [ops][2][2] complex,
// coin_p [layers].  mode: 0 optimal, 1 given, 2 Haar-optimal; layering: 0
// local, 1 global.  Returns NULL on bad arguments.
void* oracle_batch_create(int n, int layers, const int* gate_begin, const int* left, const double* gates,
                          const int* kraus_begin, const double* kraus, const double* coin_p, int64_t traj0,
                          int64_t n_traj, uint64_t seed, int chi_max, double cutoff, int mode, int layering,
                          double eps_max) {
  if (n < 2 || layers < 0 || n_traj < 0 || chi_max < 1 || mode < 0 || mode > 2 || layering < 0 || layering > 1)
    return nullptr;
  Batch* b = new Batch();
  Circuit& C = b->C;
  C.n = n;
  C.gate_begin.assign(gate_begin, gate_begin + layers + 1);
  const int ng = gate_begin[layers];
  C.left.assign(left, left + ng);
  C.gates.resize((size_t)ng * 16);
  for (size_t e = 0; e < C.gates.size(); ++e) C.gates[e] = cd(gates[2 * e], gates[2 * e + 1]);
  C.kraus_begin.assign(kraus_begin, kraus_begin + layers + 1);
  C.coin_p.assign(coin_p, coin_p + layers);
  Mat half(2, 2);
  half(0, 0) = half(1, 1) = 0.5;
  for (int l = 0; l < layers; ++l) {
    const int r = kraus_begin[l + 1] - kraus_begin[l];
    C.kraus.push_back(read_kraus(kraus + (size_t)kraus_begin[l] * 8, r));
    C.haar.push_back(mode == kHaarOptimal ? optimal_unraveling(half, C.kraus.back()) : std::vector<Mat>());
  }
  b->traj0 = traj0;
  b->seed = seed;
  b->chi = chi_max;
  b->cutoff = cutoff;
  b->mode = mode;
  b->layering = layering;
  b->eps_max = eps_max;
  b->T.resize((size_t)n_traj);
  for (auto& t : b->T) init_state(t, n);
  return b;
}

// Advance every trajectory through layers [l0, l1) (all must be at layer l0),
// n_threads OpenMP threads (<= 0: the runtime's default).  Returns 0, or -1 on
// bad arguments.
int oracle_batch_run(void* hb, int l0, int l1, int n_threads) {
  Batch* b = static_cast<Batch*>(hb);
  if (!b || l0 < 0 || l1 > b->C.layers() || l0 > l1) return -1;
  for (const auto& t : b->T)
    if (t.layer != l0) return -1;
  const int64_t nt = (int64_t)b->T.size();
#ifdef _OPENMP
  const int th = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(th)
#endif
  for (int64_t i = 0; i < nt; ++i)
    for (int l = l0; l < l1; ++l) run_layer(*b, b->T[(size_t)i], b->traj0 + i);
  (void)n_threads;
  return 0;
}

// Advance trajectories i0 .. i1-1 only (each at layer l0) through layers
// [l0, l1); the others stay where they are.  Returns 0, or -1 on bad arguments.
int oracle_batch_run_range(void* hb, int64_t i0, int64_t i1, int l0, int l1, int n_threads) {
  Batch* b = static_cast<Batch*>(hb);
  if (!b || i0 < 0 || i1 > (int64_t)b->T.size() || i0 > i1 || l0 < 0 || l1 > b->C.layers() || l0 > l1) return -1;
  for (int64_t i = i0; i < i1; ++i)
    if (b->T[(size_t)i].layer != l0) return -1;
#ifdef _OPENMP
  const int th = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(th)
#endif
  for (int64_t i = i0; i < i1; ++i)
    for (int l = l0; l < l1; ++l) run_layer(*b, b->T[(size_t)i], b->traj0 + i);
  (void)n_threads;
  return 0;
}

// Observables and the error bound of every trajectory: z [n_traj][n], zz
// [n_traj][n-1], s_half [n_traj], eps_bound [n_traj], branch [n_traj][2 *
// gates run], min_gap [n_traj] (the smallest relative gap of the squared
// Schmidt values at a truncating cut; 1 if none) (any output may be NULL).
// Every trajectory must be at the same layer (-1 otherwise).
int oracle_batch_results(void* hb, double* z, double* zz, double* s_half, double* eps_bound, int32_t* branch,
                         double* min_gap, int n_threads) {
  Batch* b = static_cast<Batch*>(hb);
  if (!b) return -1;
  for (const auto& t : b->T)   // the branch rows need one common layer
    if (t.layer != b->T.front().layer) return -1;
  const int n = b->C.n;
  const int64_t nt = (int64_t)b->T.size();
#ifdef _OPENMP
  const int th = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(th)
#endif
  for (int64_t i = 0; i < nt; ++i) {
    Trajectory T = b->T[(size_t)i];   // a copy: the sweep moves the centre
    observables(T, n);
    if (z) std::copy(T.z.begin(), T.z.end(), z + i * n);
    if (zz) std::copy(T.zz.begin(), T.zz.end(), zz + i * (n - 1));
    if (s_half) s_half[i] = T.s_half;
    if (eps_bound) eps_bound[i] = T.eps_tot <= b->eps_max - 2.0 ? T.eps_tot : b->eps_max;
    if (branch) std::copy(T.branch.begin(), T.branch.end(), branch + i * (int64_t)T.branch.size());
    if (min_gap) min_gap[i] = T.min_gap;
  }
  (void)n_threads;
  return 0;
}

// The layer every trajectory has reached, or -1 when they differ.
int oracle_batch_layer(void* hb) {
  Batch* b = static_cast<Batch*>(hb);
  if (!b || b->T.empty()) return 0;
  for (const auto& t : b->T)
    if (t.layer != b->T.front().layer) return -1;
  return b->T.front().layer;
}

// Largest bond dimension over the batch (for the tests).
int oracle_batch_max_bond(void* hb) {
  Batch* b = static_cast<Batch*>(hb);
  int m = 1;
  for (const auto& t : b->T)
    for (const auto& s : t.a) m = std::max(m, std::max(s.dl, s.dr));
  return m;
}

void oracle_batch_destroy(void* hb) { delete static_cast<Batch*>(hb); }

}  // extern "C"
