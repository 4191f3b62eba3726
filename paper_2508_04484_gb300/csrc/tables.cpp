// Host tables: real spherical harmonics, streaming matrices and their absolute
// values (Sec. 3.3.1, Sec. 3.3.2), screened-Rutherford Legendre moments (Sec. 3.3.1),
// Gauss quadratures. FP64; computed once per context.
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace dlra {

namespace {

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major, destroyed).
// Eigenvalues into lam, eigenvectors into the columns of V (row-major n x n).
void jacobi_eigen(int n, std::vector<double>& a, std::vector<double>& lam, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = a[(size_t)i * n + j] * a[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = a[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = a[(size_t)i * n + i];
}

// Fully normalised associated Legendre values Nt[l][k] = N_lk P_l^k(mu) (no
// Condon-Shortley phase), k = 0..l, stored at l*(l+1)/2 + k.
void norm_legendre(int N, double mu, std::vector<double>& out) {
  out.assign((size_t)(N + 1) * (N + 2) / 2, 0.0);
  auto at = [&](int l, int k) -> double& { return out[(size_t)l * (l + 1) / 2 + k]; };
  double s = std::sqrt(std::max(0.0, 1.0 - mu * mu));
  double pkk = 1.0 / std::sqrt(4.0 * M_PI);
  for (int k = 0; k <= N; ++k) {
    if (k > 0) pkk *= std::sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
    at(k, k) = pkk;
    if (k + 1 <= N) at(k + 1, k) = std::sqrt(2.0 * k + 3.0) * mu * pkk;
    for (int l = k + 2; l <= N; ++l) {
      double a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)k * k));
      double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)k * k) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
      at(l, k) = a * (mu * at(l - 1, k) - b * at(l - 2, k));
    }
  }
}

void real_sh(int N, double mu, double phi, std::vector<double>& nl, double* out) {
  norm_legendre(N, mu, nl);
  const double r2 = std::sqrt(2.0);
  for (int l = 0; l <= N; ++l) {
    int p0 = l * l + l;
    out[p0] = nl[(size_t)l * (l + 1) / 2];
    for (int k = 1; k <= l; ++k) {
      double v = r2 * nl[(size_t)l * (l + 1) / 2 + k];
      out[p0 + k] = v * std::cos(k * phi);
      out[p0 - k] = v * std::sin(k * phi);
    }
  }
}

void tridiag_gauss(int n, const std::vector<double>& diag, const std::vector<double>& off, double mu0,
                   double* x, double* w) {
  std::vector<double> a((size_t)n * n, 0.0), lam, V;
  for (int i = 0; i < n; ++i) a[(size_t)i * n + i] = diag[i];
  for (int i = 0; i + 1 < n; ++i) a[(size_t)i * n + i + 1] = a[(size_t)(i + 1) * n + i] = off[i];
  jacobi_eigen(n, a, lam, V);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int p, int q) { return lam[p] < lam[q]; });
  for (int i = 0; i < n; ++i) {
    x[i] = lam[idx[i]];
    double v0 = V[idx[i]];  // first component of eigenvector idx[i]
    w[i] = mu0 * v0 * v0;
  }
}

}  // namespace

void gauss_legendre(int n, double* x, double* w) {
  // Golub-Welsch: Jacobi matrix of the Legendre polynomials
  std::vector<double> d(n, 0.0), o(std::max(n - 1, 0));
  for (int k = 1; k < n; ++k) o[k - 1] = k / std::sqrt(4.0 * k * k - 1.0);
  tridiag_gauss(n, d, o, 2.0, x, w);
}

void gauss_hermite(int n, double* x, double* w) {
  std::vector<double> d(n, 0.0), o(std::max(n - 1, 0));
  for (int k = 1; k < n; ++k) o[k - 1] = std::sqrt(k / 2.0);
  tridiag_gauss(n, d, o, std::sqrt(M_PI), x, w);
}

void real_sh_dir(int N, const double dir[3], double* out) {
  double mu = std::max(-1.0, std::min(1.0, dir[2]));
  double phi = std::atan2(dir[1], dir[0]);
  std::vector<double> nl;
  real_sh(N, mu, phi, nl, out);
}

bool build_angular(int N, AngularTables& T, char* msg, int msg_len) {
  const int m = (N + 1) * (N + 1);
  T.N = N;
  T.m = m;
  T.degree.resize(m);
  for (int l = 0; l <= N; ++l)
    for (int k = -l; k <= l; ++k) T.degree[l * l + l + k] = l;
  // product quadrature exact for polynomial integrands of degree <= 2N + 2
  const int nmu = N + 2, nphi = 2 * N + 4;
  std::vector<double> xg(nmu), wg(nmu);
  gauss_legendre(nmu, xg.data(), wg.data());
  std::vector<double> mv(m), mr(m), nl;
  for (int d = 0; d < 3; ++d) T.A[d].assign((size_t)m * m, 0.0);
  // rotations mapping e_z to e_x (about y by +90 deg) and to e_y (about x by -90 deg)
  const double Qx[9] = {0, 0, 1, 0, 1, 0, -1, 0, 0};
  const double Qy[9] = {1, 0, 0, 0, 0, 1, 0, -1, 0};
  std::vector<double> Dx((size_t)m * m, 0.0), Dy((size_t)m * m, 0.0);
  std::vector<double> mx(m), my(m);
  for (int a = 0; a < nmu; ++a)
    for (int b = 0; b < nphi; ++b) {
      double mu = xg[a], phi = (b + 0.5) * 2.0 * M_PI / nphi;
      double wq = wg[a] * 2.0 * M_PI / nphi;
      double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
      double om[3] = {st * std::cos(phi), st * std::sin(phi), mu};
      real_sh(N, mu, phi, nl, mv.data());
      for (int d = 0; d < 3; ++d) {
        double f = wq * om[d];
        double* Ad = T.A[d].data();
        for (int p = 0; p < m; ++p) {
          double fp = f * mv[p];
          if (fp == 0.0) continue;
          for (int q = 0; q < m; ++q) Ad[(size_t)p * m + q] += fp * mv[q];
        }
      }
      // rotated directions Q om
      double ox[3], oy[3];
      for (int i = 0; i < 3; ++i) {
        ox[i] = Qx[3 * i] * om[0] + Qx[3 * i + 1] * om[1] + Qx[3 * i + 2] * om[2];
        oy[i] = Qy[3 * i] * om[0] + Qy[3 * i + 1] * om[1] + Qy[3 * i + 2] * om[2];
      }
      real_sh_dir(N, ox, mx.data());
      real_sh_dir(N, oy, my.data());
      for (int l = 0; l <= N; ++l) {
        int p0 = l * l;
        for (int p = p0; p < p0 + 2 * l + 1; ++p)
          for (int q = p0; q < p0 + 2 * l + 1; ++q) {
            Dx[(size_t)p * m + q] += wq * mx[p] * mv[q];
            Dy[(size_t)p * m + q] += wq * my[p] * mv[q];
          }
      }
    }
  for (int d = 0; d < 3; ++d)
    for (size_t i = 0; i < (size_t)m * m; ++i) {
      double& v = T.A[d][i];
      if (std::fabs(v) < 1e-14) v = 0.0;
    }
  // |A_z| block by block: A_z couples only moments of equal order k
  T.absA[2].assign((size_t)m * m, 0.0);
  double lmax = 0.0;
  for (int k = -N; k <= N; ++k) {
    std::vector<int> idx;
    for (int l = std::abs(k); l <= N; ++l) idx.push_back(l * l + l + k);
    int b = (int)idx.size();
    std::vector<double> blk((size_t)b * b), lam, V;
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) blk[(size_t)i * b + j] = T.A[2][(size_t)idx[i] * m + idx[j]];
    jacobi_eigen(b, blk, lam, V);
    for (int e = 0; e < b; ++e) lmax = std::max(lmax, std::fabs(lam[e]));
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) {
        double s = 0.0;
        for (int e = 0; e < b; ++e) s += V[(size_t)i * b + e] * std::fabs(lam[e]) * V[(size_t)j * b + e];
        T.absA[2][(size_t)idx[i] * m + idx[j]] = s;
      }
  }
  T.lam_max = lmax;
  // |A_x| = D_x |A_z| D_x^T, |A_y| = D_y |A_z| D_y^T; check A_x = D_x A_z D_x^T on the way
  const std::vector<double>* Ds[2] = {&Dx, &Dy};
  for (int d = 0; d < 2; ++d) {
    const std::vector<double>& D = *Ds[d];
    std::vector<double> tmpA((size_t)m * m, 0.0), tmpB((size_t)m * m, 0.0);
    // tmp = Az D^T, tmpB = |Az| D^T
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < m; ++q) {
        int lq = T.degree[q], q0 = lq * lq;
        double sa = 0.0, sb = 0.0;
        for (int j = q0; j < q0 + 2 * lq + 1; ++j) {
          sa += T.A[2][(size_t)p * m + j] * D[(size_t)q * m + j];
          sb += T.absA[2][(size_t)p * m + j] * D[(size_t)q * m + j];
        }
        tmpA[(size_t)p * m + q] = sa;
        tmpB[(size_t)p * m + q] = sb;
      }
    T.absA[d].assign((size_t)m * m, 0.0);
    double err = 0.0;
    for (int p = 0; p < m; ++p) {
      int lp = T.degree[p], p0 = lp * lp;
      for (int q = 0; q < m; ++q) {
        double sa = 0.0, sb = 0.0;
        for (int j = p0; j < p0 + 2 * lp + 1; ++j) {
          sa += D[(size_t)p * m + j] * tmpA[(size_t)j * m + q];
          sb += D[(size_t)p * m + j] * tmpB[(size_t)j * m + q];
        }
        err = std::max(err, std::fabs(sa - T.A[d][(size_t)p * m + q]));
        T.absA[d][(size_t)p * m + q] = sb;
      }
    }
    if (err > 1e-10) {
      std::snprintf(msg, msg_len, "angular tables: rotation check failed for d=%d (err %.3e)", d, err);
      return false;
    }
  }
  return true;
}

void screened_rutherford_moments(double eta, int lmax, double* s, double* xi) {
  // Legendre functions of the second kind Q_l(a), a = 1 + 2 eta > 1, by Miller's
  // backward recurrence (Q_l is the minimal solution), normalised by
  // Q_0(a) = 0.5 ln((a+1)/(a-1)); then 2 pi int P_l(mu)/(a - mu)^2 dmu = -4 pi Q_l'(a)
  // with (a^2 - 1) Q_l' = l (a Q_l - Q_{l-1}) and Q_0' = -1/(a^2 - 1).
  const double a = 1.0 + 2.0 * eta;
  const double a21 = (a - 1.0) * (a + 1.0);
  const int L = lmax + 2 + (int)(40.0 / std::max(std::acosh(a), 1e-3));
  std::vector<double> Q(L + 2, 0.0);
  Q[L + 1] = 0.0;
  Q[L] = 1e-280;
  for (int l = L; l >= 1; --l) {
    Q[l - 1] = ((2.0 * l + 1.0) * a * Q[l] - (l + 1.0) * Q[l + 1]) / l;
    if (std::fabs(Q[l - 1]) > 1e250) {
      for (int j = l - 1; j <= L + 1; ++j) Q[j] *= 1e-250;
    }
  }
  const double q0 = 0.5 * std::log((a + 1.0) / (a - 1.0));
  const double scale = q0 / Q[0];
  for (int l = 0; l <= L + 1; ++l) Q[l] *= scale;
  s[0] = -4.0 * M_PI * (-1.0 / a21);
  for (int l = 1; l <= lmax; ++l) s[l] = -4.0 * M_PI * (l * (a * Q[l] - Q[l - 1]) / a21);
  *xi = s[0] - s[1];
}

}  // namespace dlra
