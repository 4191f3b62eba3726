// Crank-Nicolson march of one ray's energy distribution through a voxel segment (Sec. 3.2), on
// the block-tridiagonal energy-DG operators of dlra_straggling_tables: with a stopping factor f
// and removal factor tau the system M dc/dz = -G c, G = -f ADV + f SIPG + tau REM, advances by
// (M + h/2 G) c_{n+1} = (M - h/2 G) c_n, the left side solved by block Thomas elimination
// (G elements of 3 x 3 blocks, factored once per segment). Plain arithmetic on raw pointers,
// callable from a device thread.
#pragma once

#include <cmath>
#include <cstddef>

#ifndef DLRA_HD
#define DLRA_HD __host__ __device__
#endif

namespace dlra {
namespace strag {

// 3 x 3 helpers (row-major)
DLRA_HD inline void mat3_inv(const double* a, double* inv) {
  const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  const double r = 1.0 / det;
  inv[0] = c00 * r;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) * r;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) * r;
  inv[3] = c01 * r;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) * r;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) * r;
  inv[6] = c02 * r;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) * r;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) * r;
}

DLRA_HD inline void mat3_mul(const double* a, const double* b, double* c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

// block b of row e of G = -f ADV + f SIPG + tau REM (tables [e][b][3][3])
DLRA_HD inline void g_block(const double* adv, const double* sipg, const double* rem, int e, int b, double f,
                            double tau, double* out) {
  const double* A = adv + ((size_t)e * 3 + b) * 9;
  const double* K = sipg + ((size_t)e * 3 + b) * 9;
  const double* R = rem + ((size_t)e * 3 + b) * 9;
  for (int q = 0; q < 9; ++q) out[q] = -f * A[q] + f * K[q] + tau * R[q];
}

// Factor (M + h/2 G): Wi[e] = (D_e - L_e X_{e-1})^{-1}, X[e] = Wi[e] U_e (each 9 doubles).
DLRA_HD inline void factor(int G, const double* mass, const double* adv, const double* sipg, const double* rem,
                           double f, double tau, double h, double* Wi, double* X) {
  double L[9], D[9], U[9], T[9];
  for (int e = 0; e < G; ++e) {
    g_block(adv, sipg, rem, e, 1, f, tau, D);
    for (int q = 0; q < 9; ++q) D[q] *= 0.5 * h;
    for (int i = 0; i < 3; ++i) D[4 * i] += mass[3 * e + i];
    if (e > 0) {
      g_block(adv, sipg, rem, e, 0, f, tau, L);
      for (int q = 0; q < 9; ++q) L[q] *= 0.5 * h;
      mat3_mul(L, X + (size_t)(e - 1) * 9, T);
      for (int q = 0; q < 9; ++q) D[q] -= T[q];
    }
    mat3_inv(D, Wi + (size_t)e * 9);
    if (e + 1 < G) {
      g_block(adv, sipg, rem, e, 2, f, tau, U);
      for (int q = 0; q < 9; ++q) U[q] *= 0.5 * h;
      mat3_mul(Wi + (size_t)e * 9, U, X + (size_t)e * 9);
    }
  }
}

// One step: cn = (M + h/2 G)^{-1} (M - h/2 G) c, with y as work space (3 G doubles).
DLRA_HD inline void step(int G, const double* mass, const double* adv, const double* sipg, const double* rem,
                         double f, double tau, double h, const double* Wi, const double* X, const double* c, double* y,
                         double* cn) {
  double B[9], r[3], t[3];
  // right side and forward elimination: y_e = Wi_e (r_e - L_e y_{e-1})
  for (int e = 0; e < G; ++e) {
    for (int i = 0; i < 3; ++i) r[i] = mass[3 * e + i] * c[3 * e + i];
    for (int b = 0; b < 3; ++b) {
      const int col = e - 1 + b;
      if (col < 0 || col >= G) continue;
      g_block(adv, sipg, rem, e, b, f, tau, B);
      for (int i = 0; i < 3; ++i)
        r[i] -= 0.5 * h * (B[3 * i] * c[3 * col] + B[3 * i + 1] * c[3 * col + 1] + B[3 * i + 2] * c[3 * col + 2]);
    }
    if (e > 0) {
      g_block(adv, sipg, rem, e, 0, f, tau, B);
      for (int i = 0; i < 3; ++i)
        r[i] -= 0.5 * h * (B[3 * i] * y[3 * (e - 1)] + B[3 * i + 1] * y[3 * (e - 1) + 1] + B[3 * i + 2] * y[3 * (e - 1) + 2]);
    }
    const double* W = Wi + (size_t)e * 9;
    for (int i = 0; i < 3; ++i) y[3 * e + i] = W[3 * i] * r[0] + W[3 * i + 1] * r[1] + W[3 * i + 2] * r[2];
  }
  // back substitution: c_e = y_e - X_e c_{e+1}
  for (int i = 0; i < 3; ++i) cn[3 * (G - 1) + i] = y[3 * (G - 1) + i];
  for (int e = G - 2; e >= 0; --e) {
    const double* Xe = X + (size_t)e * 9;
    for (int i = 0; i < 3; ++i) t[i] = Xe[3 * i] * cn[3 * (e + 1)] + Xe[3 * i + 1] * cn[3 * (e + 1) + 1] + Xe[3 * i + 2] * cn[3 * (e + 1) + 2];
    for (int i = 0; i < 3; ++i) cn[3 * e + i] = y[3 * e + i] - t[i];
  }
}

// int f S_w psi dE = f sum_e,j c_ej SW_ej
DLRA_HD inline double deposit_rate(int G, const double* SW, double f, const double* c) {
  double s = 0.0;
  for (int q = 0; q < 3 * G; ++q) s += SW[q] * c[q];
  return f * s;
}

constexpr int kMaxBinsPerElem = 8;

struct MarchTables {
  int G, K, n;
  const double *mass, *adv, *sipg, *rem, *SW;   // tables of dlra_straggling_tables and int S_w P_j
  const int* bin0;                               // first bin overlapping element e
  const int* nbin;                               // number of bins overlapping element e (<= 8)
  const double* bw;                              // [e][t][j] int over (element e and bin bin0+t) of P_j dE
  const double* c0;                              // initial coefficients (3 G)
  double inv_vh;                                 // 1 / (voxel volume x bin width)
  double inv_v;                                  // 1 / voxel volume
  double h_max;
};

// adds v to *p: atomically on the device
struct AddTo {
  DLRA_HD void operator()(double* p, double v) const {
#ifdef __CUDA_ARCH__
    atomicAdd(p, v);
#else
    *p += v;
#endif
  }
};

// doubles of work space per ray
DLRA_HD inline size_t work_per_ray(int G) { return 4 * (size_t)(3 * G) + 18 * (size_t)G; }

// March ray r through its segments [seg_ptr[r], seg_ptr[r+1]) and add each segment's energy
// lost to slowing down to e_u(cell) and its track integral over every energy bin to psi(k, cell).
template <class Add>
DLRA_HD void march_ray(int r, const int* seg_ptr, const int* seg_cell, const double* seg_len, const double* ray_w,
                       const MarchTables& t, const double* f_cell, const double* tau_cell, double* scratch,
                       double* psi, double* e_u, Add add) {
  const int N3 = 3 * t.G;
  double* c = scratch + (size_t)r * work_per_ray(t.G);
  double* cn = c + N3;
  double* y = cn + N3;
  double* track = y + N3;
  double* Wi = track + N3;
  double* X = Wi + 9 * (size_t)t.G;
  for (int q = 0; q < N3; ++q) c[q] = t.c0[q];
  const double wr = ray_w[r];
  for (int s = seg_ptr[r]; s < seg_ptr[r + 1]; ++s) {
    const int cell = seg_cell[s];
    const double len = seg_len[s], f = f_cell[cell], tau = tau_cell[cell];
    int nst = (int)ceil(len / t.h_max - 1e-12);
    if (nst < 1) nst = 1;
    const double h = len / nst;
    factor(t.G, t.mass, t.adv, t.sipg, t.rem, f, tau, h, Wi, X);
    for (int q = 0; q < N3; ++q) track[q] = 0.0;
    double dep = 0.0, prev = deposit_rate(t.G, t.SW, f, c);
    for (int k = 0; k < nst; ++k) {
      step(t.G, t.mass, t.adv, t.sipg, t.rem, f, tau, h, Wi, X, c, y, cn);
      const double cur = deposit_rate(t.G, t.SW, f, cn);
      dep += 0.5 * h * (prev + cur);
      for (int q = 0; q < N3; ++q) {
        track[q] += 0.5 * h * (c[q] + cn[q]);
        c[q] = cn[q];
      }
      prev = cur;
    }
    add(e_u + cell, wr * dep * t.inv_v);
    for (int e = 0; e < t.G; ++e) {
      for (int b = 0; b < t.nbin[e]; ++b) {
        const double* w = t.bw + ((size_t)e * kMaxBinsPerElem + b) * 3;
        const double v = w[0] * track[3 * e] + w[1] * track[3 * e + 1] + w[2] * track[3 * e + 2];
        if (v != 0.0) add(psi + (size_t)(t.bin0[e] + b) * t.n + cell, wr * v * t.inv_vh);
      }
    }
  }
}

}  // namespace strag
}  // namespace dlra
