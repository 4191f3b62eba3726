// Host-side tables of the low-rank proton transport library (FP64, built once per context).
#pragma once
#include <cstdint>
#include <vector>

namespace dlra {

// Angular tables for degree N (Sec. 3.3.1, Sec. 3.3.2).
struct AngularTables {
  int N = 0, m = 0;
  std::vector<double> A[3];     // A_d = int m m^T Omega_d dOmega, m x m row-major
  std::vector<double> absA[3];  // |A_d| = V_d |Lambda_d| V_d^T, m x m row-major
  double lam_max = 0.0;         // spectral radius of every A_d
  std::vector<int> degree;      // l(p)
};

// Builds the tables; returns false (with msg) if an internal consistency check fails.
bool build_angular(int N, AngularTables& out, char* msg, int msg_len);

// m(Omega) for a unit direction (real spherical harmonics, index p = l^2 + l + k).
void real_sh_dir(int N, const double dir[3], double* out);

// Screened-Rutherford kernel 1/(1 - mu + 2 eta)^2: s_l = 2 pi int P_l k dmu for
// l = 0..lmax via Legendre functions of the second kind; xi = s_0 - s_1.
void screened_rutherford_moments(double eta, int lmax, double* s, double* xi);

// Gauss-Legendre nodes/weights on [-1, 1] and Gauss-Hermite nodes/weights (weight e^{-x^2}).
void gauss_legendre(int n, double* x, double* w);
void gauss_hermite(int n, double* x, double* w);

}  // namespace dlra
