// Host tables of the uncollided straggling model along a ray (Sec. 3.2): the energy
// discretisation of d psi/dz + Sigma_t psi = d(S* psi)/dE + (1/2) d/dE (T d psi/dE),
// S* = S + (1/2) dT/dE, by discontinuous Galerkin on equal elements with the Legendre
// polynomials P_0, P_1, P_2 of the element coordinate (diagonal mass matrix Delta / (2j + 1)),
// a Lax-Friedrichs face flux for the slowing-down term (alpha = |S*| at the face: the value
// from the higher-energy side; no inflow above E_max, outflow below E_min) and SIPG for the
// straggling term (kappa = T / 2, penalty 18 kappa / Delta, no diffusive flux through either
// end). Element integrals by 6-point Gauss-Legendre. For a material factor f and removal
// factor tau along the ray the system is M dc/dz = -(-f ADV + f SIPG + tau REM) c.
//
// Water data: S_w(E) = E^(1-p) / (p alpha) (Bragg-Kleeman), straggling
// T_w(E) = T_Bohr (1 + 4 I / (3 m_e v^2) ln(2 m_e v^2 / I)) with T_Bohr = 4 pi r_e^2 (m_e c^2)^2 N_e
// and I = 75 eV (the paper's Williams formula read with the leading term of its bracket), and
// removal Sigma_t = tau T_scat(E) / 2 with T_scat = t100 (100 / E)^2 (the ray tracer's model).
#include <cmath>
#include <cstddef>
#include <cstring>

#include "dlra.h"
#include "tables.h"

namespace dlra {
void set_context_free_error(const char* msg);

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMeC2 = 0.51099895;        // MeV
constexpr double kMpC2 = 938.27208816;      // MeV
constexpr double kRe = 2.8179403262e-13;    // cm
constexpr double kNA = 6.02214076e23;
constexpr double kIWater = 75.0e-6;         // MeV

double t_bohr_water() {
  const double ne = kNA * 10.0 / 18.015;   // electrons per cm^3 of water
  return 4.0 * kPi * kRe * kRe * kMeC2 * kMeC2 * ne;
}

// T_w(E) and its derivative in E
void straggling_water(double E, double& T, double& dT) {
  const double gam = 1.0 + E / kMpC2;
  const double y = kMeC2 * (1.0 - 1.0 / (gam * gam));          // m_e v^2
  const double dy = kMeC2 * 2.0 / (gam * gam * gam * kMpC2);    // dy/dE
  const double a = 4.0 * kIWater / 3.0;
  const double L = 2.0 * y / kIWater;
  const double tb = t_bohr_water();
  if (L > 1.0) {
    const double lg = std::log(L);
    T = tb * (1.0 + a * lg / y);
    dT = tb * a * (1.0 - lg) / (y * y) * dy;
  } else {
    T = tb;
    dT = 0.0;
  }
}

void legendre3(double xi, double P[3], double dP[3]) {
  P[0] = 1.0;
  P[1] = xi;
  P[2] = 0.5 * (3.0 * xi * xi - 1.0);
  dP[0] = 0.0;
  dP[1] = 1.0;
  dP[2] = 3.0 * xi;
}

}  // namespace
}  // namespace dlra

extern "C" dlra_status dlra_straggling_tables(const dlra_straggling_args* a, double* mass, double* adv, double* sipg,
                                              double* rem) {
  using namespace dlra;
  if (!a || !mass || !adv || !sipg || !rem) {
    set_context_free_error("null arguments");
    return DLRA_ERR_ARG;
  }
  if (!(a->e_min > 0.0) || !(a->e_max > a->e_min) || a->n_elem < 1 || a->n_elem > (1 << 16) || !(a->bk_p > 1.0) ||
      !(a->bk_alpha > 0.0) || !(a->t100 >= 0.0)) {
    set_context_free_error("need 0 < e_min < e_max, 1 <= n_elem <= 65536, bk_p > 1, bk_alpha > 0, t100 >= 0");
    return DLRA_ERR_ARG;
  }
  const int G = a->n_elem;
  const double D = (a->e_max - a->e_min) / G;
  const double p = a->bk_p, alpha = a->bk_alpha;
  const size_t nb = (size_t)G * 27;
  std::memset(adv, 0, sizeof(double) * nb);
  std::memset(sipg, 0, sizeof(double) * nb);
  std::memset(rem, 0, sizeof(double) * nb);
  // block (e, b, i, j): row dof i of element e, column dof j of element e - 1 + b
  auto blk = [&](double* M, int e, int b, int i, int j) -> double& {
    return M[(((size_t)e * 3 + b) * 3 + i) * 3 + j];
  };
  auto strag = [&](double E, double& T, double& dT) {
    if (a->straggling) {
      straggling_water(E, T, dT);
    } else {
      T = 0.0;
      dT = 0.0;
    }
  };
  auto s_star = [&](double E) {
    double T, dT;
    strag(E, T, dT);
    return std::pow(E, 1.0 - p) / (p * alpha) + 0.5 * dT;
  };
  double xq[6], wq[6];
  gauss_legendre(6, xq, wq);
  for (int e = 0; e < G; ++e) {
    for (int j = 0; j < 3; ++j) mass[3 * e + j] = D / (2.0 * j + 1.0);
    const double Ec = a->e_min + (e + 0.5) * D;
    for (int q = 0; q < 6; ++q) {
      const double E = Ec + 0.5 * D * xq[q], w = 0.5 * D * wq[q];
      double P[3], dP[3];
      legendre3(xq[q], P, dP);
      for (int i = 0; i < 3; ++i) dP[i] *= 2.0 / D;
      double T, dT;
      strag(E, T, dT);
      const double ss = s_star(E), kap = 0.5 * T, sig = 0.5 * a->t100 * (100.0 / E) * (100.0 / E);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          blk(adv, e, 1, i, j) -= w * ss * P[j] * dP[i];
          blk(sipg, e, 1, i, j) += w * kap * dP[i] * dP[j];
          blk(rem, e, 1, i, j) += w * sig * P[i] * P[j];
        }
    }
  }
  // face traces: top of an element (xi = +1) and bottom (xi = -1), values and d/dE
  const double vt[3] = {1.0, 1.0, 1.0}, vb[3] = {1.0, -1.0, 1.0};
  const double dvt[3] = {0.0, 2.0 / D, 6.0 / D}, dvb[3] = {0.0, 2.0 / D, -6.0 / D};
  // slowing down: F = 1/2 s (psi_lo + psi_hi) + 1/2 |s| (psi_hi - psi_lo) enters the lower
  // element as + F v(top) and the upper one as - F v(bottom)
  for (int f = 0; f <= G; ++f) {
    const double s = s_star(a->e_min + f * D), al = std::fabs(s);
    const double clo = 0.5 * s - 0.5 * al, chi = 0.5 * s + 0.5 * al;
    const int lo = f - 1, hi = f;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        if (lo >= 0) {
          blk(adv, lo, 1, i, j) += vt[i] * clo * vt[j];
          if (hi < G) blk(adv, lo, 2, i, j) += vt[i] * chi * vb[j];
        }
        if (hi < G) {
          if (lo >= 0) blk(adv, hi, 0, i, j) -= vb[i] * clo * vt[j];
          blk(adv, hi, 1, i, j) -= vb[i] * chi * vb[j];
        }
      }
  }
  // straggling, interior faces: - {kappa psi'}[v] - {kappa v'}[psi] + sigma [psi][v], with the
  // jump [u] = u(lower element's top) - u(upper element's bottom)
  for (int f = 1; f < G; ++f) {
    double T, dT;
    strag(a->e_min + f * D, T, dT);
    const double kf = 0.5 * T, sg = 18.0 * kf / D;
    const int lo = f - 1, hi = f;
    const int el[2] = {lo, hi};
    for (int ia = 0; ia < 2; ++ia)
      for (int ib = 0; ib < 2; ++ib) {
        const int ea = el[ia], eb = el[ib];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            const double va = ia == 0 ? vt[i] : -vb[i], vbj = ib == 0 ? vt[j] : -vb[j];
            const double da = ia == 0 ? 0.5 * dvt[i] : 0.5 * dvb[i], db = ib == 0 ? 0.5 * dvt[j] : 0.5 * dvb[j];
            blk(sipg, ea, eb - ea + 1, i, j) += -kf * db * va - kf * da * vbj + sg * vbj * va;
          }
      }
  }
  return DLRA_OK;
}
