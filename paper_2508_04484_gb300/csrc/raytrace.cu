// CSDA ray tracer for the uncollided flux (Sec. 3.2 without straggling), FP64.
// One thread per ray: an Amanatides-Woo voxel walk; per voxel segment the energy
// follows from the water range R_w(E) = alpha E^p, which decreases by f(x) per cm
// (S(x, E) = f(x) S_w(E)); the particle weight decays with Sigma_t(x, E) =
// tau(x) T_w(E)/2, whose integral along the ray has the closed form
// (tau/f) (Lam(E) - Lam(E_in)), Lam(E) = klam E^(p-2) / (2 - p). Each segment is split
// at the energy-grid nodes and its track length and energy loss are integrated in E
// (6-point Gauss-Legendre) into the bin-averaged fluence and the uncollided deposit.
// The adjoint kernel records each ray's segments and walks them backwards, differentiating
// the same formulas with respect to the stopping factor f(x) and the removal factor tau(x).
#include <cuda_runtime.h>
#include <math.h>

#include "kernels.h"

namespace dlra {

namespace {

__constant__ double c_glx[6] = {-0.9324695142031521, -0.6612093864662645, -0.2386191860831969,
                                0.2386191860831969,  0.6612093864662645,  0.9324695142031521};
__constant__ double c_glw[6] = {0.1713244923791704, 0.3607615730481386, 0.4679139345726910,
                                0.4679139345726910, 0.3607615730481386, 0.1713244923791704};

__device__ __forceinline__ double lam_fn(double E, double p, double klam) { return klam * pow(E, p - 2.0) / (2.0 - p); }

}  // namespace

// One recorded voxel segment of a ray: entry range, entry weight, length, cell index.
struct SegRec {
  double R, N, ell, cell;
};

// Walk one ray through the grid. RECORD = false: accumulate the bin-averaged fluence and
// the deposit. RECORD = true: store every voxel segment's entry range R, entry weight N,
// length and cell in rec (at most nx + ny + nz + 8 segments) and return their number.
template <bool RECORD>
__device__ int walk_ray(const double* __restrict__ ry, const RayGeo& g, const double* __restrict__ f_cell,
                        const double* __restrict__ tau_cell, double* __restrict__ psi, double* __restrict__ e_u,
                        SegRec* __restrict__ rec) {
  const double o[3] = {ry[0], ry[1], ry[2]};
  const double v[3] = {ry[3], ry[4], ry[5]};
  const double E0 = ry[6], wr = ry[7];
  const double Lb[3] = {g.nx * g.dx, g.ny * g.dy, g.nz * g.dz};
  const double dd[3] = {g.dx, g.dy, g.dz};
  const int nd[3] = {g.nx, g.ny, g.nz};
  const long long n = (long long)g.nx * g.ny * g.nz;
  int nrec = 0;
  double t0 = 0.0, t1 = 1e300;
  for (int a = 0; a < 3; ++a) {
    if (a == 1 && g.two_d) continue;
    if (fabs(v[a]) < 1e-300) {
      if (o[a] < 0.0 || o[a] > Lb[a]) return nrec;
      continue;
    }
    double ta = (0.0 - o[a]) / v[a], tb = (Lb[a] - o[a]) / v[a];
    t0 = fmax(t0, fmin(ta, tb));
    t1 = fmin(t1, fmax(ta, tb));
  }
  if (!(t1 > t0)) return nrec;
  int idx[3];
  double tmax[3], tdel[3];
  int stp[3];
  for (int a = 0; a < 3; ++a) {
    if (a == 1 && g.two_d) {
      idx[a] = 0;
      tmax[a] = 1e300;
      tdel[a] = 1e300;
      stp[a] = 0;
      continue;
    }
    double pa = o[a] + t0 * v[a];
    int i = (int)floor(pa / dd[a]);
    if (v[a] < 0.0 && pa == i * dd[a]) i -= 1;
    if (i < 0) i = 0;
    if (i > nd[a] - 1) i = nd[a] - 1;
    idx[a] = i;
    if (v[a] > 0.0) {
      stp[a] = 1;
      tmax[a] = ((i + 1) * dd[a] - o[a]) / v[a];
      tdel[a] = dd[a] / v[a];
    } else if (v[a] < 0.0) {
      stp[a] = -1;
      tmax[a] = (i * dd[a] - o[a]) / v[a];
      tdel[a] = -dd[a] / v[a];
    } else {
      stp[a] = 0;
      tmax[a] = 1e300;
      tdel[a] = 1e300;
    }
  }
  const double p = g.p, alpha = g.alpha;
  const double Rmin = alpha * pow(g.e_min, p);
  double R = alpha * pow(E0, p);
  double N = 1.0;
  double t = t0;
  const double inv_vh = 1.0 / (g.volume * g.h);
  const int maxit = g.nx + g.ny + g.nz + 8;
  for (int it = 0; it < maxit; ++it) {
    double tn = fmin(fmin(tmax[0], tmax[1]), fmin(tmax[2], t1));
    double ell = tn - t;
    if (ell > 0.0) {
      const long long cell = ((long long)idx[2] * g.ny + idx[1]) * g.nx + idx[0];
      if (RECORD) rec[nrec++] = SegRec{R, N, ell, (double)cell};
      const double f = f_cell[cell], tau = tau_cell[cell];
      double Rb = R - f * ell;
      const bool stop = Rb <= Rmin;
      if (stop) Rb = Rmin;
      const double Ea = pow(R / alpha, 1.0 / p);
      const double Eb = pow(Rb / alpha, 1.0 / p);
      int k = (int)floor((g.e_max - Ea) / g.h);
      if (k < 0) k = 0;
      double Ecur = Ea;
      const double a_tf = (f > 0.0) ? tau / f : 0.0;
      while (Ecur > Eb && k < g.K) {
        const double Ek1 = g.e_max - (k + 1) * g.h;
        const double Elo = fmax(Eb, Ek1);
        if (Elo < Ecur) {
          double Is, Ie, Nn;
          if (a_tf == 0.0) {
            Is = N * (alpha * pow(Ecur, p) - alpha * pow(Elo, p)) / f;
            Ie = N * (Ecur - Elo);
            Nn = N;
          } else {
            const double lc = lam_fn(Ecur, p, g.klam);
            const double hm = 0.5 * (Ecur - Elo), cm = 0.5 * (Ecur + Elo);
            Is = 0.0;
            Ie = 0.0;
            for (int q = 0; q < 6; ++q) {
              const double E = cm + hm * c_glx[q];
              const double NE = N * exp(-a_tf * (lam_fn(E, p, g.klam) - lc));
              Ie += c_glw[q] * NE;
              Is += c_glw[q] * NE * pow(E, p - 1.0);
            }
            Ie *= hm;
            Is *= hm * p * alpha / f;
            Nn = N * exp(-a_tf * (lam_fn(Elo, p, g.klam) - lc));
          }
          if (!RECORD) {
            atomicAdd(psi + (long long)k * n + cell, wr * Is * inv_vh);
            atomicAdd(e_u + cell, wr * Ie / g.volume);
          }
          N = Nn;
        }
        Ecur = Elo;
        ++k;
      }
      R = Rb;
      if (stop) return nrec;
    }
    if (tn >= t1) return nrec;
    int a = 0;
    if (tmax[1] < tmax[a]) a = 1;
    if (tmax[2] < tmax[a]) a = 2;
    idx[a] += stp[a];
    if (idx[a] < 0 || idx[a] >= nd[a]) return nrec;
    t = tn;
    tmax[a] += tdel[a];
  }
  return nrec;
}

__global__ void raytrace_kernel(const double* __restrict__ rays, int nray, RayGeo g,
                                const double* __restrict__ f_cell, const double* __restrict__ tau_cell,
                                double* __restrict__ psi, double* __restrict__ e_u) {
  const int rid = blockIdx.x * blockDim.x + threadIdx.x;
  if (rid >= nray) return;
  walk_ray<false>(rays + 8 * (long long)rid, g, f_cell, tau_cell, psi, e_u, nullptr);
}

// Reverse-mode derivative of one recorded segment (entry range R, entry weight N, length ell,
// cell c): given the adjoints Rbar of the range and Nbar of the weight leaving the segment,
// returns through them the adjoints of R and N entering it, and adds d/df(c) and d/dtau(c)
// of the loss <gpsi, psi> + <geu, e_u> to fbar, taubar. Each bin sub-segment's 6-point
// Gauss-Legendre rule is differentiated as written (nodes move with its end energies).
__device__ void segment_adjoint(double R, double N, double ell, long long cell, double wr, const RayGeo& g,
                                const double* __restrict__ f_cell, const double* __restrict__ tau_cell,
                                const double* __restrict__ gpsi, const double* __restrict__ geu, double& Rbar,
                                double& Nbar, double& fbar, double& taubar) {
  const double p = g.p, alpha = g.alpha, klam = g.klam;
  const long long n = (long long)g.nx * g.ny * g.nz;
  const double Rmin = alpha * pow(g.e_min, p);
  const double f = f_cell[cell], tau = tau_cell[cell];
  double Rb = R - f * ell;
  const bool stop = Rb <= Rmin;
  if (stop) Rb = Rmin;
  const double Ea = pow(R / alpha, 1.0 / p);
  const double Eb = pow(Rb / alpha, 1.0 / p);
  const double a_tf = (f > 0.0) ? tau / f : 0.0;
  int k0 = (int)floor((g.e_max - Ea) / g.h);
  if (k0 < 0) k0 = 0;
  int J = 0;
  {
    double Ecur = Ea;
    int k = k0;
    while (Ecur > Eb && k < g.K) {
      Ecur = fmax(Eb, g.e_max - (k + 1) * g.h);
      ++k;
      ++J;
    }
  }
  const double lamA = lam_fn(Ea, p, klam);
  const double sp = wr / (g.volume * g.h), se = wr / g.volume;
  double EaBar = 0.0, EbBar = 0.0, aBar = 0.0;
  for (int j = J - 1; j >= 0; --j) {
    const int k = k0 + j;
    const double Ecur = j == 0 ? Ea : g.e_max - k * g.h;
    const double Ek1 = g.e_max - (k + 1) * g.h;
    const double Elo = fmax(Eb, Ek1);
    if (!(Elo < Ecur)) continue;
    const bool lo_is_Eb = Eb >= Ek1;
    const double Nj = N * exp(-a_tf * (lam_fn(Ecur, p, klam) - lamA));
    const double pb = gpsi[(long long)k * n + cell] * sp;   // adjoint of Is
    const double eb = geu[cell] * se;                       // adjoint of Ie
    const double nb = Nbar;                                 // adjoint of Nn
    const double lc = lam_fn(Ecur, p, klam);
    const double dlc = -klam * pow(Ecur, p - 3.0);          // Lam'(Ecur)
    const double hm = 0.5 * (Ecur - Elo), cm = 0.5 * (Ecur + Elo);
    // per unit entry weight: sums of the rule and their derivatives
    double sI = 0, sS = 0, sIa = 0, sSa = 0, sIc = 0, sSc = 0, sIl = 0, sSl = 0;
    for (int q = 0; q < 6; ++q) {
      const double x = c_glx[q], wq = c_glw[q];
      const double E = cm + hm * x;
      const double dl = lam_fn(E, p, klam) - lc;
      const double G = exp(-a_tf * dl);
      const double Ep = pow(E, p - 1.0);
      const double dEp = (p - 1.0) * pow(E, p - 2.0);
      const double lamp = -klam * pow(E, p - 3.0);
      const double dGc = G * (-a_tf) * (lamp * 0.5 * (1.0 + x) - dlc);
      const double dGl = G * (-a_tf) * (lamp * 0.5 * (1.0 - x));
      sI += wq * G;
      sS += wq * G * Ep;
      sIa += wq * G * (-dl);
      sSa += wq * G * Ep * (-dl);
      sIc += wq * dGc;
      sSc += wq * (dGc * Ep + G * dEp * 0.5 * (1.0 + x));
      sIl += wq * dGl;
      sSl += wq * (dGl * Ep + G * dEp * 0.5 * (1.0 - x));
    }
    const double cs = p * alpha / f;
    double Ie1, Is1, dIe_c, dIe_l, dIs_c, dIs_l, dIs_f;
    if (a_tf == 0.0) {
      // closed forms used by the forward walk (Sigma_t = 0 in this cell)
      Ie1 = Ecur - Elo;
      Is1 = alpha * (pow(Ecur, p) - pow(Elo, p)) / f;
      dIe_c = 1.0;
      dIe_l = -1.0;
      dIs_c = cs * pow(Ecur, p - 1.0);
      dIs_l = -cs * pow(Elo, p - 1.0);
    } else {
      Ie1 = hm * sI;
      Is1 = cs * hm * sS;
      dIe_c = 0.5 * sI + hm * sIc;
      dIe_l = -0.5 * sI + hm * sIl;
      dIs_c = cs * (0.5 * sS + hm * sSc);
      dIs_l = cs * (-0.5 * sS + hm * sSl);
    }
    dIs_f = -Is1 / f;
    const double Gn = exp(-a_tf * (lam_fn(Elo, p, klam) - lc));   // Nn = Nj Gn
    // weight: d(Is, Ie, Nn)/dNj
    const double NjBar = pb * Is1 + eb * Ie1 + nb * Gn;
    // a = tau / f (derivatives of the general rule, valid at a = 0 too)
    aBar += Nj * (pb * cs * hm * sSa + eb * hm * sIa + nb * Gn * (-(lam_fn(Elo, p, klam) - lc)));
    fbar += Nj * pb * dIs_f;
    const double EcBar = Nj * (pb * dIs_c + eb * dIe_c + nb * Gn * (a_tf * dlc));
    const double ElBar = Nj * (pb * dIs_l + eb * dIe_l + nb * Gn * (-a_tf * (-klam * pow(Elo, p - 3.0))));
    if (j == 0) EaBar += EcBar;
    if (lo_is_Eb) EbBar += ElBar;
    Nbar = NjBar;
  }
  // Ea = (R/alpha)^(1/p), Eb = (Rb/alpha)^(1/p), Rb = R - f ell
  double RbBar = stop ? 0.0 : Rbar + EbBar * Eb / (p * Rb);
  Rbar = RbBar + EaBar * Ea / (p * R);
  fbar += -ell * RbBar;
  if (f > 0.0) {
    taubar += aBar / f;
    fbar += -aBar * tau / (f * f);
  }
}

__global__ void raytrace_adjoint_kernel(const double* __restrict__ rays, int nray, RayGeo g,
                                        const double* __restrict__ f_cell, const double* __restrict__ tau_cell,
                                        const double* __restrict__ gpsi, const double* __restrict__ geu,
                                        SegRec* __restrict__ rec_all, double* __restrict__ grad_f,
                                        double* __restrict__ grad_tau) {
  const int rid = blockIdx.x * blockDim.x + threadIdx.x;
  if (rid >= nray) return;
  const int maxit = g.nx + g.ny + g.nz + 8;
  SegRec* rec = rec_all + (long long)rid * maxit;
  const double* ry = rays + 8 * (long long)rid;
  const int ns = walk_ray<true>(ry, g, f_cell, tau_cell, nullptr, nullptr, rec);
  double Rbar = 0.0, Nbar = 0.0;
  for (int s = ns - 1; s >= 0; --s) {
    const SegRec r = rec[s];
    const long long cell = (long long)r.cell;
    double fb = 0.0, tb = 0.0;
    segment_adjoint(r.R, r.N, r.ell, cell, ry[7], g, f_cell, tau_cell, gpsi, geu, Rbar, Nbar, fb, tb);
    atomicAdd(grad_f + cell, fb);
    atomicAdd(grad_tau + cell, tb);
  }
}

void launch_raytrace(cudaStream_t st, const double* rays, int nray, RayGeo g, const double* f_cell,
                     const double* tau_cell, double* psi, double* e_u) {
  if (nray <= 0) return;
  // few, long-running threads: small blocks spread the rays over all SMs
  raytrace_kernel<<<(nray + 31) / 32, 32, 0, st>>>(rays, nray, g, f_cell, tau_cell, psi, e_u);
}

size_t raytrace_adjoint_scratch_bytes(int nray, RayGeo g) {
  return (size_t)nray * (g.nx + g.ny + g.nz + 8) * sizeof(SegRec);
}

void launch_raytrace_adjoint(cudaStream_t st, const double* rays, int nray, RayGeo g, const double* f_cell,
                             const double* tau_cell, const double* gpsi, const double* geu, void* scratch,
                             double* grad_f, double* grad_tau) {
  if (nray <= 0) return;
  raytrace_adjoint_kernel<<<(nray + 31) / 32, 32, 0, st>>>(rays, nray, g, f_cell, tau_cell, gpsi, geu,
                                                           reinterpret_cast<SegRec*>(scratch), grad_f, grad_tau);
}

}  // namespace dlra
