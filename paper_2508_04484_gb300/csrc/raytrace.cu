// CSDA ray tracer for the uncollided flux (Sec. 3.2 without straggling), FP64.
// One thread per ray: an Amanatides-Woo voxel walk; per voxel segment the energy
// follows from the water range R_w(E) = alpha E^p, which decreases by f(x) per cm
// (S(x, E) = f(x) S_w(E)); the particle weight decays with Sigma_t(x, E) =
// tau(x) T_w(E)/2, whose integral along the ray has the closed form
// (tau/f) (Lam(E) - Lam(E_in)), Lam(E) = klam E^(p-2) / (2 - p). Each segment is split
// at the energy-grid nodes and its track length and energy loss are integrated in E
// (6-point Gauss-Legendre) into the bin-averaged fluence and the uncollided deposit.
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

__global__ void raytrace_kernel(const double* __restrict__ rays, int nray, RayGeo g,
                                const double* __restrict__ f_cell, const double* __restrict__ tau_cell,
                                double* __restrict__ psi, double* __restrict__ e_u) {
  const int rid = blockIdx.x * blockDim.x + threadIdx.x;
  if (rid >= nray) return;
  const double* ry = rays + 8 * (long long)rid;
  const double o[3] = {ry[0], ry[1], ry[2]};
  const double v[3] = {ry[3], ry[4], ry[5]};
  const double E0 = ry[6], wr = ry[7];
  const double Lb[3] = {g.nx * g.dx, g.ny * g.dy, g.nz * g.dz};
  const double dd[3] = {g.dx, g.dy, g.dz};
  const int nd[3] = {g.nx, g.ny, g.nz};
  const long long n = (long long)g.nx * g.ny * g.nz;
  double t0 = 0.0, t1 = 1e300;
  for (int a = 0; a < 3; ++a) {
    if (a == 1 && g.two_d) continue;
    if (fabs(v[a]) < 1e-300) {
      if (o[a] < 0.0 || o[a] > Lb[a]) return;
      continue;
    }
    double ta = (0.0 - o[a]) / v[a], tb = (Lb[a] - o[a]) / v[a];
    t0 = fmax(t0, fmin(ta, tb));
    t1 = fmin(t1, fmax(ta, tb));
  }
  if (!(t1 > t0)) return;
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
          atomicAdd(psi + (long long)k * n + cell, wr * Is * inv_vh);
          atomicAdd(e_u + cell, wr * Ie / g.volume);
          N = Nn;
        }
        Ecur = Elo;
        ++k;
      }
      R = Rb;
      if (stop) return;
    }
    if (tn >= t1) return;
    int a = 0;
    if (tmax[1] < tmax[a]) a = 1;
    if (tmax[2] < tmax[a]) a = 2;
    idx[a] += stp[a];
    if (idx[a] < 0 || idx[a] >= nd[a]) return;
    t = tn;
    tmax[a] += tdel[a];
  }
}

void launch_raytrace(cudaStream_t st, const double* rays, int nray, RayGeo g, const double* f_cell,
                     const double* tau_cell, double* psi, double* e_u) {
  if (nray <= 0) return;
  // few, long-running threads: small blocks spread the rays over all SMs
  raytrace_kernel<<<(nray + 31) / 32, 32, 0, st>>>(rays, nray, g, f_cell, tau_cell, psi, e_u);
}

}  // namespace dlra
