// Uncollided transport with energy straggling along the rays of one beam (Sec. 3.2), on the GPU:
// the stand-alone entry point dlra_straggling_trace. The host builds the beam's transverse rays
// (spot grid of pitch min(delta)/4 within 3.5 sigma, Gaussian weights normalised to a unit beam;
// the energy spread is carried by the initial energy distribution), walks each ray through the
// voxel grid into segments, and builds the energy-DG tables (dlra_straggling_tables), the
// projections int_e S_w P_j dE of the water stopping power, the overlaps of every element with
// the K energy bins and the initial distribution. One device thread marches one ray through its
// segments (Crank-Nicolson, block Thomas factorisation per segment, FP64, work space in global
// memory) and adds the segment's energy lost to slowing down to e_u(cell) and its track integral
// over every energy bin to psi(k, cell), with the definitions of the CSDA ray tracer.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <vector>

#include "dlra.h"
#include "straggling_march.cuh"
#include "tables.h"

namespace dlra {
void set_context_free_error(const char* msg);

namespace {

using strag::kMaxBinsPerElem;
using strag::MarchTables;

// Upper bound on the Crank-Nicolson steps of one ray (sum over its segments of ceil(len / h_max)):
// a 40 cm ray at h_max = 0.001 cm takes 4e4.
constexpr double kMaxStepsPerRay = 1.0e6;

__global__ void __launch_bounds__(64) straggling_march_kernel(int nray, const int* __restrict__ seg_ptr,
                                                            const int* __restrict__ seg_cell,
                                                            const double* __restrict__ seg_len,
                                                            const double* __restrict__ ray_w, MarchTables t,
                                                            const double* __restrict__ f_cell,
                                                            const double* __restrict__ tau_cell, double* scratch,
                                                            double* __restrict__ psi, double* __restrict__ e_u) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nray) return;
  strag::march_ray(r, seg_ptr, seg_cell, seg_len, ray_w, t, f_cell, tau_cell, scratch, psi, e_u, strag::AddTo{});
}

// Voxel segments (cell, length) of the ray o + s v through the box [0, L]^3 (x-z slab: y
// ignored), in order along the ray; segments shorter than 1e-14 cm are dropped.
void ray_segments(const double o[3], const double v[3], const dlra_straggling_trace_args& a, bool two_d,
                  std::vector<int>& cells, std::vector<double>& lens) {
  const double Lx[3] = {a.nx * a.dx, a.ny * (two_d ? 1.0 : a.dy), a.nz * a.dz};
  const double dl[3] = {a.dx, two_d ? 1.0 : a.dy, a.dz};
  const int nd[3] = {a.nx, a.ny, a.nz};
  double t0 = 0.0, t1 = INFINITY;
  for (int ax = 0; ax < 3; ++ax) {
    if (two_d && ax == 1) continue;
    if (std::fabs(v[ax]) < 1e-300) {
      if (o[ax] < 0.0 || o[ax] > Lx[ax]) return;
      continue;
    }
    const double ta = (0.0 - o[ax]) / v[ax], tb = (Lx[ax] - o[ax]) / v[ax];
    t0 = std::max(t0, std::min(ta, tb));
    t1 = std::min(t1, std::max(ta, tb));
  }
  if (!(t1 > t0)) return;
  std::vector<double> ts = {t0, t1};
  for (int ax = 0; ax < 3; ++ax) {
    if ((two_d && ax == 1) || std::fabs(v[ax]) < 1e-300) continue;
    for (int p = 0; p <= nd[ax]; ++p) {
      const double tp = (p * dl[ax] - o[ax]) / v[ax];
      if (tp > t0 && tp < t1) ts.push_back(tp);
    }
  }
  std::sort(ts.begin(), ts.end());
  ts.erase(std::unique(ts.begin(), ts.end()), ts.end());
  for (size_t q = 0; q + 1 < ts.size(); ++q) {
    const double ta = ts[q], tb = ts[q + 1];
    if (tb - ta <= 1e-14) continue;
    const double tm = 0.5 * (ta + tb);
    const int i = std::min(std::max((int)std::floor((o[0] + tm * v[0]) / a.dx), 0), a.nx - 1);
    const int k = std::min(std::max((int)std::floor((o[2] + tm * v[2]) / a.dz), 0), a.nz - 1);
    const int j = two_d ? 0 : std::min(std::max((int)std::floor((o[1] + tm * v[1]) / a.dy), 0), a.ny - 1);
    cells.push_back((k * a.ny + j) * a.nx + i);
    lens.push_back(tb - ta);
  }
}

struct HostTrace {
  int G = 0, K = 0;
  long long n = 0;
  std::vector<double> mass, adv, sipg, rem, SW, c0, bw, seg_len, ray_w;
  std::vector<int> bin0, nbin, seg_ptr, seg_cell;
  double inv_v = 0.0, inv_vh = 0.0;
};

// Host side of the trace: checks the arguments and builds the tables, the rays and their
// segments.
dlra_status prepare_trace(const dlra_straggling_trace_args& a, HostTrace& h) {
  const bool two_d = a.ny == 1 && a.dy == 0.0;
  const long long n = (long long)a.nx * a.ny * a.nz;
  if (a.nx < 1 || a.ny < 1 || a.nz < 1 || !(a.dx > 0) || !(a.dz > 0) || !(two_d || a.dy > 0) || n >= (1LL << 31) ||
      a.n_bins < 1 || a.n_elem < 1 || a.n_elem > 4096 || !(a.h_max > 0) || !(a.e_min > 0) || !(a.e_max > a.e_min) ||
      !(a.energy > a.e_min) || a.energy > a.e_max + 1e-12 || !(a.energy_sigma >= 0) || !(a.spot_sigma >= 0) ||
      !a.f_cell || !a.tau_cell || !a.psi || !a.e_u) {
    set_context_free_error("bad straggling-trace arguments");
    return DLRA_ERR_ARG;
  }
  const int G = a.n_elem, K = a.n_bins;
  const double D = (a.e_max - a.e_min) / G, hb = (a.e_max - a.e_min) / K;
  // energy-DG tables
  dlra_straggling_args ta{a.e_min, a.e_max, G, a.bk_p, a.bk_alpha, a.t100, a.straggling};
  std::vector<double> mass(3 * G), adv((size_t)G * 27), sipg((size_t)G * 27), rem((size_t)G * 27);
  dlra_status s = dlra_straggling_tables(&ta, mass.data(), adv.data(), sipg.data(), rem.data());
  if (s != DLRA_OK) return s;
  double xq[6], wq[6];
  gauss_legendre(6, xq, wq);
  auto legendre = [](double xi, double P[3]) {
    P[0] = 1.0;
    P[1] = xi;
    P[2] = 0.5 * (3.0 * xi * xi - 1.0);
  };
  std::vector<double> SW(3 * G, 0.0), c0(3 * G, 0.0);
  for (int e = 0; e < G; ++e) {
    const double Ec = a.e_min + (e + 0.5) * D;
    for (int q = 0; q < 6; ++q) {
      const double E = Ec + 0.5 * D * xq[q], w = 0.5 * D * wq[q];
      double P[3];
      legendre(xq[q], P);
      const double S = std::pow(E, 1.0 - a.bk_p) / (a.bk_p * a.bk_alpha);
      for (int j = 0; j < 3; ++j) SW[3 * e + j] += w * S * P[j];
      if (a.energy_sigma > 0) {
        const double z = (E - a.energy) / a.energy_sigma;
        const double g = std::exp(-0.5 * z * z) / (std::sqrt(2.0 * M_PI) * a.energy_sigma);
        for (int j = 0; j < 3; ++j) c0[3 * e + j] += w * g * P[j] / mass[3 * e + j];
      }
    }
  }
  if (a.energy_sigma > 0) {
    double num = 0.0;
    for (int e = 0; e < G; ++e) num += c0[3 * e] * D;
    for (double& v : c0) v /= num;
  } else {
    const int e = std::min(std::max((int)((a.energy - a.e_min) / D), 0), G - 1);
    const double xi = (a.energy - (a.e_min + (e + 0.5) * D)) / (0.5 * D);
    double P[3];
    legendre(xi, P);
    for (int j = 0; j < 3; ++j) c0[3 * e + j] = P[j] / mass[3 * e + j];
  }
  // overlaps of element e with bin k = [E_{k+1}, E_k], E_k = e_max - k hb: int P_j dE
  std::vector<int> bin0(G), nbin(G);
  std::vector<double> bw((size_t)G * kMaxBinsPerElem * 3, 0.0);
  for (int e = 0; e < G; ++e) {
    const double lo = a.e_min + e * D, hi = lo + D;
    int kf = std::max(0, (int)std::floor((a.e_max - hi) / hb + 1e-12));
    int kl = std::min(K - 1, (int)std::floor((a.e_max - lo) / hb - 1e-12));
    if (kl < kf) kl = kf;
    if (kl - kf + 1 > kMaxBinsPerElem) {
      set_context_free_error("more than 8 energy bins per element: use more elements");
      return DLRA_ERR_ARG;
    }
    bin0[e] = kf;
    nbin[e] = kl - kf + 1;
    const double Ec = lo + 0.5 * D;
    for (int k = kf; k <= kl; ++k) {
      const double blo = std::max(lo, a.e_max - (k + 1) * hb), bhi = std::min(hi, a.e_max - k * hb);
      if (!(bhi > blo)) continue;
      const double xa = (blo - Ec) / (0.5 * D), xb = (bhi - Ec) / (0.5 * D);
      // antiderivatives of P_0, P_1, P_2: xi, xi^2/2, (xi^3 - xi)/2
      const double pr[3] = {xb - xa, 0.5 * (xb * xb - xa * xa), 0.5 * ((xb * xb * xb - xb) - (xa * xa * xa - xa))};
      for (int j = 0; j < 3; ++j) bw[((size_t)e * kMaxBinsPerElem + (k - kf)) * 3 + j] = 0.5 * D * pr[j];
    }
  }
  // transverse rays of the beam (unit beam weight)
  double d[3] = {a.dir[0], a.dir[1], a.dir[2]};
  const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (!(dn > 0.0) || (two_d && std::fabs(d[1]) > 1e-12)) {
    set_context_free_error("bad beam direction");
    return DLRA_ERR_ARG;
  }
  for (double& v : d) v /= dn;
  double u1[3], u2[3] = {0, 0, 0};
  if (two_d) {
    const double l = std::sqrt(d[2] * d[2] + d[0] * d[0]);
    u1[0] = d[2] / l;
    u1[1] = 0.0;
    u1[2] = -d[0] / l;
  } else {
    double er[3] = {0, 1, 0};
    if (std::fabs(d[1]) >= 0.9) {
      er[0] = 1;
      er[1] = 0;
    }
    u1[0] = er[1] * d[2] - er[2] * d[1];
    u1[1] = er[2] * d[0] - er[0] * d[2];
    u1[2] = er[0] * d[1] - er[1] * d[0];
    const double l = std::sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    for (double& v : u1) v /= l;
    u2[0] = d[1] * u1[2] - d[2] * u1[1];
    u2[1] = d[2] * u1[0] - d[0] * u1[2];
    u2[2] = d[0] * u1[1] - d[1] * u1[0];
  }
  const double pitch = two_d ? std::min(a.dx, a.dz) / 4.0 : std::min(a.dx, std::min(a.dy, a.dz)) / 4.0;
  std::vector<double> offs, gw;
  if (a.spot_sigma > 0.0) {
    const int nh = (int)std::ceil(3.5 * a.spot_sigma / pitch);
    for (int j = -nh; j < nh; ++j) {
      const double o = (j + 0.5) * pitch;
      offs.push_back(o);
      gw.push_back(std::exp(-0.5 * (o / a.spot_sigma) * (o / a.spot_sigma)));
    }
  } else {
    offs.push_back(0.0);
    gw.push_back(1.0);
  }
  std::vector<std::array<double, 3>> pts;
  std::vector<double> pw;
  double wsum = 0.0;
  for (size_t i = 0; i < offs.size(); ++i) {
    if (two_d) {
      pts.push_back({a.pos[0] + offs[i] * u1[0], a.pos[1] + offs[i] * u1[1], a.pos[2] + offs[i] * u1[2]});
      pw.push_back(gw[i]);
      wsum += gw[i];
    } else {
      for (size_t j = 0; j < offs.size(); ++j) {
        std::array<double, 3> p;
        for (int q = 0; q < 3; ++q) p[q] = a.pos[q] + offs[i] * u1[q] + offs[j] * u2[q];
        pts.push_back(p);
        pw.push_back(gw[i] * gw[j]);
        wsum += gw[i] * gw[j];
      }
    }
  }
  std::vector<int> seg_ptr(1, 0), seg_cell;
  std::vector<double> seg_len, ray_w;
  for (size_t r = 0; r < pts.size(); ++r) {
    std::vector<int> cells;
    std::vector<double> lens;
    ray_segments(pts[r].data(), d, a, two_d, cells, lens);
    if (cells.empty()) continue;
    // Crank-Nicolson steps of this ray: one device thread takes them one after the other, so a
    // step length far below the voxel size would keep that thread busy for minutes
    double steps = 0.0;
    for (double l : lens) steps += std::max(1.0, std::ceil(l / a.h_max - 1e-12));
    if (steps > kMaxStepsPerRay) {
      char msg[200];
      std::snprintf(msg, sizeof msg,
                    "straggling trace: h_max = %g cm gives %.0f Crank-Nicolson steps on one ray (limit %.0f)", a.h_max,
                    steps, kMaxStepsPerRay);
      set_context_free_error(msg);
      return DLRA_ERR_ARG;
    }
    seg_cell.insert(seg_cell.end(), cells.begin(), cells.end());
    seg_len.insert(seg_len.end(), lens.begin(), lens.end());
    seg_ptr.push_back((int)seg_cell.size());
    ray_w.push_back(pw[r] / wsum);
  }
  h.G = G;
  h.K = K;
  h.n = n;
  h.mass = std::move(mass);
  h.adv = std::move(adv);
  h.sipg = std::move(sipg);
  h.rem = std::move(rem);
  h.SW = std::move(SW);
  h.c0 = std::move(c0);
  h.bin0 = std::move(bin0);
  h.nbin = std::move(nbin);
  h.bw = std::move(bw);
  h.seg_ptr = std::move(seg_ptr);
  h.seg_cell = std::move(seg_cell);
  h.seg_len = std::move(seg_len);
  h.ray_w = std::move(ray_w);
  const double vol = a.dx * (two_d ? 1.0 : a.dy) * a.dz;
  h.inv_v = 1.0 / vol;
  h.inv_vh = 1.0 / (vol * hb);
  return DLRA_OK;
}

}  // namespace
}  // namespace dlra

extern "C" dlra_status dlra_straggling_trace(const dlra_straggling_trace_args* args) {
  using namespace dlra;
  if (!args) {
    set_context_free_error("null arguments");
    return DLRA_ERR_ARG;
  }
  const dlra_straggling_trace_args& a = *args;
  HostTrace h;
  dlra_status s = prepare_trace(a, h);
  if (s != DLRA_OK) return s;
  cudaStream_t st = (cudaStream_t)a.cuda_stream;
  const int G = h.G, K = h.K;
  const long long n = h.n;
  const int nray = (int)h.ray_w.size();
  cudaError_t err = cudaMemsetAsync(a.psi, 0, sizeof(double) * (size_t)K * n, st);
  if (err == cudaSuccess) err = cudaMemsetAsync(a.e_u, 0, sizeof(double) * n, st);
  if (err != cudaSuccess || nray == 0) {
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) {
      set_context_free_error("straggling trace: CUDA error");
      return DLRA_ERR_CUDA;
    }
    return DLRA_OK;
  }
  // device copies: tables, rays, work space (one slice per ray)
  const size_t per_ray = strag::work_per_ray(G);
  std::vector<void*> bufs;
  cudaError_t copy_err = cudaSuccess;
  auto dev = [&](const void* src, size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    if (src) {
      const cudaError_t e = cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess && copy_err == cudaSuccess) copy_err = e;
    }
    return p;
  };
  MarchTables t;
  t.G = G;
  t.K = K;
  t.n = (int)n;
  t.mass = (const double*)dev(h.mass.data(), sizeof(double) * h.mass.size());
  t.adv = (const double*)dev(h.adv.data(), sizeof(double) * h.adv.size());
  t.sipg = (const double*)dev(h.sipg.data(), sizeof(double) * h.sipg.size());
  t.rem = (const double*)dev(h.rem.data(), sizeof(double) * h.rem.size());
  t.SW = (const double*)dev(h.SW.data(), sizeof(double) * h.SW.size());
  t.bin0 = (const int*)dev(h.bin0.data(), sizeof(int) * h.bin0.size());
  t.nbin = (const int*)dev(h.nbin.data(), sizeof(int) * h.nbin.size());
  t.bw = (const double*)dev(h.bw.data(), sizeof(double) * h.bw.size());
  t.c0 = (const double*)dev(h.c0.data(), sizeof(double) * h.c0.size());
  t.inv_v = h.inv_v;
  t.inv_vh = h.inv_vh;
  t.h_max = a.h_max;
  const int* d_ptr = (const int*)dev(h.seg_ptr.data(), sizeof(int) * h.seg_ptr.size());
  const int* d_cell = (const int*)dev(h.seg_cell.data(), sizeof(int) * h.seg_cell.size());
  const double* d_len = (const double*)dev(h.seg_len.data(), sizeof(double) * h.seg_len.size());
  const double* d_w = (const double*)dev(h.ray_w.data(), sizeof(double) * h.ray_w.size());
  double* scratch = (double*)dev(nullptr, sizeof(double) * per_ray * nray);
  bool ok = t.mass && t.adv && t.sipg && t.rem && t.SW && t.bin0 && t.nbin && t.bw && t.c0 && d_ptr && d_cell &&
            d_len && d_w && scratch;
  if (ok && copy_err != cudaSuccess) err = copy_err;
  if (ok && err == cudaSuccess) {
    straggling_march_kernel<<<(nray + 63) / 64, 64, 0, st>>>(nray, d_ptr, d_cell, d_len, d_w, t, a.f_cell,
                                                             a.tau_cell, scratch, a.psi, a.e_u);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  }
  for (void* p : bufs) cudaFree(p);
  if (!ok) {
    cudaGetLastError();
    set_context_free_error("straggling trace: cudaMalloc failed");
    return DLRA_ERR_OOM;
  }
  if (err != cudaSuccess) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "straggling trace failed: %s", cudaGetErrorString(err));
    set_context_free_error(buf);
    return DLRA_ERR_CUDA;
  }
  return DLRA_OK;
}
