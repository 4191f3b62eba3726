// Stencil Gram on the tensor cores (FP32 path), the contraction of the S-step and L-step
// Galerkin blocks (Sec. 3.3.2-3.3.3):
//   G_k[a][b] = sum_i A(i, a) D_k(rho^-1 B(:, b))(i),   k = 2 da + s,
// written as D[j][a] = sum_t S[j][t] A[t][a] with j = k nb + b and the cells t as the
// contraction index. A CTA owns a slice of up to 256 rows j (two 128-row MMA tiles, TMEM
// lanes = j, TMEM columns = a) and walks a contiguous run of 32-cell chunks of the grid: its
// warps form the stencil values S of the chunk (where nx % 4 == 0 a lane takes four
// x-consecutive cells of one column from eleven float4 loads of the column and of rho^-1;
// otherwise one cell per lane from per-lane neighbour tables), split them and the chunk's A
// rows into TF32 high and low parts and store both K-major in shared memory; one thread (of
// the last warp, which forms no stencil values on the float4 path) issues three
// tcgen05.mma kind::tf32 per 8-cell K-slice (hi*hi + hi*lo + lo*hi, FP32-accurate products,
// FP32 accumulation in tensor memory). Two operand buffers: the next chunk is staged while the
// tensor core reads the current one. The slice's partial sums are added to the FP64 output
// with one atomic per entry at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace dlra {

namespace {

constexpr int GT_TC = 32;  // cells per chunk: four K-slices of 8

struct GsTcShape {
  int NP;       // MMA N: na rounded up to 16
  int MT;       // 128-row MMA tiles per slice
  int tcols;    // TMEM columns (power of two, >= 32)
  int nslice;   // slices of j (grid y)
  size_t smem;  // dynamic shared memory
};

GsTcShape gs_tc_shape(int na, int nj) {
  GsTcShape s;
  s.NP = (na + 15) / 16 * 16;
  s.MT = nj > 128 ? 2 : 1;
  s.nslice = (nj + 255) / 256;
  s.tcols = 32;
  while (s.tcols < s.MT * s.NP) s.tcols *= 2;
  const size_t buf = (size_t)2 * s.MT * 128 * GT_TC + (size_t)2 * s.NP * GT_TC;
  s.smem = 2 * buf * sizeof(float);
  return s;
}

constexpr int GT_THREADS = 512;  // 16 warps: four per 8-cell group of the chunk

// This lane's cell of the chunk: the linear offsets of the 12 stencil neighbours and rho^-1
// at the 13 points (0 outside the grid or beyond the last cell, so that ghost layers and the
// ragged tail read zeros without branches). Direction list fixed at compile time: x, y, z, or
// x, z on a slab.
template <int NACT>
struct CellStencil {
  int off[4 * NACT];
  float rr[1 + 4 * NACT];
  __device__ __forceinline__ void init(long long r, long long rows, const float* __restrict__ inv_rho, const Geo& g) {
#pragma unroll
    for (int p = 0; p < 4 * NACT; ++p) off[p] = 0;
#pragma unroll
    for (int p = 0; p < 1 + 4 * NACT; ++p) rr[p] = 0.f;
    if (r >= rows) return;
    const int ri = (int)r, nxy = (int)g.nxy;
    const int iz = ri / nxy, rem = ri - iz * nxy;
    const int iy = rem / g.nx, ix = rem - iy * g.nx;
    rr[0] = inv_rho[r];
#pragma unroll
    for (int da = 0; da < NACT; ++da) {
      const int d = NACT == 3 ? da : (da == 0 ? 0 : 2);
      const int c = d == 0 ? ix : (d == 1 ? iy : iz);
      const int L = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
      const int st = d == 0 ? 1 : (d == 1 ? g.nx : nxy);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int delta = q == 0 ? -1 : (q == 1 ? -2 : (q == 2 ? 1 : 2));
        if (c + delta >= 0 && c + delta < L) {
          off[4 * da + q] = delta * st;
          rr[1 + 4 * da + q] = inv_rho[r + delta * st];
        }
      }
    }
  }
};

// One lane's float4 stencil inputs: four x-consecutive cells (a quad; nx % 4 == 0) of column b,
// the quads on either side along x and the quads one and two cells away along y and z, each
// with rho^-1. Every load is issued unconditionally (from the centre quad where the neighbour
// lies outside the grid, masked to zero afterwards), so that all of them are in flight at once.
template <int NACT>
struct QuadIn {
  static constexpr int NPOS = 3 + 4 * (NACT - 1);  // centre, x -4 / +4, then -1, -2, +1, +2 per y / z
  float4 vb[NPOS], vr[NPOS];
  unsigned valid;
  int b, q;
  bool store;
  __device__ __forceinline__ void load(int it, int nb, int Bact, long long r0, long long rows,
                                       const float* __restrict__ B, long long ldb,
                                       const float* __restrict__ inv_rho, const Geo& g, int lane) {
    b = (it >> 1) * 8 + (lane & 7);
    q = (it & 1) * 4 + (lane >> 3);
    const long long rq = r0 + 4 * q;
    store = b < Bact;
    const bool in = store && rq < rows;
    const long long rc = in ? rq : 0;
    const int ri = (int)rc, nxy = (int)g.nxy;
    const int iz = ri / nxy, rem = ri - iz * nxy;
    const int iy = rem / g.nx, ix = rem - iy * g.nx;
    int off[NPOS];
    valid = in ? 1u : 0u;
    off[0] = 0;
    const bool xm = in && ix >= 4, xp = in && ix + 4 < g.nx;
    off[1] = xm ? -4 : 0;
    off[2] = xp ? 4 : 0;
    valid |= (xm ? 2u : 0u) | (xp ? 4u : 0u);
#pragma unroll
    for (int da = 1; da < NACT; ++da) {
      const int d = NACT == 3 ? da : 2;
      const int c = d == 1 ? iy : iz, L = d == 1 ? g.ny : g.nz;
      const int st = d == 1 ? g.nx : nxy;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int delta = s == 0 ? -1 : (s == 1 ? -2 : (s == 2 ? 1 : 2));
        const bool ok = in && c + delta >= 0 && c + delta < L;
        const int p = 3 + 4 * (da - 1) + s;
        off[p] = ok ? delta * st : 0;
        valid |= ok ? (1u << p) : 0u;
      }
    }
    const float* col = B + (long long)(store ? b : 0) * ldb + rc;
    const float* rho = inv_rho + rc;
#pragma unroll
    for (int p = 0; p < NPOS; ++p) {
      vb[p] = *reinterpret_cast<const float4*>(col + off[p]);
      vr[p] = *reinterpret_cast<const float4*>(rho + off[p]);
    }
  }
  // sv[k][i]: stencil k = 2 da + s of cell i of the quad
  template <int NK>
  __device__ __forceinline__ void stencils(const float* inv2, float (&sv)[NK][4]) const {
    float4 v[NPOS];
#pragma unroll
    for (int p = 0; p < NPOS; ++p) {
      const bool ok = (valid >> p) & 1u;
      v[p] = ok ? make_float4(vb[p].x * vr[p].x, vb[p].y * vr[p].y, vb[p].z * vr[p].z, vb[p].w * vr[p].w)
                : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float4 c = v[0];
    {
      const float w[8] = {v[1].z, v[1].w, c.x, c.y, c.z, c.w, v[2].x, v[2].y};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        sv[0][i] = (-3.f * w[i + 2] + 4.f * w[i + 1] - w[i]) * inv2[0];
        sv[1][i] = (3.f * w[i + 2] - 4.f * w[i + 3] + w[i + 4]) * inv2[0];
      }
    }
#pragma unroll
    for (int da = 1; da < NACT; ++da) {
      const int p = 3 + 4 * (da - 1);
      const float4 m1 = v[p], m2 = v[p + 1], p1 = v[p + 2], p2 = v[p + 3];
      const float iv = inv2[da];
      sv[2 * da][0] = (-3.f * c.x + 4.f * m1.x - m2.x) * iv;
      sv[2 * da][1] = (-3.f * c.y + 4.f * m1.y - m2.y) * iv;
      sv[2 * da][2] = (-3.f * c.z + 4.f * m1.z - m2.z) * iv;
      sv[2 * da][3] = (-3.f * c.w + 4.f * m1.w - m2.w) * iv;
      sv[2 * da + 1][0] = (3.f * c.x - 4.f * p1.x + p2.x) * iv;
      sv[2 * da + 1][1] = (3.f * c.y - 4.f * p1.y + p2.y) * iv;
      sv[2 * da + 1][2] = (3.f * c.z - 4.f * p1.z + p2.z) * iv;
      sv[2 * da + 1][3] = (3.f * c.w - 4.f * p1.w + p2.w) * iv;
    }
  }
};

template <int NACT, bool VEC>
__global__ void __launch_bounds__(GT_THREADS, 1) gram_stencil_tc_kernel(
    long long rows, const float* __restrict__ A, long long lda, int na, const int* adim, const float* __restrict__ B,
    long long ldb, int nb, const int* bdim, const float* __restrict__ inv_rho, Geo g, int NP, int MT, int tcols,
    int a_vec, double* __restrict__ out, int ldj, long long ldo, int* err) {
  constexpr int NK = 2 * NACT;
  constexpr int NPT = 1 + 4 * NACT;  // stencil points
  constexpr int NW = GT_THREADS / 32;
  extern __shared__ __align__(1024) unsigned char raw[];
  float* base = reinterpret_cast<float*>(raw);
  const int SROWS = MT * 128;
  const int BUF = 2 * SROWS * GT_TC + 2 * NP * GT_TC;  // floats per operand buffer
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tslot, (uint32_t)tcols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_fence_init();
    s_bad = 0;
  }
  // rows j beyond the slice's last entry and padded a read zeros, never stale data
  for (int e = tid; e < 2 * BUF; e += GT_THREADS) base[e] = 0.f;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const int Aact = dev_dim(adim, na), Bact = dev_dim(bdim, nb);
  float inv2[NACT];
#pragma unroll
  for (int da = 0; da < NACT; ++da) inv2[da] = (float)g.inv2d[NACT == 3 ? da : (da == 0 ? 0 : 2)];
  const int nj = NK * nb;
  const int j0 = blockIdx.y * 256;
  const uint32_t idesc = tc::idesc_tf32(128, NP);
  const uint32_t sLBO = (128 / 8) * 128, aLBO = (uint32_t)(NP / 8) * 128;
  const long long nchunks = (rows + GT_TC - 1) / GT_TC;
  const int ag = NP >> 3;         // 8-row groups of a
  const int nbq = (nb + 3) >> 2;  // column quads of b
  // float4 path: the last warp only issues the MMAs (it forms no stencil values), so that the
  // issue never delays a staging warp; the other warps take the stencil items
  const int nbo = (nb + 7) >> 3;
  const int sw = VEC ? NW - 1 : NW;  // staging warps
  const int issuer = VEC ? (NW - 1) * 32 : 0;
  // S staging: warp w covers cells t = 8 (w % 4) + lane / 4 and the column quads w / 4, w / 4 + 4, ...
  const int t = 8 * (warp & 3) + (lane >> 2);
  const int bq0 = warp >> 2;
  bool alive = true;
  int u = 0;
  // a contiguous run of chunks per CTA: the y neighbours of a chunk were loaded by the
  // chunks just before it and are still in L1
  const long long per = (nchunks + gridDim.x - 1) / gridDim.x;
  const long long c_end = min(nchunks, (long long)(blockIdx.x + 1) * per);
  for (long long ch = (long long)blockIdx.x * per; ch < c_end; ++ch, ++u) {
    const int bsel = u & 1;
    float* Shi = base + bsel * BUF;
    float* Slo = Shi + SROWS * GT_TC;
    float* Ahi = Slo + SROWS * GT_TC;
    float* Alo = Ahi + NP * GT_TC;
    const long long r0 = ch * GT_TC;
    CellStencil<NACT> cs;
    if (!VEC) cs.init(r0 + t, rows, inv_rho, g);
    // A rows of the chunk, item (a, quad q of 4 cells), at most two per thread (NP <= 128);
    // 8 consecutive a fill one core matrix. Loads now, stores once the buffer is free.
    float4 av[2];
    int ao[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + h * GT_THREADS;
      av[h] = make_float4(0.f, 0.f, 0.f, 0.f);
      ao[h] = -1;
      if (e < NP * (GT_TC / 4)) {
        const int a = (e & 7) + 8 * ((e >> 3) % ag), q = (e >> 3) / ag;
        const long long rq = r0 + 4 * q;
        ao[h] = tc::kmajor(a, 4 * q, NP);
        if (a < Aact) {
          const float* src = A + (long long)a * lda + rq;
          if (a_vec && rq + 3 < rows) {
            av[h] = *reinterpret_cast<const float4*>(src);
          } else {
            av[h].x = rq < rows ? src[0] : 0.f;
            av[h].y = rq + 1 < rows ? src[1] : 0.f;
            av[h].z = rq + 2 < rows ? src[2] : 0.f;
            av[h].w = rq + 3 < rows ? src[3] : 0.f;
          }
        }
      }
    }
    // float4 stencil path: this warp's first item is loaded before the wait
    QuadIn<NACT> qin;
    if (VEC && warp < sw && warp < 2 * nbo) qin.load(warp, nb, Bact, r0, rows, B, ldb, inv_rho, g, lane);
    // the buffer is free once the MMAs of chunk u - 2 (its previous use) are done
    if (u >= 2 && !tc::mbar_wait(&mbar[bsel], (uint32_t)(((u - 2) >> 1) & 1), tc::kWaitLimit)) alive = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (ao[h] < 0) continue;
      float4 hi, lo;
      tc::split_tf32(av[h].x, hi.x, lo.x);
      tc::split_tf32(av[h].y, hi.y, lo.y);
      tc::split_tf32(av[h].z, hi.z, lo.z);
      tc::split_tf32(av[h].w, hi.w, lo.w);
      *reinterpret_cast<float4*>(Ahi + ao[h]) = hi;
      *reinterpret_cast<float4*>(Alo + ao[h]) = lo;
    }
    if (VEC) {
      // four x-consecutive cells per lane (nx % 4 == 0, so a quad never straddles a row): eleven
      // float4 loads of the column and of rho^-1 give its 13-point stencils, and each of the nk
      // values of the quad is one 16-byte store (four consecutive K of a core-matrix row).
      // Item (column octet, half of the chunk): lanes = 8 columns x 4 quads.
      for (int it = warp; warp < sw && it < 2 * nbo; it += sw) {
        if (it != warp) qin.load(it, nb, Bact, r0, rows, B, ldb, inv_rho, g, lane);
        if (!qin.store) continue;
        float sv[NK][4];
        qin.stencils(inv2, sv);
#pragma unroll
        for (int k = 0; k < NK; ++k) {
          const int jl = k * nb + qin.b - j0;
          if (jl < 0 || jl >= SROWS) continue;
          float4 h, l;
          tc::split_tf32(sv[k][0], h.x, l.x);
          tc::split_tf32(sv[k][1], h.y, l.y);
          tc::split_tf32(sv[k][2], h.z, l.z);
          tc::split_tf32(sv[k][3], h.w, l.w);
          const int o = (jl >> 7) * (128 * GT_TC) + tc::kmajor(jl & 127, 4 * qin.q, 128);
          *reinterpret_cast<float4*>(Shi + o) = h;
          *reinterpret_cast<float4*>(Slo + o) = l;
        }
      }
    } else
    // S rows: the nk stencil values of column b at cell t go to rows j = k nb + b of the slice;
    // two column quads per pass, their 26 loads issued before any use
    for (int bq = bq0; bq < nbq; bq += 8) {
      float v[2][NPT];
      int bb[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int b = (bq + 4 * h) * 4 + (lane & 3);
        bb[h] = (bq + 4 * h < nbq && b < Bact) ? b : -1;
        const float* col = B + (long long)(bb[h] >= 0 ? b : 0) * ldb + (r0 + t < rows ? r0 + t : 0);
        const bool ld = bb[h] >= 0 && r0 + t < rows;
        v[h][0] = ld ? col[0] : 0.f;
#pragma unroll
        for (int p = 1; p < NPT; ++p) v[h][p] = ld ? col[cs.off[p - 1]] : 0.f;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (bb[h] < 0) continue;
        const float v0 = v[h][0] * cs.rr[0];
#pragma unroll
        for (int da = 0; da < NACT; ++da) {
          const int p = 1 + 4 * da;
          const float vm1 = v[h][p] * cs.rr[p], vm2 = v[h][p + 1] * cs.rr[p + 1];
          const float vp1 = v[h][p + 2] * cs.rr[p + 2], vp2 = v[h][p + 3] * cs.rr[p + 3];
          const float sv[2] = {(-3.f * v0 + 4.f * vm1 - vm2) * inv2[da], (3.f * v0 - 4.f * vp1 + vp2) * inv2[da]};
#pragma unroll
          for (int s2 = 0; s2 < 2; ++s2) {
            const int jl = (2 * da + s2) * nb + bb[h] - j0;
            if (jl < 0 || jl >= SROWS) continue;
            float hi, lo;
            tc::split_tf32(sv[s2], hi, lo);
            const int o = (jl >> 7) * (128 * GT_TC) + tc::kmajor(jl & 127, t, 128);
            Shi[o] = hi;
            Slo[o] = lo;
          }
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    // a timeout anywhere stops the whole block at the same point
    if (!__syncthreads_and(alive)) {
      alive = false;
      break;
    }
    if (tid == issuer) {
      tc::fence_after();
      // a K-slice further is a fixed byte offset: added to the descriptors' address field
      // (addresses stay below 256 KB, so the 14-bit field never carries)
      const uint64_t dAh = tc::smem_desc(tc::su32(Ahi), aLBO, 128), dAl = tc::smem_desc(tc::su32(Alo), aLBO, 128);
      for (int mt = 0; mt < MT; ++mt) {
        const uint64_t dSh = tc::smem_desc(tc::su32(Shi + mt * 128 * GT_TC), sLBO, 128);
        const uint64_t dSl = tc::smem_desc(tc::su32(Slo + mt * 128 * GT_TC), sLBO, 128);
        const uint32_t d = tmem + (uint32_t)(mt * NP);
#pragma unroll
        for (int ks = 0; ks < GT_TC / 8; ++ks) {
          const uint64_t so = (uint64_t)((ks * 2 * sLBO) >> 4), ao = (uint64_t)((ks * 2 * aLBO) >> 4);
          const uint32_t acc = (u == 0 && ks == 0) ? 0u : 1u;
          tc::mma_tf32(d, dSh + so, dAh + ao, idesc, acc);
          tc::mma_tf32(d, dSh + so, dAl + ao, idesc, 1u);
          tc::mma_tf32(d, dSl + so, dAh + ao, idesc, 1u);
        }
      }
      tc::mma_commit(&mbar[bsel]);
    }
  }
  // the last commit arrives once every MMA issued before it is done
  if (u > 0 && !tc::mbar_wait(&mbar[(u - 1) & 1], (uint32_t)(((u - 1) >> 1) & 1), tc::kWaitLimit)) alive = false;
  if (!alive) s_bad = 1;
  __syncthreads();
  alive = s_bad == 0;  // tcgen05.ld is warp-collective: decide for the whole block
  tc::fence_after();
  if (alive && u > 0) {
    // warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 of tile (w / 4) % MT, and a share
    // of the 16-column groups
    const int quarter = warp & 3, grp = warp >> 2;
    const int parts = (NW / 4) / MT, part = grp / MT, mt = grp % MT;
    const int ngroups = NP / 16;
    const int cg0 = part * ngroups / parts, cg1 = (part + 1) * ngroups / parts;
    const int jl = mt * 128 + quarter * 32 + lane;
    const int j = j0 + jl;
    const int k = j / nb, b = j - k * nb;
    const bool rowok = j < nj && b < Bact;
    for (int cgi = cg0; cgi < cg1; ++cgi) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(mt * NP + cgi * 16), v);
      if (!rowok) continue;
      double* o = out + ((long long)k * ldj + b) * ldo;
#pragma unroll
      for (int w = 0; w < 16; ++w) {
        const int a = cgi * 16 + w;
        if (a < Aact && v[w] != 0.f) atomicAdd(o + a, (double)v[w]);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid == 0 && s_bad && err) atomicOr(err, ERR_TIMEOUT);
  if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)tcols);
}

}  // namespace

bool gram_stencil_tc_supported(int na, long long rows) { return na >= 1 && na <= 128 && rows < (1LL << 31); }

void launch_gram_stencil_tc(cudaStream_t st, long long rows, const float* A, long long lda, int na, const int* adim,
                            const float* B, long long ldb, int nb, const int* bdim, const float* inv_rho,
                            const Geo& g, double* out, int ldj, long long ldo, int waves_x2, int* err) {
  const int nk = 2 * g.nact;
  const GsTcShape s = gs_tc_shape(na, nk * nb);
  // float4 stencil loads: x-extent and column stride multiples of 4, 16-byte aligned bases
  const bool vec = g.nx % 4 == 0 && (ldb & 3) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(inv_rho) & 15) == 0;
  auto kern = g.nact == 3 ? (vec ? gram_stencil_tc_kernel<3, true> : gram_stencil_tc_kernel<3, false>)
                          : (vec ? gram_stencil_tc_kernel<2, true> : gram_stencil_tc_kernel<2, false>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GT_THREADS, s.smem);
  // resident CTAs never ask for more than the 512 TMEM columns of an SM
  per_sm = std::max(1, std::min(per_sm, 512 / s.tcols));
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long chunks = (rows + GT_TC - 1) / GT_TC;
  const long long want = std::max(1LL, (long long)sms * per_sm * std::max(1, waves_x2) / 2 / s.nslice);
  const int gx = (int)std::max(1LL, std::min(chunks, want));
  // the float4 path of the A rows needs 16-byte aligned column starts
  const int a_vec = ((lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) ? 1 : 0;
  kern<<<dim3(gx, s.nslice), GT_THREADS, s.smem, st>>>(rows, A, lda, na, adim, B, ldb, nb, bdim, inv_rho, g, s.NP, s.MT,
                                                s.tcols, a_vec, out, ldj, ldo, err);
}

}  // namespace dlra
