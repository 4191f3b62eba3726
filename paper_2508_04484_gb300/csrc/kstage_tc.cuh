// K-stage on the tensor cores (FP32 path): acc(i, :) = sum_k D_k(v)(i, :) P_k, the r x r
// mixing of the six (four in 2-D) stencil values of every column, written as a product
// D[cells x N] = A[cells x K] * B[K x N] with K = (column c', stencil k) = c' NK + k and
// B[K][c] = P_k[c'][c].
//
// A CTA owns a brick of 256 cells (8 x 8 x 4 in 3-D, 16 x 1 x 16 in a 2-D slab), one thread
// per cell, and two 128-row MMA tiles (TMEM lanes = cells). K is processed in chunks of four
// columns: the CTA stages the chunk's input values of the brick and its two-cell halo in
// shared memory (each value read from global memory once instead of up to 13 times), every
// thread forms its cell's stencil values from there, splits them into TF32 high and low parts
// and stores them K-major; three tcgen05.mma kind::tf32 per K-slice (hi*hi + hi*lo + lo*hi)
// give an FP32-accurate product. The halo of the next chunk is loaded while the tensor core
// still reads the current operands.
#pragma once
#include "device.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace dlra {

template <int NACT, int RM>
struct KsTc {
  static constexpr int NP = ((RM + 15) / 16) * 16;                 // MMA N (multiple of 16 for M = 128)
  static constexpr int TCOLS = 2 * NP <= 32 ? 32 : (2 * NP <= 64 ? 64 : 128);   // two accumulators
  static constexpr int NK = 2 * NACT;
  static constexpr int CC = 4;                                      // columns per K chunk
  static constexpr int KC = CC * NK;
  static constexpr int TX = NACT == 3 ? 8 : 16, TY = NACT == 3 ? 8 : 1, TZ = NACT == 3 ? 4 : 16;
  static constexpr int HX = TX + 4, HY = NACT == 3 ? TY + 4 : 1, HZ = TZ + 4;
  static constexpr int HALO = HX * HY * HZ;                        // staged values per column
  static constexpr int ASZ = 256 * KC, BSZ = NP * KC;              // floats per operand buffer
  static constexpr size_t SMEM = (size_t)(CC * HALO + 2 * ASZ + 2 * BSZ) * sizeof(float);
};

template <int NACT, int RM>
size_t kstage_tc_smem() {
  return KsTc<NACT, RM>::SMEM;
}

template <int NACT, int RM>
unsigned kstage_tc_grid(const Geo& g) {
  using C = KsTc<NACT, RM>;
  return (unsigned)(((g.nx + C::TX - 1) / C::TX) * ((g.ny + C::TY - 1) / C::TY) * ((g.nz + C::TZ - 1) / C::TZ));
}

// mode: 0 vout = rho^-1 (y + beta acc); 1 also yout = y + beta acc (last stage), vout = rho^-1 yout;
// 2 (transposed operator, unscaled input) vout = beta rho^-1 acc, yout = y + vout.
template <int NACT, int RM>
__global__ void __launch_bounds__(256) kstage_tc_kernel(const float* __restrict__ vin, const float* __restrict__ y,
                                                        float* __restrict__ yout, float* __restrict__ vout,
                                                        long long ld, const float* __restrict__ inv_rho, Geo g,
                                                        const float* __restrict__ Pst, const int* __restrict__ rdim,
                                                        float beta, int mode, int* err) {
  using C = KsTc<NACT, RM>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, NP = C::NP, TCOLS = C::TCOLS;
  constexpr int TX = C::TX, TY = C::TY, TZ = C::TZ, HX = C::HX, HY = C::HY, HALO = C::HALO;
  extern __shared__ __align__(1024) unsigned char raw[];
  float* Ahi = reinterpret_cast<float*>(raw);   // 256 rows (two 128-row tiles), K-major
  float* Alo = Ahi + C::ASZ;
  float* Bhi = Alo + C::ASZ;
  float* Blo = Bhi + C::BSZ;
  float* sH = Blo + C::BSZ;                      // [CC][HZ][HY][HX] staged inputs
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_fence_init();
    s_bad = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const int r = dev_dim(rdim, RM);
  const int nch = (r + CC - 1) / CC;
  // brick origin and this thread's cell (row = lx + TX (ly + TY lz); rows 0..127 are tile 0)
  const int bx = (g.nx + TX - 1) / TX, by = (g.ny + TY - 1) / TY;
  const int blk = blockIdx.x;
  const int x0 = (blk % bx) * TX, y0 = ((blk / bx) % by) * TY, z0 = (blk / (bx * by)) * TZ;
  const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
  const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
  const bool ok = ix < g.nx && iy < g.ny && iz < g.nz;
  const long long i = ((long long)iz * g.ny + iy) * g.nx + ix;
  float inv2[NACT];
#pragma unroll
  for (int da = 0; da < NACT; ++da) inv2[da] = (float)g.inv2d[(NACT == 3) ? da : (da == 0 ? 0 : 2)];
  // halo strides in the staged brick (x fastest) and this cell's centre
  constexpr int SXH = 1, SYH = HX, SZH = HX * HY;
  const int hc = (lz + 2) * SZH + (NACT == 3 ? (ly + 2) * SYH : 0) + (lx + 2);
  constexpr uint32_t idesc = tc::idesc_tf32(128, NP);
  constexpr uint32_t aLBO = (128 / 8) * 128, bLBO = (NP / 8) * 128;
  // the halo elements this thread stages (the same for every column): cell index, or -1
  // outside the grid
  constexpr int HPT = (HALO + 255) / 256;
  int hcell[HPT];
#pragma unroll
  for (int u = 0; u < HPT; ++u) {
    const int h = tid + 256 * u;
    hcell[u] = -2;   // beyond the staged brick
    if (h < HALO) {
      const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
      const int gx = x0 + hx - 2, gy = NACT == 3 ? y0 + hy - 2 : y0, gz = z0 + hz - 2;
      hcell[u] = (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz)
                     ? (int)(((long long)gz * g.ny + gy) * g.nx + gx)
                     : -1;
    }
  }
  bool alive = true;
  for (int ch = 0; ch < nch; ++ch) {
    // stage the chunk's columns over the brick and its halo (zero outside the grid); the
    // previous chunk's stencil values were formed before the last barrier, so sH is free
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
      const int c = ch * CC + cc;
      const float* col = vin + (long long)c * ld;
#pragma unroll
      for (int u = 0; u < HPT; ++u) {
        if (hcell[u] == -2) continue;
        sH[cc * HALO + tid + 256 * u] = (c < r && hcell[u] >= 0) ? col[hcell[u]] : 0.f;
      }
    }
    // the operand buffers are free once the previous chunk's MMAs are done
    if (ch >= 1 && !tc::mbar_wait(&mbar, (uint32_t)((ch - 1) & 1), tc::kWaitLimit)) alive = false;
    __syncthreads();
    // A row of this cell: the stencil values of the chunk's columns, K = cc NK + k
    float sv[KC];
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
      const float* hv = sH + cc * HALO + hc;
      const float v0 = hv[0];
#pragma unroll
      for (int da = 0; da < NACT; ++da) {
        const int st = NACT == 3 ? (da == 0 ? SXH : (da == 1 ? SYH : SZH)) : (da == 0 ? SXH : SZH);
        sv[cc * NK + 2 * da] = ok ? (-3.f * v0 + 4.f * hv[-st] - hv[-2 * st]) * inv2[da] : 0.f;
        sv[cc * NK + 2 * da + 1] = ok ? (3.f * v0 - 4.f * hv[st] + hv[2 * st]) * inv2[da] : 0.f;
      }
    }
    // 16-byte stores: four consecutive K of one row are contiguous in a core matrix
    {
      const int base = (tid >> 7) * (128 * KC) + tc::kmajor(tid & 127, 0, 128);
#pragma unroll
      for (int kg = 0; kg < KC / 4; ++kg) {
        float4 h4, l4;
        tc::split_tf32(sv[4 * kg + 0], h4.x, l4.x);
        tc::split_tf32(sv[4 * kg + 1], h4.y, l4.y);
        tc::split_tf32(sv[4 * kg + 2], h4.z, l4.z);
        tc::split_tf32(sv[4 * kg + 3], h4.w, l4.w);
        // kmajor(row, 4 kg, 128) = kmajor(row, 0, 128) + kg * 16 * 32
        *reinterpret_cast<float4*>(Ahi + base + kg * 512) = h4;
        *reinterpret_cast<float4*>(Alo + base + kg * 512) = l4;
      }
    }
    // B rows: B[n][K] = P_k[c][n] = Pst[(c NK + k) RM + n], zero for padded n
    for (int e = tid; e < NP * KC; e += 256) {
      const int n = e / KC, K = e - n * KC;
      const int cc = K / NK, k = K - cc * NK, c = ch * CC + cc;
      const float pv = (n < RM && c < RM) ? Pst[((long long)c * NK + k) * RM + n] : 0.f;
      float hi, lo;
      tc::split_tf32(pv, hi, lo);
      const int o = tc::kmajor(n, K, NP);
      Bhi[o] = hi;
      Blo[o] = lo;
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const uint32_t ah = tc::su32(Ahi + mt * 128 * KC), al = tc::su32(Alo + mt * 128 * KC);
        const uint32_t bh = tc::su32(Bhi), bl = tc::su32(Blo);
        const uint32_t d = tmem + mt * NP;
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint32_t ao = ks * 2 * aLBO, bo = ks * 2 * bLBO;
          const uint64_t dAh = tc::smem_desc(ah + ao, aLBO, 128), dAl = tc::smem_desc(al + ao, aLBO, 128);
          const uint64_t dBh = tc::smem_desc(bh + bo, bLBO, 128), dBl = tc::smem_desc(bl + bo, bLBO, 128);
          const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
          tc::mma_tf32(d, dAh, dBh, idesc, first);
          tc::mma_tf32(d, dAh, dBl, idesc, 1u);
          tc::mma_tf32(d, dAl, dBh, idesc, 1u);
        }
      }
      tc::mma_commit(&mbar);
    }
  }
  // the last commit arrives after every MMA of this thread
  if (nch > 0 && !tc::mbar_wait(&mbar, (uint32_t)((nch - 1) & 1), tc::kWaitLimit)) alive = false;
  if (!alive) s_bad = 1;
  __syncthreads();
  // tcgen05.ld is warp-collective: decide for the whole block
  alive = s_bad == 0;
  tc::fence_after();
  if (alive) {
    // warp w reads TMEM lanes 32 (w % 4) .. of accumulator w / 4: exactly its own cells
    const float ir0 = ok ? inv_rho[i] : 0.f;
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float acc[16];
      if (nch > 0) {
        tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (warp >> 2) * NP + c0, acc);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = 0.f;
      }
      if (!ok) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = c0 + j;
        if (c >= RM) break;
        const long long e = (long long)c * ld + i;
        if (mode == 2) {
          const float lam = beta * ir0 * acc[j];
          vout[e] = lam;
          yout[e] = y[e] + lam;
        } else if (mode == 1) {
          const float yn = y[e] + beta * acc[j];
          yout[e] = yn;
          vout[e] = ir0 * yn;
        } else {
          vout[e] = ir0 * (y[e] + beta * acc[j]);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid == 0 && s_bad && err) atomicOr(err, ERR_TIMEOUT);
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

}  // namespace dlra
