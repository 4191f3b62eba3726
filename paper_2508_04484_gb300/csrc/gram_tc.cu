// Stencil Gram on the tensor cores (FP32 path), the contraction of the S-step and L-step
// Galerkin blocks (Sec. 3.3.2-3.3.3):
//   G_k[a][b] = sum_i A(i, a) D_k(rho^-1 B(:, b))(i),   k = 2 da + s,
// written as D[j][a] = sum_t S[j][t] A[t][a] with j = k nb + b and the cells t as the
// contraction index. A CTA owns a slice of up to 256 rows j (two 128-row MMA tiles, TMEM
// lanes = j, TMEM columns = a) and walks 32-cell chunks of the grid: it forms the stencil
// values S of the chunk (13 neighbour loads per column and cell, as in the FMA kernel), splits
// them and the chunk's A rows into TF32 high and low parts, stores both K-major in shared
// memory and issues three tcgen05.mma kind::tf32 per 8-cell K-slice (hi*hi + hi*lo + lo*hi,
// FP32-accurate products, FP32 accumulation in tensor memory). Two operand buffers: the next
// chunk is staged while the tensor core reads the current one. The slice's partial sums are
// added to the FP64 output with one atomic per entry at the end.
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
  s.smem = 2 * buf * sizeof(float) + (size_t)13 * GT_TC * (sizeof(int) + sizeof(float));
  return s;
}

template <int NACT>
__global__ void __launch_bounds__(256) gram_stencil_tc_kernel(long long rows, const float* __restrict__ A,
                                                              long long lda, int na, const int* adim,
                                                              const float* __restrict__ B, long long ldb, int nb,
                                                              const int* bdim, const float* __restrict__ inv_rho,
                                                              Geo g, int NP, int MT, int tcols, int a_vec,
                                                              double* __restrict__ out, int ldj, long long ldo,
                                                              int* err) {
  constexpr int NK = 2 * NACT;
  extern __shared__ __align__(1024) unsigned char raw[];
  float* base = reinterpret_cast<float*>(raw);
  const int SROWS = MT * 128;
  const int BUF = 2 * SROWS * GT_TC + 2 * NP * GT_TC;  // floats per operand buffer
  int* sOff = reinterpret_cast<int*>(base + 2 * BUF);
  float* sR = reinterpret_cast<float*>(sOff + 13 * GT_TC);
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
  // rows j beyond the slice's last tile entry and padded a read zeros, never stale data
  for (int e = tid; e < 2 * BUF; e += 256) base[e] = 0.f;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const int Aact = dev_dim(adim, na), Bact = dev_dim(bdim, nb);
  const int nj = NK * nb;
  const int j0 = blockIdx.y * 256;
  const uint32_t idesc = tc::idesc_tf32(128, NP);
  const uint32_t sLBO = (128 / 8) * 128, aLBO = (uint32_t)(NP / 8) * 128;
  const long long nchunks = (rows + GT_TC - 1) / GT_TC;
  const int ag = NP >> 3;                    // 8-row groups of a
  const int nbq = (nb + 3) >> 2;             // column quads of b
  const int items = nbq * (GT_TC / 8);       // warp items: 4 columns x 8 cells
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
    // the buffer is free once the MMAs of chunk u - 2 (its previous use) are done
    if (u >= 2 && !tc::mbar_wait(&mbar[bsel], (uint32_t)(((u - 2) >> 1) & 1), tc::kWaitLimit)) alive = false;
    stencil_tables<float, GT_TC>(sOff, sR, r0, rows, inv_rho, g, tid, 256);
    // A rows of the chunk: item (a, quad q of 4 cells); 8 consecutive a fill one core matrix
    for (int e = tid; e < NP * (GT_TC / 4); e += 256) {
      const int a = (e & 7) + 8 * ((e >> 3) % ag), q = (e >> 3) / ag;
      const long long rr = r0 + 4 * q;
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (a < Aact) {
        const float* src = A + (long long)a * lda + rr;
        if (a_vec && rr + 3 < rows) {
          const float4 f = *reinterpret_cast<const float4*>(src);
          v[0] = f.x;
          v[1] = f.y;
          v[2] = f.z;
          v[3] = f.w;
        } else {
#pragma unroll
          for (int w = 0; w < 4; ++w) v[w] = rr + w < rows ? src[w] : 0.f;
        }
      }
      float4 h, l;
      tc::split_tf32(v[0], h.x, l.x);
      tc::split_tf32(v[1], h.y, l.y);
      tc::split_tf32(v[2], h.z, l.z);
      tc::split_tf32(v[3], h.w, l.w);
      const int o = tc::kmajor(a, 4 * q, NP);
      *reinterpret_cast<float4*>(Ahi + o) = h;
      *reinterpret_cast<float4*>(Alo + o) = l;
    }
    // a timeout anywhere stops the whole block at the same point
    if (!__syncthreads_and(alive)) {
      alive = false;
      break;
    }
    // S rows: the nk stencil values of column b at cell t go to rows j = k nb + b of the slice
    for (int it = warp; it < items; it += 8) {
      const int b = (it % nbq) * 4 + (lane & 3);
      const int t = (it / nbq) * 8 + (lane >> 2);
      if (b >= Bact) continue;
      float sv[NK];
      if (r0 + t < rows) {
        stencil_values<float, GT_TC>(B + (long long)b * ldb + r0 + t, sOff, sR, t, g, sv);
      } else {
#pragma unroll
        for (int k = 0; k < NK; ++k) sv[k] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        const int jl = k * nb + b - j0;
        if (jl < 0 || jl >= SROWS) continue;
        float hi, lo;
        tc::split_tf32(sv[k], hi, lo);
        const int o = (jl >> 7) * (128 * GT_TC) + tc::kmajor(jl & 127, t, 128);
        Shi[o] = hi;
        Slo[o] = lo;
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t ah = tc::su32(Ahi), al = tc::su32(Alo);
      for (int mt = 0; mt < MT; ++mt) {
        const uint32_t sh = tc::su32(Shi + mt * 128 * GT_TC), sl = tc::su32(Slo + mt * 128 * GT_TC);
        const uint32_t d = tmem + (uint32_t)(mt * NP);
#pragma unroll
        for (int ks = 0; ks < GT_TC / 8; ++ks) {
          const uint32_t so = ks * 2 * sLBO, ao = ks * 2 * aLBO;
          const uint64_t dSh = tc::smem_desc(sh + so, sLBO, 128), dSl = tc::smem_desc(sl + so, sLBO, 128);
          const uint64_t dAh = tc::smem_desc(ah + ao, aLBO, 128), dAl = tc::smem_desc(al + ao, aLBO, 128);
          const uint32_t acc = (u == 0 && ks == 0) ? 0u : 1u;
          tc::mma_tf32(d, dSh, dAh, idesc, acc);
          tc::mma_tf32(d, dSh, dAl, idesc, 1u);
          tc::mma_tf32(d, dSl, dAh, idesc, 1u);
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
    // warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 of one tile: rows j of the slice
    const int quarter = warp & 3;
    const int ngroups = NP / 16;
    int mt = 0, cg0 = 0, cg1 = ngroups;
    if (MT == 2) {
      mt = warp >> 2;
    } else {
      const int h = (ngroups + 1) / 2;
      cg0 = (warp >> 2) ? h : 0;
      cg1 = (warp >> 2) ? ngroups : h;
    }
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
  auto kern = g.nact == 3 ? gram_stencil_tc_kernel<3> : gram_stencil_tc_kernel<2>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, s.smem);
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
  kern<<<dim3(gx, s.nslice), 256, s.smem, st>>>(rows, A, lda, na, adim, B, ldb, nb, bdim, inv_rho, g, s.NP, s.MT,
                                                s.tcols, a_vec, out, ldj, ldo, err);
}

}  // namespace dlra
