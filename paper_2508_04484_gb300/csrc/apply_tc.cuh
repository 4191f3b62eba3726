// Tall-skinny apply on the tensor cores (FP32 path): C(i, c) = alpha sum_q A(i, q) M(q, c) +
// beta Cin(i, c) (and V = rho^-1 C), the products of the augmentation and truncation steps
// (Sec. 2.2: X^ = [X, orth(...)], X = X^ P) with a column-major A of n rows and Q <= 128
// columns, M (Q x N) in FP64, N <= 64.
//
// Persistent blocks (two per SM) loop over 128-row tiles (one TMEM lane per row). The B operand
// (M^T split into TF32 high and low parts, K-major, built once per launch by
// apply_tc_bimg_kernel) is loaded once per block with one bulk copy. A producer thread loads each
// tile's A in chunks of 32 columns with 2-D TMA copies (rows beyond n read zeros); four
// formation warps split their row's 32 values into TF32 high and low parts and write them into
// the row's TMEM lane (tcgen05.st); one thread issues three tcgen05.mma kind::tf32 per 8-wide K
// slice (A from TMEM, B from shared memory: hi*hi + hi*lo + lo*hi, FP32-accurate products, FP32
// accumulation in TMEM) into one of two accumulators; four epilogue warps read tile i's
// accumulator and write C (and V) while tile i + 1 accumulates in the other. A may overlap C
// (a tile's rows are read before they are written, and no other tile reads them). Every wait
// gives up after about a second (ERR_TIMEOUT).
#pragma once
#include "device.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace dlra {

template <int NP>
struct ApTc {
  static constexpr int KCH = 32;                                   // columns per chunk
  static constexpr int QMAX = 128;
  static constexpr int NS = 2;                                     // ring stages
  static constexpr int TCOLS = 256, ACOL = 128;                    // sums at 0 / 64, A stage s at 128 + 64 s
  static constexpr int THREADS = 320;                              // 4 formation, 4 epilogue warps, copies, products
  static constexpr size_t al(size_t b) { return (b + 1023) / 1024 * 1024; }
  static constexpr size_t BPART = al((size_t)NP * QMAX * 4);      // B hi (or lo) for all 128 K
  static constexpr uint32_t BBYTES = (uint32_t)(2 * BPART);
  static constexpr size_t ATILE = (size_t)KCH * 128 * 4;          // 16 KB
  static constexpr size_t OFF_B = 0;
  static constexpr size_t OFF_A = BBYTES;
  static constexpr size_t SMEM = OFF_A + NS * ATILE + 1024;
  static_assert(ACOL + 64 * NS <= TCOLS, "A stages exceed the TMEM allocation");
  static_assert(NP <= 64, "accumulator columns");
};

// B image: B[n][q] = M(q, n) (zero for n >= N or q >= Q) as TF32 high and low parts, K-major for
// an N = NP operand with K = 128, high part then low part
template <int NP>
__global__ void __launch_bounds__(256) apply_tc_bimg_kernel(const double* __restrict__ M, long long ldm, int Q,
                                                            const int* __restrict__ qdim, int N,
                                                            float* __restrict__ img) {
  using C = ApTc<NP>;
  const int Qa = dev_dim(qdim, Q);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NP * C::QMAX) return;
  const int n = e / C::QMAX, q = e - n * C::QMAX;
  const float v = (n < N && q < Qa) ? (float)M[(long long)n * ldm + q] : 0.f;
  float hi, lo;
  tc::split_tf32(v, hi, lo);
  const int o = tc::kmajor(n, q, NP);
  img[o] = hi;
  img[C::BPART / 4 + o] = lo;
}

template <int NP>
__global__ void __launch_bounds__(320, 2) apply_tc_kernel(const __grid_constant__ CUtensorMap tmap, long long rows,
                                                          int Q, const int* __restrict__ qdim,
                                                          const float* __restrict__ Bimg, int N, float* __restrict__ Cm,
                                                          long long ldc, const float* __restrict__ Cin, float alpha,
                                                          float beta, float* __restrict__ V,
                                                          const float* __restrict__ inv_rho, int* err) {
  using C = ApTc<NP>;
  constexpr int KCH = C::KCH, NS = C::NS, TCOLS = C::TCOLS, ACOL = C::ACOL;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 1023) & ~(uintptr_t)1023);
  // full / afull / free: a chunk's A tile landed / is in TMEM / was consumed; accfull: a tile's
  // sums are done; accfree: the epilogue has read them (one arrival per epilogue warp)
  __shared__ __align__(8) uint64_t bfull, full_bar[NS], afull_bar[NS], free_bar[NS], accfull[2], accfree[2], mdone;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Qa = dev_dim(qdim, Q);
  const int nch = (Qa + KCH - 1) / KCH;
  const long long tiles = (rows + 127) / 128;
  const int ntl = (int)((tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);  // this block's tiles
  if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
  if (tid == 0) {
    tc::mbar_init(&bfull, 1);
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&afull_bar[s], 4);
      tc::mbar_init(&free_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accfull[b], 1);
      tc::mbar_init(&accfree[b], 4);
    }
    tc::mbar_init(&mdone, 1);
    tc::mbar_fence_init();
    s_bad = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  auto At = [&](int s) { return reinterpret_cast<float*>(base + C::OFF_A + s * C::ATILE); };
  auto tile_row = [&](int i) { return ((long long)blockIdx.x + (long long)i * gridDim.x) * 128; };

  if (warp == 8) {
    // ---------------- copies: B once, then every tile's A chunks ----------------
    if (lane == 0) {
      int issued = 0;
      if (nch > 0) {
        tc::mbar_arrive_expect_tx(&bfull, C::BBYTES);
        tc::bulk_load(base + C::OFF_B, Bimg, C::BBYTES, &bfull);
      }
      bool ok = true;
      for (int i = 0; i < ntl && ok; ++i) {
        for (int ch = 0; ch < nch; ++ch) {
          const int g = i * nch + ch, s = g % NS;
          if (g >= NS &&
              (s_bad || !tc::mbar_wait_ns(&free_bar[s], (uint32_t)(((g - NS) / NS) & 1), tc::kWaitNs))) {
            s_bad = 1;
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&full_bar[s], (uint32_t)C::ATILE);
          tc::tma_load_2d(At(s), &tmap, (int)tile_row(i), ch * KCH, &full_bar[s]);
          issued = g + 1;
        }
      }
      for (int g = (issued >= NS ? issued - NS : 0); g < issued; ++g)
        tc::mbar_wait_ns(&full_bar[g % NS], (uint32_t)((g / NS) & 1), tc::kWaitNs);
      if (nch > 0) tc::mbar_wait_ns(&bfull, 0u, tc::kWaitNs);
    }
  } else if (warp == 9) {
    // ---------------- products: tile i into accumulator i % 2 ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_tf32(128, NP);
      constexpr uint32_t bLBO = (NP / 8) * 128;
      bool ok = nch == 0 || tc::mbar_wait_ns(&bfull, 0u, tc::kWaitNs);
      if (!ok) s_bad = 1;
      const uint32_t bh = tc::su32(base + C::OFF_B), bl = bh + (uint32_t)C::BPART;
      for (int i = 0; i < ntl && ok; ++i) {
        const int ab = i & 1;
        // the epilogue has read this accumulator's previous tile
        if (i >= 2 && (s_bad || !tc::mbar_wait_ns(&accfree[ab], (uint32_t)(((i >> 1) - 1) & 1), tc::kWaitNs))) {
          s_bad = 1;
          break;
        }
        const uint32_t dacc = tmem + ab * 64;
        for (int ch = 0; ch < nch; ++ch) {
          const int g = i * nch + ch, s = g % NS;
          if (s_bad || !tc::mbar_wait_ns(&afull_bar[s], (uint32_t)((g / NS) & 1), tc::kWaitNs)) {
            s_bad = 1;
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t ahi = tmem + ACOL + s * 64, alo = ahi + 32;
#pragma unroll
          for (int ks = 0; ks < KCH / 8; ++ks) {
            const uint32_t bk = (uint32_t)(ch * (KCH / 8) + ks) * 2 * bLBO;
            const uint64_t dBh = tc::smem_desc(bh + bk, bLBO, 128), dBl = tc::smem_desc(bl + bk, bLBO, 128);
            const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
            tc::mma_tf32_ta(dacc, ahi + ks * 8, dBh, idesc, first);
            tc::mma_tf32_ta(dacc, ahi + ks * 8, dBl, idesc, 1u);
            tc::mma_tf32_ta(dacc, alo + ks * 8, dBh, idesc, 1u);
          }
          tc::mma_commit(&free_bar[s]);
        }
        if (ok) tc::mma_commit(&accfull[ab]);
      }
      tc::mma_commit(&mdone);
      if (!tc::mbar_wait_ns(&mdone, 0u, tc::kWaitNs)) s_bad = 1;
    }
  } else if (warp < 4) {
    // ---------------- A rows into TMEM: one row (TMEM lane) per thread ----------------
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    bool go = true;
    for (int i = 0; i < ntl && go; ++i) {
      for (int ch = 0; ch < nch; ++ch) {
        const int g = i * nch + ch, s = g % NS;
        bool ok = !s_bad && tc::mbar_wait_ns(&full_bar[s], (uint32_t)((g / NS) & 1), tc::kWaitNs);
        if (!__all_sync(0xffffffffu, ok)) {  // tcgen05.st is warp-collective
          s_bad = 1;
          go = false;
          break;
        }
        const float* a = At(s) + tid;  // [q][row]
        float hi[KCH], lo[KCH];
#pragma unroll
        for (int q = 0; q < KCH; ++q) {
          const float v = (ch * KCH + q < Qa) ? a[q * 128] : 0.f;
          tc::split_tf32(v, hi[q], lo[q]);
        }
        const uint32_t ahi = lane_base + ACOL + s * 64;
#pragma unroll
        for (int q = 0; q < KCH / 8; ++q) {
          tc::tmem_st8(ahi + q * 8, hi + q * 8);
          tc::tmem_st8(ahi + 32 + q * 8, lo + q * 8);
        }
        tc::tmem_st_wait();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&afull_bar[s]);
      }
    }
  } else {
    // ---------------- epilogue: tile i's sums from accumulator i % 2 ----------------
    const int quarter = warp & 3;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int i = 0; i < ntl; ++i) {
      const int ab = i & 1;
      bool ok = !s_bad && tc::mbar_wait_ns(&accfull[ab], (uint32_t)((i >> 1) & 1), tc::kWaitNs);
      if (!__all_sync(0xffffffffu, ok)) {  // tcgen05.ld is warp-collective
        s_bad = 1;
        break;
      }
      tc::fence_after();
      const long long row = tile_row(i) + 32 * quarter + lane;
      const bool inrow = row < rows;
      const float ir = (V && inrow) ? inv_rho[row] : 0.f;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float acc[16];
        if (nch > 0) {
          tc::tmem_ld16(lane_base + ab * 64 + c0, acc);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = 0.f;
        }
        if (!inrow) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          if (c >= N) break;
          float v = alpha * acc[j];
          if (Cin) v += beta * Cin[(long long)c * ldc + row];
          Cm[(long long)c * ldc + row] = v;
          if (V) V[(long long)c * ldc + row] = ir * v;
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&accfree[ab]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid == 0 && s_bad && err) atomicOr(err, ERR_TIMEOUT);
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

}  // namespace dlra
