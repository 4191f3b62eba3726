// Tall-skinny apply on the tensor cores (FP32 path): C(i, c) = alpha sum_q A(i, q) M(q, c) +
// beta Cin(i, c) (and V = rho^-1 C), the products of the augmentation and truncation steps
// (Sec. 2.2: X^ = [X, orth(...)], X = X^ P) with a column-major A of n rows and Q <= 128
// columns, M (Q x N) in FP64, N <= 64.
//
// A CTA owns 128 rows (one TMEM lane each) and walks A's columns in chunks of 32: a producer
// thread loads each chunk's 128 x 32 tile with one 2-D TMA copy (rows beyond n read zeros) and
// the B operand (M^T split into TF32 high and low parts, K-major, built once per launch by
// apply_tc_bimg_kernel) with one bulk copy; four warps split their row's 32 values into TF32
// high and low parts and write them into the row's TMEM lane (tcgen05.st); one thread issues
// three tcgen05.mma kind::tf32 per 8-wide K slice (A from TMEM, B from shared memory: hi*hi +
// hi*lo + lo*hi, FP32-accurate products, FP32 accumulation in TMEM); the epilogue reads each
// row's accumulator and writes C (and V). A may overlap C (the CTA reads all of its rows before
// it writes any). Every wait gives up after about a second (ERR_TIMEOUT).
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
  static constexpr int TCOLS = 256, ACOL = 64;                     // acc [0, NP), A stage s at 64 + 64 s
  static constexpr int THREADS = 192;                              // 4 formation / epilogue warps, copies, products
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
__global__ void __launch_bounds__(192) apply_tc_kernel(const __grid_constant__ CUtensorMap tmap, long long rows,
                                                       int Q, const int* __restrict__ qdim,
                                                       const float* __restrict__ Bimg, int N, float* __restrict__ Cm,
                                                       long long ldc, const float* __restrict__ Cin, float alpha,
                                                       float beta, float* __restrict__ V,
                                                       const float* __restrict__ inv_rho, int* err) {
  using C = ApTc<NP>;
  constexpr int KCH = C::KCH, NS = C::NS, TCOLS = C::TCOLS, ACOL = C::ACOL;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bfull, full_bar[NS], afull_bar[NS], free_bar[NS], acc_bar;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Qa = dev_dim(qdim, Q);
  const int nch = (Qa + KCH - 1) / KCH;
  const long long r0 = (long long)blockIdx.x * 128;
  if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
  if (tid == 0) {
    tc::mbar_init(&bfull, 1);
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&afull_bar[s], 4);
      tc::mbar_init(&free_bar[s], 1);
    }
    tc::mbar_init(&acc_bar, 1);
    tc::mbar_fence_init();
    s_bad = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  auto At = [&](int s) { return reinterpret_cast<float*>(base + C::OFF_A + s * C::ATILE); };

  if (warp == 4) {
    // ---------------- copies ----------------
    if (lane == 0) {
      int issued = 0;
      if (nch > 0) {
        tc::mbar_arrive_expect_tx(&bfull, C::BBYTES);
        tc::bulk_load(base + C::OFF_B, Bimg, C::BBYTES, &bfull);
      }
      for (int ch = 0; ch < nch; ++ch) {
        const int s = ch % NS;
        if (ch >= NS &&
            (s_bad || !tc::mbar_wait_ns(&free_bar[s], (uint32_t)(((ch - NS) / NS) & 1), tc::kWaitNs))) {
          s_bad = 1;
          break;
        }
        tc::mbar_arrive_expect_tx(&full_bar[s], (uint32_t)C::ATILE);
        tc::tma_load_2d(At(s), &tmap, (int)r0, ch * KCH, &full_bar[s]);
        issued = ch + 1;
      }
      for (int ch = (issued >= NS ? issued - NS : 0); ch < issued; ++ch)
        tc::mbar_wait_ns(&full_bar[ch % NS], (uint32_t)((ch / NS) & 1), tc::kWaitNs);
      if (nch > 0) tc::mbar_wait_ns(&bfull, 0u, tc::kWaitNs);
    }
  } else if (warp == 5) {
    // ---------------- products ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_tf32(128, NP);
      constexpr uint32_t bLBO = (NP / 8) * 128;
      bool ok = nch == 0 || tc::mbar_wait_ns(&bfull, 0u, tc::kWaitNs);
      if (!ok) s_bad = 1;
      const uint32_t bh = tc::su32(base + C::OFF_B), bl = bh + (uint32_t)C::BPART;
      for (int ch = 0; ch < nch && ok; ++ch) {
        const int s = ch % NS;
        if (s_bad || !tc::mbar_wait_ns(&afull_bar[s], (uint32_t)((ch / NS) & 1), tc::kWaitNs)) {
          s_bad = 1;
          break;
        }
        tc::fence_after();
        const uint32_t ahi = tmem + ACOL + s * 64, alo = ahi + 32;
#pragma unroll
        for (int ks = 0; ks < KCH / 8; ++ks) {
          const uint32_t bk = (uint32_t)(ch * (KCH / 8) + ks) * 2 * bLBO;
          const uint64_t dBh = tc::smem_desc(bh + bk, bLBO, 128), dBl = tc::smem_desc(bl + bk, bLBO, 128);
          const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
          tc::mma_tf32_ta(tmem, ahi + ks * 8, dBh, idesc, first);
          tc::mma_tf32_ta(tmem, ahi + ks * 8, dBl, idesc, 1u);
          tc::mma_tf32_ta(tmem, alo + ks * 8, dBh, idesc, 1u);
        }
        tc::mma_commit(&free_bar[s]);
      }
      tc::mma_commit(&acc_bar);
      if (!tc::mbar_wait_ns(&acc_bar, 0u, tc::kWaitNs)) s_bad = 1;
    }
  } else {
    // ---------------- A rows into TMEM: one row (TMEM lane) per thread ----------------
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int ch = 0; ch < nch; ++ch) {
      const int s = ch % NS;
      bool go = !s_bad && tc::mbar_wait_ns(&full_bar[s], (uint32_t)((ch / NS) & 1), tc::kWaitNs);
      go = __all_sync(0xffffffffu, go);   // tcgen05.st is warp-collective
      if (!go) {
        s_bad = 1;
        break;
      }
      const float* a = At(s) + tid;        // [q][row]
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
  __syncthreads();
  const bool alive = s_bad == 0;
  if (warp < 4) {
    const long long i = r0 + tid;
    const bool row = i < rows;
    tc::fence_after();
    // every lane of the warp takes part in tcgen05.ld (warp-collective); rows beyond the
    // matrix (the ragged last tile) only skip the stores
    if (alive) {
      const float ir = (V && row) ? inv_rho[i] : 0.f;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float acc[16];
        if (nch > 0) {
          tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, acc);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = 0.f;
        }
        if (!row) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          if (c >= N) break;
          float v = alpha * acc[j];
          if (Cin) v += beta * Cin[(long long)c * ldc + i];
          Cm[(long long)c * ldc + i] = v;
          if (V) V[(long long)c * ldc + i] = ir * v;
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid == 0 && !alive && err) atomicOr(err, ERR_TIMEOUT);
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

}  // namespace dlra
