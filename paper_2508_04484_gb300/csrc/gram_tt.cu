// Tall-skinny Grams on the tensor cores (FP32 path): out[j ldo + a] += sum_t A(t, a) F(t, j) over
// the n cells t, with F(t, j) = B(t, j) (the augmentation's projections X^T K and the Gram of the
// pivoted CholeskyQR2 passes, Sec. 2.2) or F(t, k nb + b) = w_k(t) B(t, b) (the material Grams
// X^T diag(w_k) X of the collided scattering step, Sec. 3.3.1).
//
// D[a][j] = sum_t A^T[a][t] F[t][j]: A's columns on the MMA's M side (TMEM lanes, up to 128), 64
// columns of F per slice on N (grid y: slice k takes F columns 64 k ..). A block walks a
// contiguous run of 32-row chunks: a producer thread loads each chunk of A (and of B and the
// weights where B is not a column block of A) with 2-D TMA copies (128-byte swizzle; rows beyond
// n read zeros) into a ring; eight formation warps split the chunk's A values into TF32 high and
// low parts and write them into TMEM (tcgen05.st, the MMA's A operand), and form F's values
// (weighted where asked), split them and store them K-major into shared memory (the B operand);
// one thread issues three tcgen05.mma kind::tf32 per 8-row K-slice (hi*hi + hi*lo + lo*hi). The
// tensor core's FP32 accumulation rounds toward zero, so the products go to one of two short
// accumulators, a fresh one every F chunks, whose sums the formation warps add into a long FP32
// accumulator in TMEM with round-to-nearest additions (drift bounded by F x 12 roundings). Each
// block adds its long sums to the FP64 output with one atomic per entry. Every wait gives up
// after about a second (ERR_TIMEOUT).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace dlra {

namespace {

// NA: A columns loaded per chunk (64 or 128); F columns per slice: 64
template <int NA>
struct GtShape {
  static constexpr int NJ = 64;                                    // MMA N
  static constexpr int R = 4;                                      // chunk slots of the copy ring (a power of 2)
  static constexpr int NS = 4;                                     // chunk stages (A in TMEM, F in smem)
  static constexpr int F = 8;                                      // chunks per short accumulation
  static constexpr int TCOLS = 512;
  static constexpr int LCOL = 2 * NJ;                              // long sums; short ones at 0 and NJ
  static constexpr int SCOL = 3 * NJ;                              // A stage st at SCOL + 64 st (hi, lo + 32)
  static constexpr int NFORM = 8;                                  // formation warps (two per lane quarter)
  static constexpr int THREADS = 32 * (NFORM + 2);
  static constexpr uint32_t ABYTES = NA * 128;                     // 32 rows of NA columns (swizzled)
  static constexpr uint32_t BBYTES = NJ * 128;                     // 32 rows of 64 columns of B
  static constexpr int NKMAX = 8;                                  // weight columns (materials)
  static constexpr size_t SLOT = (size_t)ABYTES + BBYTES + 1024;   // + 32 rows of the weights
  static constexpr size_t OFF_P = (size_t)R * SLOT;
  static constexpr size_t PPART = (size_t)NJ * 32 * 4;             // F hi (or lo) of one chunk
  static constexpr size_t SMEM = OFF_P + (size_t)NS * 2 * PPART + 1024;
  static_assert(SCOL + NS * 64 <= TCOLS, "TMEM columns");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// A(t, a) for a < NA from tmA; F columns of slice blockIdx.y: j = 64 blockIdx.y + jj. Plain
// (nbw == 0): F(t, j) = B(t, j); weighted: F(t, k nbw + b) = w_k(t) B(t, b). B's chunk comes
// from its own map (bsame == 0, columns b0 ..) or from A's chunk (bsame: B(t, b) = A(t, boff + b)).
template <int NA>
__global__ void __launch_bounds__(GtShape<NA>::THREADS, 1) gram_tt_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const __grid_constant__ CUtensorMap tmW, long long rows, const int* __restrict__ adim, int acap,
    const int* __restrict__ jdim, int jcap, int ncols, int nbw, int nk, int bsame, int boff,
    double* __restrict__ out, long long ldo, int* err) {
  using C = GtShape<NA>;
  constexpr int NJ = C::NJ, NS = C::NS, R = C::R, F = C::F, NFORM = C::NFORM;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t rfull[R], rfree[R], afull[NS], sfree[NS], hfull[2], hfree[2], mdone;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long nchunks_all = (rows + 31) / 32;
  const long long c0 = nchunks_all * blockIdx.x / gridDim.x, c1 = nchunks_all * (blockIdx.x + 1) / gridDim.x;
  const int nchunks = (int)(c1 - c0);
  const int ngroups = (nchunks + F - 1) / F;
  const int j0 = NJ * (int)blockIdx.y;
  const int Aact = dev_dim(adim, acap), Jact = dev_dim(jdim, jcap);
  const uint32_t txb = C::ABYTES + (bsame ? 0u : C::BBYTES) + (nbw > 0 ? (uint32_t)nk * 128u : 0u);
  if (warp == 0) tc::tmem_alloc(&tslot, C::TCOLS);
  if (tid == 0) {
    for (int q = 0; q < R; ++q) {
      tc::mbar_init(&rfull[q], 1);
      tc::mbar_init(&rfree[q], NFORM);
    }
    for (int q = 0; q < NS; ++q) {
      tc::mbar_init(&afull[q], NFORM);
      tc::mbar_init(&sfree[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&hfull[q], 1);
      tc::mbar_init(&hfree[q], NFORM);
    }
    tc::mbar_init(&mdone, 1);
    tc::mbar_fence_init();
    s_bad = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  auto slot_ptr = [&](int u) { return base + (size_t)(u & (R - 1)) * C::SLOT; };

  if (warp == NFORM) {
    // ---------------- copies: A's chunk (and B's, the weights') per 32 rows ----------------
    if (lane == 0) {
      int issued = 0;
      for (int u = 0; u < nchunks; ++u) {
        const int slot = u & (R - 1);
        if (u >= R && (s_bad || !tc::mbar_wait_ns(&rfree[slot], (uint32_t)(((u / R) - 1) & 1), tc::kWaitNs))) {
          s_bad = 1;
          break;
        }
        const int t0 = (int)((c0 + u) * 32);
        unsigned char* sp = slot_ptr(u);
        tc::mbar_arrive_expect_tx(&rfull[slot], txb);
        tc::tma_load_2d(sp, &tmA, t0, 0, &rfull[slot]);
        if (!bsame) tc::tma_load_2d(sp + C::ABYTES, &tmB, t0, nbw > 0 ? 0 : j0, &rfull[slot]);
        if (nbw > 0) tc::tma_load_2d(sp + C::ABYTES + C::BBYTES, &tmW, t0, 0, &rfull[slot]);
        issued = u + 1;
      }
      for (int q = (issued > R ? issued - R : 0); q < issued; ++q)
        tc::mbar_wait_ns(&rfull[q & (R - 1)], (uint32_t)((q / R) & 1), tc::kWaitNs);
    }
  } else if (warp == NFORM + 1) {
    // ---------------- products: A from TMEM, F from shared memory ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_tf32(128, NJ);
      constexpr uint32_t bLBO = (NJ / 8) * 128;
      for (int u = 0; u < nchunks; ++u) {
        const int st = u % NS, grp = u / F, hb = grp & 1;
        if (u % F == 0 && grp >= 2 &&
            (s_bad || !tc::mbar_wait_ns(&hfree[hb], (uint32_t)(((grp >> 1) - 1) & 1), tc::kWaitNs))) {
          s_bad = 1;
          break;
        }
        if (s_bad || !tc::mbar_wait_ns(&afull[st], (uint32_t)((u / NS) & 1), tc::kWaitNs)) {
          s_bad = 1;
          break;
        }
        tc::fence_after();
        const uint32_t ph = tc::su32(base + C::OFF_P + (size_t)st * 2 * C::PPART), pl = ph + (uint32_t)C::PPART;
        const uint32_t shi = tmem + C::SCOL + st * 64, slo = shi + 32, dacc = tmem + hb * NJ;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t bk = ks * 2 * bLBO;
          const uint64_t dPh = tc::smem_desc(ph + bk, bLBO, 128), dPl = tc::smem_desc(pl + bk, bLBO, 128);
          const uint32_t first = (u % F == 0 && ks == 0) ? 0u : 1u;
          tc::mma_tf32_ta(dacc, shi + ks * 8, dPh, idesc, first);
          tc::mma_tf32_ta(dacc, shi + ks * 8, dPl, idesc, 1u);
          tc::mma_tf32_ta(dacc, slo + ks * 8, dPh, idesc, 1u);
        }
        tc::mma_commit(&sfree[st]);
        if (u % F == F - 1 || u == nchunks - 1) tc::mma_commit(&hfull[hb]);
      }
      tc::mma_commit(&mdone);
      if (!tc::mbar_wait_ns(&mdone, 0u, tc::kWaitNs)) s_bad = 1;
    }
  } else {
    // ---------------- formation: lane = A column a (TMEM lane), 16 rows of the chunk per warp ----------------
    constexpr int FCOLS = NJ / 2;  // sum columns per warp (flush, epilogue)
    const int quarter = warp & 3, half = warp >> 2;
    const int L = 32 * quarter + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    // F column jj = L (L < 64): its B row in the chunk (B's own, or A's with bsame) and weight
    const bool frow = L < NJ;
    const int j = j0 + L;
    const int wk = nbw > 0 ? j / nbw : 0;
    const int bcol = nbw > 0 ? j - wk * nbw : (bsame ? j : L);
    const int fr = bsame ? boff + bcol : bcol;
    const bool fok = frow && fr < (bsame ? NA : NJ) && wk < nk;
    auto sw_off = [](int r, int q) { return (uint32_t)(r * 128) + ((((uint32_t)q) ^ (uint32_t)(r & 7)) << 4); };
    // long (+)= short sums of group gi: this warp's lanes, FCOLS columns
    auto flush = [&](int gi) -> bool {
      bool ok = !s_bad && tc::mbar_wait_ns(&hfull[gi & 1], (uint32_t)((gi >> 1) & 1), tc::kWaitNs);
      if (!__all_sync(0xffffffffu, ok)) return false;  // tcgen05.ld / st are warp-collective
      tc::fence_after();
#pragma unroll 1
      for (int c8 = 0; c8 < FCOLS; c8 += 8) {
        const uint32_t col = (uint32_t)(half * FCOLS + c8);
        float sv[8], lv[8];
        tc::tmem_ld8(lane_base + (uint32_t)((gi & 1) * NJ) + col, sv);
        if (gi > 0) {
          tc::tmem_ld8(lane_base + C::LCOL + col, lv);
#pragma unroll
          for (int q = 0; q < 8; ++q) sv[q] += lv[q];
        }
        tc::tmem_st8(lane_base + C::LCOL + col, sv);
      }
      tc::tmem_st_wait();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&hfree[gi & 1]);
      return true;
    };
    int gdone = 0;
    bool go = true;
    for (int u = 0; u < nchunks && go; ++u) {
      const int st = u % NS;
      // the products finished chunk u - NS: take the short sums of the group it closed
      if (u >= NS && (u - NS) % F == F - 1) {
        if (!flush(gdone)) {
          s_bad = 1;
          go = false;
          break;
        }
        ++gdone;
      }
      bool ok = !s_bad && tc::mbar_wait_ns(&rfull[u & (R - 1)], (uint32_t)((u / R) & 1), tc::kWaitNs);
      if (ok && u >= NS) ok = tc::mbar_wait_ns(&sfree[st], (uint32_t)(((u - NS) / NS) & 1), tc::kWaitNs);
      if (!__all_sync(0xffffffffu, ok)) {
        s_bad = 1;
        go = false;
        break;
      }
      tc::fence_after();
      const unsigned char* sp = slot_ptr(u);
      // every shared-memory load first
      float4 xa[4], xf[4], wf[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int q = 4 * half + i;
        xa[i] = L < NA ? *reinterpret_cast<const float4*>(sp + sw_off(L, q)) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (fok) {
          xf[i] = *reinterpret_cast<const float4*>((bsame ? sp : sp + C::ABYTES) + sw_off(fr, q));
          wf[i] = nbw > 0 ? *reinterpret_cast<const float4*>(sp + C::ABYTES + C::BBYTES + wk * 128 + 16 * q)
                          : make_float4(1.f, 1.f, 1.f, 1.f);
        } else {
          xf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          wf[i] = xf[i];
        }
      }
      // A rows into TMEM (hi, lo), rows 16 half .. of the chunk
      const uint32_t scol = lane_base + C::SCOL + st * 64 + 16 * half;
#pragma unroll
      for (int g8 = 0; g8 < 2; ++g8) {
        const float v[8] = {xa[2 * g8].x, xa[2 * g8].y, xa[2 * g8].z, xa[2 * g8].w,
                            xa[2 * g8 + 1].x, xa[2 * g8 + 1].y, xa[2 * g8 + 1].z, xa[2 * g8 + 1].w};
        float hv[8], lv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) tc::split_tf32(v[t], hv[t], lv[t]);
        tc::tmem_st8(scol + 8 * g8, hv);
        tc::tmem_st8(scol + 32 + 8 * g8, lv);
      }
      // F row jj = L, K-major (two core-matrix rows per 8 cells)
      if (frow) {
        float* Phi = reinterpret_cast<float*>(base + C::OFF_P + (size_t)st * 2 * C::PPART);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = 4 * half + i;
          float4 hi, lo;
          tc::split_tf32(xf[i].x * wf[i].x, hi.x, lo.x);
          tc::split_tf32(xf[i].y * wf[i].y, hi.y, lo.y);
          tc::split_tf32(xf[i].z * wf[i].z, hi.z, lo.z);
          tc::split_tf32(xf[i].w * wf[i].w, hi.w, lo.w);
          const int o = ((q * (NJ / 8) + (L >> 3)) << 5) + ((L & 7) << 2);
          *reinterpret_cast<float4*>(Phi + o) = hi;
          *reinterpret_cast<float4*>(Phi + C::PPART / 4 + o) = lo;
        }
      }
      tc::tmem_st_wait();
      tc::fence_before();
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&afull[st]);
        tc::mbar_arrive(&rfree[u & (R - 1)]);
      }
    }
    // the short sums still to take
    while (go && gdone < ngroups) {
      if (!flush(gdone)) {
        s_bad = 1;
        go = false;
        break;
      }
      ++gdone;
    }
  }
  __syncthreads();
  const bool alive = s_bad == 0;
  if (warp < NFORM && alive && nchunks > 0) {
    // this block's long sums: warp (quarter, half) reads its lanes' rows (A columns), half of the
    // 64 columns; every lane loads (warp-collective), only the atomics are guarded
    tc::fence_after();
    const int quarter = warp & 3, half = warp >> 2;
    const int a = 32 * quarter + lane;
#pragma unroll
    for (int c16 = 0; c16 < NJ / 2; c16 += 16) {
      const int jj0 = half * (NJ / 2) + c16;
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + C::LCOL + (uint32_t)jj0, v);
      if (a >= Aact) continue;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int jg = j0 + jj0 + q;
        if (jg >= ncols || v[q] == 0.f) continue;
        const int kk = nbw > 0 ? jg / nbw : 0, bb = nbw > 0 ? jg - kk * nbw : jg;
        if (kk >= nk || bb >= Jact) continue;
        atomicAdd(out + (long long)jg * ldo + a, (double)v[q]);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid == 0 && !alive && err) atomicOr(err, ERR_TIMEOUT);
  if (warp == 0) tc::tmem_dealloc(tmem, C::TCOLS);
}

}  // namespace

}  // namespace dlra

namespace dlra {

bool launch_gram_tt(cudaStream_t st, long long rows, const float* A, long long lda, const int* adim, int acap,
                    const float* B, long long ldb, const int* jdim, int jcap, int ncols, const float* wv, int nbw,
                    int nk, double* out, long long ldo, int* err) {
  if (rows <= 0 || rows >= (1LL << 31) || acap < 1 || acap > 128 || ncols < 1) return false;
  if (nbw > 0 && (nbw > 64 || nk < 1 || nk > GtShape<64>::NKMAX || !wv || ((uintptr_t)wv & 15u) != 0 || rows % 4 != 0)) return false;
  if (lda % 4 != 0 || ldb % 4 != 0 || ((uintptr_t)A & 15u) != 0 || ((uintptr_t)B & 15u) != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encode_fn();
  if (!enc) return false;
  const int NA = acap > 64 ? 128 : 64;
  const int bcols = nbw > 0 ? nbw : ncols;  // B columns read
  // B a column block of A (the Grams of the CholeskyQR2 passes, the material Grams): read from
  // A's chunk
  int bsame = 0, boff = 0;
  if (ldb == lda && B >= A) {
    const long long d = (long long)(B - A);
    if (d % lda == 0 && d / lda + bcols <= NA && d / lda < acap) bsame = 1, boff = (int)(d / lda);
  }
  auto map2 = [&](CUtensorMap* m, const float* p, long long ld, int cols, int box_cols, CUtensorMapSwizzle sw) {
    const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {32, (cuuint32_t)box_cols};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  CUtensorMap ma, mb, mw;
  if (!map2(&ma, A, lda, acap, NA, CU_TENSOR_MAP_SWIZZLE_128B)) return false;
  mb = ma;
  mw = ma;
  if (!bsame && !map2(&mb, B, ldb, bcols, 64, CU_TENSOR_MAP_SWIZZLE_128B)) return false;
  if (nbw > 0 && !map2(&mw, wv, rows, nk, nk, CU_TENSOR_MAP_SWIZZLE_NONE)) return false;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nsl = (ncols + 63) / 64;
  const long long chunks = (rows + 31) / 32;
  // one block per SM (the TMEM allocation takes all 512 columns), shared among the slices
  const int gx = (int)std::max(1LL, std::min(chunks, (long long)std::max(1, sms / nsl)));
  auto go = [&](auto kern, size_t smem, int threads) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<dim3(gx, nsl), threads, smem, st>>>(ma, mb, mw, rows, adim, acap, jdim, jcap, ncols, nbw, nk, bsame, boff,
                                              out, ldo, err);
  };
  if (NA == 128)
    go(gram_tt_kernel<128>, GtShape<128>::SMEM, GtShape<128>::THREADS);
  else
    go(gram_tt_kernel<64>, GtShape<64>::SMEM, GtShape<64>::THREADS);
  return true;
}

}  // namespace dlra
