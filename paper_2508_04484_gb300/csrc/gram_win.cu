// Stencil Gram on the tensor cores with a sliding TMA window (FP32 path, 3-D grids, A == B):
//   G_k[a][b] = sum_i X(i, a) D_k(rho^-1 X(:, b))(i),   k = 2 d + s  (Sec. 3.3.2-3.3.3),
// the Galerkin blocks of the L-step (r x r) and of the S-step (2r x 2r), as the product
// D[j][a] = sum_t S[j][t] P[a][t] over the cells t, with S[j][t] = D_k(rho^-1 X(:, b))(t),
// j = (s, b), and P[a][t] = X(t, a).
//
// The grid is cut into runs of 32 x-consecutive cells. The CTAs of slice d (one slice per axis)
// own the two stencils of axis d and walk lines of runs along that axis: along y (z) a run at
// (x0, y, z) needs the runs two cells before and after it, along x the runs on either side. A
// producer thread loads each run of all columns once (one 4-D TMA copy, 32 cells x NB columns,
// 128-byte swizzle, so that a warp reading one column per lane meets no bank conflicts; runs
// outside the grid read zeros, the vacuum ghost layer) and its rho^-1 (one 3-D copy) into a
// ring of R slots; a run's slot is released once the last chunk that reads it is formed. Eight
// formation warps (lane = TMEM lane = column b, two warps per lane quarter, 16 cells each) form
// the chunk's stencil values, split them into TF32 high and low parts and write them into TMEM
// (tcgen05.st: S is the MMA's A operand, M = j), and write the chunk's X values (split) K-major
// into shared memory (P, the B operand, N = a). One thread issues three tcgen05.mma kind::tf32
// per 8-cell K-slice and tile (hi*hi + hi*lo + lo*hi, FP32-accurate products, FP32 sums in
// TMEM). The CTAs are persistent (one per SM at 2r = 128); each adds its sums to the FP64
// output with one atomic per entry at the end. Every wait gives up after about a second
// (ERR_TIMEOUT).
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

// NB = 128: j = (s, b) on two 128-lane tiles (tile s, lane b); NB = 64: one tile, lane 64 s + b
template <int NB>
struct GwShape {
  static constexpr int NT = NB == 128 ? 2 : 1;                    // M tiles
  static constexpr int NPA = NB;                                   // MMA N (a)
  static constexpr int NS = NB == 128 ? 2 : 3;                     // chunk stages (S in TMEM, P in smem)
  static constexpr int R = NB == 128 ? 8 : 7;                      // run slots of the window ring
  static constexpr int TCOLS = NB == 128 ? 512 : 256;
  static constexpr int SCOL = NT * NPA;                            // first S column (after the sums)
  static constexpr int SSTAGE = NT * 64;                           // S columns per stage (hi 32 + lo 32 per tile)
  static constexpr int NFORM = 8;                                  // formation warps
  static constexpr int THREADS = 32 * (NFORM + 2);
  static constexpr uint32_t RUN_BYTES = NB * 128;                  // one run of NB columns
  static constexpr uint32_t RHO_BYTES = 128;
  static constexpr size_t OFF_RUN = 0;
  static constexpr size_t OFF_RHO = OFF_RUN + (size_t)R * RUN_BYTES;
  static constexpr size_t OFF_P = (OFF_RHO + (size_t)R * RHO_BYTES + 1023) / 1024 * 1024;
  static constexpr size_t PPART = (size_t)NPA * 32 * 4;            // P hi (or lo) of one chunk
  static constexpr size_t SMEM = OFF_P + (size_t)NS * 2 * PPART + 1024;
  static_assert(SCOL + NS * SSTAGE <= TCOLS, "TMEM columns");
};

// The chunks of slice d: lines of runs along axis d (x: lines (y, z) of nxr runs; y: lines
// (x-run, z) of ny runs; z: lines (x-run, y) of nz runs), numbered line-major. A CTA owns a
// contiguous range of them, cut into segments that stay within one line.
struct GwWalk {
  int d, nxr, len;  // axis, runs per x row, chunks per line
  long long lines;
  __device__ GwWalk(int d_, const Geo& g) : d(d_) {
    nxr = (g.nx + 31) / 32;
    len = d == 0 ? nxr : (d == 1 ? g.ny : g.nz);
    lines = d == 0 ? (long long)g.ny * g.nz : (long long)nxr * (d == 1 ? g.nz : g.ny);
  }
  __device__ long long total() const { return lines * len; }
  // TMA coordinates (x, y, z) of position p along the line
  __device__ void coords(long long line, int p, const Geo& g, int& x, int& y, int& z) const {
    if (d == 0) {
      x = 32 * p, y = (int)(line % g.ny), z = (int)(line / g.ny);
    } else if (d == 1) {
      x = 32 * (int)(line % nxr), y = p, z = (int)(line / nxr);
    } else {
      x = 32 * (int)(line % nxr), y = (int)(line / nxr), z = p;
    }
  }
};

template <int NB>
__global__ void __launch_bounds__(GwShape<NB>::THREADS, 1) gram_win_kernel(
    const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmR, Geo g, int na,
    const int* __restrict__ adim, double* __restrict__ out, int ldj, long long ldo, int* err) {
  using C = GwShape<NB>;
  constexpr int NT = C::NT, NPA = C::NPA, NS = C::NS, R = C::R, NFORM = C::NFORM;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 1023) & ~(uintptr_t)1023);
  // rfull: a run's copies landed; rfree: the run's last reader is done (one arrival per
  // formation warp); afull: a chunk's S (TMEM) and P (smem) are written; sfree: the chunk's
  // products are done with them
  __shared__ __align__(8) uint64_t rfull[R], rfree[R], afull[NS], sfree[NS], acc_bar;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = (int)(blockIdx.x % 3);
  const int nci = (int)((gridDim.x - d + 2) / 3), ci = (int)(blockIdx.x / 3);
  const GwWalk wk(d, g);
  const long long tot = wk.total();
  const long long c0 = tot * ci / nci, c1 = tot * (ci + 1) / nci;
  const int W = d == 0 ? 1 : 2;  // window radius in runs
  const int Aact = dev_dim(adim, na);
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
    tc::mbar_init(&acc_bar, 1);
    tc::mbar_fence_init();
    s_bad = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  auto run_ptr = [&](int e) { return base + C::OFF_RUN + (size_t)(e % R) * C::RUN_BYTES; };
  auto rho_ptr = [&](int e) {
    return reinterpret_cast<const float*>(base + C::OFF_RHO + (size_t)(e % R) * C::RHO_BYTES);
  };

  if (warp == NFORM) {
    // ---------------- copies: every run of the window once, in walking order ----------------
    if (lane == 0) {
      int e = 0;  // runs issued (a block walks far fewer than 2^31)
      bool ok = true;
      for (long long c = c0; c < c1 && ok;) {
        const long long line = c / wk.len;
        const int p0 = (int)(c % wk.len);
        const int p1 = (int)min((long long)wk.len, p0 + (c1 - c));
        for (int i = 0; i < p1 - p0 + 2 * W; ++i) {
          const int slot = (int)(e % R);
          if (e >= R &&
              (s_bad || !tc::mbar_wait_ns(&rfree[slot], (uint32_t)(((e / R) - 1) & 1), tc::kWaitNs))) {
            s_bad = 1;
            ok = false;
            break;
          }
          int x, y, z;
          wk.coords(line, p0 - W + i, g, x, y, z);
          tc::mbar_arrive_expect_tx(&rfull[slot], C::RUN_BYTES + C::RHO_BYTES);
          tc::tma_load_4d(base + C::OFF_RUN + (size_t)slot * C::RUN_BYTES, &tmX, x, y, z, 0, &rfull[slot]);
          tc::tma_load_3d(base + C::OFF_RHO + (size_t)slot * C::RHO_BYTES, &tmR, x, y, z, &rfull[slot]);
          ++e;
        }
        c += p1 - p0;
      }
      // no copy is still in flight when the block moves on
      for (int q = (e > R ? e - R : 0); q < e; ++q)
        tc::mbar_wait_ns(&rfull[q % R], (uint32_t)((q / R) & 1), tc::kWaitNs);
    }
  } else if (warp == NFORM + 1) {
    // ---------------- products: S from TMEM, P from shared memory ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_tf32(128, NPA);
      constexpr uint32_t bLBO = (NPA / 8) * 128;
      const int nchunks = (int)(c1 - c0);
      for (int u = 0; u < nchunks; ++u) {
        const int st = (int)(u % NS);
        if (s_bad || !tc::mbar_wait_ns(&afull[st], (uint32_t)((u / NS) & 1), tc::kWaitNs)) {
          s_bad = 1;
          break;
        }
        tc::fence_after();
        const uint32_t ph = tc::su32(base + C::OFF_P + (size_t)st * 2 * C::PPART), pl = ph + (uint32_t)C::PPART;
        const uint32_t sc = tmem + C::SCOL + st * C::SSTAGE;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const uint32_t shi = sc + t * 64, slo = shi + 32, dacc = tmem + t * NPA;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t bk = ks * 2 * bLBO;
            const uint64_t dPh = tc::smem_desc(ph + bk, bLBO, 128), dPl = tc::smem_desc(pl + bk, bLBO, 128);
            const uint32_t first = (u == 0 && ks == 0) ? 0u : 1u;
            tc::mma_tf32_ta(dacc, shi + ks * 8, dPh, idesc, first);
            tc::mma_tf32_ta(dacc, shi + ks * 8, dPl, idesc, 1u);
            tc::mma_tf32_ta(dacc, slo + ks * 8, dPh, idesc, 1u);
          }
        }
        tc::mma_commit(&sfree[st]);
      }
      tc::mma_commit(&acc_bar);
      if (!tc::mbar_wait_ns(&acc_bar, 0u, tc::kWaitNs)) s_bad = 1;
    }
  } else {
    // ---------------- formation: lane = TMEM lane, 16 cells of the chunk per warp ----------------
    const int quarter = warp & 3, half = warp >> 2;
    const int L = 32 * quarter + lane;
    const int b = NB == 128 ? L : (L & 63);   // column of the stencil rows this lane writes
    const int sN = NB == 128 ? 0 : (L >> 6);  // its stencil (NB = 64: one per lane)
    const bool bval = b < Aact;
    const bool prow = L < NPA;                // this lane also writes P row a = L
    const uint32_t sw = (uint32_t)(b & 7);    // 128-byte swizzle of this column's row
    const float iv = (float)g.inv2d[d];
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    int e_seg = 0, u = 0;
    bool go = true;
    for (long long c = c0; c < c1 && go;) {
      const int p0 = (int)(c % wk.len);
      const int nch = (int)min((long long)wk.len, p0 + (c1 - c)) - p0;
      for (int cc = 0; cc < nch; ++cc, ++u) {
        const int st = (int)(u % NS);
        bool ok = !s_bad;
        for (int j = 0; j <= 2 * W && ok; ++j) {
          const int q = e_seg + cc + j;
          ok = tc::mbar_wait_ns(&rfull[q % R], (uint32_t)((q / R) & 1), tc::kWaitNs);
        }
        if (ok && u >= NS) ok = tc::mbar_wait_ns(&sfree[st], (uint32_t)(((u - NS) / NS) & 1), tc::kWaitNs);
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.st is warp-collective
        if (!ok) {
          s_bad = 1;
          go = false;
          break;
        }
        tc::fence_after();
        float* Phi = reinterpret_cast<float*>(base + C::OFF_P + (size_t)st * 2 * C::PPART);
        float* Plo = Phi + C::PPART / 4;
        const uint32_t scol = lane_base + C::SCOL + st * C::SSTAGE + 16 * half;
        // eight cells at a time: their stencil values (hi, lo) go to TMEM with one st.x8 each
        float h0[8], l0[8], h1[8], l1[8];
        auto emit = [&](int t, float vm2, float vm1, float v0, float vp1, float vp2) {
          const float s0 = (-3.f * v0 + 4.f * vm1 - vm2) * iv;
          const float s1 = (3.f * v0 - 4.f * vp1 + vp2) * iv;
          if (NB == 128) {
            tc::split_tf32(s0, h0[t], l0[t]);
            tc::split_tf32(s1, h1[t], l1[t]);
          } else {
            tc::split_tf32(sN ? s1 : s0, h0[t], l0[t]);
          }
        };
        auto store8 = [&](int g8) {
          const uint32_t c8 = scol + 8 * g8;
          tc::tmem_st8(c8, h0);
          tc::tmem_st8(c8 + 32, l0);
          if (NB == 128) {
            tc::tmem_st8(c8 + 64, h1);
            tc::tmem_st8(c8 + 96, l1);
          }
        };
        // P row a = L, cells 4 q .. 4 q + 3 of the chunk (raw values, split)
        auto put_p = [&](int q, float4 x) {
          if (!prow) return;
          if (!bval) x = make_float4(0.f, 0.f, 0.f, 0.f);
          float4 hi, lo;
          tc::split_tf32(x.x, hi.x, lo.x);
          tc::split_tf32(x.y, hi.y, lo.y);
          tc::split_tf32(x.z, hi.z, lo.z);
          tc::split_tf32(x.w, hi.w, lo.w);
          const int o = ((q * (NPA / 8) + (L >> 3)) << 5) + ((L & 7) << 2);
          *reinterpret_cast<float4*>(Phi + o) = hi;
          *reinterpret_cast<float4*>(Plo + o) = lo;
        };
        auto ldx = [&](int e, int q) {
          return *reinterpret_cast<const float4*>(run_ptr(e) + b * 128 + (((uint32_t)q ^ sw) << 4));
        };
        auto ldr = [&](int e, int q) { return *reinterpret_cast<const float4*>(rho_ptr(e) + 4 * q); };
        const int ec = e_seg + cc + W;  // the chunk's own run
        if (W == 2) {
          // stencil along y or z: the same cell of the runs two before .. two after
#pragma unroll
          for (int g8 = 0; g8 < 2; ++g8) {
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
              const int q = 4 * half + 2 * g8 + qq;
              float4 xv[5], rv[5];
#pragma unroll
              for (int j = 0; j < 5; ++j) {
                xv[j] = ldx(ec - 2 + j, q);
                rv[j] = ldr(ec - 2 + j, q);
              }
              put_p(q, xv[2]);
              float v[5][4];
#pragma unroll
              for (int j = 0; j < 5; ++j) {
                v[j][0] = bval ? xv[j].x * rv[j].x : 0.f;
                v[j][1] = bval ? xv[j].y * rv[j].y : 0.f;
                v[j][2] = bval ? xv[j].z * rv[j].z : 0.f;
                v[j][3] = bval ? xv[j].w * rv[j].w : 0.f;
              }
#pragma unroll
              for (int i = 0; i < 4; ++i) emit(4 * qq + i, v[0][i], v[1][i], v[2][i], v[3][i], v[4][i]);
            }
            store8(g8);
          }
        } else {
          // stencil along x: cells 16 half - 4 .. 16 half + 19 from this run and its neighbours
          float w[24];
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            const int Q = 4 * half - 1 + i;
            const int e = Q < 0 ? ec - 1 : (Q >= 8 ? ec + 1 : ec);
            const float4 xv = ldx(e, Q & 7), rv = ldr(e, Q & 7);
            if (i >= 1 && i <= 4) put_p(Q, xv);
            w[4 * i] = bval ? xv.x * rv.x : 0.f;
            w[4 * i + 1] = bval ? xv.y * rv.y : 0.f;
            w[4 * i + 2] = bval ? xv.z * rv.z : 0.f;
            w[4 * i + 3] = bval ? xv.w * rv.w : 0.f;
          }
#pragma unroll
          for (int g8 = 0; g8 < 2; ++g8) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int c = 8 * g8 + t;
              emit(t, w[c + 2], w[c + 3], w[c + 4], w[c + 5], w[c + 6]);
            }
            store8(g8);
          }
        }
        tc::tmem_st_wait();
        tc::fence_before();
        tc::fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          tc::mbar_arrive(&afull[st]);
          // the runs this chunk reads for the last time
          const int jr = cc == nch - 1 ? 2 * W : 0;
          for (int j = 0; j <= jr; ++j) tc::mbar_arrive(&rfree[(e_seg + cc + j) % R]);
        }
      }
      e_seg += nch + 2 * W;
      c += nch;
    }
  }
  __syncthreads();
  const bool alive = s_bad == 0;
  if (warp < NFORM && alive && c1 > c0) {
    // the sums of this block: warp (quarter, half) reads its lanes' rows, half of the columns;
    // tcgen05.ld is warp-collective, so every lane loads and only the atomics are guarded
    tc::fence_after();
    const int quarter = warp & 3, half = warp >> 2;
    const int L = 32 * quarter + lane;
    const int b = NB == 128 ? L : (L & 63);
    constexpr int G16 = NT * NPA / 16;
    for (int gi = half * G16 / 2; gi < (half + 1) * G16 / 2; ++gi) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(gi * 16), v);
      const int t = gi * 16 / NPA, a0 = gi * 16 - t * NPA;
      const int s = NB == 128 ? t : (L >> 6);
      if (b >= Aact) continue;
      double* o = out + ((long long)(2 * d + s) * ldj + b) * ldo;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (a0 + j < Aact && v[j] != 0.f) atomicAdd(o + a0 + j, (double)v[j]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid == 0 && !alive && err) atomicOr(err, ERR_TIMEOUT);
  if (warp == 0) tc::tmem_dealloc(tmem, C::TCOLS);
}

}  // namespace

// The windowed kernel where it applies (A == B, 3-D, nx and the column stride multiples of 4,
// 16-byte aligned bases, at most 128 columns); false otherwise (nothing launched).
bool launch_gram_stencil_win(cudaStream_t st, long long rows, const float* A, long long lda, int na,
                             const int* adim, const float* B, long long ldb, int nb, const int* bdim,
                             const float* inv_rho, const Geo& g, double* out, int ldj, long long ldo, int* err) {
  if (A != B || lda != ldb || na != nb || adim != bdim || g.nact != 3 || nb < 1 || nb > 128) return false;
  if (g.nx % 4 != 0 || lda % 4 != 0 || ((uintptr_t)A & 15u) != 0 || ((uintptr_t)inv_rho & 15u) != 0) return false;
  if (rows != (long long)g.nx * g.ny * g.nz) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encode_fn();
  if (!enc) return false;
  const int NB = nb > 64 ? 128 : 64;
  CUtensorMap mx, mr;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)nb};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nxy * 4, (cuuint64_t)lda * 4};
    const cuuint32_t box[4] = {32, 1, 1, (cuuint32_t)NB};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(A), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nxy * 4};
    const cuuint32_t box[3] = {32, 1, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    if (enc(&mr, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(inv_rho), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto go = [&](auto kern, size_t smem, int threads, int tcols) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    // resident blocks never ask for more than the 512 TMEM columns of an SM
    per_sm = std::max(1, std::min(per_sm, 512 / tcols));
    const int grid = std::max(3, sms * per_sm);
    kern<<<grid, threads, smem, st>>>(mx, mr, g, na, adim, out, ldj, ldo, err);
  };
  if (NB == 128)
    go(gram_win_kernel<128>, GwShape<128>::SMEM, GwShape<128>::THREADS, GwShape<128>::TCOLS);
  else
    go(gram_win_kernel<64>, GwShape<64>::SMEM, GwShape<64>::THREADS, GwShape<64>::TCOLS);
  return true;
}

PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

}  // namespace dlra
