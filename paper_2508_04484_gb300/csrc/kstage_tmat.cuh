// The tensor-core stage with A in TMEM (kstage_tmaa_kernel) on bricks of T 128-cell tiles
// stacked along z (8 x 4 x 4T cells): one TMA halo box (16 x 8 x (4T + 4) x 4 columns) and one
// B image serve all T tiles of a chunk, so the L2 reads per cell and chunk drop from
// (16 x 8 x 8 x 4 + 3 K) / 128 (halo + B image) to (16 x 8 x (4T + 4) x 4 + 3 K) / 128 T.
// TMEM: the T accumulators in columns [0, T NP), the A stages after them (tile t of stage s at
// T NP + s T 48 + 48 t: hi at +0, lo at +24); 4T formation warps (tile w / 4, lane quarter
// w % 4), one producer and one MMA warp. One block per SM (the allocation takes all 512
// columns). Every wait gives up after about a second (ERR_TIMEOUT).
#pragma once
#include "kstage_tma.cuh"

namespace dlra {

template <int RM, int T>
struct KsTmaT {
  using Base = KsTma<RM, 1>;
  static constexpr int NK = 6, CC = 4, KC = 24, NP = Base::NP;
  static constexpr int TX = 8, TY = 4, TZ = 4 * T;                   // brick
  static constexpr int BX = 16, BY = 8, BZ = TZ + 4, HALO = BX * BY * BZ;
  static constexpr int ACOL = T * NP;                                // first A column
  static constexpr int TCOLS = 512;
  // ring stages (halo, B, A in TMEM): as many as the TMEM left after the sums holds, at most 3
  static constexpr int NS = (TCOLS - ACOL) / (T * 48) < 3 ? (TCOLS - ACOL) / (T * 48) : 3;
  static constexpr int NFORM = 4 * T;
  static constexpr int THREADS = 32 * (NFORM + 2);
  static constexpr size_t al(size_t b) { return (b + 1023) / 1024 * 1024; }
  static constexpr uint32_t BIMG_BYTES = Base::BIMG_BYTES;
  static constexpr size_t OFF_B = 0;
  static constexpr size_t OFF_H = al(BIMG_BYTES);
  static constexpr size_t STAGE = OFF_H + al((size_t)CC * HALO * 4);
  static constexpr size_t SMEM = NS * STAGE + 1024;
  static constexpr uint32_t HALO_BYTES = CC * HALO * 4;
  static_assert(ACOL + NS * T * 48 <= TCOLS, "A stages exceed the TMEM allocation");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <int RM, int T>
unsigned kstage_tmat_grid(const Geo& g) {
  using C = KsTmaT<RM, T>;
  return (unsigned)(((g.nx + C::TX - 1) / C::TX) * ((g.ny + C::TY - 1) / C::TY) * ((g.nz + C::TZ - 1) / C::TZ));
}


// mode: as kstage_kernel (0 vout = rho^-1 (y + beta acc); 1 also yout = y + beta acc, vout =
// rho^-1 yout; 2 transposed operator: vout = beta rho^-1 acc, yout = y + vout)
template <int RM, int T>
__global__ void __launch_bounds__(KsTmaT<RM, T>::THREADS, 1) kstage_tmat_kernel(
    const __grid_constant__ CUtensorMap tmap, const float* __restrict__ y, float* __restrict__ yout,
    float* __restrict__ vout, long long ld, const float* __restrict__ inv_rho, Geo g,
    const float* __restrict__ Bimg, const int* __restrict__ rdim, float beta, int mode, int* err) {
  using C = KsTmaT<RM, T>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, NP = C::NP, TCOLS = C::TCOLS, ACOL = C::ACOL, NS = C::NS;
  constexpr int TX = C::TX, TY = C::TY, BX = C::BX, BY = C::BY, HALO = C::HALO, NFORM = C::NFORM;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[NS], afull_bar[NS], free_bar[NS], acc_bar;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = dev_dim(rdim, RM);
  const int nch = (r + CC - 1) / CC;
  if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&afull_bar[s], NFORM);
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
  const int bxn = (g.nx + TX - 1) / TX, byn = (g.ny + TY - 1) / TY;
  const int blk = blockIdx.x;
  const int x0 = (blk % bxn) * TX, y0 = ((blk / bxn) % byn) * TY, z0 = (blk / (bxn * byn)) * C::TZ;
  auto stage_ptr = [&](int s, size_t off) { return reinterpret_cast<float*>(base + s * C::STAGE + off); };
  // this formation thread's cell: tile warp / 4, lane quarter warp % 4, 32 cells per quarter
  const int tt = warp >> 2, tl = 32 * (warp & 3) + lane;
  const int lx = tl % TX, ly = (tl / TX) % TY, lz = 4 * tt + tl / (TX * TY);

  if (warp == NFORM) {
    // ---------------- producer: halo (TMA) and B image (bulk copy) of each chunk ----------------
    if (lane == 0) {
      int issued = 0;
      for (int ch = 0; ch < nch; ++ch) {
        const int s = ch % NS;
        if (ch >= NS &&
            (s_bad || !tc::mbar_wait_ns(&free_bar[s], (uint32_t)(((ch - NS) / NS) & 1), tc::kWaitNs))) {
          s_bad = 1;
          break;
        }
        tc::mbar_arrive_expect_tx(&full_bar[s], C::HALO_BYTES + C::BIMG_BYTES);
        tc::tma_load_4d(stage_ptr(s, C::OFF_H), &tmap, x0 - 4, y0 - 2, z0 - 2, ch * CC, &full_bar[s]);
        tc::bulk_load(stage_ptr(s, C::OFF_B), Bimg + (size_t)ch * (C::BIMG_BYTES / 4), C::BIMG_BYTES, &full_bar[s]);
        issued = ch + 1;
      }
      for (int ch = (issued >= NS ? issued - NS : 0); ch < issued; ++ch)
        tc::mbar_wait_ns(&full_bar[ch % NS], (uint32_t)((ch / NS) & 1), tc::kWaitNs);
    }
  } else if (warp == NFORM + 1) {
    // ---------------- products: A from TMEM, B from shared memory, T tiles per chunk ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_tf32(128, NP);
      constexpr uint32_t bLBO = (NP / 8) * 128;
      for (int ch = 0; ch < nch; ++ch) {
        const int s = ch % NS;
        if (s_bad || !tc::mbar_wait_ns(&afull_bar[s], (uint32_t)((ch / NS) & 1), tc::kWaitNs)) {
          s_bad = 1;
          break;
        }
        tc::fence_after();
        const uint32_t bh = tc::su32(stage_ptr(s, C::OFF_B));
        const uint32_t bl = bh + (uint32_t)(KsTma<RM, 1>::OFF_BLO - KsTma<RM, 1>::OFF_BHI);
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint32_t bk = ks * 2 * bLBO;
          const uint64_t dBh = tc::smem_desc(bh + bk, bLBO, 128), dBl = tc::smem_desc(bl + bk, bLBO, 128);
          const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
#pragma unroll
          for (int t = 0; t < T; ++t) {
            const uint32_t ahi = tmem + ACOL + (s * T + t) * 48, alo = ahi + 24, d = tmem + t * NP;
            tc::mma_tf32_ta(d, ahi + ks * 8, dBh, idesc, first);
            tc::mma_tf32_ta(d, ahi + ks * 8, dBl, idesc, 1u);
            tc::mma_tf32_ta(d, alo + ks * 8, dBh, idesc, 1u);
          }
        }
        tc::mma_commit(&free_bar[s]);
      }
      tc::mma_commit(&acc_bar);
      if (!tc::mbar_wait_ns(&acc_bar, 0u, tc::kWaitNs)) s_bad = 1;
    }
  } else {
    // ---------------- formation: one cell (TMEM lane of its tile) per thread ----------------
    const bool ok = x0 + lx < g.nx && y0 + ly < g.ny && z0 + lz < g.nz;
    float inv2[3];
#pragma unroll
    for (int da = 0; da < 3; ++da) inv2[da] = (float)g.inv2d[da];
    constexpr int SY = BX, SZ = BX * BY;
    const int hc = (lz + 2) * SZ + (ly + 2) * SY + (lx + 4);
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    for (int ch = 0; ch < nch; ++ch) {
      const int s = ch % NS;
      // the warp decides together: tcgen05.st is warp-collective
      bool go = !s_bad && tc::mbar_wait_ns(&full_bar[s], (uint32_t)((ch / NS) & 1), tc::kWaitNs);
      go = __all_sync(0xffffffffu, go);
      if (!go) {
        s_bad = 1;
        break;
      }
      const float* H = stage_ptr(s, C::OFF_H);
      float hi[KC], lo[KC];
#pragma unroll
      for (int cc = 0; cc < CC; ++cc) {
        const float* hv = H + cc * HALO + hc;
        const float v0 = hv[0];
#pragma unroll
        for (int da = 0; da < 3; ++da) {
          const int st = da == 0 ? 1 : (da == 1 ? SY : SZ);
          const float dm = ok ? (-3.f * v0 + 4.f * hv[-st] - hv[-2 * st]) * inv2[da] : 0.f;
          const float dp = ok ? (3.f * v0 - 4.f * hv[st] + hv[2 * st]) * inv2[da] : 0.f;
          tc::split_tf32(dm, hi[cc * NK + 2 * da], lo[cc * NK + 2 * da]);
          tc::split_tf32(dp, hi[cc * NK + 2 * da + 1], lo[cc * NK + 2 * da + 1]);
        }
      }
      const uint32_t ahi = lane_base + ACOL + (s * T + tt) * 48;
#pragma unroll
      for (int q = 0; q < KC / 8; ++q) {
        tc::tmem_st8(ahi + q * 8, hi + q * 8);
        tc::tmem_st8(ahi + 24 + q * 8, lo + q * 8);
      }
      tc::tmem_st_wait();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&afull_bar[s]);
    }
  }
  // the epilogue's state values, loaded while the last products run
  const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
  const bool cell = warp < NFORM && ix < g.nx && iy < g.ny && iz < g.nz;
  const long long i = cell ? ((long long)iz * g.ny + iy) * g.nx + ix : 0;
  float yv[NP];
  if (warp < NFORM) {
#pragma unroll
    for (int c = 0; c < NP; ++c) yv[c] = (cell && c < RM) ? y[(long long)c * ld + i] : 0.f;
  }
  __syncthreads();
  const bool alive = s_bad == 0;
  if (warp < NFORM) {
    tc::fence_after();
    if (alive) {
      const float ir0 = cell ? inv_rho[i] : 0.f;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float acc[16];
        if (nch > 0) {
          tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + tt * NP + c0, acc);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = 0.f;
        }
        if (!cell) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          if (c >= RM) break;
          const long long e = (long long)c * ld + i;
          if (mode == 2) {
            const float lam = beta * ir0 * acc[j];
            vout[e] = lam;
            yout[e] = yv[c] + lam;
          } else if (mode == 1) {
            const float yn = yv[c] + beta * acc[j];
            yout[e] = yn;
            vout[e] = ir0 * yn;
          } else {
            vout[e] = ir0 * (yv[c] + beta * acc[j]);
          }
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
