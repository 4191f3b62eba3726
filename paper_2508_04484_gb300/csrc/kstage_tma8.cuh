// The tensor-core stage with A in TMEM (kstage_tmaa_kernel) on chunks of eight input columns
// (K = 48 per chunk) instead of four: one TMA halo box of 8 columns and two consecutive 4-column B
// images (one bulk copy) per chunk, a two-stage ring, A stages of 96 TMEM columns (hi 48, lo 48)
// at 64 + 96 s. Half as many chunks per brick (barrier round trips, copy issues); the same
// products. Two blocks per SM (112 KB of shared memory each, 128-byte aligned parts).
#pragma once
#include "kstage_tma.cuh"

namespace dlra {

template <int RM>
struct KsTmaA8 {
  using Base = KsTma<RM, 1>;
  static constexpr int NK = 6, CC = 8, KC = 48, NP = Base::NP;
  static constexpr int TX = 8, TY = 4, TZ = 4, BX = 16, BY = 8, BZ = 8, HALO = BX * BY * BZ;
  static constexpr int NS = 2;                                     // ring stages (halo, B, A in TMEM)
  static constexpr int TCOLS = 256, ACOL = 64;                     // A stage s at ACOL + 96 s
  static constexpr int THREADS = 192;                              // 4 formation, producer, MMA warps
  static constexpr size_t al(size_t b) { return (b + 127) / 128 * 128; }
  static constexpr uint32_t BIMG_BYTES = 2 * Base::BIMG_BYTES;     // two consecutive 4-column images
  static constexpr size_t OFF_B = 0;
  static constexpr size_t OFF_H = al(BIMG_BYTES);
  static constexpr size_t STAGE = OFF_H + al((size_t)CC * HALO * 4);
  static constexpr size_t SMEM = NS * STAGE + 128;
  static constexpr uint32_t HALO_BYTES = CC * HALO * 4;
  static_assert(ACOL + 2 * KC * NS <= TCOLS, "A stages exceed the TMEM allocation");
};

template <int RM>
__global__ void __launch_bounds__(192) kstage_tmaa8_kernel(
    const __grid_constant__ CUtensorMap tmap, const float* __restrict__ y, float* __restrict__ yout,
    float* __restrict__ vout, long long ld, const float* __restrict__ inv_rho, Geo g,
    const float* __restrict__ Bimg, const int* __restrict__ rdim, float beta, int mode, int* err) {
  using C = KsTmaA8<RM>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, NP = C::NP, TCOLS = C::TCOLS, ACOL = C::ACOL, NS = C::NS;
  constexpr int TX = C::TX, TY = C::TY, BX = C::BX, BY = C::BY, HALO = C::HALO;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 127) & ~(uintptr_t)127);
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
  const int bxn = (g.nx + TX - 1) / TX, byn = (g.ny + TY - 1) / TY;
  const int blk = blockIdx.x;
  const int x0 = (blk % bxn) * TX, y0 = ((blk / bxn) % byn) * TY, z0 = (blk / (bxn * byn)) * C::TZ;
  auto stage_ptr = [&](int s, size_t off) { return reinterpret_cast<float*>(base + s * C::STAGE + off); };

  if (warp == 4) {
    // ---------------- producer: halo (TMA) and B image (bulk copy) of each chunk ----------------
    int issued = 0;
    if (lane == 0) {
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
  } else if (warp == 5) {
    // ---------------- products: A from TMEM, B from shared memory ----------------
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
        const uint32_t b0 = tc::su32(stage_ptr(s, C::OFF_B));
        const uint32_t ahi = tmem + ACOL + s * (2 * KC), alo = ahi + KC;
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          // K-slice ks: slice ks % 3 of the chunk's 4-column image ks / 3
          const uint32_t bh = b0 + (uint32_t)(ks / 3) * KsTma<RM, 1>::BIMG_BYTES + (uint32_t)(ks % 3) * 2 * bLBO;
          const uint32_t bl = bh + (uint32_t)(KsTma<RM, 1>::OFF_BLO - KsTma<RM, 1>::OFF_BHI);
          const uint64_t dBh = tc::smem_desc(bh, bLBO, 128), dBl = tc::smem_desc(bl, bLBO, 128);
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
    // ---------------- formation: one cell (TMEM lane) per thread ----------------
    const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
    const bool ok = x0 + lx < g.nx && y0 + ly < g.ny && z0 + lz < g.nz;
    float inv2[3];
#pragma unroll
    for (int da = 0; da < 3; ++da) inv2[da] = (float)g.inv2d[da];
    constexpr int SY = BX, SZ = BX * BY;
    const int hc = (lz + 2) * SZ + (ly + 2) * SY + (lx + 4);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
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
      const uint32_t ahi = lane_base + ACOL + s * (2 * KC);
#pragma unroll
      for (int q = 0; q < KC / 8; ++q) {
        tc::tmem_st8(ahi + q * 8, hi + q * 8);
        tc::tmem_st8(ahi + KC + q * 8, lo + q * 8);
      }
      tc::tmem_st_wait();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&afull_bar[s]);
    }
  }
  // the epilogue's state values, loaded while the last products run
  float yv[NP];
  if (warp < 4) {
    const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
    const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
    const bool ok = ix < g.nx && iy < g.ny && iz < g.nz;
    const long long i = ((long long)iz * g.ny + iy) * g.nx + ix;
#pragma unroll
    for (int c = 0; c < NP; ++c) yv[c] = (ok && c < RM) ? y[(long long)c * ld + i] : 0.f;
  }
  __syncthreads();
  const bool alive = s_bad == 0;
  if (warp < 4) {
    const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
    const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
    const bool ok = ix < g.nx && iy < g.ny && iz < g.nz;
    const long long i = ((long long)iz * g.ny + iy) * g.nx + ix;
    tc::fence_after();
    if (alive) {
      const float ir0 = ok ? inv_rho[i] : 0.f;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float acc[16];
        if (nch > 0) {
          tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, acc);
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
