// The tensor-core stage with A in TMEM (kstage_tmaa_kernel) on clusters of two CTAs that own
// y-adjacent 128-cell bricks (8 x 4 x 4 each): their halo boxes overlap in y, so the leader
// loads one 16 x 12 x 8 x 4 box covering both bricks and multicasts it, together with the
// chunk's B image, into both CTAs' shared memory (TMA multicast within this GPU's memory).
// Per cell and chunk that is 96 + 48 bytes of L2 reads instead of 128 + 96. A stage is
// refilled only once the products of both CTAs have consumed it: each CTA's MMA thread commits
// to a cluster-wide free barrier (multicast arrive) on which the leader waits. Each CTA keeps
// its own TMEM accumulator and A stages, formation, products and epilogue. Every wait gives up
// after about a second (ERR_TIMEOUT); both CTAs meet at a cluster barrier before they exit, so
// neither leaves while copies or arrivals aimed at it may be in flight.
#pragma once
#include <cooperative_groups.h>

#include "kstage_tma.cuh"

namespace dlra {

template <int RM>
struct KsTmaC {
  using Base = KsTma<RM, 1>;
  static constexpr int NK = 6, CC = 4, KC = 24, NP = Base::NP;
  static constexpr int TX = 8, TY = 4, TZ = 4;                     // one brick
  static constexpr int BX = 16, BY = 12, BZ = 8, HALO = BX * BY * BZ;   // the pair's box
  static constexpr int NS = 3;
  static constexpr int TCOLS = 256, ACOL = 64;
  static constexpr int THREADS = 192;
  static constexpr size_t al(size_t b) { return (b + 1023) / 1024 * 1024; }
  static constexpr uint32_t BIMG_BYTES = Base::BIMG_BYTES;
  static constexpr size_t OFF_B = 0;
  static constexpr size_t OFF_H = al(BIMG_BYTES);
  static constexpr size_t STAGE = OFF_H + al((size_t)CC * HALO * 4);
  static constexpr size_t SMEM = NS * STAGE + 1024;
  static constexpr uint32_t HALO_BYTES = CC * HALO * 4;
  static_assert(ACOL + 48 * NS <= TCOLS, "A stages exceed the TMEM allocation");
};

// bricks of the pair grid: x fastest, then y pairs, then z; CTA 2 p + rank owns brick row
// 2 (p's y pair) + rank (a ragged last pair's second brick lies outside the grid and writes
// nothing)
template <int RM>
unsigned kstage_tmac_grid(const Geo& g) {
  const unsigned bxn = (g.nx + 7) / 8, bpn = ((g.ny + 3) / 4 + 1) / 2, bzn = (g.nz + 3) / 4;
  return 2u * bxn * bpn * bzn;
}

// launched with clusters of (2, 1, 1); arguments and modes as kstage_tmaa_kernel, the tensor map
// with a 16 x 12 x 8 x 4 box
template <int RM>
__global__ void __launch_bounds__(192) kstage_tmac_kernel(
    const __grid_constant__ CUtensorMap tmap, const float* __restrict__ y, float* __restrict__ yout,
    float* __restrict__ vout, long long ld, const float* __restrict__ inv_rho, Geo g,
    const float* __restrict__ Bimg, const int* __restrict__ rdim, float beta, int mode, int* err) {
  using C = KsTmaC<RM>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, NP = C::NP, TCOLS = C::TCOLS, ACOL = C::ACOL, NS = C::NS;
  constexpr int TX = C::TX, TY = C::TY, BX = C::BX, BY = C::BY, HALO = C::HALO;
  constexpr uint16_t BOTH = 0x3;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 1023) & ~(uintptr_t)1023);
  // full: this CTA's expect_tx arrival + the multicast copies' bytes; free: the products of both
  // CTAs (multicast commits); afull / acc as in kstage_tmaa_kernel
  __shared__ __align__(8) uint64_t full_bar[NS], afull_bar[NS], free_bar[NS], acc_bar;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = tc::cluster_ctarank();
  const int r = dev_dim(rdim, RM);
  const int nch = (r + CC - 1) / CC;
  if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&afull_bar[s], 4);
      tc::mbar_init(&free_bar[s], 2);
    }
    tc::mbar_init(&acc_bar, 1);
    tc::mbar_fence_init();
    s_bad = 0;
  }
  tc::fence_before();
  // both CTAs' barriers are initialised before either CTA's copies or commits reach them
  tc::cluster_sync();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const int bxn = (g.nx + TX - 1) / TX, bpn = ((g.ny + TY - 1) / TY + 1) / 2;
  const int pair = blockIdx.x >> 1;
  const int x0 = (pair % bxn) * TX, yp = ((pair / bxn) % bpn) * 2 * TY, z0 = (pair / (bxn * bpn)) * C::TZ;
  const int y0 = yp + (int)rank * TY;
  auto stage_ptr = [&](int s, size_t off) { return reinterpret_cast<float*>(base + s * C::STAGE + off); };

  if (warp == 4) {
    // ---------------- copies: the leader multicasts the pair's halo box and the B image ----------------
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
        if (rank == 0) {
          tc::tma_load_4d_mc(stage_ptr(s, C::OFF_H), &tmap, x0 - 4, yp - 2, z0 - 2, ch * CC, &full_bar[s], BOTH);
          tc::bulk_load_mc(stage_ptr(s, C::OFF_B), Bimg + (size_t)ch * (C::BIMG_BYTES / 4), C::BIMG_BYTES,
                           &full_bar[s], BOTH);
        }
        issued = ch + 1;
      }
      // this CTA's copies of the last chunks have landed and both CTAs' last commits reached
      // this CTA's free barriers
      for (int ch = (issued >= NS ? issued - NS : 0); ch < issued; ++ch)
        tc::mbar_wait_ns(&full_bar[ch % NS], (uint32_t)((ch / NS) & 1), tc::kWaitNs);
      if (!s_bad)
        for (int ch = (nch >= NS ? nch - NS : 0); ch < nch; ++ch)
          if (!tc::mbar_wait_ns(&free_bar[ch % NS], (uint32_t)((ch / NS) & 1), tc::kWaitNs)) {
            s_bad = 1;
            break;
          }
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
        const uint32_t bh = tc::su32(stage_ptr(s, C::OFF_B));
        const uint32_t bl = bh + (uint32_t)(KsTma<RM, 1>::OFF_BLO - KsTma<RM, 1>::OFF_BHI);
        const uint32_t ahi = tmem + ACOL + s * 48, alo = ahi + 24;
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint32_t bk = ks * 2 * bLBO;
          const uint64_t dBh = tc::smem_desc(bh + bk, bLBO, 128), dBl = tc::smem_desc(bl + bk, bLBO, 128);
          const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
          tc::mma_tf32_ta(tmem, ahi + ks * 8, dBh, idesc, first);
          tc::mma_tf32_ta(tmem, ahi + ks * 8, dBl, idesc, 1u);
          tc::mma_tf32_ta(tmem, alo + ks * 8, dBh, idesc, 1u);
        }
        // the stage is free in both CTAs once both CTAs' products are done with it
        tc::mma_commit_mc(&free_bar[s], BOTH);
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
    const int hc = (lz + 2) * SZ + (ly + 2 + (int)rank * TY) * SY + (lx + 4);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int ch = 0; ch < nch; ++ch) {
      const int s = ch % NS;
      bool go = !s_bad && tc::mbar_wait_ns(&full_bar[s], (uint32_t)((ch / NS) & 1), tc::kWaitNs);
      go = __all_sync(0xffffffffu, go);   // tcgen05.st is warp-collective
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
      const uint32_t ahi = lane_base + ACOL + s * 48;
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
  const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
  const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
  const bool cell = warp < 4 && ix < g.nx && iy < g.ny && iz < g.nz;
  const long long i = cell ? ((long long)iz * g.ny + iy) * g.nx + ix : 0;
  float yv[NP];
  if (warp < 4) {
#pragma unroll
    for (int c = 0; c < NP; ++c) yv[c] = (cell && c < RM) ? y[(long long)c * ld + i] : 0.f;
  }
  __syncthreads();
  const bool alive = s_bad == 0;
  if (warp < 4) {
    tc::fence_after();
    if (alive) {
      const float ir0 = cell ? inv_rho[i] : 0.f;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float acc[16];
        if (nch > 0) {
          tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, acc);
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
  // neither CTA leaves while a copy or a commit of the other may still be aimed at it
  tc::cluster_sync();
  if (tid == 0 && !alive && err) atomicOr(err, ERR_TIMEOUT);
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

}  // namespace dlra
