// The tensor-core stage with A in TMEM (kstage_tmaa_kernel) with eight formation warps: warp w
// forms the stencil values of two of the chunk's four input columns (column pair w / 4) for the
// 32 cells of TMEM lane quarter w % 4, so twice as many warps share the halo reads, their
// latency and the TF32 splits of a chunk; the epilogue splits the output columns between the two
// warp groups the same way (16-column blocks alternating). Halo box, B image, TMEM layout
// (accumulator in [0, NP), A stage s at 64 + 48 s: hi at +0, lo at +24, K index 6 c + 2 a + s
// for chunk column c, axis a and side s), three-stage ring and bounded waits as
// kstage_tmaa_kernel; 320 threads (8 formation, producer, MMA warps), two blocks per SM.
#pragma once
#include "kstage_tma.cuh"

namespace dlra {

template <int RM>
struct KsTmaW {
  using A = KsTmaA<RM>;
  static constexpr int NK = A::NK, CC = A::CC, KC = A::KC, NP = A::NP;
  static constexpr int TX = A::TX, TY = A::TY, TZ = A::TZ, BX = A::BX, BY = A::BY, HALO = A::HALO;
  static constexpr int NS = A::NS, TCOLS = A::TCOLS, ACOL = A::ACOL;
  static constexpr int NFORM = 8, THREADS = 32 * (NFORM + 2);
  static constexpr int KH = KC / 2;                                // K values a warp group forms
  static constexpr size_t OFF_B = A::OFF_B, OFF_H = A::OFF_H, STAGE = A::STAGE, SMEM = A::SMEM;
  static constexpr uint32_t BIMG_BYTES = A::BIMG_BYTES, HALO_BYTES = A::HALO_BYTES;
  static_assert(KH == 12, "two chunk columns of six stencil values per warp group");
};

// mode: as kstage_kernel (0 vout = rho^-1 (y + beta acc); 1 also yout = y + beta acc, vout =
// rho^-1 yout; 2 transposed operator: vout = beta rho^-1 acc, yout = y + vout)
template <int RM>
__global__ void __launch_bounds__(320, 2) kstage_tmaw_kernel(
    const __grid_constant__ CUtensorMap tmap, const float* __restrict__ y, float* __restrict__ yout,
    float* __restrict__ vout, long long ld, const float* __restrict__ inv_rho, Geo g,
    const float* __restrict__ Bimg, const int* __restrict__ rdim, float beta, int mode, int* err) {
  using C = KsTmaW<RM>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, KH = C::KH, NP = C::NP, TCOLS = C::TCOLS, ACOL = C::ACOL;
  constexpr int NS = C::NS, TX = C::TX, TY = C::TY, BX = C::BX, BY = C::BY, HALO = C::HALO, NFORM = C::NFORM;
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
  // formation and epilogue warps: the cell of this lane (TMEM lane quarter warp % 4) and the
  // warp's column group
  const int q = warp & 3, grp = (warp >> 2) & 1;
  const int cid = q * 32 + lane;
  const int lx = cid % TX, ly = (cid / TX) % TY, lz = cid / (TX * TY);

  if (warp == NFORM) {
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
  } else if (warp == NFORM + 1) {
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
        tc::mma_commit(&free_bar[s]);
      }
      tc::mma_commit(&acc_bar);
      if (!tc::mbar_wait_ns(&acc_bar, 0u, tc::kWaitNs)) s_bad = 1;
    }
  } else {
    // ---------------- formation: one cell (TMEM lane) per thread, two chunk columns ----------------
    const bool ok = x0 + lx < g.nx && y0 + ly < g.ny && z0 + lz < g.nz;
    float inv2[3];
#pragma unroll
    for (int da = 0; da < 3; ++da) inv2[da] = (float)g.inv2d[da];
    constexpr int SY = BX, SZ = BX * BY;
    const int hc = (lz + 2) * SZ + (ly + 2) * SY + (lx + 4) + grp * 2 * HALO;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
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
      float hi[KH], lo[KH];
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
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
      const uint32_t ahi = lane_base + ACOL + s * 48 + grp * KH;
      // four-column stores: every TMEM column offset here is a multiple of four
#pragma unroll
      for (int j = 0; j < KH; j += 4) {
        tc::tmem_st4(ahi + j, hi + j);
        tc::tmem_st4(ahi + 24 + j, lo + j);
      }
      tc::tmem_st_wait();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&afull_bar[s]);
    }
  }
  // the epilogue's state values (this warp group's 16-column blocks), loaded while the last
  // products run
  constexpr int NB = (NP / 16 + 1) / 2;                            // blocks per warp group
  float yv[NB * 16];
  const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
  const bool okc = ix < g.nx && iy < g.ny && iz < g.nz;
  const long long i = ((long long)iz * g.ny + iy) * g.nx + ix;
  if (warp < NFORM) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = (2 * b + grp) * 16 + j;
        yv[b * 16 + j] = (okc && c < RM && c < NP) ? y[(long long)c * ld + i] : 0.f;
      }
    }
  }
  __syncthreads();
  const bool alive = s_bad == 0;
  if (warp < NFORM) {
    tc::fence_after();
    if (alive) {
      const float ir0 = okc ? inv_rho[i] : 0.f;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int c0 = (2 * b + grp) * 16;
        if (c0 >= NP) break;                                       // uniform over the warp
        float acc[16];
        if (nch > 0) {
          tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + c0, acc);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = 0.f;
        }
        if (!okc) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          if (c >= RM) break;
          const long long e = (long long)c * ld + i;
          const float yc = yv[b * 16 + j];
          if (mode == 2) {
            const float lam = beta * ir0 * acc[j];
            vout[e] = lam;
            yout[e] = yc + lam;
          } else if (mode == 1) {
            const float yn = yc + beta * acc[j];
            yout[e] = yn;
            vout[e] = ir0 * yn;
          } else {
            vout[e] = ir0 * (yc + beta * acc[j]);
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
