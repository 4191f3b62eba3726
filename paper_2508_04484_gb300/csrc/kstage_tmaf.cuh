// The tensor-core stage with A in TMEM and eight formation warps (kstage_tmaw_kernel) on a
// lighter staging of each chunk: five TMA boxes instead of the 16 x 8 x 8 halo box (the brick
// with its x halo, 24 x 4 x 4, and its four y and z faces, 8 x 2 x 4 and 8 x 4 x 2: 640 values
// per column instead of 1,024, the stencil being a cross), and the chunk's B operand copied as
// one FP32 image (6 KB at N = 64 instead of the 12 KB of high and low parts) that the formation
// warps split into TF32 high and low parts in shared memory. The x box is 24 values wide (x0 - 4
// to x0 + 19; 12 are needed) so that the four rows a warp reads (24 apart) fall in distinct bank
// octets: its halo reads are free of bank conflicts. Each chunk reads 15 of the 28 KB that
// kstage_tmaw_kernel's reads from L2. Four-stage ring (22 KB of shared memory per stage, A stages
// at 64 + 48 s in TMEM), 320 threads (8 formation, producer, MMA warps), two blocks per SM;
// every wait gives up after about a second (ERR_TIMEOUT). Without SPLIT the chunk's B operand is
// copied as the image of TF32 high and low parts (kstage_tma_bimg_kernel's, 12 KB at N = 64), so
// the formation warps only form A.
#pragma once
#include "kstage_tmaw.cuh"

namespace dlra {

template <int RM, bool SPLIT = true>
struct KsTmaF {
  using A = KsTmaA<RM>;
  static constexpr int NK = A::NK, CC = A::CC, KC = A::KC, NP = A::NP;
  static constexpr int TX = 8, TY = 4, TZ = 4;                    // brick
  static constexpr int XW = 24;                                    // x box width (from x0 - 4)
  static constexpr int XCOL = TZ * TY * XW;                        // x box values per column
  static constexpr int FCOL = TX * 2 * TZ;                          // values per column of a y face box
  static constexpr int NS = 4, TCOLS = 256, ACOL = 64;
  static constexpr int NFORM = 8, THREADS = 32 * (NFORM + 2);
  static constexpr int KH = KC / 2;
  static constexpr int BSZ = NP * KC;                              // floats of one B part
  static constexpr size_t al(size_t b) { return (b + 1023) / 1024 * 1024; }
  static constexpr size_t OFF_BH = 0, OFF_BL = al(BSZ * 4);
  static constexpr size_t OFF_X = OFF_BL + al(BSZ * 4);
  static constexpr size_t OFF_YL = OFF_X + al(CC * XCOL * 4);
  static constexpr size_t OFF_YH = OFF_YL + al(CC * FCOL * 4);
  static constexpr size_t OFF_ZL = OFF_YH + al(CC * FCOL * 4);
  static constexpr size_t OFF_ZH = OFF_ZL + al(CC * FCOL * 4);
  static constexpr size_t STAGE = OFF_ZH + al(CC * FCOL * 4);
  static constexpr size_t SMEM = NS * STAGE + 1024;
  // one chunk's B image: FP32 (split in shared memory) or the high and low parts
  static constexpr uint32_t BIMG_BYTES = SPLIT ? BSZ * 4 : (uint32_t)(OFF_X - OFF_BH);
  static constexpr uint32_t TX_BYTES = (CC * XCOL + 4 * CC * FCOL) * 4 + BIMG_BYTES;
  static constexpr int NCH = RM / CC;
  static_assert(ACOL + 48 * NS <= TCOLS, "A stages exceed the TMEM allocation");
  static_assert(SPLIT || OFF_BL - OFF_BH == KsTma<RM, 1>::OFF_BLO - KsTma<RM, 1>::OFF_BHI,
                "the high and low parts lie as in the split image");
  static_assert(TX * TY * 2 == FCOL, "the y and z face boxes (8 x 2 x 4, 8 x 4 x 2) hold as many values");
};

// The FP32 B image of every chunk, K-major as the stage keeps B_hi in shared memory:
// image[ch][kmajor(n, K)] = P_k[c][n] with K = cc NK + k, c = ch CC + cc (zero for n >= RM or
// c >= r). Built once per launch from the stacked P (rows (c NK + k), RM columns).
template <int RM>
__global__ void __launch_bounds__(256) kstage_tmaf_bimg_kernel(const float* __restrict__ Pst,
                                                               const int* __restrict__ rdim, float* __restrict__ img) {
  using C = KsTmaF<RM>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, NP = C::NP, BSZ = C::BSZ;
  const int r = dev_dim(rdim, RM);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= C::NCH * BSZ) return;
  const int ch = e / BSZ, q = e - ch * BSZ;
  const int n = q / KC, K = q - n * KC;
  const int cc = K / NK, k = K - cc * NK, c = ch * CC + cc;
  img[(size_t)ch * BSZ + tc::kmajor(n, K, NP)] = (n < RM && c < r) ? Pst[((long long)c * NK + k) * RM + n] : 0.f;
}

// Float offsets (from the stage base) of a formation thread's cell (lx, ly, lz) and its 12
// stencil neighbours in the five boxes of configuration C, for its warp group's first column
// (column 2 grp of the chunk): 0 the cell, then per axis x, y, z the minus side (-1, -2) and the
// plus side (+1, +2). The group's second column adds strd[j], the column stride of the box the
// neighbour lies in (XCOL in the x box, FCOL in a face box). Host-callable so that the layout
// can be checked on the CPU.
template <class C>
__host__ __device__ __forceinline__ void tmaf_offsets(int lx, int ly, int lz, int grp, int* off, int* strd) {
  constexpr int TX = C::TX, TY = C::TY, TZ = C::TZ, XW = C::XW, XCOL = C::XCOL, FCOL = C::FCOL;
  constexpr int OX = (int)(C::OFF_X / 4), OYL = (int)(C::OFF_YL / 4), OYH = (int)(C::OFF_YH / 4);
  constexpr int OZL = (int)(C::OFF_ZL / 4), OZH = (int)(C::OFF_ZH / 4);
  const int ca = 2 * grp;
  auto xoff = [&](int zz, int yy, int xx) { return OX + ca * XCOL + (zz * TY + yy) * XW + xx + 4; };
  off[0] = xoff(lz, ly, lx);
  strd[0] = XCOL;
  off[1] = off[0] - 1; off[2] = off[0] - 2; off[3] = off[0] + 1; off[4] = off[0] + 2;
  strd[1] = strd[2] = strd[3] = strd[4] = XCOL;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int d = e < 2 ? -(e + 1) : e - 1;                        // -1, -2, +1, +2
    const int yy = ly + d, zz = lz + d;
    if (yy < 0) {
      off[5 + e] = OYL + ca * FCOL + (lz * 2 + yy + 2) * TX + lx;
      strd[5 + e] = FCOL;
    } else if (yy >= TY) {
      off[5 + e] = OYH + ca * FCOL + (lz * 2 + yy - TY) * TX + lx;
      strd[5 + e] = FCOL;
    } else {
      off[5 + e] = xoff(lz, yy, lx);
      strd[5 + e] = XCOL;
    }
    if (zz < 0) {
      off[9 + e] = OZL + ca * FCOL + ((zz + 2) * TY + ly) * TX + lx;
      strd[9 + e] = FCOL;
    } else if (zz >= TZ) {
      off[9 + e] = OZH + ca * FCOL + ((zz - TZ) * TY + ly) * TX + lx;
      strd[9 + e] = FCOL;
    } else {
      off[9 + e] = xoff(zz, ly, lx);
      strd[9 + e] = XCOL;
    }
  }
}

// mode: as kstage_kernel (0 vout = rho^-1 (y + beta acc); 1 also yout = y + beta acc, vout =
// rho^-1 yout; 2 transposed operator: vout = beta rho^-1 acc, yout = y + vout). Tensor maps of
// the stage input: mx with box (XW, 4, 4, CC), my (8, 2, 4, CC), mz (8, 4, 2, CC).
template <int RM, bool SPLIT>
__global__ void __launch_bounds__(320, 2) kstage_tmaf_kernel(
    const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap my,
    const __grid_constant__ CUtensorMap mz, const float* __restrict__ y, float* __restrict__ yout,
    float* __restrict__ vout, long long ld, const float* __restrict__ inv_rho, Geo g,
    const float* __restrict__ Bimg, const int* __restrict__ rdim, float beta, int mode, int* err) {
  using C = KsTmaF<RM, SPLIT>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, KH = C::KH, NP = C::NP, TCOLS = C::TCOLS, ACOL = C::ACOL;
  constexpr int NS = C::NS, TX = C::TX, TY = C::TY, TZ = C::TZ, XW = C::XW, NFORM = C::NFORM, BSZ = C::BSZ;
  constexpr int XCOL = C::XCOL, FCOL = C::FCOL;
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
  const int x0 = (blk % bxn) * TX, y0 = ((blk / bxn) % byn) * TY, z0 = (blk / (bxn * byn)) * TZ;
  auto stage_ptr = [&](int s, size_t off) { return reinterpret_cast<float*>(base + s * C::STAGE + off); };
  const int q = warp & 3, grp = (warp >> 2) & 1;
  const int cid = q * 32 + lane;
  const int lx = cid % TX, ly = (cid / TX) % TY, lz = cid / (TX * TY);

  if (warp == NFORM) {
    // ---------------- producer: five boxes (TMA) and the B image (bulk copy) of each chunk ----------------
    int issued = 0;
    if (lane == 0) {
      for (int ch = 0; ch < nch; ++ch) {
        const int s = ch % NS;
        if (ch >= NS &&
            (s_bad || !tc::mbar_wait_ns(&free_bar[s], (uint32_t)(((ch - NS) / NS) & 1), tc::kWaitNs))) {
          s_bad = 1;
          break;
        }
        const int c0 = ch * CC;
        tc::mbar_arrive_expect_tx(&full_bar[s], C::TX_BYTES);
        tc::tma_load_4d(stage_ptr(s, C::OFF_X), &mx, x0 - 4, y0, z0, c0, &full_bar[s]);
        tc::tma_load_4d(stage_ptr(s, C::OFF_YL), &my, x0, y0 - 2, z0, c0, &full_bar[s]);
        tc::tma_load_4d(stage_ptr(s, C::OFF_YH), &my, x0, y0 + TY, z0, c0, &full_bar[s]);
        tc::tma_load_4d(stage_ptr(s, C::OFF_ZL), &mz, x0, y0, z0 - 2, c0, &full_bar[s]);
        tc::tma_load_4d(stage_ptr(s, C::OFF_ZH), &mz, x0, y0, z0 + TZ, c0, &full_bar[s]);
        tc::bulk_load(stage_ptr(s, C::OFF_BH), Bimg + (size_t)ch * (C::BIMG_BYTES / 4), C::BIMG_BYTES, &full_bar[s]);
        issued = ch + 1;
      }
      for (int ch = (issued >= NS ? issued - NS : 0); ch < issued; ++ch)
        tc::mbar_wait_ns(&full_bar[ch % NS], (uint32_t)((ch / NS) & 1), tc::kWaitNs);
    }
  } else if (warp == NFORM + 1) {
    // ---------------- products: A from TMEM, B (split in place) from shared memory ----------------
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
        const uint32_t bh = tc::su32(stage_ptr(s, C::OFF_BH));
        const uint32_t bl = bh + (uint32_t)(C::OFF_BL - C::OFF_BH);
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
    int off[13], strd[13];
    tmaf_offsets<C>(lx, ly, lz, grp, off, strd);
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    const int ftid = warp * 32 + lane;                               // 0 .. 255
    for (int ch = 0; ch < nch; ++ch) {
      const int s = ch % NS;
      // the warp decides together: tcgen05.st is warp-collective
      bool go = !s_bad && tc::mbar_wait_ns(&full_bar[s], (uint32_t)((ch / NS) & 1), tc::kWaitNs);
      go = __all_sync(0xffffffffu, go);
      if (!go) {
        s_bad = 1;
        break;
      }
      const float* S = stage_ptr(s, 0);
      // this thread's share of the B split: B_hi in place, B_lo beside it
      if constexpr (SPLIT) {
        float* bh = stage_ptr(s, C::OFF_BH);
        float* bl = stage_ptr(s, C::OFF_BL);
        for (int e = ftid; e < BSZ; e += 32 * NFORM) {
          float hi, lo;
          tc::split_tf32(bh[e], hi, lo);
          bh[e] = hi;
          bl[e] = lo;
        }
        tc::fence_async_smem();
      }
      float hi[KH], lo[KH];
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        auto at = [&](int j) { return S[off[j] + cc * strd[j]]; };
        const float v0 = at(0);
        // neighbours: minus side (j, j + 1) = (-1, -2) and plus side (j + 2, j + 3) = (+1, +2)
#pragma unroll
        for (int da = 0; da < 3; ++da) {
          const int j = 1 + 4 * da;
          const float dm = ok ? (-3.f * v0 + 4.f * at(j) - at(j + 1)) * inv2[da] : 0.f;
          const float dp = ok ? (3.f * v0 - 4.f * at(j + 2) + at(j + 3)) * inv2[da] : 0.f;
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
  constexpr int NB = (NP / 16 + 1) / 2;
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
