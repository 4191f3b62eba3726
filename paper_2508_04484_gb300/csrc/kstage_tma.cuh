// K-stage on the tensor cores with TMA halo staging (FP32 path, 3-D grids, rank capacity >= 32):
// acc(i, :) = sum_k D_k(v)(i, :) P_k, the r x r mix of the six stencil values of every input
// column (Sec. 3.3.2, Eq. KLS first line), as the product D[cells x N] = A[cells x K] B[K x N]
// with K = (column c, stencil k) = c NK + k and B[K][n] = P_k[c][n].
//
// A CTA owns a brick of 128 TILES cells (8 x 4 TILES x 4, one TMEM lane per cell) and walks the
// input columns in chunks of four (K = 24 per chunk) through a two-stage ring:
//   * the producer warp loads the chunk's input values of the brick and its two-cell halo with
//     one 4-D TMA copy (box 16 x (4 TILES + 4) x 8 x 4; the zero fill outside the grid is the
//     vacuum ghost layer) and the chunk's B rows (TF32 high and low parts, K-major, prepared
//     once per launch by kstage_tma_bimg_kernel) with one bulk copy;
//   * 4 TILES formation warps (one thread per cell) form the cell's 24 stencil values from the
//     staged halo, split them into TF32 high and low parts and store them K-major;
//   * one thread of the MMA warp issues three tcgen05.mma kind::tf32 per 8-wide K slice and
//     tile (hi*hi + hi*lo + lo*hi: FP32-accurate products, FP32 accumulation in tensor memory)
//     and commits to the stage's free barrier.
// The epilogue reads each cell's accumulator row from tensor memory and applies the Horner
// update of kstage_kernel. Every wait is bounded: a wait that runs out marks the block, stops
// the issue of new work, lets the copies and products in flight finish (bounded), frees the
// tensor memory and sets ERR_TIMEOUT.
#pragma once
#include "device.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace dlra {

template <int RM, int TILES>
struct KsTma {
  static constexpr int NACT = 3, NK = 6;
  static constexpr int NP = ((RM + 15) / 16) * 16;                  // MMA N
  static constexpr int TCOLS = TILES * NP <= 32 ? 32 : (TILES * NP <= 64 ? 64 : (TILES * NP <= 128 ? 128 : 256));
  static constexpr int CC = 4;                                       // columns per chunk
  static constexpr int KC = CC * NK;                                 // 24
  static constexpr int TX = 8, TY = 4 * TILES, TZ = 4;               // brick
  static constexpr int BX = 16, BY = TY + 4, BZ = TZ + 4;            // TMA box (x from x0 - 4)
  static constexpr int HALO = BX * BY * BZ;                          // values per column
  static constexpr int NFORM = 4 * TILES;                            // formation warps
  static constexpr int THREADS = 32 * (NFORM + 2);                   // + producer + MMA warps
  static constexpr int ASZ = 128 * TILES * KC;                       // floats per A part (hi or lo)
  static constexpr int BSZ = NP * KC;                                // floats per B part
  static constexpr int HSZ = CC * HALO;                              // floats per halo stage
  // per stage: Ahi, Alo, Bhi, Blo, halo; 1024-byte aligned parts
  static constexpr size_t al(size_t b) { return (b + 1023) / 1024 * 1024; }
  static constexpr size_t OFF_AHI = 0;
  static constexpr size_t OFF_ALO = al(ASZ * 4);
  static constexpr size_t OFF_BHI = OFF_ALO + al(ASZ * 4);
  static constexpr size_t OFF_BLO = OFF_BHI + al(BSZ * 4);
  static constexpr size_t OFF_H = OFF_BLO + al(BSZ * 4);
  static constexpr size_t STAGE = OFF_H + al(HSZ * 4);
  static constexpr size_t SMEM = 2 * STAGE + 1024;                   // + alignment slack
  static constexpr uint32_t HALO_BYTES = HSZ * 4;
  // B of one chunk as laid out in shared memory (hi part, then lo part): the image one bulk
  // copy loads
  static constexpr uint32_t BIMG_BYTES = (uint32_t)(OFF_H - OFF_BHI);
  static constexpr int NCH = RM / CC;                                // chunks at full capacity
};

// The B operand of every chunk, split into TF32 high and low parts and laid out K-major as the
// stage kernel keeps it in shared memory: image[ch] = [B_hi | B_lo], B[n][K] = P_k[c][n] with
// K = cc NK + k, c = ch CC + cc (zero for n >= RM or c >= r). Built once per launch from the
// stacked P (rows (c NK + k), RM columns).
template <int RM, int TILES>
__global__ void __launch_bounds__(256) kstage_tma_bimg_kernel(const float* __restrict__ Pst,
                                                              const int* __restrict__ rdim, float* __restrict__ img) {
  using C = KsTma<RM, TILES>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, NP = C::NP;
  const int r = dev_dim(rdim, RM);
  const int per = NP * KC;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= C::NCH * per) return;
  const int ch = e / per, q = e - ch * per;
  const int n = q / KC, K = q - n * KC;
  const int cc = K / NK, k = K - cc * NK, c = ch * CC + cc;
  const float pv = (n < RM && c < r) ? Pst[((long long)c * NK + k) * RM + n] : 0.f;
  float hi, lo;
  tc::split_tf32(pv, hi, lo);
  float* base = img + (size_t)ch * (C::BIMG_BYTES / 4);
  const int o = tc::kmajor(n, K, NP);
  base[o] = hi;
  base[(C::OFF_BLO - C::OFF_BHI) / 4 + o] = lo;
}

template <int RM, int TILES>
unsigned kstage_tma_grid(const Geo& g) {
  using C = KsTma<RM, TILES>;
  return (unsigned)(((g.nx + C::TX - 1) / C::TX) * ((g.ny + C::TY - 1) / C::TY) * ((g.nz + C::TZ - 1) / C::TZ));
}

// mode: as kstage_kernel (0 vout = rho^-1 (y + beta acc); 1 also yout = y + beta acc, vout =
// rho^-1 yout; 2 transposed operator: vout = beta rho^-1 acc, yout = y + vout)
template <int RM, int TILES>
__global__ void __launch_bounds__(KsTma<RM, TILES>::THREADS) kstage_tma_kernel(
    const __grid_constant__ CUtensorMap tmap, const float* __restrict__ y, float* __restrict__ yout,
    float* __restrict__ vout, long long ld, const float* __restrict__ inv_rho, Geo g,
    const float* __restrict__ Bimg, const int* __restrict__ rdim, float beta, int mode, int* err) {
  using C = KsTma<RM, TILES>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, NP = C::NP, TCOLS = C::TCOLS;
  constexpr int TX = C::TX, TY = C::TY, BX = C::BX, BY = C::BY, HALO = C::HALO;
  constexpr int NFORM = C::NFORM;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[2], afull_bar[2], free_bar[2], acc_bar;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = dev_dim(rdim, RM);
  const int nch = (r + CC - 1) / CC;
  if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&full_bar[s], 1);        // the producer's expect_tx arrival (halo and B copies)
      tc::mbar_init(&afull_bar[s], NFORM);   // one arrival per formation warp
      tc::mbar_init(&free_bar[s], 1);        // tcgen05.commit of the stage's products
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

  if (warp == NFORM) {
    // ---------------- producer: TMA halo + B rows of each chunk ----------------
    int issued = 0;
    for (int ch = 0; ch < nch; ++ch) {
      const int s = ch & 1;
      if (ch >= 2) {
        bool ok = true;
        if (lane == 0) ok = s_bad == 0 && tc::mbar_wait(&free_bar[s], (uint32_t)(((ch - 2) >> 1) & 1), tc::kWaitLimit);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) {
          s_bad = 1;
          break;
        }
      }
      if (lane == 0) {
        tc::mbar_arrive_expect_tx(&full_bar[s], C::HALO_BYTES + C::BIMG_BYTES);
        tc::tma_load_4d(stage_ptr(s, C::OFF_H), &tmap, x0 - 4, y0 - 2, z0 - 2, ch * CC, &full_bar[s]);
        tc::bulk_load(stage_ptr(s, C::OFF_BHI), Bimg + (size_t)ch * (C::BIMG_BYTES / 4), C::BIMG_BYTES, &full_bar[s]);
      }
      issued = ch + 1;
    }
    // copies in flight must land before the block leaves: wait (bounded) for the last phase
    // of each stage that this warp started
    if (lane == 0) {
      for (int ch = (issued >= 2 ? issued - 2 : 0); ch < issued; ++ch)
        tc::mbar_wait(&full_bar[ch & 1], (uint32_t)((ch >> 1) & 1), tc::kWaitLimit);
    }
  } else if (warp == NFORM + 1) {
    // ---------------- MMA issue ----------------
    int issued = 0;
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_tf32(128, NP);
      constexpr uint32_t aLBO = (128 / 8) * 128, bLBO = (NP / 8) * 128;
      for (int ch = 0; ch < nch; ++ch) {
        const int s = ch & 1;
        if (s_bad || !tc::mbar_wait(&afull_bar[s], (uint32_t)((ch >> 1) & 1), tc::kWaitLimit)) {
          s_bad = 1;
          break;
        }
        tc::fence_after();
        const uint32_t ah = tc::su32(stage_ptr(s, C::OFF_AHI)), al = tc::su32(stage_ptr(s, C::OFF_ALO));
        const uint32_t bh = tc::su32(stage_ptr(s, C::OFF_BHI)), bl = tc::su32(stage_ptr(s, C::OFF_BLO));
#pragma unroll
        for (int mt = 0; mt < TILES; ++mt) {
          const uint32_t d = tmem + mt * NP;
          const uint32_t ao = mt * 128 * KC * 4;
#pragma unroll
          for (int ks = 0; ks < KC / 8; ++ks) {
            const uint32_t ak = ao + ks * 2 * aLBO, bk = ks * 2 * bLBO;
            const uint64_t dAh = tc::smem_desc(ah + ak, aLBO, 128), dAl = tc::smem_desc(al + ak, aLBO, 128);
            const uint64_t dBh = tc::smem_desc(bh + bk, bLBO, 128), dBl = tc::smem_desc(bl + bk, bLBO, 128);
            const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
            tc::mma_tf32(d, dAh, dBh, idesc, first);
            tc::mma_tf32(d, dAh, dBl, idesc, 1u);
            tc::mma_tf32(d, dAl, dBh, idesc, 1u);
          }
        }
        tc::mma_commit(&free_bar[s]);
        ++issued;
      }
      // the accumulator is complete (or, after a failure, every issued product is done)
      tc::mma_commit(&acc_bar);
      if (!tc::mbar_wait(&acc_bar, 0u, tc::kWaitLimit)) s_bad = 1;
    }
    (void)issued;
  } else {
    // ---------------- formation: one cell per thread ----------------
    const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
    const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
    const bool ok = ix < g.nx && iy < g.ny && iz < g.nz;
    float inv2[3];
#pragma unroll
    for (int da = 0; da < 3; ++da) inv2[da] = (float)g.inv2d[da];
    constexpr int SY = BX, SZ = BX * BY;
    const int hc = (lz + 2) * SZ + (ly + 2) * SY + (lx + 4);
    const int tile = tid >> 7, row = tid & 127;
    const int abase = tile * 128 * KC + tc::kmajor(row, 0, 128);
    for (int ch = 0; ch < nch; ++ch) {
      const int s = ch & 1;
      if (s_bad || !tc::mbar_wait(&full_bar[s], (uint32_t)((ch >> 1) & 1), tc::kWaitLimit)) {
        s_bad = 1;
        break;
      }
      const float* H = stage_ptr(s, C::OFF_H);
      float sv[KC];
#pragma unroll
      for (int cc = 0; cc < CC; ++cc) {
        const float* hv = H + cc * HALO + hc;
        const float v0 = hv[0];
#pragma unroll
        for (int da = 0; da < 3; ++da) {
          const int st = da == 0 ? 1 : (da == 1 ? SY : SZ);
          sv[cc * NK + 2 * da] = ok ? (-3.f * v0 + 4.f * hv[-st] - hv[-2 * st]) * inv2[da] : 0.f;
          sv[cc * NK + 2 * da + 1] = ok ? (3.f * v0 - 4.f * hv[st] + hv[2 * st]) * inv2[da] : 0.f;
        }
      }
      float* Ah = stage_ptr(s, C::OFF_AHI);
      float* Al = stage_ptr(s, C::OFF_ALO);
#pragma unroll
      for (int kg = 0; kg < KC / 4; ++kg) {
        float4 h4, l4;
        tc::split_tf32(sv[4 * kg + 0], h4.x, l4.x);
        tc::split_tf32(sv[4 * kg + 1], h4.y, l4.y);
        tc::split_tf32(sv[4 * kg + 2], h4.z, l4.z);
        tc::split_tf32(sv[4 * kg + 3], h4.w, l4.w);
        // kmajor(row, 4 kg, 128) = kmajor(row, 0, 128) + kg * 16 * 32
        *reinterpret_cast<float4*>(Ah + abase + kg * 512) = h4;
        *reinterpret_cast<float4*>(Al + abase + kg * 512) = l4;
      }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&afull_bar[s]);
    }
  }
  // every role is done issuing; the MMA thread has waited for the last products
  __syncthreads();
  const bool alive = s_bad == 0;
  if (warp < NFORM) {
    const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
    const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
    const bool ok = ix < g.nx && iy < g.ny && iz < g.nz;
    const long long i = ((long long)iz * g.ny + iy) * g.nx + ix;
    tc::fence_after();
    if (alive) {
      // warp w reads TMEM lanes 32 (w % 4) .. of accumulator w / 4: exactly its own cells
      const float ir0 = ok ? inv_rho[i] : 0.f;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float acc[16];
        if (nch > 0) {
          tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (warp >> 2) * NP + c0, acc);
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
            yout[e] = y[e] + lam;
          } else if (mode == 1) {
            const float yn = y[e] + beta * acc[j];
            yout[e] = yn;
            vout[e] = ir0 * yn;
          } else {
            vout[e] = ir0 * (y[e] + beta * acc[j]);
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

namespace dlra {

// The same stage as kstage_tma_kernel (128-cell bricks) in a persistent form: one CTA per SM
// walks its bricks' chunks as one stream, through a ring of NH halo stages (TMA) and two A/B
// stages, and accumulates brick b in one of two TMEM accumulators while four epilogue warps
// drain the other (brick b - 1): the copies of later chunks, the products and the epilogue
// overlap. Warps 0-3 form the A operand, 4-7 run the epilogue (TMEM lanes = their cells), warp
// 8 issues the halo copies, warp 9 the B copies and the products. Every wait gives up after
// about a second (global timer): the block then stops issuing, waits (bounded) for its copies
// and products in flight, frees its tensor memory and sets ERR_TIMEOUT.
template <int RM>
struct KsTmaP {
  using Base = KsTma<RM, 1>;
  static constexpr int NK = 6, CC = 4, KC = 24, NP = Base::NP;
  static constexpr int TX = 8, TY = 4, TZ = 4, BX = 16, BY = 8, BZ = 8, HALO = BX * BY * BZ;
  static constexpr int NH = 4;                                     // halo stages
  static constexpr int TCOLS = 2 * NP <= 64 ? 64 : (2 * NP <= 128 ? 128 : 256);   // two accumulators
  static constexpr int THREADS = 320;
  static constexpr size_t al(size_t b) { return (b + 1023) / 1024 * 1024; }
  static constexpr size_t HBYTES = al((size_t)CC * HALO * 4);     // one halo stage
  static constexpr size_t ABYTES = al((size_t)128 * KC * 4);      // one A part (hi or lo)
  static constexpr uint32_t BIMG_BYTES = Base::BIMG_BYTES;        // one B stage (hi and lo)
  static constexpr size_t OFF_H = 0;
  static constexpr size_t OFF_A = NH * HBYTES;                     // [stage][hi, lo]
  static constexpr size_t OFF_B = OFF_A + 2 * 2 * ABYTES;          // [stage] hi, lo
  static constexpr size_t SMEM = OFF_B + 2 * (size_t)BIMG_BYTES + 1024;
  static constexpr uint32_t HALO_BYTES = CC * HALO * 4;
};

template <int RM>
__global__ void __launch_bounds__(320, 1) kstage_tmap_kernel(
    const __grid_constant__ CUtensorMap tmap, const float* __restrict__ y, float* __restrict__ yout,
    float* __restrict__ vout, long long ld, const float* __restrict__ inv_rho, Geo g,
    const float* __restrict__ Bimg, const int* __restrict__ rdim, float beta, int mode, int* err) {
  using C = KsTmaP<RM>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, NP = C::NP, NH = C::NH, TCOLS = C::TCOLS;
  constexpr int TX = C::TX, TY = C::TY, BX = C::BX, BY = C::BY, HALO = C::HALO;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t hfull[NH], hfree[NH], afull[2], abfree[2], bfull[2], accfull[2], accfree[2], fin;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = dev_dim(rdim, RM);
  const int nch = (r + CC - 1) / CC;
  const int bxn = (g.nx + TX - 1) / TX, byn = (g.ny + TY - 1) / TY, bzn = (g.nz + C::TZ - 1) / C::TZ;
  const int nbricks = bxn * byn * bzn;
  const int nb = blockIdx.x < nbricks ? (nbricks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = nb * nch;                                      // chunks this block streams
  if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
  if (tid == 0) {
    for (int s = 0; s < NH; ++s) {
      tc::mbar_init(&hfull[s], 1);
      tc::mbar_init(&hfree[s], 4);
    }
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&afull[s], 4);
      tc::mbar_init(&abfree[s], 1);
      tc::mbar_init(&bfull[s], 1);
      tc::mbar_init(&accfull[s], 1);
      tc::mbar_init(&accfree[s], 4);
    }
    tc::mbar_init(&fin, 1);
    tc::mbar_fence_init();
    s_bad = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  auto brick_origin = [&](int bl, int& x0, int& y0, int& z0) {
    const int b = (int)blockIdx.x + bl * (int)gridDim.x;
    x0 = (b % bxn) * TX;
    y0 = ((b / bxn) % byn) * TY;
    z0 = (b / (bxn * byn)) * C::TZ;
  };
  auto H = [&](int s) { return reinterpret_cast<float*>(base + C::OFF_H + s * C::HBYTES); };
  auto A = [&](int s, int part) { return reinterpret_cast<float*>(base + C::OFF_A + (2 * s + part) * C::ABYTES); };
  auto Bs = [&](int s) { return reinterpret_cast<float*>(base + C::OFF_B + s * (size_t)C::BIMG_BYTES); };

  if (warp == 8) {
    // ---------------- halo copies ----------------
    int issued = 0;
    if (lane == 0) {
      for (int q = 0; q < total; ++q) {
        const int h = q % NH;
        if (q >= NH && (s_bad || !tc::mbar_wait_ns(&hfree[h], (uint32_t)(((q - NH) / NH) & 1), tc::kWaitNs))) {
          s_bad = 1;
          break;
        }
        int x0, y0, z0;
        brick_origin(q / nch, x0, y0, z0);
        tc::mbar_arrive_expect_tx(&hfull[h], C::HALO_BYTES);
        tc::tma_load_4d(H(h), &tmap, x0 - 4, y0 - 2, z0 - 2, (q % nch) * CC, &hfull[h]);
        issued = q + 1;
      }
      // copies in flight land before the block leaves
      for (int q = (issued > NH ? issued - NH : 0); q < issued; ++q)
        tc::mbar_wait_ns(&hfull[q % NH], (uint32_t)((q / NH) & 1), tc::kWaitNs);
    }
  } else if (warp == 9) {
    // ---------------- B copies and products ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_tf32(128, NP);
      constexpr uint32_t aLBO = (128 / 8) * 128, bLBO = (NP / 8) * 128;
      int bissued = 0;
      if (total > 0) {
        tc::mbar_arrive_expect_tx(&bfull[0], C::BIMG_BYTES);
        tc::bulk_load(Bs(0), Bimg, C::BIMG_BYTES, &bfull[0]);
        bissued = 1;
      }
      for (int q = 0; q < total; ++q) {
        const int a = q & 1, bl = q / nch, ch = q % nch, t = bl & 1;
        bool ok = !s_bad;
        ok = ok && tc::mbar_wait_ns(&afull[a], (uint32_t)((q >> 1) & 1), tc::kWaitNs);
        ok = ok && tc::mbar_wait_ns(&bfull[a], (uint32_t)((q >> 1) & 1), tc::kWaitNs);
        if (ok && ch == 0 && bl >= 2) ok = tc::mbar_wait_ns(&accfree[t], (uint32_t)(((bl - 2) >> 1) & 1), tc::kWaitNs);
        if (!ok) {
          s_bad = 1;
          break;
        }
        tc::fence_after();
        const uint32_t ah = tc::su32(A(a, 0)), al = tc::su32(A(a, 1));
        const uint32_t bh = tc::su32(Bs(a)), blo = bh + (uint32_t)(KsTma<RM, 1>::OFF_BLO - KsTma<RM, 1>::OFF_BHI);
        const uint32_t d = tmem + t * NP;
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint32_t ak = ks * 2 * aLBO, bk = ks * 2 * bLBO;
          const uint64_t dAh = tc::smem_desc(ah + ak, aLBO, 128), dAl = tc::smem_desc(al + ak, aLBO, 128);
          const uint64_t dBh = tc::smem_desc(bh + bk, bLBO, 128), dBl = tc::smem_desc(blo + bk, bLBO, 128);
          const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
          tc::mma_tf32(d, dAh, dBh, idesc, first);
          tc::mma_tf32(d, dAh, dBl, idesc, 1u);
          tc::mma_tf32(d, dAl, dBh, idesc, 1u);
        }
        tc::mma_commit(&abfree[a]);
        if (ch == nch - 1) tc::mma_commit(&accfull[t]);
        // next chunk's B into the other stage, once the products that read it (chunk q - 1) are done
        if (q + 1 < total) {
          const int a1 = (q + 1) & 1;
          if (q >= 1 && !tc::mbar_wait_ns(&abfree[a1], (uint32_t)(((q - 1) >> 1) & 1), tc::kWaitNs)) {
            s_bad = 1;
            break;
          }
          tc::mbar_arrive_expect_tx(&bfull[a1], C::BIMG_BYTES);
          tc::bulk_load(Bs(a1), Bimg + (size_t)((q + 1) % nch) * (C::BIMG_BYTES / 4), C::BIMG_BYTES, &bfull[a1]);
          bissued = q + 2;
        }
      }
      // every product issued so far is done, and the B copies in flight have landed
      tc::mma_commit(&fin);
      tc::mbar_wait_ns(&fin, 0u, tc::kWaitNs);
      for (int q = (bissued > 2 ? bissued - 2 : 0); q < bissued; ++q)
        tc::mbar_wait_ns(&bfull[q & 1], (uint32_t)((q >> 1) & 1), tc::kWaitNs);
    }
  } else if (warp < 4) {
    // ---------------- formation: one cell per thread ----------------
    const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
    float inv2[3];
#pragma unroll
    for (int da = 0; da < 3; ++da) inv2[da] = (float)g.inv2d[da];
    constexpr int SY = BX, SZ = BX * BY;
    const int hc = (lz + 2) * SZ + (ly + 2) * SY + (lx + 4);
    const int abase = tc::kmajor(tid, 0, 128);
    for (int q = 0; q < total; ++q) {
      const int h = q % NH, a = q & 1;
      int x0, y0, z0;
      brick_origin(q / nch, x0, y0, z0);
      const bool ok = x0 + lx < g.nx && y0 + ly < g.ny && z0 + lz < g.nz;
      bool go = !s_bad && tc::mbar_wait_ns(&hfull[h], (uint32_t)((q / NH) & 1), tc::kWaitNs);
      if (go && q >= 2) go = tc::mbar_wait_ns(&abfree[a], (uint32_t)(((q - 2) >> 1) & 1), tc::kWaitNs);
      if (!go) {
        s_bad = 1;
        break;
      }
      const float* Hs = H(h);
      float sv[KC];
#pragma unroll
      for (int cc = 0; cc < CC; ++cc) {
        const float* hv = Hs + cc * HALO + hc;
        const float v0 = hv[0];
#pragma unroll
        for (int da = 0; da < 3; ++da) {
          const int st = da == 0 ? 1 : (da == 1 ? SY : SZ);
          sv[cc * NK + 2 * da] = ok ? (-3.f * v0 + 4.f * hv[-st] - hv[-2 * st]) * inv2[da] : 0.f;
          sv[cc * NK + 2 * da + 1] = ok ? (3.f * v0 - 4.f * hv[st] + hv[2 * st]) * inv2[da] : 0.f;
        }
      }
      // the halo stage is free once every formation warp has read it
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&hfree[h]);
      float* Ah = A(a, 0);
      float* Al = A(a, 1);
#pragma unroll
      for (int kg = 0; kg < KC / 4; ++kg) {
        float4 h4, l4;
        tc::split_tf32(sv[4 * kg + 0], h4.x, l4.x);
        tc::split_tf32(sv[4 * kg + 1], h4.y, l4.y);
        tc::split_tf32(sv[4 * kg + 2], h4.z, l4.z);
        tc::split_tf32(sv[4 * kg + 3], h4.w, l4.w);
        *reinterpret_cast<float4*>(Ah + abase + kg * 512) = h4;
        *reinterpret_cast<float4*>(Al + abase + kg * 512) = l4;
      }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&afull[a]);
    }
  } else {
    // ---------------- epilogue: warps 4-7, TMEM lanes 32 (warp % 4) .. ----------------
    const int row = tid - 128;
    const int lx = row % TX, ly = (row / TX) % TY, lz = row / (TX * TY);
    const bool has = nch > 0;   // rank 0: no products, the update with a zero accumulator
    for (int bl = 0; bl < nb; ++bl) {
      const int t = bl & 1;
      if (has && (s_bad || !tc::mbar_wait_ns(&accfull[t], (uint32_t)((bl >> 1) & 1), tc::kWaitNs))) {
        s_bad = 1;
        break;
      }
      tc::fence_after();
      int x0, y0, z0;
      brick_origin(bl, x0, y0, z0);
      const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
      const bool ok = ix < g.nx && iy < g.ny && iz < g.nz;
      const long long i = ((long long)iz * g.ny + iy) * g.nx + ix;
      const float ir0 = ok ? inv_rho[i] : 0.f;
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 16) {
        float acc[16];
        if (has) {
          tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + t * NP + c0, acc);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = 0.f;
        }
        if (!ok) continue;
        float yv[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) yv[j] = (c0 + j < RM) ? y[(long long)(c0 + j) * ld + i] : 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          if (c >= RM) break;
          const long long e = (long long)c * ld + i;
          if (mode == 2) {
            const float lam = beta * ir0 * acc[j];
            vout[e] = lam;
            yout[e] = yv[j] + lam;
          } else if (mode == 1) {
            const float yn = yv[j] + beta * acc[j];
            yout[e] = yn;
            vout[e] = ir0 * yn;
          } else {
            vout[e] = ir0 * (yv[j] + beta * acc[j]);
          }
        }
      }
      // the accumulator is free for brick bl + 2 once every epilogue warp has read it
      tc::fence_before();
      __syncwarp();
      if (has && lane == 0) tc::mbar_arrive(&accfree[t]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (tid == 0 && s_bad && err) atomicOr(err, ERR_TIMEOUT);
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

}  // namespace dlra

namespace dlra {

// The 128-cell TMA-staged stage with its A operand in tensor memory: the formation warps write
// each cell's 24 stencil values (TF32 high and low parts) into TMEM columns of the cell's lane
// (tcgen05.st) and the products read A from there (tcgen05.mma with an A address in TMEM), so
// neither the operand stores nor the tensor core's A reads use shared memory, which the halo
// reads and the B reads keep to themselves. TMEM: the accumulator in columns [0, NP), the A
// stages at 64 + 48 s (hi at +0, lo at +24), a three-stage ring; 256 columns, two blocks per SM.
// The formation threads load their cell's state row for the epilogue while the last products run.
template <int RM>
struct KsTmaA {
  using Base = KsTma<RM, 1>;
  static constexpr int NK = 6, CC = 4, KC = 24, NP = Base::NP;
  static constexpr int TX = 8, TY = 4, TZ = 4, BX = 16, BY = 8, BZ = 8, HALO = BX * BY * BZ;
  static constexpr int NS = 3;                                     // ring stages (halo, B, A in TMEM)
  static constexpr int TCOLS = 256, ACOL = 64;                     // A stage s at ACOL + 48 s
  static constexpr int THREADS = 192;                              // 4 formation, producer, MMA warps
  static constexpr size_t al(size_t b) { return (b + 1023) / 1024 * 1024; }
  static constexpr uint32_t BIMG_BYTES = Base::BIMG_BYTES;
  static constexpr size_t OFF_B = 0;
  static constexpr size_t OFF_H = al(BIMG_BYTES);
  static constexpr size_t STAGE = OFF_H + al((size_t)CC * HALO * 4);
  static constexpr size_t SMEM = NS * STAGE + 1024;
  static constexpr uint32_t HALO_BYTES = CC * HALO * 4;
  static_assert(ACOL + 48 * NS <= TCOLS, "A stages exceed the TMEM allocation");
};

template <int RM>
__global__ void __launch_bounds__(192) kstage_tmaa_kernel(
    const __grid_constant__ CUtensorMap tmap, const float* __restrict__ y, float* __restrict__ yout,
    float* __restrict__ vout, long long ld, const float* __restrict__ inv_rho, Geo g,
    const float* __restrict__ Bimg, const int* __restrict__ rdim, float beta, int mode, int* err) {
  using C = KsTmaA<RM>;
  constexpr int NK = C::NK, CC = C::CC, KC = C::KC, NP = C::NP, TCOLS = C::TCOLS, ACOL = C::ACOL, NS = C::NS;
  constexpr int TX = C::TX, TY = C::TY, BX = C::BX, BY = C::BY, HALO = C::HALO;
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
