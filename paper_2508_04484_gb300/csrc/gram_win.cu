// Stencil Gram on the tensor cores with a sliding TMA window (FP32 path, 3-D grids, A == B):
//   G_k[a][b] = sum_i X(i, a) D_k(rho^-1 X(:, b))(i),   k = 2 d + s  (Sec. 3.3.2-3.3.3),
// the Galerkin blocks of the L-step (r x r) and of the S-step (2r x 2r), as the product
// D[j][a] = sum_t S[j][t] P[a][t] over the cells t, with S[j][t] = D_k(rho^-1 X(:, b))(t),
// j = (s, b), and P[a][t] = X(t, a).
//
// The grid is cut into runs of 32 x-consecutive cells. A slice of CTAs owns the stencils of one
// axis d (both, s = 0 and 1, on one 128-lane tile when there are at most 64 columns; one stencil
// per slice otherwise, the two slices of an axis walking the same runs side by side so that the
// second reads them from L2) and walks lines of runs along d: along y (z) a run at (x0, y, z)
// needs the runs two cells before or after it, along x the runs on either side. A producer
// thread loads each run of all columns once (one 4-D TMA copy, 32 cells x NB columns, 128-byte
// swizzle, so that a warp reading one column per lane meets no bank conflicts; runs outside the
// grid read zeros, the vacuum ghost layer) and its rho^-1 (one 3-D copy) into a ring of R slots,
// released once no chunk reads them any more. Eight formation warps (lane = TMEM lane = column
// b; two warps per lane quarter, 16 cells of the chunk each) keep the three runs their stencil
// needs along y or z in registers (one new run per chunk), form the chunk's stencil values,
// split them into TF32 high and low parts and write them into TMEM (tcgen05.st: S is the MMA's A
// operand, M = j), and write the chunk's X values (split) K-major into shared memory (P, the B
// operand, N = a). One thread issues three tcgen05.mma kind::tf32 per 8-cell K-slice (hi*hi +
// hi*lo + lo*hi, FP32-accurate products).
//
// The tensor core's FP32 accumulation rounds toward zero, so a long sum in one TMEM accumulator
// drifts toward zero by up to an ulp per MMA (measured: 4.8e-4 of the entries at 2.1M cells).
// The products therefore go to one of two short accumulators, a fresh one every F chunks; the
// formation warps add each finished short sum into a long FP32 accumulator in TMEM (round to
// nearest) while the MMAs fill the other, which bounds the drift to F x 12 roundings (~3e-6).
// The CTAs are persistent (one per SM); each adds its long sums to the FP64 output with one
// atomic per entry at the end. Every wait gives up after about a second (ERR_TIMEOUT).
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

// NB = 128: one stencil per slice, lane b; NB = 64: both stencils, lane 64 s + b
template <int NB>
struct GwShape {
  static constexpr int NPA = NB;                                   // MMA N (a)
  static constexpr int NSL = NB == 128 ? 6 : 3;                    // slices
  static constexpr int NS = NB == 128 ? 2 : 4;                     // chunk stages (S in TMEM, P in smem)
  static constexpr int R = 8;                                      // run slots of the window ring (a power of 2)
  static constexpr int F = 8;                                      // chunks per short accumulation
  static constexpr int TCOLS = 512;
  static constexpr int LCOL = 2 * NPA;                             // long sums; short ones at 0 and NPA
  static constexpr int SCOL = 3 * NPA;                             // S stage st at SCOL + 64 st (hi, lo + 32)
  static constexpr int NFORM = 8;                                  // formation warps (two per lane quarter)
  static constexpr int THREADS = 32 * (NFORM + 2);
  static constexpr uint32_t RUN_BYTES = NB * 128;                  // one run of NB columns
  static constexpr uint32_t RHO_BYTES = 128;
  static constexpr size_t OFF_RUN = 0;
  static constexpr size_t OFF_RHO = OFF_RUN + (size_t)R * RUN_BYTES;
  static constexpr size_t OFF_P = (OFF_RHO + (size_t)R * RHO_BYTES + 1023) / 1024 * 1024;
  static constexpr size_t PPART = (size_t)NPA * 32 * 4;            // P hi (or lo) of one chunk
  static constexpr size_t SMEM = OFF_P + (size_t)NS * 2 * PPART + 1024;
  static_assert(SCOL + NS * 64 <= TCOLS, "TMEM columns");
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
  constexpr int NPA = C::NPA, NS = C::NS, R = C::R, F = C::F, NFORM = C::NFORM, NSL = C::NSL;
  extern __shared__ unsigned char raw_dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)raw_dyn + 1023) & ~(uintptr_t)1023);
  // rfull: a run's copies landed; rfree: no chunk reads the run any more (one arrival per
  // formation warp); afull: a chunk's S (TMEM) and P (smem) are written; sfree: the chunk's
  // products are done with them; hfull: a short accumulator's F chunks are summed; hfree: its
  // sums were added into the long accumulator (one arrival per formation warp)
  __shared__ __align__(8) uint64_t rfull[R], rfree[R], afull[NS], sfree[NS], hfull[2], hfree[2], mdone;
  __shared__ uint32_t tslot;
  __shared__ volatile int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sl = (int)(blockIdx.x % NSL);
  const int d = NB == 128 ? sl >> 1 : sl;
  const int nci = (int)((gridDim.x - sl + NSL - 1) / NSL), ci = (int)(blockIdx.x / NSL);
  const GwWalk wk(d, g);
  const long long tot = wk.total();
  const long long c0 = tot * ci / nci, c1 = tot * (ci + 1) / nci;
  const int nchunks = (int)(c1 - c0);
  const int ngroups = (nchunks + F - 1) / F;
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
          const int slot = e % R;
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
      for (int u = 0; u < nchunks; ++u) {
        const int st = u % NS, grp = u / F, hb = grp & 1;
        // a short accumulator is reused once its sums of two groups ago were taken
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
        const uint32_t shi = tmem + C::SCOL + st * 64, slo = shi + 32, dacc = tmem + hb * NPA;
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
      // every product issued is done before tensor memory is read or freed
      tc::mma_commit(&mdone);
      if (!tc::mbar_wait_ns(&mdone, 0u, tc::kWaitNs)) s_bad = 1;
    }
  } else {
    // ---------------- formation: lane = TMEM lane, CPW cells of the chunk per warp ----------------
    constexpr int NPART = NFORM / 4, CPW = 32 / NPART, QPW = CPW / 4;  // warps per lane quarter, cells, quads
    constexpr int FCOLS = NPA / NPART;                                // sum columns per warp (flush, epilogue)
    const int quarter = warp & 3, part = warp >> 2;
    const int L = 32 * quarter + lane;
    const int b = NB == 128 ? L : (L & 63);          // column of this lane's stencil row
    const int s = NB == 128 ? (sl & 1) : (L >> 6);   // its stencil (uniform over the warp)
    const bool prow = L < NPA;                       // this lane also writes P row a = L
    // rows b >= rank and columns a >= rank of the product are never read out: their inputs
    // (stale values beyond the rank) need no masking
    const float iv = (float)g.inv2d[d];
    // stencil s = k0 v(-2 or 0) + k1 v(-1 or +1) + k2 v(0 or +2), oldest run first
    const float k0 = s == 0 ? -iv : 3.f * iv, k1 = s == 0 ? 4.f * iv : -4.f * iv, k2 = s == 0 ? -3.f * iv : iv;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const unsigned char* colp = base + C::OFF_RUN + b * 128;  // column b in slot 0
    const unsigned char* rhop = base + C::OFF_RHO;
    const uint32_t sw = (uint32_t)(b & 7);
    auto qoff = [&](int q) { return (uint32_t)(((uint32_t)q ^ sw) << 4); };
    const int q0 = QPW * part;  // first quad of this warp's cells
    // x values of this warp's cells of run e (quads q0 ..)
    auto rawq = [&](int e, int i) {
      return *reinterpret_cast<const float4*>(colp + (size_t)(e & (R - 1)) * C::RUN_BYTES + qoff(q0 + i));
    };
    auto rhoq = [&](int e, int q) {
      return *reinterpret_cast<const float4*>(rhop + (size_t)(e & (R - 1)) * C::RHO_BYTES + 16 * q);
    };
    // P row a = L, cells 4 q .. 4 q + 3 of chunk stage st (raw values, split)
    auto put_p = [&](int st, int q, float4 x) {
      float* Phi = reinterpret_cast<float*>(base + C::OFF_P + (size_t)st * 2 * C::PPART) +
                   (((q * (NPA / 8) + (L >> 3)) << 5) + ((L & 7) << 2));
      float4 hi, lo;
      tc::split_tf32(x.x, hi.x, lo.x);
      tc::split_tf32(x.y, hi.y, lo.y);
      tc::split_tf32(x.z, hi.z, lo.z);
      tc::split_tf32(x.w, hi.w, lo.w);
      *reinterpret_cast<float4*>(Phi) = hi;
      *reinterpret_cast<float4*>(Phi + C::PPART / 4) = lo;
    };
    auto full_wait = [&](int e) {
      return tc::mbar_wait_ns(&rfull[e & (R - 1)], (uint32_t)((e / R) & 1), tc::kWaitNs);
    };
    // long (+)= short sums of group gi: this warp's lanes, FCOLS columns
    auto flush = [&](int gi) -> bool {
      bool ok = !s_bad && tc::mbar_wait_ns(&hfull[gi & 1], (uint32_t)((gi >> 1) & 1), tc::kWaitNs);
      if (!__all_sync(0xffffffffu, ok)) return false;  // tcgen05.ld / st are warp-collective
      tc::fence_after();
#pragma unroll 1
      for (int c8 = 0; c8 < FCOLS; c8 += 8) {
        const uint32_t col = (uint32_t)(part * FCOLS + c8);
        float sv[8], lv[8];
        tc::tmem_ld8(lane_base + (uint32_t)((gi & 1) * NPA) + col, sv);
        if (gi > 0) {
          tc::tmem_ld8(lane_base + C::LCOL + col, lv);
#pragma unroll
          for (int j = 0; j < 8; ++j) sv[j] += lv[j];
        }
        tc::tmem_st8(lane_base + C::LCOL + col, sv);
      }
      tc::tmem_st_wait();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&hfree[gi & 1]);
      return true;
    };
    int e_seg = 0, u = 0, gdone = 0;  // first run of the segment, chunks formed, short sums taken
    bool go = true;
    float w0[CPW], w1[CPW], w2[CPW];  // along y or z: the scaled runs of this lane's stencil, oldest first
    for (long long c = c0; c < c1 && go;) {
      const int p0 = (int)(c % wk.len);
      const int nch = (int)min((long long)wk.len, p0 + (c1 - c)) - p0;
      for (int cc = 0; cc < nch; ++cc, ++u) {
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
        // the runs that arrive for this chunk: all of the window at a segment's start, then the
        // newest one (along y / z this lane's stencil reads cc + 2 + 2 s, along x cc + 2)
        bool ok = !s_bad;
        if (cc == 0) {
          for (int j = 0; j <= 2 * W && ok; ++j) ok = full_wait(e_seg + j);
        } else {
          ok = ok && full_wait(e_seg + cc + 2 * W);
        }
        if (ok && u >= NS) ok = tc::mbar_wait_ns(&sfree[st], (uint32_t)(((u - NS) / NS) & 1), tc::kWaitNs);
        if (!__all_sync(0xffffffffu, ok)) {
          s_bad = 1;
          go = false;
          break;
        }
        tc::fence_after();
        float sv[CPW];  // stencil values
        if (W == 2) {
          if (cc == 0) {
            // the two older runs of the window: rows 2 s, 2 s + 1 of the segment
#pragma unroll
            for (int i = 0; i < QPW; ++i) {
              const float4 xa = rawq(e_seg + 2 * s, i), ra = rhoq(e_seg + 2 * s, q0 + i);
              const float4 xb = rawq(e_seg + 2 * s + 1, i), rb = rhoq(e_seg + 2 * s + 1, q0 + i);
              w1[4 * i] = xa.x * ra.x, w1[4 * i + 1] = xa.y * ra.y, w1[4 * i + 2] = xa.z * ra.z, w1[4 * i + 3] = xa.w * ra.w;
              w2[4 * i] = xb.x * rb.x, w2[4 * i + 1] = xb.y * rb.y, w2[4 * i + 2] = xb.z * rb.z, w2[4 * i + 3] = xb.w * rb.w;
            }
          }
          // every shared-memory load of the chunk first (stores to P would order them otherwise)
          const int en = e_seg + cc + 2 + 2 * s;
          float4 xq[QPW], rq[QPW], pq[QPW];
#pragma unroll
          for (int i = 0; i < QPW; ++i) xq[i] = rawq(en, i), rq[i] = rhoq(en, q0 + i);
          // P: the chunk's own run is the newest for s = 0, two runs back for s = 1
          if (s != 0 && prow) {
#pragma unroll
            for (int i = 0; i < QPW; ++i) pq[i] = rawq(e_seg + cc + 2, i);
          }
          if (prow) {
#pragma unroll
            for (int i = 0; i < QPW; ++i) put_p(st, q0 + i, s == 0 ? xq[i] : pq[i]);
          }
#pragma unroll
          for (int i = 0; i < QPW; ++i) {
            const float xv[4] = {xq[i].x * rq[i].x, xq[i].y * rq[i].y, xq[i].z * rq[i].z, xq[i].w * rq[i].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int t = 4 * i + k;
              w0[t] = w1[t], w1[t] = w2[t], w2[t] = xv[k];
              sv[t] = k0 * w0[t] + k1 * w1[t] + k2 * w2[t];
            }
          }
        } else {
          // along x: cells CPW part - 4 .. CPW part + CPW + 3 from the chunk's run and its neighbours
          const int ec = e_seg + cc + 1;
          float4 xq[QPW + 2], rq[QPW + 2];
#pragma unroll
          for (int i = 0; i < QPW + 2; ++i) {
            const int Q = q0 - 1 + i;
            const int e = Q < 0 ? ec - 1 : (Q >= 8 ? ec + 1 : ec);
            xq[i] = *reinterpret_cast<const float4*>(colp + (size_t)(e & (R - 1)) * C::RUN_BYTES + qoff(Q & 7));
            rq[i] = rhoq(e, Q & 7);
          }
          if (prow) {
#pragma unroll
            for (int i = 1; i <= QPW; ++i) put_p(st, q0 - 1 + i, xq[i]);
          }
          float wv[CPW + 8];
#pragma unroll
          for (int i = 0; i < QPW + 2; ++i) {
            wv[4 * i] = xq[i].x * rq[i].x, wv[4 * i + 1] = xq[i].y * rq[i].y;
            wv[4 * i + 2] = xq[i].z * rq[i].z, wv[4 * i + 3] = xq[i].w * rq[i].w;
          }
          // cell t: s = 0 reads t - 2, t - 1, t; s = 1 reads t, t + 1, t + 2 (wv index t + 4 = cell t)
#pragma unroll
          for (int t = 0; t < CPW; ++t)
            sv[t] = s == 0 ? k0 * wv[t + 2] + k1 * wv[t + 3] + k2 * wv[t + 4]
                           : k0 * wv[t + 4] + k1 * wv[t + 5] + k2 * wv[t + 6];
        }
        const uint32_t scol = lane_base + C::SCOL + st * 64 + CPW * part;
#pragma unroll
        for (int g8 = 0; g8 < CPW / 8; ++g8) {
          float hv[8], lv[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) tc::split_tf32(sv[8 * g8 + t], hv[t], lv[t]);
          tc::tmem_st8(scol + 8 * g8, hv);
          tc::tmem_st8(scol + 32 + 8 * g8, lv);
        }
        tc::tmem_st_wait();
        tc::fence_before();
        tc::fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          tc::mbar_arrive(&afull[st]);
          // the runs no later chunk reads
          const bool last = cc == nch - 1;
          if (W == 1) {
            tc::mbar_arrive(&rfree[(e_seg + cc) & (R - 1)]);
            if (last) {
              tc::mbar_arrive(&rfree[(e_seg + cc + 1) & (R - 1)]);
              tc::mbar_arrive(&rfree[(e_seg + cc + 2) & (R - 1)]);
            }
          } else {
            tc::mbar_arrive(&rfree[(e_seg + cc + 2) & (R - 1)]);
            if (cc == 0) {
              tc::mbar_arrive(&rfree[e_seg & (R - 1)]);
              tc::mbar_arrive(&rfree[(e_seg + 1) & (R - 1)]);
            }
            if (last) {
              tc::mbar_arrive(&rfree[(e_seg + cc + 3) & (R - 1)]);
              tc::mbar_arrive(&rfree[(e_seg + cc + 4) & (R - 1)]);
            }
          }
        }
      }
      e_seg += nch + 2 * W;
      c += nch;
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
    // this block's long sums: warp (quarter, part) reads its lanes' rows, its share of the
    // columns; every lane loads (warp-collective), only the atomics are guarded
    tc::fence_after();
    const int quarter = warp & 3, part = warp >> 2;
    const int L = 32 * quarter + lane;
    const int b = NB == 128 ? L : (L & 63);
    const int s = NB == 128 ? (sl & 1) : (L >> 6);
    double* o = out + ((long long)(2 * d + s) * ldj + b) * ldo;
    constexpr int FCOLS = NPA / (NFORM / 4);
#pragma unroll
    for (int c16 = 0; c16 < FCOLS; c16 += 16) {
      const int a0 = part * FCOLS + c16;
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + C::LCOL + (uint32_t)a0, v);
      if (b >= Aact) continue;
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
  auto go = [&](auto kern, size_t smem, int threads, int tcols, int nsl) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    // resident blocks never ask for more than the 512 TMEM columns of an SM
    per_sm = std::max(1, std::min(per_sm, 512 / tcols));
    // an even count keeps the two one-stencil slices of an axis at the same number of blocks
    const int grid = std::max(nsl, sms * per_sm / 2 * 2);
    kern<<<grid, threads, smem, st>>>(mx, mr, g, na, adim, out, ldj, ldo, err);
  };
  if (NB == 128)
    go(gram_win_kernel<128>, GwShape<128>::SMEM, GwShape<128>::THREADS, GwShape<128>::TCOLS, GwShape<128>::NSL);
  else
    go(gram_win_kernel<64>, GwShape<64>::SMEM, GwShape<64>::THREADS, GwShape<64>::TCOLS, GwShape<64>::NSL);
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
