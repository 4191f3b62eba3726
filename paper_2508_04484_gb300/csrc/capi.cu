// C ABI and energy-step driver of the GB300 low-rank collided-proton transport
// library (arXiv 2508.04484). Every step of the method runs in the kernels of
// device.cuh, small.cu and raytrace.cu; this file owns the device state, builds
// the per-energy tables and enqueues one energy step (Sec. 3.3.3) per beam:
//
//   streaming (augmented BUG, Sec. 2.2, Eq. KLS; RK4 in Horner form)
//     P_k = W^T A^s_d W, G_k = X^T D^s_d rho^-1 X      (k = 2 d + s)
//     K' = sum_k D_k(rho^-1 K) P_k c(t)                  (n-side, fused stencil x mix)
//     L' = sum_k A^s_d L G_k^T c(t)                      (m-side)
//     X^ = [X, orth((I - X X^T) K1)], W^ = [W, orth((I - W W^T) L1)]
//     S' = sum_k G^_k S P^_k c(t), then truncated SVD
//   collided scattering (implicit Euler L-step at E_{k+1}, QR)
//   first-collision source (augmented K/L/S with explicit Euler, truncated SVD)
//   dose e_c += dE sqrt(4 pi) (X S W^T)(:, 0)
//
// The stopping power of the mixture is S(x, E) = rho_s(x) S_w(E): every base
// material has the water energy dependence, so S^-1 = rho_s^-1 c(t) with the
// scalar c(t) = 1/S_w(E(t)) folded into the Horner coefficients.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dlra.h"
#include "device.cuh"
#include "kernels.h"
#include "kstage_tc.cuh"
#include "kstage_tma.cuh"
#include "kstage_tmac.cuh"
#include "kstage_tmat.cuh"
#include "kstage_tma8.cuh"
#include "kstage_tmaw.cuh"
#include "kstage_tmaf.cuh"
#include "apply_tc.cuh"
#include "tables.h"

using namespace dlra;

namespace {

// ---------------------------------------------------------------------------
// small helper kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void pstack_kernel(const double* __restrict__ P, int RB, int nk, T* __restrict__ Pst, int adj) {
  // Pst[(c' * nk + k) * RB + c] = P_k[c'][c], P_k[a][b] at P[(k*RB + b)*RB + a].
  // adj: the transposed streaming operator pairs D^-_d with -P^-_d and D^+_d with -P^+_d
  // ((D^-)^T = -D^+ for the zero-ghost stencils), i.e. block k takes -P_{k xor 1}.
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int tot = nk * RB * RB;
  if (e >= tot) return;
  int c = e % RB, row = e / RB;
  int k = row % nk, cp = row / nk;
  const double v = P[((long long)(adj ? (k ^ 1) : k) * RB + c) * RB + cp];
  Pst[e] = T(adj ? -v : v);
}

template <typename T>
__global__ void gt_kernel(const double* __restrict__ G, int RB, int nk, T* __restrict__ GT, int adj) {
  // GT[(k*RB + c)*RB + a] = G_k[c][a] = G[(k*RB + a)*RB + c]; adj (transposed operator): GT_k = G_k
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int tot = nk * RB * RB;
  if (e >= tot) return;
  int a = e % RB, j = e / RB;
  int k = j / RB, c = j % RB;
  GT[e] = T(adj ? G[e] : G[((long long)k * RB + a) * RB + c]);
}

template <typename T>
__global__ void src_vec_kernel(const T* __restrict__ w, const double* __restrict__ psi, long long n, int M,
                               T* __restrict__ A) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ps = psi[i];
  for (int j = 0; j < M; ++j) A[(long long)j * n + i] = T((double)w[(long long)j * n + i] * ps);
}

// A[:, col0 + j] = scale w_j(x) psi(x), j < M: one beam's rank-M source factor placed among the
// stacked factors of a joint state
template <typename T>
__global__ void src_vec_scaled_kernel(const T* __restrict__ w, const double* __restrict__ psi, long long n, int M,
                                      double scale, T* __restrict__ A) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double ps = scale * psi[i];
  for (int j = 0; j < M; ++j) A[(long long)j * n + i] = T((double)w[(long long)j * n + i] * ps);
}

template <typename T>
__global__ void dose_kernel(const T* __restrict__ X, long long n, const double* __restrict__ S,
                            const T* __restrict__ W, int m, int RB, const BeamDims* __restrict__ dims, double fac,
                            double* __restrict__ e) {
  __shared__ double v[64];
  int r = dims->r < RB ? dims->r : RB;
  for (int c = threadIdx.x; c < RB; c += blockDim.x) {
    double s = 0.0;
    if (c < r)
      for (int j = 0; j < r; ++j) s += S[j * RB + c] * (double)W[(long long)j * m];
    v[c] = s;
  }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < r; ++c) acc += (double)X[(long long)c * n + i] * v[c];
    e[i] += fac * acc;
  }
}

__global__ void bin_flags_kernel(const double* __restrict__ psi, long long n, int K, int* __restrict__ flags) {
  int k = blockIdx.y;
  int any = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (psi[(long long)k * n + i] != 0.0) any = 1;
  any = __syncthreads_or(any);
  if (any && threadIdx.x == 0) atomicOr(flags + k, 1);
}

template <typename T>
__global__ void convert_kernel(const double* __restrict__ in, T* __restrict__ out, long long cnt) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = T(in[i]);
}

template <typename T>
__global__ void to_double_kernel(const T* __restrict__ in, double* __restrict__ out, long long cnt) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = (double)in[i];
}

__global__ void dose_total_kernel(const double* __restrict__ ec, const double* __restrict__ eu, long long n,
                                  int first, double weight, double* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (first ? 0.0 : out[i]) + weight * (ec[i] + eu[i]);
}

__global__ void scale_kernel(const double* __restrict__ in, double a, long long n, double* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * in[i];
}

__global__ void div_kernel(double* __restrict__ out, const double* __restrict__ rho, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = rho[i] > 0.0 ? out[i] / rho[i] : 0.0;
}

inline unsigned nblk(long long cnt, int bs) { return (unsigned)((cnt + bs - 1) / bs); }

// Pst[(c*nk + k)*RB + c2] = P_k[c][c2] from column-major r x r blocks, zero padded
__global__ void kstep_pack_p(const float* __restrict__ P, int r, int nk, int RB, float* __restrict__ Pst) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int tot = nk * RB * RB;
  if (e >= tot) return;
  int c2 = e % RB, row = e / RB;
  int k = row % nk, c = row / nk;
  Pst[e] = (c < r && c2 < r) ? P[(long long)k * r * r + (long long)c2 * r + c] : 0.f;
}

// y = K0 (zero columns beyond r), v = rho^-1 y
__global__ void kstep_load(const float* __restrict__ K0, long long n, int r, int RB, const float* __restrict__ inv_rho,
                           float* __restrict__ y, float* __restrict__ v) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * RB) return;
  long long i = e % n;
  int c = (int)(e / n);
  float val = c < r ? K0[(long long)c * n + i] : 0.f;
  y[e] = val;
  v[e] = inv_rho[i] * val;
}

__global__ void kstep_store(const float* __restrict__ y, long long n, int r, float* __restrict__ K1) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n * r) K1[e] = y[e];
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }

// out[e] = T(in[e])
template <typename T>
__global__ void convert_kernel(const double* __restrict__ in, long long cnt, T* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < cnt) out[e] = T(in[e]);
}

// ---------------------------------------------------------------------------
// launch helpers for the tiled product and the Gram reduction
// ---------------------------------------------------------------------------
// Multiprocessors of the current device (queried once per device; 152 on a GB300).
int device_sms() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 152;
    }
    cached[dev] = v;
  }
  return cached[dev];
}

// Launch geometry chosen by dlra_autotune for the context being stepped on this thread.
struct Tuning {
  int gram_blocks = 1216;     // target number of blocks of the Gram reductions (x the 2-D tile grid)
  int gs_waves_x2 = 2;        // stencil Gram grid: (gs_waves_x2 / 2) x (blocks per SM) x SMs blocks
  int kstage_variant = 0;     // streaming stage: 0 per-cell FMA, 1 tcgen05 (FP32 path), 2 brick-staged FMA,
                              // 3 cell pairs, 4 / 5 TMA-staged tcgen05 with 128 / 256-cell bricks,
                              // 6 its persistent form, 7 with the A operand in tensor memory, 8 that on
                              // 2-CTA clusters with multicast halo and B copies, 9 that on bricks of three
                              // 128-cell tiles along z, 10 variant 7 on chunks of eight columns,
                              // 11 variant 7 with eight formation warps (two column groups), 12 variant 11
                              // staging the brick and its faces (five boxes) and an FP32 B image,
                              // 13 variant 12 with the B image of TF32 high and low parts
  int gs_variant = 0;         // stencil Gram: 0 FMA, 1 tcgen05 (FP32 path), 2 tcgen05 with a TMA window (A == B, 3-D)
  int gs_tc_waves_x2 = 2;     // grid of the tensor-core stencil Gram, as gs_waves_x2
  int gram_variant = 0;       // tall-skinny Grams: 0 FMA, 1 tcgen05 (FP32 path, tall, at least 8 columns),
                              // 2 tcgen05 at any height
  int* gram_err = nullptr;    // error word of the tensor-core Grams (the context's)
  int apply_variant = 0;      // tall-skinny applies: 0 FMA, 1 tcgen05 (FP32 path, tall, 16 <= N, Q <= 128),
                              // 2 tcgen05 at any height
};
thread_local const Tuning* t_tuning = nullptr;
const Tuning& tuning() {
  static const Tuning def;
  return t_tuning ? *t_tuning : def;
}
struct TuneScope {
  const Tuning* prev;
  explicit TuneScope(const Tuning* t) : prev(t_tuning) { t_tuning = t; }
  ~TuneScope() { t_tuning = prev; }
};

template <typename T>
__global__ void fill_pseudo_random_kernel(T* p, long long cnt, unsigned seed, T scale) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  unsigned h = (unsigned)i * 2654435761u ^ seed;
  h ^= h >> 15;
  h *= 2246822519u;
  h ^= h >> 13;
  p[i] = scale * (T((h & 0xFFFFFF) * (1.0 / 16777216.0)) - T(0.5));
}

template <typename T, int BK, class AL, class BL, class EP>
void gemm(cudaStream_t st, long long rows, int N, int Q, AL al, BL bl, EP ep, int64_t& nl) {
  if (rows <= 0 || N <= 0) return;
  int BN = std::min(64, (N + 3) / 4 * 4);
  int threads = 16 * (BN / 4);
  dim3 grid((unsigned)((rows + GM_BM - 1) / GM_BM), (unsigned)((N + BN - 1) / BN));
  size_t smem = (size_t)(BK * GM_BM + BK * BN) * sizeof(T) + AL::kExtra;
  gemm_kernel<T, BK, AL, BL, EP><<<grid, threads, smem, st>>>(rows, N, Q, al, bl, ep);
  ++nl;
}

// m-side RK4 stage of the L-step (Sec. 2.2, the L equation): out = y + beta sum_k A_k z G_k^T
// (A_k row-major m x m, G_k[c][a] at GT[(k RB + c) RB + a]; columns beyond the rank stay y)
template <typename T>
void lstage(cudaStream_t st, int m, int nk, int RB, const int* rdim, const T* Apm, const T* z, const T* y, T* out,
            const T* GT, T* U, T beta, int64_t& nl) {
  gemm<T, 16>(st, (long long)nk * m, RB, m, ALoadRowMajor<T>{Apm, m, m}, BLoadCol<T, T>{z, m, nullptr, m, rdim, RB},
              EpiStoreKBlocks<T>{U, m, RB}, nl);
  gemm<T, 16>(st, m, RB, nk * RB, ALoadPlain<T>{U, m, nullptr, nk * RB}, BLoadGt<T>{GT, RB, nk, rdim},
              EpiKStage<T>{out, y, m, beta}, nl);
}

template <typename T, class F>
void gram(cudaStream_t st, long long rows, const T* A, long long lda, const int* adim, int acap, int ncols_j, F f,
          double* out, long long ldo, int64_t& nl) {
  if (rows <= 0 || acap <= 0 || ncols_j <= 0) return;
  // on the tensor cores (FP32 path, tall, at least 8 F columns; the narrow reductions stay below)
  if constexpr (std::is_same<T, float>::value) {
    const int gv = tuning().gram_variant;
    if (((gv == 1 && rows >= 65536) || gv == 2) && ncols_j >= 8) {
      bool done = false;
      if constexpr (std::is_same<F, FPlain<T>>::value)
        done = launch_gram_tt(st, rows, A, lda, adim, acap, f.B, f.ldb, f.jdim, f.jcap, ncols_j, nullptr, 0, 1, out, ldo,
                              tuning().gram_err);
      if constexpr (std::is_same<F, FDiag<T>>::value)
        done = launch_gram_tt(st, rows, A, lda, adim, acap, f.B, f.ldb, f.bdim, f.nb, ncols_j, f.wv, f.nb, f.nk, out,
                              ldo, tuning().gram_err);
      if (done) {
        ++nl;
        return;
      }
    }
  }
  if constexpr (std::is_same<F, FPlain<T>>::value) {
    if (ncols_j <= 2 && rows >= 4096) {
      // a few columns (the source step's rank-M updates): a bandwidth-bound reduction
      // at least eight rows per thread: the block reduction at the end costs ~5 x 32 shuffles
      const unsigned gx =
          (unsigned)std::max<long long>(1, std::min<long long>((rows + 2047) / 2048, 2LL * device_sms()));
      const dim3 grid(gx, (unsigned)((acap + 31) / 32));
#define NARROW(NC)                                                                                                 \
  gram_narrow_kernel<T, NC><<<grid, 256, 0, st>>>(rows, A, lda, adim, acap, f.B, f.ldb, f.jdim, f.jcap, ncols_j, out, \
                                                  ldo)
      if (ncols_j == 1) NARROW(1);
      else NARROW(2);
#undef NARROW
      ++nl;
      return;
    }
  }
  const long long area64 = (long long)((acap + 63) / 64) * ((ncols_j + 63) / 64) * 4096;
  const long long area32 = (long long)((acap + 31) / 32) * ((ncols_j + 31) / 32) * 1024;
  const int tile = area32 < area64 ? 32 : 64;
  int gy = (acap + tile - 1) / tile, gz = (ncols_j + tile - 1) / tile;
  long long want = (rows + GR_TC - 1) / GR_TC;
  if (tile == 64) {
    long long cap = std::max(1, tuning().gram_blocks / (gy * gz));
    int gx = (int)std::max(1LL, std::min(want, cap));
    gram_kernel<T, F, 64, 1><<<dim3(gx, gy, gz), 256, 0, st>>>(rows, A, lda, adim, acap, ncols_j, f, out, ldo);
  } else {
    // row groups per block: 4 (FP32) / 2 (FP64) keep the static staging below 48 KB
    constexpr int RG = sizeof(T) == 4 ? 4 : 2;
    long long cap = std::max(1, tuning().gram_blocks / (gy * gz));
    int gx = (int)std::max(1LL, std::min((want + RG - 1) / RG, cap));
    gram_kernel<T, F, 32, RG><<<dim3(gx, gy, gz), 64 * RG, 0, st>>>(rows, A, lda, adim, acap, ncols_j, f, out, ldo);
  }
  ++nl;
}

// rank capacities with a compiled streaming-stage kernel
constexpr int kRankCaps[] = {4, 8, 12, 16, 20, 24, 32, 40, 48, 64};

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point query: the library
// links only the runtime)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return tma_encode_fn(); }

// The streaming-stage input (rcap columns of ld floats, each an nx x ny x nz grid, x fastest)
// as a 4-D tensor for TMA, box 16 x box_y x box_z x box_c (x, y, z, column). Needs nx and ld multiples
// of 4 and a 16-byte aligned base (the tensor map's stride and address rules).
bool stage_tensor_map(CUtensorMap* m, const float* vin, const Geo& g, long long ld, int rcap, int box_y,
                      int box_z = 8, int box_c = 4, int box_x = 16) {
  if (g.nx % 4 != 0 || ld % 4 != 0 || ((uintptr_t)vin & 15u) != 0 || g.nact != 3) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)rcap};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nxy * 4, (cuuint64_t)ld * 4};
  const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_z, (cuuint32_t)box_c};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(vin), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the TMA-staged tensor-core stage at a rank capacity and brick (FP32, 3-D, rcap >= 32);
// false when the grid or the buffers do not meet its layout rules (the caller falls back)
// bytes of the B-operand images of the TMA-staged stage at rank capacity RB (the larger brick)
size_t kstage_tma_bimg_bytes(int RB) {
  switch (RB) {
    case 32: return (size_t)KsTma<32, 2>::NCH * KsTma<32, 2>::BIMG_BYTES;
    case 40: return (size_t)KsTma<40, 2>::NCH * KsTma<40, 2>::BIMG_BYTES;
    case 48: return (size_t)KsTma<48, 2>::NCH * KsTma<48, 2>::BIMG_BYTES;
    case 64: return (size_t)KsTma<64, 2>::NCH * KsTma<64, 2>::BIMG_BYTES;
    default: return 0;
  }
}

template <int RM, int TILES>
bool kstage_tma_launch(cudaStream_t st, const float* vin, const float* y, float* yout, float* vout, long long n,
                       const float* inv_rho, const Geo& g, const float* Pst, const int* rdim, float beta, int last,
                       int* err, void* bimg) {
  using C = KsTma<RM, TILES>;
  if (!bimg) return false;
  CUtensorMap m;
  if (!stage_tensor_map(&m, vin, g, n, RM, C::BY)) return false;
  float* img = reinterpret_cast<float*>(bimg);
  kstage_tma_bimg_kernel<RM, TILES><<<nblk((long long)C::NCH * C::NP * C::KC, 256), 256, 0, st>>>(Pst, rdim, img);
  cudaFuncSetAttribute(kstage_tma_kernel<RM, TILES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  kstage_tma_kernel<RM, TILES><<<kstage_tma_grid<RM, TILES>(g), C::THREADS, C::SMEM, st>>>(
      m, y, yout, vout, n, inv_rho, g, img, rdim, beta, last, err);
  return true;
}

// the persistent TMA-staged tensor-core stage: one CTA per SM over the 128-cell bricks
template <int RM>
bool kstage_tmap_launch(cudaStream_t st, const float* vin, const float* y, float* yout, float* vout, long long n,
                        const float* inv_rho, const Geo& g, const float* Pst, const int* rdim, float beta, int last,
                        int* err, void* bimg) {
  using C = KsTmaP<RM>;
  using B1 = KsTma<RM, 1>;
  if (!bimg) return false;
  CUtensorMap m;
  if (!stage_tensor_map(&m, vin, g, n, RM, B1::BY)) return false;
  float* img = reinterpret_cast<float*>(bimg);
  kstage_tma_bimg_kernel<RM, 1><<<nblk((long long)B1::NCH * B1::NP * B1::KC, 256), 256, 0, st>>>(Pst, rdim, img);
  cudaFuncSetAttribute(kstage_tmap_kernel<RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  const unsigned bricks = kstage_tma_grid<RM, 1>(g);
  const unsigned grid = std::min<unsigned>(bricks, (unsigned)device_sms());
  kstage_tmap_kernel<RM><<<grid, C::THREADS, C::SMEM, st>>>(m, y, yout, vout, n, inv_rho, g, img, rdim, beta, last,
                                                             err);
  return true;
}

// the TMA-staged stage with its A operand in tensor memory (128-cell bricks)
template <int RM>
bool kstage_tmaa_launch(cudaStream_t st, const float* vin, const float* y, float* yout, float* vout, long long n,
                        const float* inv_rho, const Geo& g, const float* Pst, const int* rdim, float beta, int last,
                        int* err, void* bimg) {
  using C = KsTmaA<RM>;
  using B1 = KsTma<RM, 1>;
  if (!bimg) return false;
  CUtensorMap m;
  if (!stage_tensor_map(&m, vin, g, n, RM, B1::BY)) return false;
  float* img = reinterpret_cast<float*>(bimg);
  kstage_tma_bimg_kernel<RM, 1><<<nblk((long long)B1::NCH * B1::NP * B1::KC, 256), 256, 0, st>>>(Pst, rdim, img);
  cudaFuncSetAttribute(kstage_tmaa_kernel<RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  kstage_tmaa_kernel<RM><<<kstage_tma_grid<RM, 1>(g), C::THREADS, C::SMEM, st>>>(m, y, yout, vout, n, inv_rho, g, img,
                                                                                rdim, beta, last, err);
  return true;
}

// the A-in-TMEM stage on chunks of eight input columns (128-cell bricks)
template <int RM>
bool kstage_tmaa8_launch(cudaStream_t st, const float* vin, const float* y, float* yout, float* vout, long long n,
                         const float* inv_rho, const Geo& g, const float* Pst, const int* rdim, float beta, int last,
                         int* err, void* bimg) {
  using C = KsTmaA8<RM>;
  using B1 = KsTma<RM, 1>;
  if (!bimg) return false;
  CUtensorMap m;
  if (!stage_tensor_map(&m, vin, g, n, RM, C::BY, C::BZ, C::CC)) return false;
  float* img = reinterpret_cast<float*>(bimg);
  kstage_tma_bimg_kernel<RM, 1><<<nblk((long long)B1::NCH * B1::NP * B1::KC, 256), 256, 0, st>>>(Pst, rdim, img);
  cudaFuncSetAttribute(kstage_tmaa8_kernel<RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  kstage_tmaa8_kernel<RM><<<kstage_tma_grid<RM, 1>(g), C::THREADS, C::SMEM, st>>>(m, y, yout, vout, n, inv_rho, g,
                                                                                 img, rdim, beta, last, err);
  return true;
}

// the A-in-TMEM stage with eight formation warps (128-cell bricks)
template <int RM>
bool kstage_tmaw_launch(cudaStream_t st, const float* vin, const float* y, float* yout, float* vout, long long n,
                        const float* inv_rho, const Geo& g, const float* Pst, const int* rdim, float beta, int last,
                        int* err, void* bimg) {
  using C = KsTmaW<RM>;
  using B1 = KsTma<RM, 1>;
  if (!bimg) return false;
  CUtensorMap m;
  if (!stage_tensor_map(&m, vin, g, n, RM, B1::BY)) return false;
  float* img = reinterpret_cast<float*>(bimg);
  kstage_tma_bimg_kernel<RM, 1><<<nblk((long long)B1::NCH * B1::NP * B1::KC, 256), 256, 0, st>>>(Pst, rdim, img);
  cudaFuncSetAttribute(kstage_tmaw_kernel<RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  kstage_tmaw_kernel<RM><<<kstage_tma_grid<RM, 1>(g), C::THREADS, C::SMEM, st>>>(m, y, yout, vout, n, inv_rho, g, img,
                                                                                rdim, beta, last, err);
  return true;
}

// the eight-formation-warp stage on five boxes per chunk (128-cell bricks) with its B operand as
// one FP32 image split in shared memory (SPLIT) or as the image of TF32 high and low parts
template <int RM, bool SPLIT>
bool kstage_tmaf_launch(cudaStream_t st, const float* vin, const float* y, float* yout, float* vout, long long n,
                        const float* inv_rho, const Geo& g, const float* Pst, const int* rdim, float beta, int last,
                        int* err, void* bimg) {
  using C = KsTmaF<RM, SPLIT>;
  using B1 = KsTma<RM, 1>;
  if (!bimg) return false;
  CUtensorMap mx, my, mz;
  if (!stage_tensor_map(&mx, vin, g, n, RM, C::TY, C::TZ, C::CC, C::XW) ||
      !stage_tensor_map(&my, vin, g, n, RM, 2, C::TZ, C::CC, C::TX) ||
      !stage_tensor_map(&mz, vin, g, n, RM, C::TY, 2, C::CC, C::TX))
    return false;
  float* img = reinterpret_cast<float*>(bimg);
  if (SPLIT)
    kstage_tmaf_bimg_kernel<RM><<<nblk((long long)C::NCH * C::BSZ, 256), 256, 0, st>>>(Pst, rdim, img);
  else
    kstage_tma_bimg_kernel<RM, 1><<<nblk((long long)B1::NCH * B1::NP * B1::KC, 256), 256, 0, st>>>(Pst, rdim, img);
  cudaFuncSetAttribute(kstage_tmaf_kernel<RM, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  const unsigned grid = (unsigned)(((g.nx + C::TX - 1) / C::TX) * ((g.ny + C::TY - 1) / C::TY) *
                                   ((g.nz + C::TZ - 1) / C::TZ));
  kstage_tmaf_kernel<RM, SPLIT><<<grid, C::THREADS, C::SMEM, st>>>(mx, my, mz, y, yout, vout, n, inv_rho, g, img, rdim,
                                                                   beta, last, err);
  return true;
}

// the A-in-TMEM stage on bricks of T tiles stacked along z (one block per SM)
template <int RM, int T>
bool kstage_tmat_launch(cudaStream_t st, const float* vin, const float* y, float* yout, float* vout, long long n,
                        const float* inv_rho, const Geo& g, const float* Pst, const int* rdim, float beta, int last,
                        int* err, void* bimg) {
  using C = KsTmaT<RM, T>;
  using B1 = KsTma<RM, 1>;
  if (!bimg) return false;
  CUtensorMap m;
  if (!stage_tensor_map(&m, vin, g, n, RM, C::BY, C::BZ)) return false;
  float* img = reinterpret_cast<float*>(bimg);
  kstage_tma_bimg_kernel<RM, 1><<<nblk((long long)B1::NCH * B1::NP * B1::KC, 256), 256, 0, st>>>(Pst, rdim, img);
  cudaFuncSetAttribute(kstage_tmat_kernel<RM, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  kstage_tmat_kernel<RM, T><<<kstage_tmat_grid<RM, T>(g), C::THREADS, C::SMEM, st>>>(m, y, yout, vout, n, inv_rho, g,
                                                                                    img, rdim, beta, last, err);
  return true;
}

// cluster launches of the stage that the runtime refused (their work ran as variant 7)
std::atomic<long long> g_tmac_refused{0};

// the A-in-TMEM stage on clusters of two y-adjacent bricks sharing one multicast halo box and
// B image; false when the layout rules are not met or the cluster launch is refused
template <int RM>
bool kstage_tmac_launch(cudaStream_t st, const float* vin, const float* y, float* yout, float* vout, long long n,
                        const float* inv_rho, const Geo& g, const float* Pst, const int* rdim, float beta, int last,
                        int* err, void* bimg) {
  using C = KsTmaC<RM>;
  using B1 = KsTma<RM, 1>;
  if (!bimg) return false;
  CUtensorMap m;
  if (!stage_tensor_map(&m, vin, g, n, RM, C::BY)) return false;
  float* img = reinterpret_cast<float*>(bimg);
  kstage_tma_bimg_kernel<RM, 1><<<nblk((long long)B1::NCH * B1::NP * B1::KC, 256), 256, 0, st>>>(Pst, rdim, img);
  cudaFuncSetAttribute(kstage_tmac_kernel<RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kstage_tmac_grid<RM>(g), 1, 1);
  cfg.blockDim = dim3(C::THREADS, 1, 1);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const Geo gg = g;
  if (cudaLaunchKernelEx(&cfg, kstage_tmac_kernel<RM>, m, y, yout, vout, n, inv_rho, gg, (const float*)img, rdim, beta,
                         last, err) != cudaSuccess) {
    cudaGetLastError();
    g_tmac_refused.fetch_add(1);
    return false;
  }
  return true;
}

template <typename T, int RM, int NACT>
void kstage_launch(cudaStream_t st, const T* vin, const T* y, T* yout, T* vout, long long n, const T* inv_rho,
                   const Geo& g, const T* Pst, const int* rdim, T beta, int last, int* err, int variant,
                   void* bimg) {
  if constexpr (sizeof(T) == 4 && NACT == 3 && RM >= 32) {
    if (variant == 12) {
      if (kstage_tmaf_launch<RM, true>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, bimg)) return;
      variant = 7;
    }
    if (variant == 13) {
      if (kstage_tmaf_launch<RM, false>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, bimg))
        return;
      variant = 7;
    }
    if (variant == 11) {
      if (kstage_tmaw_launch<RM>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, bimg)) return;
      variant = 7;
    }
    if (variant == 10) {
      if (kstage_tmaa8_launch<RM>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, bimg)) return;
      variant = 7;
    }
    if (variant == 9) {
      if (kstage_tmat_launch<RM, 3>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, bimg)) return;
      variant = 7;
    }
    if (variant == 8) {
      if (kstage_tmac_launch<RM>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, bimg)) return;
      variant = 7;
    }
    if (variant == 7) {
      if (kstage_tmaa_launch<RM>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, bimg)) return;
      variant = 0;
    }
    if (variant == 6) {
      if (kstage_tmap_launch<RM>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, bimg)) return;
      variant = 0;
    }
    if (variant == 4 || variant == 5) {
      const bool done = variant == 4 ? kstage_tma_launch<RM, 1>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim,
                                                                beta, last, err, bimg)
                                     : kstage_tma_launch<RM, 2>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim,
                                                                beta, last, err, bimg);
      if (done) return;
      variant = 0;
    }
  }
  if (variant >= 4) variant = 0;
  if (variant == 2) {
    using Bk = Brick<NACT>;
    const size_t smem = ((size_t)2 * NACT * RM * RM + 2 * Bk::HALO) * sizeof(T);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(kstage_brick_kernel<T, RM, NACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned grid = (unsigned)(((g.nx + Bk::TX - 1) / Bk::TX) * ((g.ny + Bk::TY - 1) / Bk::TY) *
                                     ((g.nz + Bk::TZ - 1) / Bk::TZ));
    kstage_brick_kernel<T, RM, NACT><<<grid, 256, smem, st>>>(vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta,
                                                               last);
    return;
  }
  if constexpr (sizeof(T) == 4) {
    if (variant == 3 && g.nx % 2 == 0) {
      // FP32 path: two x-adjacent cells per thread
      const size_t smem = (size_t)2 * NACT * RM * RM * sizeof(float);
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(kstage_pair_kernel<RM, NACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kstage_pair_kernel<RM, NACT><<<nblk(n / 2, 128), 128, smem, st>>>(vin, y, yout, vout, n, inv_rho, g, Pst, rdim,
                                                                        beta, last);
      return;
    }
    if (variant == 1) {
      // FP32 path on request: the r x r mix on the tensor cores (3xTF32)
      const size_t smem = kstage_tc_smem<NACT, RM>();
      cudaFuncSetAttribute(kstage_tc_kernel<NACT, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kstage_tc_kernel<NACT, RM><<<kstage_tc_grid<NACT, RM>(g), 256, smem, st>>>(vin, y, yout, vout, n, inv_rho, g,
                                                                                 Pst, rdim, beta, last, err);
      return;
    }
  }
  size_t smem = (size_t)2 * NACT * RM * RM * sizeof(T);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kstage_kernel<T, RM, NACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kstage_kernel<T, RM, NACT><<<nblk(n, 128), 128, smem, st>>>(vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta,
                                                              last);
}

template <typename T, int NACT>
void kstage_dispatch(int RB, cudaStream_t st, const T* vin, const T* y, T* yout, T* vout, long long n,
                     const T* inv_rho, const Geo& g, const T* Pst, const int* rdim, T beta, int last, int* err,
                     int tc, void* bimg) {
  switch (RB) {
#define KS_CASE(R) \
  case R: kstage_launch<T, R, NACT>(st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, tc, bimg); break;
    KS_CASE(4) KS_CASE(8) KS_CASE(12) KS_CASE(16) KS_CASE(20) KS_CASE(24) KS_CASE(32)
    KS_CASE(40) KS_CASE(48) KS_CASE(64)
#undef KS_CASE
    default: break;
  }
}

// one RK4 Horner stage of the K-step on the scaled input vin = rho^-1 z
template <typename T>
void kstage(int RB, cudaStream_t st, const T* vin, const T* y, T* yout, T* vout, long long n, const T* inv_rho,
            const Geo& g, const T* Pst, const int* rdim, T beta, int last, int64_t& nl, int* err = nullptr,
            int tc = 0, void* bimg = nullptr) {
  if (g.nact == 3)
    kstage_dispatch<T, 3>(RB, st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, tc, bimg);
  else kstage_dispatch<T, 2>(RB, st, vin, y, yout, vout, n, inv_rho, g, Pst, rdim, beta, last, err, tc, bimg);
  ++nl;
}

// out[(k*ldj + b)*ldo + a] += sum_i A(i, a) D_k(rho^-1 B(:, b))(i)
template <typename T>
void gram_stencil(cudaStream_t st, long long rows, const T* A, long long lda, int na, const int* adim, const T* B,
                  long long ldb, int nb, const int* bdim, const T* inv_rho, const Geo& g, double* out, int ldj,
                  long long ldo, int64_t& nl, int* err = nullptr) {
  if constexpr (std::is_same<T, float>::value) {
    if (tuning().gs_variant == 2 &&
        launch_gram_stencil_win(st, rows, A, lda, na, adim, B, ldb, nb, bdim, inv_rho, g, out, ldj, ldo, err)) {
      ++nl;
      return;
    }
    if (tuning().gs_variant >= 1 && gram_stencil_tc_supported(na, rows)) {
      launch_gram_stencil_tc(st, rows, A, lda, na, adim, B, ldb, nb, bdim, inv_rho, g, out, ldj, ldo,
                             tuning().gs_tc_waves_x2, err);
      ++nl;
      return;
    }
  }
  const int nk = 2 * g.nact;
  const int nj = nk * nb;
  const int naP = (na + 3) / 4 * 4;
  const int tpa = naP / 4;
  int jslice = std::min((nj + 7) / 8 * 8, std::max(8, (512 / tpa) / 1 * 8));
  jslice = std::min(jslice, (512 / tpa) * 8);
  const int nslice = (nj + jslice - 1) / jslice;
  const int threads = tpa * ((std::min(jslice, nj) + 7) / 8);
  const int ldA = naP + (((naP / 4) & 1) ? 0 : 4);
  const int ldS = jslice + (((jslice / 4) & 1) ? 0 : 4);
  const size_t smem = (size_t)GS_TC * (ldA + ldS) * sizeof(T) + (size_t)13 * GS_TC * (sizeof(int) + sizeof(T));
  const long long chunks = (rows + GS_TC - 1) / GS_TC;
  auto kern = g.nact == 3 ? gram_stencil_kernel<T, 3> : gram_stencil_kernel<T, 2>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  per_sm = std::max(per_sm, 1);
  const int gx = (int)std::max(
      1LL, std::min(chunks, (long long)std::max(1, device_sms() * per_sm * tuning().gs_waves_x2 / 2 / nslice)));
  kern<<<dim3(gx, nslice), threads, smem, st>>>(rows, A, lda, na, adim, B, ldb, nb, bdim, inv_rho, g, jslice, out,
                                                ldj, ldo);
  ++nl;
}

template <typename T, int NM>
void apply_launch(cudaStream_t st, long long rows, const T* A, long long lda, int Q, const int* qdim, const double* M,
                  long long ldm, int N, T* C, long long ldc, const T* Cin, T alpha, T beta, T* V, const T* inv_rho) {
  const size_t smem = (size_t)Q * NM * sizeof(T);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(apply_kernel<T, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  apply_kernel<T, NM><<<nblk(rows, 128), 128, smem, st>>>(rows, A, lda, Q, qdim, M, ldm, N, C, ldc, Cin, alpha, beta,
                                                          V, inv_rho);
}

// Work space of the tensor-core apply: the B image of one launch (64 KB) and the error word.
struct ApplyTc {
  void* img = nullptr;
  int* err = nullptr;
};

// the tensor-core apply at MMA width NP (FP32, Q <= 128, N <= NP); false when A does not meet
// the tensor map's rules (the caller falls back to the FMA kernel)
template <int NP>
bool apply_tc_launch(cudaStream_t st, long long rows, const float* A, long long lda, int Q, const int* qdim,
                     const double* M, long long ldm, int N, float* C, long long ldc, const float* Cin, float alpha,
                     float beta, float* V, const float* inv_rho, const ApplyTc& tcw) {
  using Cf = ApTc<NP>;
  if (lda % 4 != 0 || ((uintptr_t)A & 15u) != 0 || Q > Cf::QMAX || N > NP) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)Q};
  const cuuint64_t strides[1] = {(cuuint64_t)lda * 4};
  const cuuint32_t box[2] = {128, (cuuint32_t)Cf::KCH};
  const cuuint32_t es[2] = {1, 1};
  if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  float* img = reinterpret_cast<float*>(tcw.img);
  apply_tc_bimg_kernel<NP><<<nblk((long long)NP * Cf::QMAX, 256), 256, 0, st>>>(M, ldm, Q, qdim, N, img);
  cudaFuncSetAttribute(apply_tc_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM);
  // persistent: two blocks per SM over the 128-row tiles
  const long long tiles = (rows + 127) / 128;
  const unsigned grid = (unsigned)std::max(1LL, std::min(tiles, 2LL * device_sms()));
  apply_tc_kernel<NP><<<grid, Cf::THREADS, Cf::SMEM, st>>>(
      m, rows, Q, qdim, img, N, C, ldc, Cin, alpha, beta, V, inv_rho, tcw.err);
  return true;
}

// C(:, :N) = alpha A(:, :Q) M + beta Cin (+ V = rho^-1 C); N <= 64. With tcw (FP32, 16 <= N,
// Q <= 128, tuning().apply_variant 1 with at least 65,536 rows or 2) on the tensor cores, else
// the FMA kernel.
template <typename T>
void apply(cudaStream_t st, long long rows, const T* A, long long lda, int Q, const int* qdim, const double* M,
           long long ldm, int N, T* C, long long ldc, const T* Cin, T alpha, T beta, int64_t& nl, T* V = nullptr,
           const T* inv_rho = nullptr, const ApplyTc* tcw = nullptr) {
  if (rows <= 0 || N <= 0) return;
  if constexpr (sizeof(T) == 4) {
    const int av = tuning().apply_variant;
    if (tcw && tcw->img && ((av == 1 && rows >= 65536) || av == 2) && N >= 16 && Q <= 128) {
      bool done = false;
      if (N <= 32)
        done = apply_tc_launch<32>(st, rows, A, lda, Q, qdim, M, ldm, N, C, ldc, Cin, alpha, beta, V, inv_rho, *tcw);
      else if (N <= 48)
        done = apply_tc_launch<48>(st, rows, A, lda, Q, qdim, M, ldm, N, C, ldc, Cin, alpha, beta, V, inv_rho, *tcw);
      else
        done = apply_tc_launch<64>(st, rows, A, lda, Q, qdim, M, ldm, N, C, ldc, Cin, alpha, beta, V, inv_rho, *tcw);
      if (done) {
        nl += 2;
        return;
      }
    }
  }
  const int nm = N <= 4 ? 4 : N <= 8 ? 8 : N <= 12 ? 12 : N <= 16 ? 16 : N <= 20 ? 20 : N <= 24 ? 24
               : N <= 32 ? 32 : N <= 40 ? 40 : N <= 48 ? 48 : 64;
  switch (nm) {
#define AP_CASE(R) \
  case R: apply_launch<T, R>(st, rows, A, lda, Q, qdim, M, ldm, N, C, ldc, Cin, alpha, beta, V, inv_rho); break;
    AP_CASE(4) AP_CASE(8) AP_CASE(12) AP_CASE(16) AP_CASE(20) AP_CASE(24) AP_CASE(32) AP_CASE(40) AP_CASE(48)
    AP_CASE(64)
#undef AP_CASE
    default: break;
  }
  ++nl;
}

// ---------------------------------------------------------------------------
// engine state
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Base {
  virtual ~Base() {}
};

// a copy of one low-rank state (checkpoints and replayed states of the reverse sweep)
template <typename T>
struct Snap {
  T* X = nullptr;
  T* W = nullptr;
  double* S = nullptr;
  BeamDims* dims = nullptr;
};

template <typename T>
struct Beam {
  T* X = nullptr;
  T* W = nullptr;
  double* S = nullptr;
  BeamDims* dims = nullptr;
  int* rank_log = nullptr;
  double* psi = nullptr;      // fluence of every energy bin at unit beam weight
  double* e_u = nullptr;      // uncollided deposit at unit weight
  double* e_c = nullptr;      // collided deposit at unit weight
  double* Bsrc = nullptr;
  std::vector<int> has_src;
  int first_src = -1;         // first energy step with a first-collision source
  double weight = 1.0;        // beam weight: the beam's deposit enters the dose times weight
  double dir[3] = {0, 0, 1};
  dlra_beam params{};         // as added (the straggling tracer re-traces from these)
  bool active = false;
  std::vector<Snap<T>> ckpt;  // states at the start of steps 0, I, 2I, ... (adjoint enabled)
};

// Work space of the reverse sweep (allocated on the first dlra_backward).
template <typename T>
struct AdjWork {
  Beam<T> mu;                 // adjoint state, its own low-rank factors and rank log
  Snap<T> alpha;              // adjoint state after the adjoint collision step
  Beam<T> rep;                // forward state replayed from a checkpoint
  std::vector<Snap<T>> seg;   // forward states at the start of each step of a segment
  T* capf = nullptr;          // forward K-stage inputs rho^-1 z of one energy step
  T* capa = nullptr;          // their adjoints
  int cap_ns = 0;
  // with room on the device, the replay keeps every step's K-stage inputs and post-collision
  // state of the segment, so that the reverse steps need not recompute them
  bool store = false;
  T* capseg = nullptr;        // [step of segment][beam] x 4 nsub_max stage buffers
  size_t capseg_stride = 0;   // elements per (step, beam)
  size_t capseg_slots = 0;
  std::vector<Snap<T>> segb;  // post-collision states [step of segment][beam]
  T* gvec = nullptr;          // dL/de in the n-side type
  double *ge = nullptr, *be0 = nullptr, *gtmp = nullptr;
  double *grad_rho = nullptr, *grad_f = nullptr, *grad_tau = nullptr, *grad_w = nullptr, *dw = nullptr;
  double *Cm = nullptr, *Cl = nullptr, *ysrc = nullptr, *mcoef = nullptr, *dbeta = nullptr;
  std::vector<double*> gpsi;  // dL/dpsi per beam (K x n)
  int nb_cap = 0;
  void* ray_scratch = nullptr;
  size_t ray_scratch_bytes = 0;
};

// Work space of one lane: the buffers of one energy step of one beam and two streams
// (cell side s0, moment side s1). Beams on different lanes advance concurrently.
struct Lane {
  cudaStream_t s0 = nullptr, s1 = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  void *Kb[3] = {nullptr, nullptr, nullptr}, *Xh = nullptr, *Asrc = nullptr;
  void *Lb[3] = {nullptr, nullptr, nullptr}, *Zm = nullptr, *Wh = nullptr, *L1T = nullptr, *Pst = nullptr;
  void* Ul = nullptr;  // L-step stages: U_k = A_k z, nk blocks of m x RB
  void* GtT = nullptr;
  double *G1 = nullptr, *Gc = nullptr, *Ph = nullptr, *P1 = nullptr, *C1 = nullptr, *Cg = nullptr, *Mapply = nullptr;
  double *Sh = nullptr, *Pt = nullptr, *Qt = nullptr, *Mg = nullptr, *XA = nullptr;
  double* mwork = nullptr;   // FP64 work space of the m-side QR (FP32 paths)
  double *C1m = nullptr, *Cgm = nullptr, *Mapplym = nullptr;   // W-side augmentation (FP32 paths)
  void* Kw = nullptr;        // the source's moment factor in the n-side type (FP32 paths)
  void* svdV = nullptr;      // right rotations of the truncation SVD when they do not fit shared memory
  void* Bimg = nullptr;      // B-operand images of the TMA-staged tensor-core stage
  ApplyTc atc;               // tensor-core applies of the cell side (B image, error word)
  SstepWork sgw;             // grid-parallel S-step (2r beyond the cluster kernel's shared memory)
};

// dlra_step(n) from a given step and beam-activity pattern, captured as a CUDA graph
struct StepGraph {
  int start = 0, n = 0;
  std::vector<char> active_before, active_after;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
};

}  // namespace

struct dlra_ctx {
  dlra_config cfg{};
  std::vector<int32_t> schedule_host;
  std::string err = "no error";
  dlra_status poisoned = DLRA_OK;
  cudaStream_t st = nullptr;
  bool fp64 = true;
  bool small64 = true;  // truncation SVD and Galerkin S-step in FP64 (FP64 and FP32-split paths)
  int n = 0, m = 0, N = 0, K = 0, M = 0, RB = 0, nk = 0, n2 = 0;
  bool two_d = false;
  Geo geo{};
  AngularTables ang;
  double h = 0.0;
  std::vector<double> E;
  std::vector<int> nsub;
  int nsub_max = 1;
  std::vector<dlra_material> mats;
  std::vector<std::vector<double>> s_unit;
  std::vector<double> xi_unit;
  std::vector<double> rho_s_host, rho_host;
  int step = 0;
  bool materials_set = false;
  int64_t launches = 0;
  std::vector<void*> allocs;
  // type-erased engine buffers
  void* beams = nullptr;   // std::vector<Beam<T>>*
  // shared device buffers (raw pointers, typed at use)
  void *inv_rho = nullptr, *wc = nullptr, *wT = nullptr, *Apm = nullptr;
  double *rho = nullptr, *f_cell = nullptr, *tau_cell = nullptr;
  double *coef = nullptr, *sbeta = nullptr;
  std::vector<Lane> lanes;
  int max_lanes = 8;
  cudaEvent_t ev_step = nullptr;
  int* dev_err = nullptr;
  int* flags_dev = nullptr;
  int* schedule_dev = nullptr;
  double* dose_tmp = nullptr;
  double* zeros = nullptr;   // n zeros
  // ray sets of the beams (for dlra_reset with retrace)
  std::vector<double*> ray_dev;
  std::vector<int> ray_count;
  // uncollided source from the energy-DG straggling tracer (dlra_set_straggling) instead of
  // the CSDA tracer
  bool strag = false;
  int strag_elems = 128, strag_on = 1;
  double strag_hmax = 0.01;
  // joint mode: every beam feeds one low-rank state (held by beam 0); stacked source factors
  bool joint = false;
  void* joint_A = nullptr;      // n x (M n_beams), n-side type
  double* joint_B = nullptr;    // m x (M n_beams)
  int joint_cols = 0;
  // reverse sweep: checkpoint interval (0 = off) and its work space (AdjWork<T>*)
  int ckpt_interval = 0;
  int adj_store = 1;  // reverse sweep keeps the replayed segment's stage inputs when they fit
  void* adj = nullptr;
  std::vector<double> tau_coef;   // per material: Sigma_t / T_w factor rho_i kappa_i g0_i
  size_t sbeta_cap = 0;
  // launch geometry and kernel variants (dlra_autotune, dlra_set_tensor_cores)
  Tuning tun;
  BeamDims* tune_dims = nullptr;
  // CUDA-graph replay of dlra_step (dlra_set_graphs)
  bool graphs = false;
  cudaStream_t cap_st = nullptr;
  std::vector<StepGraph> step_graphs;
  // streaming-stage kernel timing
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double prof_ms = 0.0;
  int64_t prof_count = 0;
};

namespace {

dlra_status fail(dlra_ctx* c, dlra_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = buf;
    if (s == DLRA_ERR_CUDA || s == DLRA_ERR_NONFINITE || s == DLRA_ERR_TIMEOUT) c->poisoned = s;
  }
  return s;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? DLRA_ERR_OOM : DLRA_ERR_CUDA,      \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                            \
  } while (0)

// frees one allocation made by dalloc (device-synchronising)
void dfree(dlra_ctx* ctx, void* p) {
  if (!p) return;
  for (auto& a : ctx->allocs)
    if (a == p) {
      cudaFree(p);
      a = ctx->allocs.back();
      ctx->allocs.pop_back();
      return;
    }
}

dlra_status dalloc(dlra_ctx* ctx, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DLRA_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  ctx->allocs.push_back(*p);
  e = cudaMemsetAsync(*p, 0, bytes, ctx->st);
  if (e != cudaSuccess) return fail(ctx, DLRA_ERR_CUDA, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
  return DLRA_OK;
}

#define ALLOC(ptr, bytes)                                                      \
  do {                                                                         \
    dlra_status s_ = dalloc(ctx, (void**)&(ptr), (size_t)(bytes));             \
    if (s_ != DLRA_OK) return s_;                                              \
  } while (0)

double Sw(const dlra_ctx* c, double E) { return std::pow(E, 1.0 - c->cfg.bk_p) / (c->cfg.bk_p * c->cfg.bk_alpha); }
double Tw(const dlra_ctx* c, double E) { return c->cfg.t100 * (100.0 / E) * (100.0 / E); }

// G_{i,l} - Sigma_{t,i} (self-scattering) and G_{i,l} (in-scattering) at energy E.
void moments_at(const dlra_ctx* c, int i, double E, std::vector<double>& self, std::vector<double>& src) {
  const dlra_material& mt = c->mats[i];
  const double xi1 = mt.density * mt.scatter_ratio * 0.5 * Tw(c, E);
  self.assign(c->N + 1, 0.0);
  src.assign(c->N + 1, 0.0);
  if (c->cfg.collision == DLRA_BOLTZMANN) {
    const double C = xi1 / c->xi_unit[i];
    const std::vector<double>& s = c->s_unit[i];
    const double corr = c->cfg.transport_correction ? s[c->N + 1] : 0.0;
    for (int l = 0; l <= c->N; ++l) {
      self[l] = C * (s[l] - s[0]);
      src[l] = C * (s[l] - corr);
    }
  } else {
    // Fokker-Planck; transport_correction == 2: the delta-function corrected expansion (the
    // moments shifted so that degree N+1 vanishes; Sigma_t = G_0), the self-scattering unchanged
    const double shift = c->cfg.transport_correction == 2 ? 0.5 * xi1 * (c->N + 1.0) * (c->N + 2.0) : 0.0;
    for (int l = 0; l <= c->N; ++l) {
      self[l] = -0.5 * xi1 * l * (l + 1.0);
      src[l] = self[l] + shift;
    }
  }
}

// Horner coefficients of one RK4 sub-step of y' = c(t) L y, c = 1/S_w(E(t)), from energy Ea.
void horner_betas_p(double bk_p, double bk_alpha, double Ea, double hs, double* beta) {
  auto sw = [&](double E) { return std::pow(E, 1.0 - bk_p) / (bk_p * bk_alpha); };
  const double c1 = 1.0 / sw(Ea), c2 = 1.0 / sw(Ea - 0.5 * hs), c4 = 1.0 / sw(Ea - hs);
  const double a1 = hs * (c1 + 4.0 * c2 + c4) / 6.0;
  const double a2 = hs * hs * (c1 * c2 + c2 * c2 + c2 * c4) / 6.0;
  const double a3 = hs * hs * hs * (c1 * c2 * c2 + c2 * c2 * c4) / 12.0;
  const double a4 = hs * hs * hs * hs * c1 * c2 * c2 * c4 / 24.0;
  beta[0] = a4 / a3;
  beta[1] = a3 / a2;
  beta[2] = a2 / a1;
  beta[3] = a1;
}

void horner_betas(const dlra_ctx* c, double Ea, double hs, double* beta) {
  horner_betas_p(c->cfg.bk_p, c->cfg.bk_alpha, Ea, hs, beta);
}

// events around the streaming-stage kernel when profiling is on
void prof_begin(dlra_ctx* c, cudaStream_t st) {
  if (!c->profiling) return;
  if (c->ev_used + 2 > c->ev_pool.size()) {
    for (int i = 0; i < 512; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->ev_pool.push_back(e);
    }
  }
  cudaEventRecord(c->ev_pool[c->ev_used], st);
}
void prof_end(dlra_ctx* c, cudaStream_t st) {
  if (!c->profiling) return;
  cudaEventRecord(c->ev_pool[c->ev_used + 1], st);
  c->ev_used += 2;
}
void prof_collect(dlra_ctx* c) {
  if (c->ev_used == 0) return;
  cudaStreamSynchronize(c->st);
  for (auto& l : c->lanes) cudaStreamSynchronize(l.s0);
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev_pool[i], c->ev_pool[i + 1]);
    c->prof_ms += ms;
    c->prof_count++;
  }
  c->ev_used = 0;
}

// ---------------------------------------------------------------------------
// the energy step, templated on the n-side precision
// ---------------------------------------------------------------------------
template <typename T>
struct Engine {
  void snap_save(const Beam<T>& B, Snap<T>& s, cudaStream_t st) {
    const long long n = ctx->n;
    const int RB = ctx->RB, m = ctx->m;
    cudaMemcpyAsync(s.X, B.X, sizeof(T) * n * RB, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s.W, B.W, sizeof(T) * (size_t)m * RB, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s.S, B.S, sizeof(double) * RB * RB, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s.dims, B.dims, sizeof(BeamDims), cudaMemcpyDeviceToDevice, st);
  }
  void snap_load(const Snap<T>& s, Beam<T>& B, cudaStream_t st) {
    const long long n = ctx->n;
    const int RB = ctx->RB, m = ctx->m;
    cudaMemcpyAsync(B.X, s.X, sizeof(T) * n * RB, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(B.W, s.W, sizeof(T) * (size_t)m * RB, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(B.S, s.S, sizeof(double) * RB * RB, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(B.dims, s.dims, sizeof(BeamDims), cudaMemcpyDeviceToDevice, st);
  }

  dlra_ctx* ctx;
  Lane* L = nullptr;
  std::vector<Beam<T>>& beams() { return *reinterpret_cast<std::vector<Beam<T>>*>(ctx->beams); }
  T* P(void* p) { return reinterpret_cast<T*>(p); }

  bool adj_rank = false;   // the reverse sweep's own rank control (no schedule replay)

  RankParams rank_params() {
    RankParams rp;
    rp.mode = ctx->cfg.rank_mode;
    if (adj_rank && rp.mode == DLRA_RANK_SCHEDULE) rp.mode = DLRA_RANK_ADAPTIVE;
    rp.rank = ctx->cfg.rank;
    // the configured maximum (the capacity RB is rank_max rounded up to a compiled tile width)
    rp.rank_max = (ctx->cfg.rank_max > 0 && ctx->cfg.rank_max < ctx->RB) ? ctx->cfg.rank_max : ctx->RB;
    rp.tol = ctx->cfg.trunc_tol;
    rp.nz_tol = sizeof(T) == 8 ? 1e-14 : 1e-6;
    rp.cluster_tol = sizeof(T) == 8 ? 1e-10 : 1e-5;
    rp.schedule = adj_rank ? nullptr : ctx->schedule_dev;
    return rp;
  }
  // truncation SVD of S^ (n2 x n2, FP64 in memory), in FP64 arithmetic where small64 is set;
  // the rank tolerances stay those of the n-side precision, which sets the noise floor of S^
  void svd_truncate(double* Sh, int n2, int RB, int k, int event, Beam<T>& B) {
    if (ctx->small64)
      launch_svd_truncate<double>(L->s0, Sh, n2, RB, rank_params(), k, event, L->Pt, L->Qt, B.S, B.dims, B.rank_log,
                                  ctx->dev_err, L->svdV);
    else
      launch_svd_truncate<T>(L->s0, Sh, n2, RB, rank_params(), k, event, L->Pt, L->Qt, B.S, B.dims, B.rank_log,
                             ctx->dev_err, L->svdV);
  }
  double drop1() const { return sizeof(T) == 8 ? 1e-12 : 3e-4; }
  double drop2() const { return sizeof(T) == 8 ? 1e-8 : 1e-3; }

  // X^ = [X, orth((I - X X^T) K)] with K (n x qcap); X^ in L->Xh (n x 2RB)
  void augment_x(Beam<T>& B, const T* K, int qcap) {
    const long long n = ctx->n;
    const int RB = ctx->RB;
    cudaStream_t st = L->s0;
    int64_t& nl = ctx->launches;
    T* Xh = P(L->Xh);
    cudaMemsetAsync(Xh + (long long)RB * n, 0, sizeof(T) * n * RB, st);
    cudaMemcpyAsync(Xh, B.X, sizeof(T) * n * RB, cudaMemcpyDeviceToDevice, st);
    const int* rdim = &B.dims->r;
    // C1 = X^T K
    cudaMemsetAsync(L->C1, 0, sizeof(double) * RB * qcap, st);
    gram<T>(st, n, B.X, n, rdim, RB, qcap, FPlain<T>{K, n, nullptr, qcap}, L->C1, RB, nl);
    // R = K - X C1 into X^[:, RB:RB+qcap]
    apply<T>(st, n, B.X, n, RB, rdim, L->C1, RB, qcap, Xh + (long long)RB * n, n, K, T(-1), T(1), nl, nullptr, nullptr,
             &L->atc);
    for (int pass = 0; pass < 2; ++pass) {
      const int lg = RB + qcap;
      cudaMemsetAsync(L->Cg, 0, sizeof(double) * lg * qcap, st);
      gram<T>(st, n, Xh, n, nullptr, lg, qcap, FPlain<T>{Xh + (long long)RB * n, n, nullptr, qcap}, L->Cg, lg, nl);
      launch_orth_factor(st, L->Cg, pass == 0 ? L->C1 : nullptr, RB, qcap, pass == 0 ? drop1() : drop2(),
                         L->Mapply, &B.dims->qx, ctx->dev_err);
      ++nl;
      apply<T>(st, n, Xh, n, lg, nullptr, L->Mapply, lg, qcap, Xh + (long long)RB * n, n, nullptr, T(1), T(0), nl,
               nullptr, nullptr, &L->atc);
    }
  }

  // W^ = [W, orth((I - W W^T) K)] with K (m x qcap, ld m) on the moment-side stream: the same
  // pivoted CholeskyQR2 as augment_x (Gram and pivoted Cholesky factor in FP64, FP32 data),
  // the count of new columns in dims->qw (FP32 paths; the FP64 path runs launch_waug)
  void augment_w(Beam<T>& B, const T* K, int qcap) {
    const int m = ctx->m, RB = ctx->RB;
    cudaStream_t sm = L->s1;
    int64_t& nl = ctx->launches;
    T* Wh = P(L->Wh);
    cudaMemsetAsync(Wh + (long long)RB * m, 0, sizeof(T) * (size_t)m * RB, sm);
    cudaMemcpyAsync(Wh, B.W, sizeof(T) * (size_t)m * RB, cudaMemcpyDeviceToDevice, sm);
    const int* rdim = &B.dims->r;
    cudaMemsetAsync(L->C1m, 0, sizeof(double) * RB * qcap, sm);
    gram<T>(sm, m, B.W, m, rdim, RB, qcap, FPlain<T>{K, m, nullptr, qcap}, L->C1m, RB, nl);
    apply<T>(sm, m, B.W, m, RB, rdim, L->C1m, RB, qcap, Wh + (long long)RB * m, m, K, T(-1), T(1), nl);
    for (int pass = 0; pass < 2; ++pass) {
      const int lg = RB + qcap;
      cudaMemsetAsync(L->Cgm, 0, sizeof(double) * lg * qcap, sm);
      gram<T>(sm, m, Wh, m, nullptr, lg, qcap, FPlain<T>{Wh + (long long)RB * m, m, nullptr, qcap}, L->Cgm, lg, nl);
      launch_orth_factor(sm, L->Cgm, pass == 0 ? L->C1m : nullptr, RB, qcap, pass == 0 ? drop1() : drop2(),
                         L->Mapplym, &B.dims->qw, ctx->dev_err);
      ++nl;
      apply<T>(sm, m, Wh, m, lg, nullptr, L->Mapplym, lg, qcap, Wh + (long long)RB * m, m, nullptr, T(1), T(0), nl);
    }
  }

  // X = X^ Pt, W = W^ Qt after a truncation
  void apply_truncation(Beam<T>& B) {
    const long long n = ctx->n;
    const int RB = ctx->RB, n2 = ctx->n2, m = ctx->m;
    int64_t& nl = ctx->launches;
    apply<T>(L->s0, n, P(L->Xh), n, n2, nullptr, L->Pt, n2, RB, B.X, n, nullptr, T(1), T(0), nl, nullptr, nullptr,
             &L->atc);
    gemm<T, 16>(L->s0, m, RB, n2, ALoadPlain<T>{P(L->Wh), m, nullptr, n2},
                BLoadCol<T, double>{L->Qt, n2, nullptr, n2, nullptr, RB}, EpiStore<T>{B.W, m, nullptr, m, T(1), T(0)},
                nl);
  }

  // fork: st2 waits for everything enqueued so far on st
  void fork() {
    cudaEventRecord(L->ev[0], L->s0);
    cudaStreamWaitEvent(L->s1, L->ev[0], 0);
  }
  // st waits for everything enqueued so far on st2
  void join() {
    cudaEventRecord(L->ev[3], L->s1);
    cudaStreamWaitEvent(L->s0, L->ev[3], 0);
  }

  // Streaming BUG step of Eq. KLS over one energy step (K-, L-, S-steps with n_sub RK4
  // sub-steps each, augmentation, truncation). adj = 1 integrates the transposed operator
  // (reverse sweep): the K-stage kernel applies sum_d rho^-1 [(D^-_d)^T K P^+_d + (D^+_d)^T K P^-_d],
  // the L-step uses G_k instead of G_k^T and the S-step G_k^T instead of G_k.
  // cap (n x RB buffers, stride n RB): forward, the stage inputs rho^-1 z of every sub-step
  // j and stage s at cap[4j + s]; adjoint (required), the adjoint of that stage input.
  void streaming(Beam<T>& B, int k, int adj = 0, T* cap = nullptr) {
    const long long n = ctx->n;
    const int RB = ctx->RB, m = ctx->m, nk = ctx->nk, n2 = ctx->n2;
    cudaStream_t st = L->s0;     // cell-side chain
    cudaStream_t sm = L->s1;    // moment-side chain
    int64_t& nl = ctx->launches;
    const int* rdim = &B.dims->r;
    T* Zm = P(L->Zm);
    const long long nrb = n * RB;
    auto capq = [&](int q) { return cap + (long long)q * nrb; };
    fork();
    // [m] P_k = W^T A^s_d W, packed for the stage kernel; L0 = W S^T
    gemm<T, 16>(sm, (long long)nk * m, RB, m, ALoadRowMajor<T>{P(ctx->Apm), m, m},
                BLoadCol<T, T>{B.W, m, nullptr, m, rdim, RB}, EpiStoreKBlocks<T>{Zm, m, RB}, nl);
    cudaMemsetAsync(L->P1, 0, sizeof(double) * nk * RB * RB, sm);
    gram<T>(sm, m, B.W, m, rdim, RB, nk * RB, FPlain<T>{Zm, m, nullptr, nk * RB}, L->P1, RB, nl);
    pstack_kernel<T><<<nblk((long long)nk * RB * RB, 256), 256, 0, sm>>>(L->P1, RB, nk, P(L->Pst), adj);
    ++nl;
    cudaEventRecord(L->ev[1], sm);
    T* ly = P(L->Lb[0]);
    T* la = P(L->Lb[1]);
    T* lb = P(L->Lb[2]);
    gemm<T, 16>(sm, m, RB, RB, ALoadPlain<T>{B.W, m, rdim, RB}, BLoadRow<T, double>{B.S, RB, RB, RB},
                EpiStore<T>{ly, m, nullptr, m, T(1), T(0)}, nl);
    // [n] G_k = X^T D_k rho^-1 X; K0 = X S (and rho^-1 K0)
    cudaMemsetAsync(L->G1, 0, sizeof(double) * nk * RB * RB, st);
    gram_stencil<T>(st, n, B.X, n, RB, rdim, B.X, n, RB, rdim, P(ctx->inv_rho), ctx->geo, L->G1, RB, RB, nl,
                    ctx->dev_err);
    gt_kernel<T><<<nblk((long long)nk * RB * RB, 256), 256, 0, st>>>(L->G1, RB, nk, P(L->GtT), adj);
    ++nl;
    cudaEventRecord(L->ev[2], st);
    T* y = P(L->Kb[0]);
    T* va = (cap && !adj) ? capq(0) : P(L->Kb[1]);
    T* vb = P(L->Kb[2]);
    if (adj) apply<T>(st, n, B.X, n, RB, rdim, B.S, RB, RB, y, n, nullptr, T(1), T(0), nl, nullptr, nullptr, &L->atc);
    else apply<T>(st, n, B.X, n, RB, rdim, B.S, RB, RB, y, n, nullptr, T(1), T(0), nl, va, P(ctx->inv_rho), &L->atc);
    cudaStreamWaitEvent(st, L->ev[1], 0);   // stage kernel needs P
    cudaStreamWaitEvent(sm, L->ev[2], 0);   // L-stage needs G
    // RK4 Horner stages: K-step on st, L-step on sm
    const int ns = ctx->nsub[k];
    const double hs = ctx->h / ns;
    for (int jj = 0; jj < ns; ++jj) {
      // the transposed K-step runs the sub-steps backwards (their adjoints pair with the
      // forward stages of the same sub-step); the polynomials of one energy step commute,
      // so the L-step keeps the forward order
      const int j = adj ? ns - 1 - jj : jj;
      double beta[4];
      horner_betas(ctx, ctx->E[k] - j * hs, hs, beta);
      if (adj) cudaMemcpyAsync(va, y, sizeof(T) * nrb, cudaMemcpyDeviceToDevice, st);
      const T* vins[4] = {va, vb, va, vb};
      T* vouts[4] = {vb, va, vb, va};
      const T* lin = ly;
      T* louts[4] = {la, lb, la, ly};
      for (int s2 = 0; s2 < 4; ++s2) {
        prof_begin(ctx, st);
        if (adj) {
          // adjoint stage s2 uses the outermost remaining Horner factor and produces the
          // adjoint of the input of forward stage 3 - s2
          const int sf = 3 - s2;
          const T* vin = s2 == 0 ? va : capq(4 * j + sf + 1);
          kstage<T>(RB, st, vin, y, y, capq(4 * j + sf), n, P(ctx->inv_rho), ctx->geo, P(L->Pst), rdim,
                    T(beta[sf]), 2, nl, ctx->dev_err, ctx->tun.kstage_variant, L->Bimg);
        } else if (cap) {
          T* vout = s2 < 3 ? capq(4 * j + s2 + 1) : (j + 1 < ns ? capq(4 * (j + 1)) : vb);
          kstage<T>(RB, st, capq(4 * j + s2), y, y, vout, n, P(ctx->inv_rho), ctx->geo, P(L->Pst), rdim,
                    T(beta[s2]), s2 == 3 ? 1 : 0, nl, ctx->dev_err, ctx->tun.kstage_variant, L->Bimg);
        } else {
          kstage<T>(RB, st, vins[s2], y, y, vouts[s2], n, P(ctx->inv_rho), ctx->geo, P(L->Pst), rdim,
                    T(beta[s2]), s2 == 3 ? 1 : 0, nl, ctx->dev_err, ctx->tun.kstage_variant, L->Bimg);
        }
        prof_end(ctx, st);
        double lbeta[4];
        horner_betas(ctx, ctx->E[k] - jj * hs, hs, lbeta);
        // the m-side stage out = y + beta sum_k A_k z G_k^T as two tiled products: U_k = A_k z
        // for all k at once (nk m x m by m x r), then y + beta [U_0 .. U_nk-1] [G_0^T; ..]
        lstage<T>(sm, m, nk, RB, rdim, P(ctx->Apm), lin, ly, louts[s2], P(L->GtT), P(L->Ul), T(lbeta[s2]), nl);
        lin = louts[s2];
      }
    }
    // augmentation of both bases, then the Galerkin operators on them
    augment_x(B, y, RB);
    if (sizeof(T) == 4) {
      augment_w(B, ly, RB);
    } else {
      launch_waug<T, T>(sm, B.W, m, RB, ly, m, RB, drop1(), P(L->Wh), B.dims);
      ++nl;
    }
    T* Xh = P(L->Xh);
    T* Wh = P(L->Wh);
    cudaMemsetAsync(L->Gc, 0, sizeof(double) * nk * n2 * n2, st);
    gram_stencil<T>(st, n, Xh, n, n2, nullptr, Xh, n, n2, nullptr, P(ctx->inv_rho), ctx->geo, L->Gc, n2, n2, nl,
                    ctx->dev_err);
    if (adj) {
      launch_transpose_blocks(st, L->Gc, n2, nk);
      ++nl;
    }
    gemm<T, 16>(sm, (long long)nk * m, n2, m, ALoadRowMajor<T>{P(ctx->Apm), m, m},
                BLoadCol<T, T>{Wh, m, nullptr, m, nullptr, n2}, EpiStoreKBlocks<T>{Zm, m, n2}, nl);
    cudaMemsetAsync(L->Ph, 0, sizeof(double) * nk * n2 * n2, sm);
    gram<T>(sm, m, Wh, m, nullptr, n2, nk * n2, FPlain<T>{Zm, m, nullptr, nk * n2}, L->Ph, n2, nl);
    join();
    if (ctx->small64)
      launch_sstep<double>(st, L->Gc, L->Ph, nk, B.S, RB, n2, ctx->sbeta + (long long)k * ctx->nsub_max * 4, ns,
                           L->Sh, &L->sgw, ctx->dev_err);
    else
      launch_sstep<T>(st, L->Gc, L->Ph, nk, B.S, RB, n2, ctx->sbeta + (long long)k * ctx->nsub_max * 4, ns, L->Sh,
                      &L->sgw, ctx->dev_err);
    ++nl;
    svd_truncate(L->Sh, n2, RB, k, 0, B);
    ++nl;
    apply_truncation(B);
  }

  void scattering(Beam<T>& B, int k) {
    const long long n = ctx->n;
    const int RB = ctx->RB, m = ctx->m, M = ctx->M, N = ctx->N;
    cudaStream_t st = L->s0;
    int64_t& nl = ctx->launches;
    const int* rdim = &B.dims->r;
    cudaMemsetAsync(L->Mg, 0, sizeof(double) * M * RB * RB, st);
    gram<T>(st, n, B.X, n, rdim, RB, M * RB, FDiag<T>{B.X, n, P(ctx->wc), n, RB, rdim, M}, L->Mg, RB, nl);
    launch_scatter_solve<T>(st, L->Mg, M, ctx->coef + (long long)k * M * (N + 1), N, B.S, B.W, m, RB,
                            P(L->L1T), ctx->dev_err);
    ++nl;
    launch_qr_lt<T>(st, P(L->L1T), m, RB, B.dims, B.W, B.S, L->mwork);
    ++nl;
  }

  void source(Beam<T>& B, int k) {
    source_with(B, k, nullptr, B.Bsrc + (long long)k * ctx->M * ctx->m, ctx->M, B.psi + (long long)k * ctx->n);
  }

  // Explicit-Euler source BUG step (Sec. 3.3.3 steps 2-4) for a rank-Ms source h A Bk^T:
  // A (n x Ms) given, or (A == nullptr) w_i(x) psi(x) built from the fluence psi.
  void source_with(Beam<T>& B, int k, const T* Ain, const double* Bk, int Ms, const double* psi) {
    const long long n = ctx->n;
    const int RB = ctx->RB, m = ctx->m, n2 = ctx->n2;
    cudaStream_t st = L->s0;
    int64_t& nl = ctx->launches;
    fork();
    if (sizeof(T) == 4) {
      convert_kernel<T><<<nblk((long long)m * Ms, 256), 256, 0, L->s1>>>(Bk, (long long)m * Ms, P(L->Kw));
      ++nl;
      augment_w(B, P(L->Kw), Ms);
    } else {
      launch_waug<T, double>(L->s1, B.W, m, RB, Bk, m, Ms, drop1(), P(L->Wh), B.dims);
      ++nl;
    }
    const T* A = Ain;
    if (!A) {
      src_vec_kernel<T><<<nblk(n, 256), 256, 0, st>>>(P(ctx->wT), psi, n, Ms, P(L->Asrc));
      ++nl;
      A = P(L->Asrc);
    }
    augment_x(B, A, Ms);
    cudaMemsetAsync(L->XA, 0, sizeof(double) * n2 * Ms, st);
    gram<T>(st, n, P(L->Xh), n, nullptr, n2, Ms, FPlain<T>{A, n, nullptr, Ms}, L->XA, n2, nl);
    join();
    launch_src_assemble<T>(st, B.S, RB, L->XA, Bk, P(L->Wh), m, Ms, n2, ctx->h, L->Sh);
    ++nl;
    svd_truncate(L->Sh, n2, RB, k, 1, B);
    ++nl;
    apply_truncation(B);
  }

  void dose(Beam<T>& B) {
    dose_kernel<T><<<std::min<unsigned>(nblk(ctx->n, 256), 2048), 256, 0, L->s0>>>(
        B.X, ctx->n, B.S, B.W, ctx->m, ctx->RB, B.dims, ctx->h * std::sqrt(4.0 * M_PI), B.e_c);
    ++ctx->launches;
  }

  // One energy step of the joint state (held by beam 0): streaming and collided scattering once,
  // then the first-collision source of every beam that has one at this step, each beam's rank-M
  // factor scaled by its weight and stacked into one source of rank M x (active beams)
  void joint_step(int k) {
    auto& bs = beams();
    Beam<T>& J = bs[0];
    L = &ctx->lanes[0];
    const long long n = ctx->n;
    const int M = ctx->M, m = ctx->m;
    if (J.active) {
      streaming(J, k);
      scattering(J, k);
    }
    int cols = 0;
    for (size_t b = 0; b < bs.size(); ++b) {
      if (!bs[b].has_src[k]) continue;
      src_vec_scaled_kernel<T><<<nblk(n, 256), 256, 0, L->s0>>>(P(ctx->wT), bs[b].psi + (long long)k * n, n, M,
                                                                bs[b].weight, P(ctx->joint_A) + (long long)cols * n);
      ++ctx->launches;
      cudaMemcpyAsync(ctx->joint_B + (long long)cols * m, bs[b].Bsrc + (long long)k * M * m,
                      sizeof(double) * (size_t)M * m, cudaMemcpyDeviceToDevice, L->s0);
      cols += M;
    }
    if (cols > 0) {
      source_with(J, k, P(ctx->joint_A), ctx->joint_B, cols, nullptr);
      J.active = true;
    }
    if (J.active) dose(J);
  }

  dlra_status step_all(int nsteps) {
    const int nlanes = (int)ctx->lanes.size();
    for (int s = 0; s < nsteps; ++s) {
      const int k = ctx->step;
      // every lane starts after the work enqueued so far on the context stream
      cudaEventRecord(ctx->ev_step, ctx->st);
      for (int l = 0; l < nlanes; ++l) cudaStreamWaitEvent(ctx->lanes[l].s0, ctx->ev_step, 0);
      auto& bs = beams();
      if (ctx->joint && !bs.empty()) joint_step(k);
      for (size_t b = 0; b < bs.size() && !ctx->joint; ++b) {
        Beam<T>& B = bs[b];
        L = &ctx->lanes[b % nlanes];
        if (ctx->ckpt_interval > 0 && k % ctx->ckpt_interval == 0)
          snap_save(B, B.ckpt[k / ctx->ckpt_interval], L->s0);
        if (B.active) {
          streaming(B, k);
          scattering(B, k);
        }
        if (B.has_src[k]) {
          source(B, k);
          B.active = true;
        }
        if (B.active) dose(B);
      }
      // the context stream waits for every lane
      for (int l = 0; l < nlanes; ++l) {
        cudaEventRecord(ctx->lanes[l].ev[2], ctx->lanes[l].s0);
        cudaStreamWaitEvent(ctx->st, ctx->lanes[l].ev[2], 0);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return fail(ctx, DLRA_ERR_CUDA, "kernel launch failed at step %d: %s", k, cudaGetErrorString(e));
      ctx->step++;
      if (ctx->ev_used > 4096) prof_collect(ctx);
    }
    return DLRA_OK;
  }
};

dlra_status check_device_errors(dlra_ctx* ctx) {
  if (ctx->poisoned != DLRA_OK) return ctx->poisoned;
  cudaError_t e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) return fail(ctx, DLRA_ERR_CUDA, "stream failed: %s", cudaGetErrorString(e));
  int h = 0;
  e = cudaMemcpy(&h, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(ctx, DLRA_ERR_CUDA, "error flag read failed: %s", cudaGetErrorString(e));
  if (h & ERR_NONFINITE) return fail(ctx, DLRA_ERR_NONFINITE, "the low-rank state became non-finite");
  if (h & ERR_CHOLESKY) return fail(ctx, DLRA_ERR_NONFINITE, "implicit scattering matrix is not positive definite");
  if (h & ERR_CAPACITY) return fail(ctx, DLRA_ERR_RANK, "rank capacity rank_max exceeded");
  if (h & ERR_TIMEOUT) return fail(ctx, DLRA_ERR_TIMEOUT, "a bounded device-side wait gave up");
  return DLRA_OK;
}

template <typename T>
std::vector<Beam<T>>& beams_of(dlra_ctx* ctx) {
  return *reinterpret_cast<std::vector<Beam<T>>*>(ctx->beams);
}

void drop_graphs(dlra_ctx* ctx) {
  for (auto& g : ctx->step_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  ctx->step_graphs.clear();
}

template <typename T>
std::vector<char> active_flags(dlra_ctx* ctx) {
  std::vector<char> a;
  for (auto& B : beams_of<T>(ctx)) a.push_back(B.active ? 1 : 0);
  return a;
}

template <typename T>
void set_active_flags(dlra_ctx* ctx, const std::vector<char>& a) {
  auto& bs = beams_of<T>(ctx);
  for (size_t b = 0; b < bs.size() && b < a.size(); ++b) bs[b].active = a[b] != 0;
}

// dlra_step through a CUDA graph: the work of n energy steps from the current step (ranks
// live on the device, so the launch sequence depends only on the step range and on which
// beams are active) is captured once on a private stream and replayed on the context stream.
// A capture that fails falls back to launching the kernels directly.
template <typename T>
dlra_status step_graph(dlra_ctx* ctx, int n) {
  const std::vector<char> before = active_flags<T>(ctx);
  for (auto& g : ctx->step_graphs)
    if (g.start == ctx->step && g.n == n && g.active_before == before) {
      CK(cudaGraphLaunch(g.exec, ctx->st));
      ctx->launches += g.launches;
      ctx->step += n;
      set_active_flags<T>(ctx, g.active_after);
      return DLRA_OK;
    }
  if (!ctx->cap_st) CK(cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking));
  const int step0 = ctx->step;
  const int64_t l0 = ctx->launches;
  cudaStream_t user = ctx->st;
  CK(cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeRelaxed));
  ctx->st = ctx->cap_st;
  dlra_status s = Engine<T>{ctx}.step_all(n);
  ctx->st = user;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->cap_st, &graph);
  cudaGraphExec_t exec = nullptr;
  if (s == DLRA_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (s != DLRA_OK || e != cudaSuccess || !exec) {
    cudaGetLastError();
    if (ctx->poisoned == DLRA_ERR_CUDA) ctx->poisoned = DLRA_OK;
    ctx->step = step0;
    ctx->launches = l0;
    set_active_flags<T>(ctx, before);
    ctx->graphs = false;
    return Engine<T>{ctx}.step_all(n);
  }
  StepGraph g;
  g.start = step0;
  g.n = n;
  g.active_before = before;
  g.active_after = active_flags<T>(ctx);
  g.exec = exec;
  g.launches = ctx->launches - l0;
  ctx->step_graphs.push_back(std::move(g));
  CK(cudaGraphLaunch(exec, ctx->st));
  return DLRA_OK;
}

template <typename T>
dlra_status alloc_shared(dlra_ctx* ctx) {
  const long long n = ctx->n;
  const int m = ctx->m, nk = ctx->nk;
  ALLOC(ctx->inv_rho, sizeof(T) * n);
  ALLOC(ctx->rho, sizeof(double) * n);
  ALLOC(ctx->f_cell, sizeof(double) * n);
  ALLOC(ctx->tau_cell, sizeof(double) * n);
  ALLOC(ctx->Apm, sizeof(T) * (size_t)nk * m * m);
  ALLOC(ctx->dev_err, sizeof(int));
  ctx->tun.gram_err = ctx->dev_err;
  ALLOC(ctx->flags_dev, sizeof(int) * ctx->K);
  ALLOC(ctx->dose_tmp, sizeof(double) * n);
  ALLOC(ctx->zeros, sizeof(double) * n);
  return DLRA_OK;
}

// a new lane (work space and streams); needs the number of materials
template <typename T>
dlra_status alloc_lane(dlra_ctx* ctx) {
  const long long n = ctx->n;
  const int m = ctx->m, RB = ctx->RB, nk = ctx->nk, n2 = ctx->n2, M = ctx->M;
  ctx->lanes.emplace_back();
  Lane& L = ctx->lanes.back();
  CK(cudaStreamCreateWithFlags(&L.s0, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&L.s1, cudaStreamNonBlocking));
  for (int i = 0; i < 4; ++i) CK(cudaEventCreateWithFlags(&L.ev[i], cudaEventDisableTiming));
  for (int i = 0; i < 3; ++i) ALLOC(L.Kb[i], sizeof(T) * n * RB);
  ALLOC(L.Xh, sizeof(T) * n * n2);
  ALLOC(L.Asrc, sizeof(T) * M * n);
  for (int i = 0; i < 3; ++i) ALLOC(L.Lb[i], sizeof(T) * m * RB);
  ALLOC(L.Zm, sizeof(T) * (size_t)m * nk * n2);
  ALLOC(L.Wh, sizeof(T) * (size_t)m * n2);
  ALLOC(L.L1T, sizeof(T) * (size_t)m * RB);
  ALLOC(L.Ul, sizeof(T) * (size_t)nk * RB * m);
  ALLOC(L.Pst, sizeof(T) * (size_t)nk * RB * RB);
  ALLOC(L.GtT, sizeof(T) * (size_t)nk * RB * RB);
  ALLOC(L.G1, sizeof(double) * nk * RB * RB);
  ALLOC(L.P1, sizeof(double) * nk * RB * RB);
  ALLOC(L.Gc, sizeof(double) * nk * n2 * n2);
  ALLOC(L.Ph, sizeof(double) * nk * n2 * n2);
  ALLOC(L.C1, sizeof(double) * RB * RB);
  ALLOC(L.Cg, sizeof(double) * n2 * RB);
  ALLOC(L.Mapply, sizeof(double) * n2 * RB);
  ALLOC(L.Sh, sizeof(double) * n2 * n2);
  ALLOC(L.Pt, sizeof(double) * n2 * RB);
  ALLOC(L.Qt, sizeof(double) * n2 * RB);
  ALLOC(L.Mg, sizeof(double) * M * RB * RB);
  ALLOC(L.XA, sizeof(double) * n2 * M);
  if (sizeof(T) == 4) {
    ALLOC(L.mwork, sizeof(double) * mside_work_doubles(m, RB));
    ALLOC(L.C1m, sizeof(double) * RB * RB);
    ALLOC(L.Cgm, sizeof(double) * n2 * RB);
    ALLOC(L.Mapplym, sizeof(double) * n2 * RB);
    ALLOC(L.Kw, sizeof(T) * (size_t)m * std::max(RB, M));
  }
  if (sizeof(T) == 4 && ctx->geo.nact == 3 && kstage_tma_bimg_bytes(RB) > 0)
    ALLOC(L.Bimg, kstage_tma_bimg_bytes(RB));
  if (sizeof(T) == 4) {
    ALLOC(L.atc.img, ApTc<64>::BBYTES);
    L.atc.err = ctx->dev_err;
  }
  const size_t tsmall = ctx->small64 ? sizeof(double) : sizeof(T);   // arithmetic of the SVD and S-step
  if (svd_needs_vwork(n2, tsmall)) ALLOC(L.svdV, tsmall * (size_t)n2 * n2);
  if (sstep_needs_grid(nk, n2, tsmall)) {
    const size_t ne = (size_t)n2 * n2;
    ALLOC(L.sgw.z, tsmall * ne);
    ALLOC(L.sgw.U, tsmall * ne * nk);
    ALLOC(L.sgw.O, tsmall * ne * nk);
    ALLOC(L.sgw.bar, 4 * sizeof(unsigned));
    const int cap = sstep_grid_capacity(tsmall);
    const int nt = (n2 + 15) / 16;
    const int share = cap / std::max(1, ctx->max_lanes);
    L.sgw.grid = std::max(1, std::min(nk * nt * nt, share));
    if (cap <= 0) return fail(ctx, DLRA_ERR_CUDA, "occupancy query of the S-step kernel failed");
  }
  return DLRA_OK;
}

RayGeo ray_geo(const dlra_ctx* ctx);

template <typename T>
dlra_status alloc_snap(dlra_ctx* ctx, Snap<T>& s) {
  ALLOC(s.X, sizeof(T) * ctx->n * ctx->RB);
  ALLOC(s.W, sizeof(T) * (size_t)ctx->m * ctx->RB);
  ALLOC(s.S, sizeof(double) * ctx->RB * ctx->RB);
  ALLOC(s.dims, sizeof(BeamDims));
  return DLRA_OK;
}

// checkpoint slots of every beam for the current interval (before the first step)
template <typename T>
dlra_status ensure_checkpoints(dlra_ctx* ctx) {
  const int I = ctx->ckpt_interval;
  if (I <= 0) return DLRA_OK;
  const size_t need = (size_t)((ctx->K + I - 1) / I);
  for (auto& B : beams_of<T>(ctx))
    while (B.ckpt.size() < need) {
      B.ckpt.emplace_back();
      dlra_status s = alloc_snap<T>(ctx, B.ckpt.back());
      if (s != DLRA_OK) return s;
    }
  CK(cudaStreamSynchronize(ctx->st));
  return DLRA_OK;
}

// work space of the reverse sweep; grows with the number of beams, sub-steps and rays
template <typename T>
dlra_status alloc_adj(dlra_ctx* ctx) {
  const long long n = ctx->n;
  const int m = ctx->m, RB = ctx->RB, K = ctx->K, M = ctx->M, N = ctx->N;
  auto& bs = beams_of<T>(ctx);
  const int nb = (int)bs.size();
  if (!ctx->adj) ctx->adj = new AdjWork<T>();
  AdjWork<T>& A = *reinterpret_cast<AdjWork<T>*>(ctx->adj);
  if (!A.mu.X) {
    for (Beam<T>* B : {&A.mu, &A.rep}) {
      ALLOC(B->X, sizeof(T) * n * RB);
      ALLOC(B->W, sizeof(T) * (size_t)m * RB);
      ALLOC(B->S, sizeof(double) * RB * RB);
      ALLOC(B->dims, sizeof(BeamDims));
      ALLOC(B->rank_log, sizeof(int) * 2 * K);
    }
    dlra_status s = alloc_snap<T>(ctx, A.alpha);
    if (s != DLRA_OK) return s;
    ALLOC(A.gvec, sizeof(T) * n);
    ALLOC(A.ge, sizeof(double) * n);
    ALLOC(A.gtmp, sizeof(double) * n);
    ALLOC(A.be0, sizeof(double) * m);
    ALLOC(A.grad_rho, sizeof(double) * n);
    ALLOC(A.grad_f, sizeof(double) * n);
    ALLOC(A.grad_tau, sizeof(double) * n);
    ALLOC(A.grad_w, sizeof(double) * M * n);
    ALLOC(A.dw, sizeof(double) * M * n);
    ALLOC(A.Cm, sizeof(double) * RB * RB);
    ALLOC(A.Cl, sizeof(double) * (N + 1) * RB * RB);
    ALLOC(A.ysrc, sizeof(double) * M * RB);
    ALLOC(A.mcoef, sizeof(double) * 2 * M);
    // the dose reads the l = 0 moment: e += h sqrt(4 pi) u(., 0)
    const double s4 = std::sqrt(4.0 * M_PI);
    CK(cudaMemcpyAsync(A.be0, &s4, sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  }
  if (A.cap_ns < ctx->nsub_max) {
    ALLOC(A.capf, sizeof(T) * (size_t)4 * ctx->nsub_max * n * RB);
    ALLOC(A.capa, sizeof(T) * (size_t)4 * ctx->nsub_max * n * RB);
    A.cap_ns = ctx->nsub_max;
  }
  {
    // keep the forward stage inputs of a whole segment when they fit in a third of the free memory
    const size_t stride = (size_t)4 * ctx->nsub_max * n * RB;
    const size_t need = stride * sizeof(T) * ctx->ckpt_interval * nb +
                        (size_t)ctx->ckpt_interval * nb * (sizeof(T) * ((size_t)n + m) * RB + sizeof(double) * RB * RB);
    const size_t slots = (size_t)ctx->ckpt_interval * nb;
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    if (!ctx->adj_store) {
      A.store = false;
    } else if (A.capseg && A.capseg_stride == stride && A.capseg_slots >= slots && A.segb.size() >= slots) {
      A.store = true;
    } else if (need < freeb / 3) {
      CK(cudaStreamSynchronize(ctx->st));
      dfree(ctx, A.capseg);
      A.capseg = nullptr;
      ALLOC(A.capseg, stride * sizeof(T) * slots);
      A.capseg_stride = stride;
      A.capseg_slots = slots;
      while (A.segb.size() < slots) {
        A.segb.emplace_back();
        dlra_status s = alloc_snap<T>(ctx, A.segb.back());
        if (s != DLRA_OK) return s;
      }
      A.store = true;
    } else {
      A.store = false;
    }
  }
  while (A.seg.size() < (size_t)ctx->ckpt_interval * nb) {
    A.seg.emplace_back();
    dlra_status s = alloc_snap<T>(ctx, A.seg.back());
    if (s != DLRA_OK) return s;
  }
  while ((int)A.gpsi.size() < nb) {
    A.gpsi.push_back(nullptr);
    ALLOC(A.gpsi.back(), sizeof(double) * (size_t)K * n);
  }
  if (nb > A.nb_cap) {
    ALLOC(A.dbeta, sizeof(double) * nb);
    A.nb_cap = nb;
  }
  size_t rb = 0;
  RayGeo g = ray_geo(ctx);
  for (int c : ctx->ray_count) rb = std::max(rb, raytrace_adjoint_scratch_bytes(c, g));
  if (rb > A.ray_scratch_bytes) {
    ALLOC(A.ray_scratch, rb);
    A.ray_scratch_bytes = rb;
  }
  std::vector<double> mc(2 * M);
  for (int i = 0; i < M; ++i) {
    mc[2 * i] = ctx->mats[i].density * ctx->mats[i].sp_ratio;
    mc[2 * i + 1] = ctx->tau_coef[i];
  }
  CK(cudaMemcpyAsync(A.mcoef, mc.data(), sizeof(double) * 2 * M, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return DLRA_OK;
}

template <typename T>
dlra_status upload_apm(dlra_ctx* ctx) {
  // A^+_d = (A_d + |A_d|)/2 (s = 0) and A^-_d = (A_d - |A_d|)/2 (s = 1), row-major per k
  const int m = ctx->m;
  std::vector<T> h((size_t)ctx->nk * m * m);
  for (int da = 0; da < ctx->geo.nact; ++da) {
    const int d = ctx->geo.dirs[da];
    for (int s = 0; s < 2; ++s)
      for (int p = 0; p < m; ++p)
        for (int q = 0; q < m; ++q) {
          double a = ctx->ang.A[d][(size_t)p * m + q], b = ctx->ang.absA[d][(size_t)p * m + q];
          h[((size_t)(2 * da + s) * m + p) * m + q] = T(0.5 * (s == 0 ? a + b : a - b));
        }
  }
  CK(cudaMemcpyAsync(ctx->Apm, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return DLRA_OK;
}

template <typename T>
dlra_status set_materials_t(dlra_ctx* ctx, const double* w_host) {
  const long long n = ctx->n;
  const int M = ctx->M;
  // mixture: S(x, E) = rho_s(x) S_w(E), rho_s = sum_i w_i rho_i s_i
  std::vector<double> rho_s(n, 0.0), rho(n, 0.0), tau(n, 0.0);
  std::vector<T> inv_rho(n), wc((size_t)M * n), wT((size_t)M * n);
  ctx->tau_coef.assign(M, 0.0);
  for (int i = 0; i < M; ++i) {
    const dlra_material& mt = ctx->mats[i];
    double g0 = 0.0;
    if (ctx->cfg.collision == DLRA_BOLTZMANN) {
      const std::vector<double>& s = ctx->s_unit[i];
      g0 = (s[0] - (ctx->cfg.transport_correction ? s[ctx->N + 1] : 0.0)) / ctx->xi_unit[i];
    } else if (ctx->cfg.transport_correction == 2) {
      // corrected Fokker-Planck: Sigma_t = (xi_1/2)(N+1)(N+2) = (T_w/2) rho kappa (N+1)(N+2)/2
      g0 = 0.5 * (ctx->N + 1.0) * (ctx->N + 2.0);
    }
    ctx->tau_coef[i] = mt.density * mt.scatter_ratio * g0;
    for (long long x = 0; x < n; ++x) {
      double wv = w_host[(size_t)i * n + x];
      rho_s[x] += wv * mt.density * mt.sp_ratio;
      rho[x] += wv * mt.density;
      tau[x] += wv * mt.density * mt.scatter_ratio * g0;
    }
  }
  double rmin = 1e300;
  for (long long x = 0; x < n; ++x) {
    if (!(rho_s[x] > 0.0)) return fail(ctx, DLRA_ERR_ARG, "cell %lld has no stopping power (rho_s = %g)", x, rho_s[x]);
    rmin = std::min(rmin, rho_s[x]);
    inv_rho[x] = T(1.0 / rho_s[x]);
  }
  for (int i = 0; i < M; ++i)
    for (long long x = 0; x < n; ++x) {
      wc[(size_t)i * n + x] = T(w_host[(size_t)i * n + x] / rho_s[x]);
      wT[(size_t)i * n + x] = T(w_host[(size_t)i * n + x]);
    }
  ctx->rho_s_host = rho_s;
  ctx->rho_host = rho;
  if (!ctx->wc) ALLOC(ctx->wc, sizeof(T) * M * n);
  if (!ctx->wT) ALLOC(ctx->wT, sizeof(T) * M * n);
  CK(cudaMemcpyAsync(ctx->inv_rho, inv_rho.data(), sizeof(T) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->wc, wc.data(), sizeof(T) * wc.size(), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->wT, wT.data(), sizeof(T) * wT.size(), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->rho, rho.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->f_cell, rho_s.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->tau_cell, tau.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
  // sub-steps, Horner coefficients, scattering coefficients per energy step
  const int K = ctx->K;
  double lam = 0.0;
  for (int da = 0; da < ctx->geo.nact; ++da) {
    int d = ctx->geo.dirs[da];
    double delta = d == 0 ? ctx->cfg.dx : (d == 1 ? ctx->cfg.dy : ctx->cfg.dz);
    lam += ctx->ang.lam_max / delta;
  }
  ctx->nsub.assign(K, 1);
  for (int k = 0; k < K; ++k) {
    double nu = ctx->h * lam / (rmin * Sw(ctx, ctx->E[k]) * ctx->cfg.cfl_max);
    ctx->nsub[k] = std::max(1, (int)std::ceil(nu - 1e-9));
  }
  ctx->nsub_max = *std::max_element(ctx->nsub.begin(), ctx->nsub.end());
  std::vector<double> sbeta((size_t)K * ctx->nsub_max * 4, 0.0);
  for (int k = 0; k < K; ++k) {
    double hs = ctx->h / ctx->nsub[k];
    for (int j = 0; j < ctx->nsub[k]; ++j) horner_betas(ctx, ctx->E[k] - j * hs, hs, &sbeta[((size_t)k * ctx->nsub_max + j) * 4]);
  }
  std::vector<double> coef((size_t)K * M * (ctx->N + 1));
  std::vector<double> self, src;
  for (int k = 0; k < K; ++k) {
    double E1 = ctx->E[k + 1];
    for (int i = 0; i < M; ++i) {
      moments_at(ctx, i, E1, self, src);
      for (int l = 0; l <= ctx->N; ++l) coef[((size_t)k * M + i) * (ctx->N + 1) + l] = ctx->h * self[l] / Sw(ctx, E1);
    }
  }
  if (ctx->sbeta_cap < sbeta.size()) {
    ALLOC(ctx->sbeta, sizeof(double) * sbeta.size());
    ctx->sbeta_cap = sbeta.size();
  }
  if (!ctx->coef) ALLOC(ctx->coef, sizeof(double) * coef.size());
  CK(cudaMemcpyAsync(ctx->sbeta, sbeta.data(), sizeof(double) * sbeta.size(), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return DLRA_OK;
}

RayGeo ray_geo(const dlra_ctx* ctx) {
  const dlra_config& c = ctx->cfg;
  RayGeo g;
  g.nx = c.nx; g.ny = c.ny; g.nz = c.nz; g.two_d = ctx->two_d ? 1 : 0; g.K = ctx->K;
  g.dx = c.dx; g.dy = ctx->two_d ? 1.0 : c.dy; g.dz = c.dz;
  g.e_max = c.e_max; g.h = ctx->h; g.e_min = c.e_min; g.p = c.bk_p; g.alpha = c.bk_alpha;
  g.klam = c.t100 * 1e4 * c.bk_p * c.bk_alpha / 2.0;
  g.volume = c.dx * c.dz * (ctx->two_d ? 1.0 : c.dy);
  return g;
}

// in-scattering moment vectors B[k][i][p] = G_{i,l(p)}(E_{k+1/2}) m_p(Omega) of one beam
template <typename T>
dlra_status upload_bsrc(dlra_ctx* ctx, Beam<T>& B) {
  const int m = ctx->m, K = ctx->K, M = ctx->M;
  std::vector<double> mo(m), Bh((size_t)K * M * m), self, src;
  real_sh_dir(ctx->N, B.dir, mo.data());
  for (int k = 0; k < K; ++k) {
    double Em = 0.5 * (ctx->E[k] + ctx->E[k + 1]);
    for (int i = 0; i < M; ++i) {
      moments_at(ctx, i, Em, self, src);
      for (int p = 0; p < m; ++p) Bh[((size_t)k * M + i) * m + p] = src[ctx->ang.degree[p]] * mo[p];
    }
  }
  CK(cudaMemcpyAsync(B.Bsrc, Bh.data(), sizeof(double) * Bh.size(), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return DLRA_OK;
}

// The beam's uncollided fluence per energy bin and deposit from the energy-DG straggling tracer
// (Sec. 3.2; dlra_straggling_trace), in place of the CSDA tracer's
dlra_status straggling_source(dlra_ctx* ctx, const dlra_beam& b, double* psi, double* e_u) {
  const dlra_config& c = ctx->cfg;
  dlra_straggling_trace_args a{};
  a.nx = c.nx; a.ny = c.ny; a.nz = c.nz;
  a.dx = c.dx; a.dy = c.dy; a.dz = c.dz;
  a.e_min = c.e_min; a.e_max = c.e_max;
  a.n_bins = ctx->K;
  a.n_elem = ctx->strag_elems;
  a.h_max = ctx->strag_hmax;
  a.bk_p = c.bk_p; a.bk_alpha = c.bk_alpha; a.t100 = c.t100;
  a.straggling = ctx->strag_on;
  a.energy = b.energy; a.energy_sigma = b.energy_sigma; a.spot_sigma = b.spot_sigma;
  for (int q = 0; q < 3; ++q) {
    a.pos[q] = b.pos[q];
    a.dir[q] = b.dir[q];
  }
  a.f_cell = ctx->f_cell;
  a.tau_cell = ctx->tau_cell;
  a.psi = psi;
  a.e_u = e_u;
  a.cuda_stream = ctx->st;
  dlra_status s = dlra_straggling_trace(&a);
  if (s != DLRA_OK) return fail(ctx, s, "straggling trace: %s", dlra_last_error(nullptr));
  return DLRA_OK;
}

template <typename T>
dlra_status add_beam_t(dlra_ctx* ctx, const dlra_beam* b, int32_t* id) {
  const long long n = ctx->n;
  const int m = ctx->m, RB = ctx->RB, K = ctx->K, M = ctx->M;
  const dlra_config& c = ctx->cfg;
  // rays: transverse Gaussian grid at half-integer pitch, Gauss-Hermite energies
  double d[3] = {b->dir[0], b->dir[1], b->dir[2]};
  double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (!(dn > 0.0)) return fail(ctx, DLRA_ERR_ARG, "beam direction is zero");
  for (double& v : d) v /= dn;
  if (ctx->two_d && std::fabs(d[1]) > 1e-12) return fail(ctx, DLRA_ERR_ARG, "a 2-D slab beam must have dir[1] = 0");
  double u1[3], u2[3] = {0, 0, 0};
  if (ctx->two_d) {
    double l = std::sqrt(d[2] * d[2] + d[0] * d[0]);
    u1[0] = d[2] / l; u1[1] = 0.0; u1[2] = -d[0] / l;
  } else {
    double e[3] = {0, 1, 0};
    if (std::fabs(d[1]) >= 0.9) { e[0] = 1; e[1] = 0; }
    u1[0] = e[1] * d[2] - e[2] * d[1];
    u1[1] = e[2] * d[0] - e[0] * d[2];
    u1[2] = e[0] * d[1] - e[1] * d[0];
    double l = std::sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    for (double& v : u1) v /= l;
    u2[0] = d[1] * u1[2] - d[2] * u1[1];
    u2[1] = d[2] * u1[0] - d[0] * u1[2];
    u2[2] = d[0] * u1[1] - d[1] * u1[0];
  }
  double pitch = ctx->two_d ? std::min(c.dx, c.dz) / 4.0 : std::min(c.dx, std::min(c.dy, c.dz)) / 4.0;
  std::vector<double> offs, gw;
  if (b->spot_sigma > 0.0) {
    int nh = (int)std::ceil(3.5 * b->spot_sigma / pitch);
    for (int j = -nh; j < nh; ++j) {
      double o = (j + 0.5) * pitch;
      offs.push_back(o);
      gw.push_back(std::exp(-0.5 * (o / b->spot_sigma) * (o / b->spot_sigma)));
    }
  } else {
    offs.push_back(0.0);
    gw.push_back(1.0);
  }
  std::vector<double> ee, ew;
  if (b->energy_sigma > 0.0) {
    double x[5], w[5];
    gauss_hermite(5, x, w);
    for (int i = 0; i < 5; ++i) {
      ee.push_back(b->energy + std::sqrt(2.0) * b->energy_sigma * x[i]);
      ew.push_back(w[i] / std::sqrt(M_PI));
    }
  } else {
    ee.push_back(b->energy);
    ew.push_back(1.0);
  }
  for (double e : ee)
    if (e > c.e_max + 1e-12 || e <= c.e_min)
      return fail(ctx, DLRA_ERR_ARG, "beam energy node %.6g outside (e_min, e_max]", e);
  std::vector<double> rays;
  double wsum = 0.0;
  std::vector<std::pair<std::array<double, 3>, double>> pts;
  if (ctx->two_d) {
    for (size_t i = 0; i < offs.size(); ++i) {
      std::array<double, 3> p = {b->pos[0] + offs[i] * u1[0], b->pos[1] + offs[i] * u1[1], b->pos[2] + offs[i] * u1[2]};
      pts.push_back({p, gw[i]});
      wsum += gw[i];
    }
  } else {
    for (size_t i = 0; i < offs.size(); ++i)
      for (size_t j = 0; j < offs.size(); ++j) {
        std::array<double, 3> p;
        for (int a = 0; a < 3; ++a) p[a] = b->pos[a] + offs[i] * u1[a] + offs[j] * u2[a];
        pts.push_back({p, gw[i] * gw[j]});
        wsum += gw[i] * gw[j];
      }
  }
  for (auto& pt : pts)
    for (size_t e = 0; e < ee.size(); ++e) {
      rays.insert(rays.end(), {pt.first[0], pt.first[1], pt.first[2], d[0], d[1], d[2], ee[e],
                               pt.second / wsum * ew[e]});   // unit beam weight
    }
  const int nray = (int)(rays.size() / 8);
  if ((int)ctx->lanes.size() < ctx->max_lanes && ctx->lanes.size() <= beams_of<T>(ctx).size()) {
    dlra_status ls = alloc_lane<T>(ctx);
    if (ls != DLRA_OK) return ls;
  }
  Beam<T> B;
  B.weight = b->weight;
  B.params = *b;
  for (int a = 0; a < 3; ++a) B.dir[a] = d[a];
  ALLOC(B.X, sizeof(T) * n * RB);
  ALLOC(B.W, sizeof(T) * (size_t)m * RB);
  ALLOC(B.S, sizeof(double) * RB * RB);
  ALLOC(B.dims, sizeof(BeamDims));
  ALLOC(B.rank_log, sizeof(int) * 2 * K);
  ALLOC(B.psi, sizeof(double) * (size_t)K * n);
  ALLOC(B.e_u, sizeof(double) * n);
  ALLOC(B.e_c, sizeof(double) * n);
  ALLOC(B.Bsrc, sizeof(double) * (size_t)K * M * m);
  {
    std::vector<int> neg(2 * K, -1);
    CK(cudaMemcpyAsync(B.rank_log, neg.data(), sizeof(int) * 2 * K, cudaMemcpyHostToDevice, ctx->st));
  }
  double* rays_dev = nullptr;
  ALLOC(rays_dev, sizeof(double) * rays.size());
  CK(cudaMemcpyAsync(rays_dev, rays.data(), sizeof(double) * rays.size(), cudaMemcpyHostToDevice, ctx->st));
  RayGeo g = ray_geo(ctx);
  ctx->ray_dev.push_back(rays_dev);
  ctx->ray_count.push_back(nray);
  if (ctx->strag) {
    dlra_status ss = straggling_source(ctx, *b, B.psi, B.e_u);
    if (ss != DLRA_OK) return ss;
  } else {
    launch_raytrace(ctx->st, rays_dev, nray, g, ctx->f_cell, ctx->tau_cell, B.psi, B.e_u);
  }
  ++ctx->launches;
  int* flags = nullptr;
  ALLOC(flags, sizeof(int) * K);
  bin_flags_kernel<<<dim3(std::min<unsigned>(nblk(n, 256), 64), K), 256, 0, ctx->st>>>(B.psi, n, K, flags);
  ++ctx->launches;
  B.has_src.assign(K, 0);
  CK(cudaMemcpyAsync(B.has_src.data(), flags, sizeof(int) * K, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  B.first_src = -1;
  for (int k = 0; k < K && B.first_src < 0; ++k)
    if (B.has_src[k]) B.first_src = k;
  dlra_status us = upload_bsrc<T>(ctx, B);
  if (us != DLRA_OK) return us;
  CK(cudaGetLastError());
  beams_of<T>(ctx).push_back(B);
  *id = (int32_t)beams_of<T>(ctx).size() - 1;
  return DLRA_OK;
}

template <typename T>
dlra_status get_state_t(dlra_ctx* ctx, int id, double* X, double* S, double* W, int32_t* r) {
  Beam<T>& B = beams_of<T>(ctx)[id];
  const long long n = ctx->n;
  const int m = ctx->m, RB = ctx->RB;
  BeamDims dh;
  CK(cudaMemcpy(&dh, B.dims, sizeof(BeamDims), cudaMemcpyDeviceToHost));
  *r = dh.r;
  double* tmp = nullptr;
  CK(cudaMalloc(&tmp, sizeof(double) * std::max<long long>(n, m) * RB));
  if (X) {
    to_double_kernel<T><<<nblk(n * RB, 256), 256, 0, ctx->st>>>(B.X, tmp, n * RB);
    CK(cudaMemcpyAsync(X, tmp, sizeof(double) * n * RB, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  if (W) {
    to_double_kernel<T><<<nblk((long long)m * RB, 256), 256, 0, ctx->st>>>(B.W, tmp, (long long)m * RB);
    CK(cudaMemcpyAsync(W, tmp, sizeof(double) * m * RB, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  if (S) CK(cudaMemcpy(S, B.S, sizeof(double) * RB * RB, cudaMemcpyDeviceToHost));
  cudaFree(tmp);
  return DLRA_OK;
}

template <typename T>
dlra_status set_state_t(dlra_ctx* ctx, int id, const double* X, const double* S, const double* W, int r) {
  Beam<T>& B = beams_of<T>(ctx)[id];
  const long long n = ctx->n;
  const int m = ctx->m, RB = ctx->RB;
  double* tmp = nullptr;
  CK(cudaMalloc(&tmp, sizeof(double) * std::max<long long>(n, m) * RB));
  std::vector<double> hx((size_t)std::max<long long>(n, m) * RB, 0.0);
  for (long long c = 0; c < r; ++c)
    for (long long i = 0; i < n; ++i) hx[c * n + i] = X[c * n + i];
  CK(cudaMemcpy(tmp, hx.data(), sizeof(double) * n * RB, cudaMemcpyHostToDevice));
  convert_kernel<T><<<nblk(n * RB, 256), 256, 0, ctx->st>>>(tmp, B.X, n * RB);
  CK(cudaStreamSynchronize(ctx->st));
  std::fill(hx.begin(), hx.end(), 0.0);
  for (long long c = 0; c < r; ++c)
    for (long long i = 0; i < m; ++i) hx[c * m + i] = W[c * m + i];
  CK(cudaMemcpy(tmp, hx.data(), sizeof(double) * m * RB, cudaMemcpyHostToDevice));
  convert_kernel<T><<<nblk((long long)m * RB, 256), 256, 0, ctx->st>>>(tmp, B.W, (long long)m * RB);
  CK(cudaStreamSynchronize(ctx->st));
  std::vector<double> hs((size_t)RB * RB, 0.0);
  for (int c = 0; c < r; ++c)
    for (int a = 0; a < r; ++a) hs[(size_t)c * RB + a] = S[(size_t)c * RB + a];
  CK(cudaMemcpy(B.S, hs.data(), sizeof(double) * RB * RB, cudaMemcpyHostToDevice));
  BeamDims dh{r, 0, 0, 0};
  CK(cudaMemcpy(B.dims, &dh, sizeof(BeamDims), cudaMemcpyHostToDevice));
  B.active = r > 0;
  cudaFree(tmp);
  return DLRA_OK;
}

template <typename T>
dlra_status dose_t(dlra_ctx* ctx, double* out, int on_device, int per_mass) {
  const long long n = ctx->n;
  auto& bs = beams_of<T>(ctx);
  double* dst = on_device ? out : ctx->dose_tmp;
  if (bs.empty()) CK(cudaMemsetAsync(dst, 0, sizeof(double) * n, ctx->st));
  if (ctx->joint && !bs.empty()) {
    // the joint state's collided deposit carries the beam weights already (they scale its
    // sources); the uncollided deposits enter times their beam's weight
    scale_kernel<<<nblk(n, 256), 256, 0, ctx->st>>>(bs[0].e_c, 1.0, n, dst);
    for (size_t b = 0; b < bs.size(); ++b)
      dose_total_kernel<<<nblk(n, 256), 256, 0, ctx->st>>>(ctx->zeros, bs[b].e_u, n, 0, bs[b].weight, dst);
  } else {
    for (size_t b = 0; b < bs.size(); ++b)
      dose_total_kernel<<<nblk(n, 256), 256, 0, ctx->st>>>(bs[b].e_c, bs[b].e_u, n, b == 0 ? 1 : 0, bs[b].weight,
                                                           dst);
  }
  if (per_mass) div_kernel<<<nblk(n, 256), 256, 0, ctx->st>>>(dst, ctx->rho, n);
  CK(cudaGetLastError());
  if (!on_device) {
    CK(cudaMemcpyAsync(out, dst, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  return check_device_errors(ctx);
}

template <typename T>
dlra_status reset_t(dlra_ctx* ctx, int retrace, bool flags_changed = false) {
  const long long n = ctx->n;
  auto& bs = beams_of<T>(ctx);
  RayGeo g = ray_geo(ctx);
  for (size_t b = 0; b < bs.size(); ++b) {
    Beam<T>& B = bs[b];
    // the factors too: kernels read all rank_max columns and rely on those beyond the rank being zero
    CK(cudaMemsetAsync(B.X, 0, sizeof(T) * n * ctx->RB, ctx->st));
    CK(cudaMemsetAsync(B.W, 0, sizeof(T) * (size_t)ctx->m * ctx->RB, ctx->st));
    CK(cudaMemsetAsync(B.dims, 0, sizeof(BeamDims), ctx->st));
    CK(cudaMemsetAsync(B.e_c, 0, sizeof(double) * n, ctx->st));
    CK(cudaMemsetAsync(B.S, 0, sizeof(double) * ctx->RB * ctx->RB, ctx->st));
    CK(cudaMemsetAsync(B.rank_log, 0xff, sizeof(int) * 2 * ctx->K, ctx->st));
    if (retrace) {
      CK(cudaMemsetAsync(B.psi, 0, sizeof(double) * (size_t)ctx->K * n, ctx->st));
      CK(cudaMemsetAsync(B.e_u, 0, sizeof(double) * n, ctx->st));
      if (ctx->strag) {
        dlra_status ss = straggling_source(ctx, B.params, B.psi, B.e_u);
        if (ss != DLRA_OK) return ss;
      } else {
        launch_raytrace(ctx->st, ctx->ray_dev[b], ctx->ray_count[b], g, ctx->f_cell, ctx->tau_cell, B.psi, B.e_u);
      }
      ++ctx->launches;
      if (flags_changed || ctx->strag) {
        // the mixture or the tracer changed: the bins the beam reaches may have changed too
        CK(cudaMemsetAsync(ctx->flags_dev, 0, sizeof(int) * ctx->K, ctx->st));
        bin_flags_kernel<<<dim3(std::min<unsigned>(nblk(n, 256), 64), ctx->K), 256, 0, ctx->st>>>(B.psi, n, ctx->K,
                                                                                                  ctx->flags_dev);
        ++ctx->launches;
        CK(cudaMemcpyAsync(B.has_src.data(), ctx->flags_dev, sizeof(int) * ctx->K, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        B.first_src = -1;
        for (int k = 0; k < ctx->K && B.first_src < 0; ++k)
          if (B.has_src[k]) B.first_src = k;
      }
    }
    B.active = false;
  }
  CK(cudaGetLastError());
  ctx->step = 0;
  return DLRA_OK;
}

// Reverse sweep (discrete adjoint) of the ctx->step energy steps run so far, for the loss
// gradient dL/de already in the work space (ge, gvec). Segment by segment from the last
// checkpoint: replay the forward steps of the segment, storing every step's start state;
// then, step by step backwards, advance the adjoint state mu through the transposed step
// (dose source, collision, streaming) and pair it with the replayed forward quantities.
template <typename T>
dlra_status backward_t(dlra_ctx* ctx, double* dbeta_host, double* dw_out, int out_on_device) {
  Engine<T> E{ctx};
  AdjWork<T>& A = *reinterpret_cast<AdjWork<T>*>(ctx->adj);
  auto& bs = E.beams();
  const int nb = (int)bs.size();
  const long long n = ctx->n;
  const int RB = ctx->RB, m = ctx->m, M = ctx->M, N = ctx->N;
  const int Kp = ctx->step, I = ctx->ckpt_interval;
  E.L = &ctx->lanes[0];
  cudaStream_t st = E.L->s0;
  int64_t& nl = ctx->launches;
  cudaEventRecord(ctx->ev_step, ctx->st);
  cudaStreamWaitEvent(st, ctx->ev_step, 0);
  // dL/dbeta_b = <dL/de, e_c,b + e_u,b>: the deposit is linear in each beam weight
  cudaMemsetAsync(A.dbeta, 0, sizeof(double) * nb, st);
  for (int b = 0; b < nb; ++b) {
    launch_dot(st, A.ge, bs[b].e_c, bs[b].e_u, n, A.dbeta + b);
    ++nl;
  }
  cudaMemsetAsync(A.grad_rho, 0, sizeof(double) * n, st);
  cudaMemsetAsync(A.grad_f, 0, sizeof(double) * n, st);
  cudaMemsetAsync(A.grad_tau, 0, sizeof(double) * n, st);
  cudaMemsetAsync(A.grad_w, 0, sizeof(double) * M * n, st);
  for (int b = 0; b < nb; ++b) cudaMemsetAsync(A.gpsi[b], 0, sizeof(double) * (size_t)ctx->K * n, st);
  convert_kernel<T><<<nblk(n, 256), 256, 0, st>>>(A.ge, A.gvec, n);
  ++nl;
  cudaMemsetAsync(A.mu.X, 0, sizeof(T) * n * RB, st);
  cudaMemsetAsync(A.mu.W, 0, sizeof(T) * (size_t)m * RB, st);
  cudaMemsetAsync(A.mu.S, 0, sizeof(double) * RB * RB, st);
  cudaMemsetAsync(A.mu.dims, 0, sizeof(BeamDims), st);
  auto active_at = [&](int b, int k) { return bs[b].first_src >= 0 && k > bs[b].first_src; };
  const int nseg = (Kp + I - 1) / I;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int k0 = sg * I, k1 = std::min(Kp, k0 + I);
    // replay the segment from its checkpoint
    for (int b = 0; b < nb; ++b) {
      Beam<T>& B = bs[b];
      E.snap_load(B.ckpt[sg], A.rep, st);
      for (int k = k0; k < k1; ++k) {
        const size_t slot = (size_t)(k - k0) * nb + b;
        E.snap_save(A.rep, A.seg[slot], st);
        const bool last = k + 1 == k1;
        if (last && !A.store) break;
        if (active_at(b, k)) {
          E.streaming(A.rep, k, 0, A.store ? A.capseg + slot * A.capseg_stride : nullptr);
          E.scattering(A.rep, k);
          if (A.store) E.snap_save(A.rep, A.segb[slot], st);
        }
        if (last) break;
        if (B.has_src[k]) E.source_with(A.rep, k, nullptr, B.Bsrc + (long long)k * M * m, M, B.psi + (long long)k * n);
      }
    }
    for (int k = k1 - 1; k >= k0; --k) {
      // dose: e += h sqrt(4 pi) u_{k+1}(., 0) gives mu += h sqrt(4 pi) dL/de e_0^T
      E.adj_rank = true;
      E.source_with(A.mu, k, A.gvec, A.be0, 1, nullptr);
      E.adj_rank = false;
      // first-collision source of each beam: u_{k+1} += h beta_b sum_i diag(w_i psi_b) 1 B_i^T
      for (int b = 0; b < nb; ++b) {
        Beam<T>& B = bs[b];
        if (!B.has_src[k]) continue;
        launch_grad_source<T>(st, A.mu.X, A.mu.S, A.mu.W, n, m, RB, B.Bsrc + (long long)k * M * m, M,
                              B.psi + (long long)k * n, E.P(ctx->wT), B.weight * ctx->h, A.ysrc, A.grad_w,
                              A.gpsi[b] + (long long)k * n);
        nl += 2;
      }
      bool any = false;
      for (int b = 0; b < nb; ++b) any = any || active_at(b, k);
      if (!any) continue;
      // transposed collision (the implicit factor 1/(1 - F) is diagonal, hence self-adjoint)
      // and transposed streaming with the adjoints of the K-stage inputs captured
      E.adj_rank = true;
      E.scattering(A.mu, k);
      E.snap_save(A.mu, A.alpha, st);
      E.streaming(A.mu, k, 1, A.capa);
      E.adj_rank = false;
      const int ns = ctx->nsub[k];
      for (int b = 0; b < nb; ++b) {
        if (!active_at(b, k)) continue;
        Beam<T>& B = bs[b];
        const size_t slot = (size_t)(k - k0) * nb + b;
        // forward quantities of step k: the start state's W (K-step basis), the K-stage inputs
        // and the post-collision state; kept by the replay, or recomputed from the start state
        const T* Wf;
        const T* cf;
        const T* Xb;
        const T* Wb;
        const double* Sb;
        if (A.store) {
          Wf = A.seg[slot].W;
          cf = A.capseg + slot * A.capseg_stride;
          Xb = A.segb[slot].X;
          Wb = A.segb[slot].W;
          Sb = A.segb[slot].S;
        } else {
          E.snap_load(A.seg[slot], A.rep, st);
          Wf = A.seg[slot].W;
          E.streaming(A.rep, k, 0, A.capf);
          E.scattering(A.rep, k);
          cf = A.capf;
          Xb = A.rep.X;
          Wb = A.rep.W;
          Sb = A.rep.S;
        }
        // C = W_f^T W_alpha: the forward K-step basis against the adjoint K-step basis
        cudaMemsetAsync(A.Cm, 0, sizeof(double) * RB * RB, st);
        gram<T>(st, m, Wf, m, nullptr, RB, RB, FPlain<T>{A.alpha.W, m, nullptr, RB}, A.Cm, RB, nl);
        launch_grad_stream<T>(st, cf, A.capa, 4 * ns, n, RB, A.Cm, B.weight, A.grad_rho);
        launch_scatter_cl(st, A.alpha.S, A.alpha.W, Sb, Wb, sizeof(T) == 8 ? 1 : 0, m, N, RB, A.Cl);
        launch_grad_scatter<T>(st, A.alpha.X, Xb, n, RB, A.Cl, N, ctx->coef + (long long)k * M * (N + 1), M,
                               E.P(ctx->wc), ctx->f_cell, B.weight, A.grad_w, A.grad_rho);
        nl += 3;
      }
    }
  }
  // uncollided part: the ray tracer's reverse walk with dL/dpsi_b and dL/de_u,b = beta_b dL/de
  RayGeo g = ray_geo(ctx);
  for (int b = 0; b < nb; ++b) {
    scale_kernel<<<nblk(n, 256), 256, 0, st>>>(A.ge, bs[b].weight, n, A.gtmp);
    launch_raytrace_adjoint(st, ctx->ray_dev[b], ctx->ray_count[b], g, ctx->f_cell, ctx->tau_cell, A.gpsi[b], A.gtmp,
                            A.ray_scratch, A.grad_f, A.grad_tau);
    nl += 2;
  }
  double* dst = (dw_out && out_on_device) ? dw_out : A.dw;
  launch_grad_assemble(st, A.grad_w, A.grad_rho, A.grad_f, A.grad_tau, A.mcoef, M, n, dst);
  ++nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, DLRA_ERR_CUDA, "reverse sweep launch failed: %s", cudaGetErrorString(e));
  cudaEventRecord(E.L->ev[2], st);
  cudaStreamWaitEvent(ctx->st, E.L->ev[2], 0);
  if (dw_out && !out_on_device)
    CK(cudaMemcpyAsync(dw_out, A.dw, sizeof(double) * M * n, cudaMemcpyDeviceToHost, ctx->st));
  if (dbeta_host) CK(cudaMemcpyAsync(dbeta_host, A.dbeta, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return DLRA_OK;
}

// Times the launch variants of the heavy n-side kernels on lane 0's work space filled with
// synthetic values (rank = capacity) and keeps the fastest (streaming stages with a cold L2). report (optional, 16 doubles): ms of
// the FMA / tensor-core streaming stage, of the Gram reduction at 608 / 1216 / 2432 / 4864
// target blocks, of the stencil Gram at 0.5 / 1 / 2 waves, then the chosen stage variant,
// Gram block target and stencil-Gram waves x 2, ms of the brick stage, ms of the tensor-core
// stencil Gram, the chosen stencil-Gram kernel and ms of the cell-pair stage.
template <typename T>
dlra_status autotune_t(dlra_ctx* ctx, double* report) {
  Engine<T> E{ctx};
  E.L = &ctx->lanes[0];
  Lane& L = *E.L;
  cudaStream_t st = L.s0;
  const long long n = ctx->n;
  const int RB = ctx->RB, n2 = ctx->n2, nk = ctx->nk;
  int64_t nl = 0;
  CK(cudaStreamSynchronize(ctx->st));
  if (!ctx->tune_dims) {
    ALLOC(ctx->tune_dims, sizeof(BeamDims));
  }
  BeamDims dh{RB, RB, RB, 0};
  CK(cudaMemcpy(ctx->tune_dims, &dh, sizeof dh, cudaMemcpyHostToDevice));
  const int* rdim = &ctx->tune_dims->r;
  for (int i = 0; i < 3; ++i)
    fill_pseudo_random_kernel<T><<<nblk(n * RB, 256), 256, 0, st>>>(E.P(L.Kb[i]), n * RB, 17u + i, T(1));
  fill_pseudo_random_kernel<T><<<nblk(n * n2, 256), 256, 0, st>>>(E.P(L.Xh), n * n2, 29u, T(1));
  fill_pseudo_random_kernel<T><<<nblk((long long)nk * RB * RB, 256), 256, 0, st>>>(E.P(L.Pst), (long long)nk * RB * RB,
                                                                                  31u, T(0.1));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_ms = [&](auto&& launch) {
    for (int w = 0; w < 2; ++w) launch();
    cudaEventRecord(e0, st);
    for (int w = 0; w < 5; ++w) launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return (double)ms / 5.0;
  };
  // the streaming stage reads most of its inputs from DRAM inside a solve (the other chains of
  // the step evict them from L2): its variants are timed one launch at a time after a write of
  // 256 MB (a warm loop of launches gets their order wrong)
  const size_t flush_bytes = (size_t)256 << 20;
  void* flush = nullptr;
  CK(cudaMalloc(&flush, flush_bytes));
  auto time_cold_ms = [&](auto&& launch) {
    launch();
    double tot = 0.0;
    for (int w = 0; w < 5; ++w) {
      cudaMemsetAsync(flush, w, flush_bytes, st);
      cudaEventRecord(e0, st);
      launch();
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    return tot / 5.0;
  };
  Tuning t = ctx->tun;
  TuneScope scope(&t);
  double rep[31] = {0};
  // streaming stage: per-cell FMA, tensor cores (FP32 path), brick-staged FMA, cell pairs (FP32
  // path, nx even), TMA-staged tensor cores with 128- and 256-cell bricks (FP32 path, 3-D,
  // nx % 4 == 0, rank capacity >= 32)
  double stage_ms[14];
  for (int v = 0; v < 14; ++v) {
    if ((v == 1 || v == 3 || v >= 4) && sizeof(T) != 4) {
      stage_ms[v] = -1.0;
      continue;
    }
    if (v == 3 && ctx->geo.nx % 2 != 0) {
      stage_ms[v] = -1.0;
      continue;
    }
    if (v >= 4 && (ctx->geo.nact != 3 || ctx->geo.nx % 4 != 0 || RB < 32 || n % 4 != 0)) {
      stage_ms[v] = -1.0;
      continue;
    }
    const long long refused = g_tmac_refused.load();
    stage_ms[v] = time_cold_ms([&] {
      kstage<T>(RB, st, E.P(L.Kb[1]), E.P(L.Kb[0]), E.P(L.Kb[0]), E.P(L.Kb[2]), n, E.P(ctx->inv_rho), ctx->geo,
                E.P(L.Pst), rdim, T(1e-3), 0, nl, ctx->dev_err, v, L.Bimg);
    });
    if (v == 8 && g_tmac_refused.load() != refused) stage_ms[v] = -1.0;   // ran as variant 7
  }
  rep[0] = stage_ms[0];
  rep[1] = stage_ms[1];
  // the truncation apply X = X^ P (n x 2RB by 2RB x RB): FMA against tensor cores (FP32 path)
  double apply_ms[2] = {-1.0, -1.0};
  for (int v = 0; v < 2; ++v) {
    if (v == 1 && (sizeof(T) != 4 || n < 65536 || RB < 16)) continue;
    t.apply_variant = v;
    apply_ms[v] = time_cold_ms([&] {
      apply<T>(st, n, E.P(L.Xh), n, n2, nullptr, L.Pt, n2, RB, E.P(L.Kb[2]), n, nullptr, T(1), T(0), nl, nullptr,
               nullptr, &L.atc);
    });
  }
  t.apply_variant = 0;
  // Gram reduction X^_{:, RB:}^T X^ (the second augmentation pass's shape)
  const int gb[4] = {608, 1216, 2432, 4864};
  for (int v = 0; v < 4; ++v) {
    t.gram_blocks = gb[v];
    rep[2 + v] = time_ms([&] {
      gram<T>(st, n, E.P(L.Xh), n, nullptr, n2, RB, FPlain<T>{E.P(L.Xh) + (long long)RB * n, n, nullptr, RB}, L.Cg,
              n2, nl);
    });
  }
  // the same Gram on the tensor cores (FP32 path)
  double gram_tc_ms = -1.0;
  if (sizeof(T) == 4 && n >= 65536) {
    t.gram_blocks = gb[0];
    t.gram_variant = 1;
    gram_tc_ms = time_ms([&] {
      gram<T>(st, n, E.P(L.Xh), n, nullptr, n2, RB, FPlain<T>{E.P(L.Xh) + (long long)RB * n, n, nullptr, RB}, L.Cg,
              n2, nl);
    });
    t.gram_variant = 0;
  }
  // stencil Gram on the augmented basis
  const int gw[3] = {1, 2, 4};
  for (int v = 0; v < 3; ++v) {
    t.gs_waves_x2 = gw[v];
    rep[6 + v] = time_ms([&] {
      gram_stencil<T>(st, n, E.P(L.Xh), n, n2, nullptr, E.P(L.Xh), n, n2, nullptr, E.P(ctx->inv_rho), ctx->geo, L.Gc,
                      n2, n2, nl);
    });
  }
  // the same stencil Gram on the tensor cores (FP32 path)
  double gs_tc_ms = -1.0, gs_win_ms = -1.0;
  const bool gram_win_applies = ctx->geo.nact == 3 && ctx->geo.nx % 4 == 0 && n % 4 == 0 && n2 <= 128;
  if (sizeof(T) == 4 && gram_stencil_tc_supported(n2, n)) {
    t.gs_variant = 1;
    gs_tc_ms = time_ms([&] {
      gram_stencil<T>(st, n, E.P(L.Xh), n, n2, nullptr, E.P(L.Xh), n, n2, nullptr, E.P(ctx->inv_rho), ctx->geo, L.Gc,
                      n2, n2, nl, ctx->dev_err);
    });
    t.gs_variant = 2;
    gs_win_ms = time_ms([&] {
      gram_stencil<T>(st, n, E.P(L.Xh), n, n2, nullptr, E.P(L.Xh), n, n2, nullptr, E.P(ctx->inv_rho), ctx->geo, L.Gc,
                      n2, n2, nl, ctx->dev_err);
    });
    if (!gram_win_applies) gs_win_ms = -1.0;
    t.gs_variant = 0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  cudaFree(flush);
  Tuning best = ctx->tun;
  int sv = 0;
  for (int v = 1; v < 14; ++v)
    if (stage_ms[v] > 0.0 && stage_ms[v] < stage_ms[sv]) sv = v;
  best.kstage_variant = sv;
  int bi = 0;
  for (int v = 1; v < 4; ++v)
    if (rep[2 + v] < rep[2 + bi]) bi = v;
  best.gram_blocks = gb[bi];
  best.gram_variant = (gram_tc_ms > 0.0 && gram_tc_ms < rep[2 + bi]) ? 1 : 0;
  rep[26] = gram_tc_ms;
  int wi = 0;
  for (int v = 1; v < 3; ++v)
    if (rep[6 + v] < rep[6 + wi]) wi = v;
  best.gs_waves_x2 = gw[wi];
  best.gs_variant = (gs_tc_ms > 0.0 && gs_tc_ms < rep[6 + wi]) ? 1 : 0;
  if (gs_win_ms > 0.0 && gs_win_ms < (best.gs_variant == 1 ? gs_tc_ms : rep[6 + wi])) best.gs_variant = 2;
  rep[24] = gs_win_ms;
  rep[13] = gs_tc_ms;
  rep[14] = best.gs_variant;
  rep[9] = best.kstage_variant;
  rep[12] = stage_ms[2];
  rep[15] = stage_ms[3];
  rep[16] = stage_ms[4];
  rep[17] = stage_ms[5];
  rep[18] = stage_ms[6];
  rep[19] = stage_ms[7];
  rep[23] = stage_ms[8];
  rep[25] = stage_ms[9];
  rep[27] = stage_ms[10];
  rep[28] = stage_ms[11];
  rep[29] = stage_ms[12];
  rep[30] = stage_ms[13];
  best.apply_variant = (apply_ms[1] > 0.0 && apply_ms[1] < apply_ms[0]) ? 1 : 0;
  rep[20] = apply_ms[0];
  rep[21] = apply_ms[1];
  rep[22] = best.apply_variant;
  rep[10] = best.gram_blocks;
  rep[11] = best.gs_waves_x2;
  ctx->tun = best;
  if (report) std::memcpy(report, rep, sizeof rep);
  return DLRA_OK;
}

template <typename T>
void free_beams(dlra_ctx* ctx) {
  delete reinterpret_cast<std::vector<Beam<T>>*>(ctx->beams);
  ctx->beams = nullptr;
}

}  // namespace

// ===========================================================================
// stand-alone K-step on caller-provided work space
// ===========================================================================
namespace dlra {

static int kstep_rank_cap(int r) {
  for (int cap : kRankCaps)
    if (cap >= r) return cap;
  return -1;
}

size_t kstep_scratch_bytes(long long n, int r, int nact, int stage_kernel) {
  const int RB = kstep_rank_cap(r);
  if (RB < 0) return 0;
  const size_t al = 256;
  auto up = [&](size_t b) { return (b + al - 1) / al * al; };
  // the TMA-staged tensor-core stages read their B operand from images built per launch
  const size_t bimg = (stage_kernel >= 4 && nact == 3) ? up(kstage_tma_bimg_bytes(RB)) : 0;
  return 3 * up(sizeof(float) * (size_t)n * RB) + up(sizeof(float) * (size_t)2 * nact * RB * RB) + up(sizeof(int)) +
         bimg;
}

int run_kstep(const void* argp, void* scratch, size_t scratch_bytes, char* msg, int msg_len) {
  const dlra_kstep_args& a = *reinterpret_cast<const dlra_kstep_args*>(argp);
  const bool two_d = a.ny == 1 && a.dy == 0.0;
  const int nact = two_d ? 2 : 3;
  const long long n = (long long)a.nx * a.ny * a.nz;
  const int RB = kstep_rank_cap(a.r);
  const size_t need = kstep_scratch_bytes(n, a.r, nact, a.stage_kernel);
  if (scratch_bytes < need) {
    std::snprintf(msg, msg_len, "K-step needs %zu bytes of work space, %zu available", need, scratch_bytes);
    return DLRA_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)a.cuda_stream;
  const size_t al = 256;
  auto up = [&](size_t b) { return (b + al - 1) / al * al; };
  char* base = reinterpret_cast<char*>(scratch);
  float* y = reinterpret_cast<float*>(base);
  float* va = reinterpret_cast<float*>(base + up(sizeof(float) * (size_t)n * RB));
  float* vb = reinterpret_cast<float*>(base + 2 * up(sizeof(float) * (size_t)n * RB));
  float* Pst = reinterpret_cast<float*>(base + 3 * up(sizeof(float) * (size_t)n * RB));
  int* rdev = reinterpret_cast<int*>(base + 3 * up(sizeof(float) * (size_t)n * RB) +
                                     up(sizeof(float) * (size_t)2 * nact * RB * RB));
  void* bimg = (a.stage_kernel >= 4 && nact == 3) ? reinterpret_cast<char*>(rdev) + up(sizeof(int)) : nullptr;
  Geo g{};
  g.nx = a.nx;
  g.ny = a.ny;
  g.nz = a.nz;
  g.nxy = (long long)a.nx * a.ny;
  g.n = n;
  g.nact = nact;
  if (two_d) { g.dirs[0] = 0; g.dirs[1] = 2; g.dirs[2] = 2; }
  else { g.dirs[0] = 0; g.dirs[1] = 1; g.dirs[2] = 2; }
  g.inv2d[0] = 1.0 / (2.0 * a.dx);
  g.inv2d[1] = two_d ? 0.0 : 1.0 / (2.0 * a.dy);
  g.inv2d[2] = 1.0 / (2.0 * a.dz);
  const int nk = 2 * nact;
  int64_t nl = 0;
  set_int_kernel<<<1, 1, 0, st>>>(rdev, a.r);
  kstep_pack_p<<<nblk((long long)nk * RB * RB, 256), 256, 0, st>>>(a.P, a.r, nk, RB, Pst);
  kstep_load<<<nblk(n * RB, 256), 256, 0, st>>>(a.K0, n, a.r, RB, a.inv_rho, y, va);
  const double hs = a.de / a.n_sub;
  for (int j = 0; j < a.n_sub; ++j) {
    double beta[4];
    horner_betas_p(a.bk_p, a.bk_alpha, a.e0 - j * hs, hs, beta);
    const float* vins[4] = {va, vb, va, vb};
    float* vouts[4] = {vb, va, vb, va};
    for (int s2 = 0; s2 < 4; ++s2)
      kstage<float>(RB, st, vins[s2], y, y, vouts[s2], n, a.inv_rho, g, Pst, rdev, (float)beta[s2], s2 == 3 ? 1 : 0,
                    nl, nullptr, a.stage_kernel, bimg);
  }
  kstep_store<<<nblk(n * a.r, 256), 256, 0, st>>>(y, n, a.r, a.K1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::snprintf(msg, msg_len, "K-step launch failed: %s", cudaGetErrorString(e));
    return DLRA_ERR_CUDA;
  }
  return DLRA_OK;
}

int check_kstep_args(const dlra_kstep_args* a, char* msg, int msg_len) {
  if (!a) {
    std::snprintf(msg, msg_len, "null arguments");
    return DLRA_ERR_ARG;
  }
  const bool two_d = a->ny == 1 && a->dy == 0.0;
  if (a->nx < 1 || a->ny < 1 || a->nz < 1 || !(a->dx > 0) || !(a->dz > 0) || !(two_d || a->dy > 0)) {
    std::snprintf(msg, msg_len, "bad grid");
    return DLRA_ERR_ARG;
  }
  if (a->r < 1 || a->r > 64 || a->n_sub < 1 || !(a->de > 0) || !(a->e0 - a->de > 0) || a->stage_kernel < 0 ||
      a->stage_kernel > 13) {
    std::snprintf(msg, msg_len, "need 1 <= r <= 64, n_sub >= 1, e0 > de > 0, stage kernel 0 .. 13");
    return DLRA_ERR_ARG;
  }
  if (!a->K0 || !a->K1 || !a->inv_rho || !a->P || a->K0 == a->K1) {
    std::snprintf(msg, msg_len, "null or aliased device arrays");
    return DLRA_ERR_ARG;
  }
  return DLRA_OK;
}

}  // namespace dlra

static thread_local char g_kstep_msg[256] = "no error";

namespace dlra {
// message returned by dlra_last_error(NULL) after a failed context-free call
void set_context_free_error(const char* msg) { std::snprintf(g_kstep_msg, sizeof g_kstep_msg, "%s", msg); }
}  // namespace dlra

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

dlra_status dlra_init(const dlra_config* cfg, dlra_ctx** out) {
  if (!cfg || !out) return DLRA_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<dlra_ctx> c(new dlra_ctx());
  dlra_ctx* ctx = c.get();
  ctx->cfg = *cfg;
  const dlra_config& g = *cfg;
  if (g.nx < 1 || g.ny < 1 || g.nz < 1) return fail(ctx, DLRA_ERR_ARG, "grid sizes must be >= 1");
  ctx->two_d = (g.ny == 1 && g.dy == 0.0);
  if (!(g.dx > 0 && g.dz > 0 && (ctx->two_d || g.dy > 0))) return fail(ctx, DLRA_ERR_ARG, "voxel sizes must be > 0");
  if (g.sh_degree < 1 || g.sh_degree > 31) return fail(ctx, DLRA_ERR_ARG, "sh_degree must be in [1, 31]");
  if (g.collision != DLRA_FOKKER_PLANCK && g.collision != DLRA_BOLTZMANN) return fail(ctx, DLRA_ERR_ARG, "bad collision");
  if (g.transport_correction < 0 || g.transport_correction > 2)
    return fail(ctx, DLRA_ERR_ARG, "transport_correction must be 0, 1 or 2");
  if (g.rank_mode < 0 || g.rank_mode > 2) return fail(ctx, DLRA_ERR_ARG, "bad rank_mode");
  if (g.precision != DLRA_FP64 && g.precision != DLRA_FP32_MIXED && g.precision != DLRA_FP32_SPLIT)
    return fail(ctx, DLRA_ERR_ARG, "bad precision");
  if (g.rank_max < 1 || g.rank_max > 64) return fail(ctx, DLRA_ERR_ARG, "rank_max must be in [1, 64]");
  if (g.rank_mode == DLRA_RANK_FIXED && (g.rank < 1 || g.rank > g.rank_max))
    return fail(ctx, DLRA_ERR_ARG, "rank must be in [1, rank_max]");
  if (g.rank_mode == DLRA_RANK_ADAPTIVE && !(g.trunc_tol > 0)) return fail(ctx, DLRA_ERR_ARG, "trunc_tol must be > 0");
  if (g.n_energy_steps < 1 || !(g.e_max > g.e_min) || !(g.e_min > 0))
    return fail(ctx, DLRA_ERR_ARG, "need e_max > e_min > 0 and n_energy_steps >= 1");
  if (!(g.cfl_max > 0)) return fail(ctx, DLRA_ERR_ARG, "cfl_max must be > 0");
  if (!(g.bk_p > 1 && g.bk_p < 2 && g.bk_alpha > 0 && g.t100 >= 0))
    return fail(ctx, DLRA_ERR_ARG, "need 1 < bk_p < 2, bk_alpha > 0, t100 >= 0");
  ctx->fp64 = g.precision == DLRA_FP64;
  ctx->small64 = g.precision != DLRA_FP32_MIXED;
  if (g.max_concurrent_beams < 0) return fail(ctx, DLRA_ERR_ARG, "max_concurrent_beams must be >= 0");
  ctx->max_lanes = g.max_concurrent_beams > 0 ? g.max_concurrent_beams : 8;
  if (ctx->fp64 && g.rank_max > 32) return fail(ctx, DLRA_ERR_ARG, "FP64 precision supports rank_max <= 32");
  ctx->st = (cudaStream_t)g.cuda_stream;
  ctx->n = g.nx * g.ny * g.nz;
  ctx->N = g.sh_degree;
  ctx->m = (g.sh_degree + 1) * (g.sh_degree + 1);
  ctx->K = g.n_energy_steps;
  ctx->RB = 64;
  for (int cap : kRankCaps)
    if (cap >= g.rank_max) { ctx->RB = cap; break; }
  ctx->n2 = 2 * ctx->RB;
  const size_t tsz = ctx->fp64 ? 8 : 4;
  if ((size_t)ctx->m * ctx->RB * tsz > 160 * 1024)
    return fail(ctx, DLRA_ERR_ARG, "m * rank_max too large for the one-block QR (m=%d)", ctx->m);
  if (g.rank_mode == DLRA_RANK_SCHEDULE) {
    if (!g.rank_schedule) return fail(ctx, DLRA_ERR_ARG, "SCHEDULE mode needs rank_schedule");
    ctx->schedule_host.assign(g.rank_schedule, g.rank_schedule + 2 * ctx->K);
  }
  ctx->cfg.rank_schedule = nullptr;
  ctx->geo.nx = g.nx;
  ctx->geo.ny = g.ny;
  ctx->geo.nz = g.nz;
  ctx->geo.nxy = (long long)g.nx * g.ny;
  ctx->geo.n = ctx->n;
  if (ctx->two_d) {
    ctx->geo.nact = 2;
    ctx->geo.dirs[0] = 0;
    ctx->geo.dirs[1] = 2;
    ctx->geo.dirs[2] = 2;
  } else {
    ctx->geo.nact = 3;
    for (int i = 0; i < 3; ++i) ctx->geo.dirs[i] = i;
  }
  ctx->geo.inv2d[0] = 1.0 / (2.0 * g.dx);
  ctx->geo.inv2d[1] = ctx->two_d ? 0.0 : 1.0 / (2.0 * g.dy);
  ctx->geo.inv2d[2] = 1.0 / (2.0 * g.dz);
  ctx->nk = 2 * ctx->geo.nact;
  ctx->h = (g.e_max - g.e_min) / g.n_energy_steps;
  ctx->E.resize(ctx->K + 1);
  for (int k = 0; k <= ctx->K; ++k) ctx->E[k] = g.e_max - ctx->h * k;
  char msg[256];
  if (!build_angular(ctx->N, ctx->ang, msg, sizeof msg)) return fail(ctx, DLRA_ERR_ARG, "%s", msg);
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
    cudaGetLastError();
    return fail(ctx, DLRA_ERR_CUDA, "no CUDA device");
  }
  dlra_status s;
  if (ctx->fp64) {
    ctx->beams = new std::vector<Beam<double>>();
    s = alloc_shared<double>(ctx);
    if (s == DLRA_OK) s = upload_apm<double>(ctx);
  } else {
    ctx->beams = new std::vector<Beam<float>>();
    s = alloc_shared<float>(ctx);
    if (s == DLRA_OK) s = upload_apm<float>(ctx);
  }
  if (s != DLRA_OK) {
    *out = c.release();
    return s;
  }
  CK(cudaEventCreateWithFlags(&ctx->ev_step, cudaEventDisableTiming));
  if (!ctx->schedule_host.empty()) {
    ALLOC(ctx->schedule_dev, sizeof(int) * ctx->schedule_host.size());
    CK(cudaMemcpy(ctx->schedule_dev, ctx->schedule_host.data(), sizeof(int) * ctx->schedule_host.size(),
                  cudaMemcpyHostToDevice));
  }
  *out = c.release();
  return DLRA_OK;
}

dlra_status dlra_set_materials(dlra_ctx* ctx, int32_t n_mat, const dlra_material* mats, const double* w,
                               int32_t w_on_device) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (ctx->materials_set && n_mat != ctx->M)
    return fail(ctx, DLRA_ERR_STATE, "materials can be replaced only with the same number (%d)", ctx->M);
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  if (n_mat < 1 || !mats || !w) return fail(ctx, DLRA_ERR_ARG, "need n_mat >= 1, mats and w");
  if (n_mat > ctx->RB) return fail(ctx, DLRA_ERR_ARG, "n_mat must not exceed the rank capacity");
  for (int i = 0; i < n_mat; ++i) {
    const dlra_material& mt = mats[i];
    if (!(mt.density > 0 && mt.sp_ratio > 0 && mt.scatter_ratio >= 0 && mt.screening > 0))
      return fail(ctx, DLRA_ERR_ARG, "material %d: need density, sp_ratio, screening > 0", i);
  }
  ctx->M = n_mat;
  ctx->mats.assign(mats, mats + n_mat);
  ctx->s_unit.assign(n_mat, std::vector<double>(ctx->N + 2));
  ctx->xi_unit.assign(n_mat, 0.0);
  for (int i = 0; i < n_mat; ++i) screened_rutherford_moments(mats[i].screening, ctx->N + 1, ctx->s_unit[i].data(), &ctx->xi_unit[i]);
  std::vector<double> wh;
  const double* w_host = w;
  if (w_on_device) {
    wh.resize((size_t)n_mat * ctx->n);
    CK(cudaMemcpy(wh.data(), w, sizeof(double) * wh.size(), cudaMemcpyDeviceToHost));
    w_host = wh.data();
  }
  for (size_t i = 0; i < (size_t)n_mat * ctx->n; ++i)
    if (!(w_host[i] >= 0.0) || std::isinf(w_host[i])) return fail(ctx, DLRA_ERR_ARG, "mixture weights must be finite and >= 0");
  const bool again = ctx->materials_set;
  dlra_status s = ctx->fp64 ? set_materials_t<double>(ctx, w_host) : set_materials_t<float>(ctx, w_host);
  if (s != DLRA_OK) return s;
  ctx->materials_set = true;
  if (again) {
    // new mixture: new in-scattering vectors, ray trace and source bins; every beam restarts
    if (ctx->fp64) {
      for (auto& B : beams_of<double>(ctx))
        if ((s = upload_bsrc<double>(ctx, B)) != DLRA_OK) return s;
      s = reset_t<double>(ctx, 1, true);
    } else {
      for (auto& B : beams_of<float>(ctx))
        if ((s = upload_bsrc<float>(ctx, B)) != DLRA_OK) return s;
      s = reset_t<float>(ctx, 1, true);
    }
  }
  return s;
}

dlra_status dlra_set_beam_weight(dlra_ctx* ctx, int32_t beam_id, double weight) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  size_t nb = ctx->fp64 ? beams_of<double>(ctx).size() : beams_of<float>(ctx).size();
  if (beam_id < 0 || (size_t)beam_id >= nb) return fail(ctx, DLRA_ERR_ARG, "bad beam id");
  if (!(weight >= 0.0) || std::isinf(weight)) return fail(ctx, DLRA_ERR_ARG, "beam weight must be finite and >= 0");
  if (ctx->fp64) beams_of<double>(ctx)[beam_id].weight = weight;
  else beams_of<float>(ctx)[beam_id].weight = weight;
  return DLRA_OK;
}

dlra_status dlra_enable_adjoint(dlra_ctx* ctx, int32_t checkpoint_interval) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (checkpoint_interval < 0) return fail(ctx, DLRA_ERR_ARG, "checkpoint_interval must be >= 0");
  if (ctx->step != 0) return fail(ctx, DLRA_ERR_STATE, "the reverse sweep must be enabled before the first step");
  if (ctx->joint && checkpoint_interval > 0) return fail(ctx, DLRA_ERR_STATE, "the joint state has no reverse sweep");
  if (ctx->strag && checkpoint_interval > 0)
    return fail(ctx, DLRA_ERR_STATE, "the reverse sweep differentiates the CSDA tracer only");
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  if (checkpoint_interval != ctx->ckpt_interval) {
    if (ctx->fp64) for (auto& B : beams_of<double>(ctx)) B.ckpt.clear();
    else for (auto& B : beams_of<float>(ctx)) B.ckpt.clear();
  }
  ctx->ckpt_interval = checkpoint_interval;
  return DLRA_OK;
}

dlra_status dlra_backward(dlra_ctx* ctx, const double* dL_de, int32_t in_on_device, double* dL_dweight,
                          double* dL_dw, int32_t out_on_device) {
  if (!ctx) return DLRA_ERR_ARG;
  dlra_status s = check_device_errors(ctx);
  if (s != DLRA_OK) return s;
  if (!dL_de) return fail(ctx, DLRA_ERR_ARG, "null dL_de");
  if (!ctx->materials_set) return fail(ctx, DLRA_ERR_STATE, "no materials");
  if (ctx->ckpt_interval <= 0) return fail(ctx, DLRA_ERR_STATE, "dlra_enable_adjoint was not called before stepping");
  if (ctx->step == 0) return fail(ctx, DLRA_ERR_STATE, "no energy step to differentiate");
  const size_t nb = ctx->fp64 ? beams_of<double>(ctx).size() : beams_of<float>(ctx).size();
  const long long n = ctx->n;
  std::vector<double> gh(n);
  if (in_on_device) CK(cudaMemcpy(gh.data(), dL_de, sizeof(double) * n, cudaMemcpyDeviceToHost));
  else std::memcpy(gh.data(), dL_de, sizeof(double) * n);
  bool zero = true;
  for (double v : gh) {
    if (!std::isfinite(v)) return fail(ctx, DLRA_ERR_ARG, "dL_de must be finite");
    zero = zero && v == 0.0;
  }
  s = ctx->fp64 ? alloc_adj<double>(ctx) : alloc_adj<float>(ctx);
  if (s != DLRA_OK) return s;
  const size_t Mn = (size_t)ctx->M * n;
  if (zero) {
    // a zero loss gradient has zero gradients (and an adjoint state of rank 0)
    if (dL_dweight) std::fill(dL_dweight, dL_dweight + nb, 0.0);
    if (dL_dw) {
      if (out_on_device) CK(cudaMemset(dL_dw, 0, sizeof(double) * Mn));
      else std::fill(dL_dw, dL_dw + Mn, 0.0);
    }
    return DLRA_OK;
  }
  double* ge = ctx->fp64 ? reinterpret_cast<AdjWork<double>*>(ctx->adj)->ge
                         : reinterpret_cast<AdjWork<float>*>(ctx->adj)->ge;
  CK(cudaMemcpyAsync(ge, gh.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
  TuneScope scope(&ctx->tun);
  s = ctx->fp64 ? backward_t<double>(ctx, dL_dweight, dL_dw, out_on_device)
                : backward_t<float>(ctx, dL_dweight, dL_dw, out_on_device);
  if (s != DLRA_OK) return s;
  return check_device_errors(ctx);
}

dlra_status dlra_add_beam(dlra_ctx* ctx, const dlra_beam* beam, int32_t* beam_id) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (!beam || !beam_id) return fail(ctx, DLRA_ERR_ARG, "null beam or beam_id");
  if (!ctx->materials_set) return fail(ctx, DLRA_ERR_STATE, "dlra_set_materials must precede dlra_add_beam");
  if (ctx->step > 0) return fail(ctx, DLRA_ERR_STATE, "beams must be added before the first step");
  if (!(beam->weight >= 0) || !(beam->spot_sigma >= 0) || !(beam->energy_sigma >= 0))
    return fail(ctx, DLRA_ERR_ARG, "beam weight and sigmas must be >= 0");
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  return ctx->fp64 ? add_beam_t<double>(ctx, beam, beam_id) : add_beam_t<float>(ctx, beam, beam_id);
}

// Work space of the joint state for nb beams: the stacked source factors (n x M nb and
// m x M nb) and lane 0's source-projection buffer widened to M nb columns. The stacked source
// augments the basis by up to M nb columns, which must fit the augmentation's rank capacity.
dlra_status ensure_joint(dlra_ctx* ctx, int nb) {
  const int cols = ctx->M * nb;
  if (cols > ctx->RB)
    return fail(ctx, DLRA_ERR_ARG, "joint state: %d beams x %d materials = %d source columns exceed the rank capacity %d",
                nb, ctx->M, cols, ctx->RB);
  if (cols <= ctx->joint_cols) return DLRA_OK;
  CK(cudaStreamSynchronize(ctx->st));
  const size_t tsz = ctx->fp64 ? sizeof(double) : sizeof(float);
  dfree(ctx, ctx->joint_A);
  dfree(ctx, ctx->joint_B);
  dfree(ctx, ctx->lanes[0].XA);
  ALLOC(ctx->joint_A, tsz * (size_t)ctx->n * cols);
  ALLOC(ctx->joint_B, sizeof(double) * (size_t)ctx->m * cols);
  ALLOC(ctx->lanes[0].XA, sizeof(double) * (size_t)ctx->n2 * cols);
  ctx->joint_cols = cols;
  return DLRA_OK;
}

dlra_status dlra_set_straggling(dlra_ctx* ctx, int32_t enable, int32_t n_elem, double h_max, int32_t straggling) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (enable && (n_elem < 1 || n_elem > 4096 || !(h_max > 0.0)))
    return fail(ctx, DLRA_ERR_ARG, "straggling source: n_elem in [1, 4096] and h_max > 0 required");
  if (enable && ctx->ckpt_interval > 0)
    return fail(ctx, DLRA_ERR_STATE, "the reverse sweep differentiates the CSDA tracer only");
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  ctx->strag = enable != 0;
  ctx->strag_elems = n_elem;
  ctx->strag_hmax = h_max;
  ctx->strag_on = straggling != 0;
  return DLRA_OK;
}

dlra_status dlra_set_joint(dlra_ctx* ctx, int32_t enable) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (ctx->step != 0) return fail(ctx, DLRA_ERR_STATE, "the beam mode must be set before the first step");
  if (enable && ctx->ckpt_interval > 0) return fail(ctx, DLRA_ERR_STATE, "the joint state has no reverse sweep");
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  ctx->joint = enable != 0;
  return DLRA_OK;
}

dlra_status dlra_step(dlra_ctx* ctx, int32_t n_steps) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (n_steps < 0) return fail(ctx, DLRA_ERR_ARG, "n_steps must be >= 0");
  if (!ctx->materials_set) return fail(ctx, DLRA_ERR_STATE, "no materials");
  size_t nb = ctx->fp64 ? beams_of<double>(ctx).size() : beams_of<float>(ctx).size();
  if (nb == 0) return fail(ctx, DLRA_ERR_STATE, "no beam added");
  if (ctx->step + n_steps > ctx->K) return fail(ctx, DLRA_ERR_STATE, "only %d energy steps remain", ctx->K - ctx->step);
  if (ctx->ckpt_interval > 0) {
    dlra_status s = ctx->fp64 ? ensure_checkpoints<double>(ctx) : ensure_checkpoints<float>(ctx);
    if (s != DLRA_OK) return s;
  }
  if (ctx->joint) {
    dlra_status s = ensure_joint(ctx, (int)nb);
    if (s != DLRA_OK) return s;
  }
  TuneScope scope(&ctx->tun);
  if (ctx->graphs && !ctx->joint && !ctx->profiling && n_steps > 0)
    return ctx->fp64 ? step_graph<double>(ctx, n_steps) : step_graph<float>(ctx, n_steps);
  return ctx->fp64 ? Engine<double>{ctx}.step_all(n_steps) : Engine<float>{ctx}.step_all(n_steps);
}

dlra_status dlra_autotune(dlra_ctx* ctx, double* report) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (!ctx->materials_set || ctx->lanes.empty()) return fail(ctx, DLRA_ERR_STATE, "autotuning needs materials and a beam");
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  return ctx->fp64 ? autotune_t<double>(ctx, report) : autotune_t<float>(ctx, report);
}

dlra_status dlra_set_stage_kernel(dlra_ctx* ctx, int32_t variant) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (variant < 0 || variant > 13) return fail(ctx, DLRA_ERR_ARG, "stage kernel variant must be 0 .. 13");
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  ctx->tun.kstage_variant = variant;
  return DLRA_OK;
}

dlra_status dlra_set_gram_kernel(dlra_ctx* ctx, int32_t variant) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (variant < 0 || variant > 2) return fail(ctx, DLRA_ERR_ARG, "Gram kernel variant must be 0, 1 or 2");
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  ctx->tun.gram_variant = variant;
  return DLRA_OK;
}

dlra_status dlra_set_apply_kernel(dlra_ctx* ctx, int32_t variant) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (variant < 0 || variant > 2) return fail(ctx, DLRA_ERR_ARG, "apply kernel variant must be 0, 1 or 2");
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  ctx->tun.apply_variant = variant;
  return DLRA_OK;
}

dlra_status dlra_set_tensor_cores(dlra_ctx* ctx, int32_t enable) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  ctx->tun.kstage_variant = enable != 0 ? 1 : 0;
  return DLRA_OK;
}

dlra_status dlra_set_stencil_gram_kernel(dlra_ctx* ctx, int32_t variant) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (variant < 0 || variant > 2) return fail(ctx, DLRA_ERR_ARG, "stencil Gram variant must be 0, 1 or 2");
  CK(cudaStreamSynchronize(ctx->st));
  drop_graphs(ctx);
  ctx->tun.gs_variant = variant;
  return DLRA_OK;
}

dlra_status dlra_set_adjoint_store(dlra_ctx* ctx, int32_t keep) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  ctx->adj_store = keep != 0;
  return DLRA_OK;
}

dlra_status dlra_set_graphs(dlra_ctx* ctx, int32_t enable) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  ctx->graphs = enable != 0;
  if (!ctx->graphs) {
    CK(cudaStreamSynchronize(ctx->st));
    drop_graphs(ctx);
  }
  return DLRA_OK;
}

dlra_status dlra_dose(dlra_ctx* ctx, double* out, int32_t out_on_device, int32_t per_mass) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (!out) return fail(ctx, DLRA_ERR_ARG, "null output");
  if (!ctx->materials_set) return fail(ctx, DLRA_ERR_STATE, "no materials");
  return ctx->fp64 ? dose_t<double>(ctx, out, out_on_device, per_mass) : dose_t<float>(ctx, out, out_on_device, per_mass);
}

dlra_status dlra_query(dlra_ctx* ctx, int32_t* step, int32_t* ranks) {
  if (!ctx) return DLRA_ERR_ARG;
  dlra_status s = check_device_errors(ctx);
  if (s != DLRA_OK) return s;
  if (step) *step = ctx->step;
  if (ranks) {
    size_t nb = ctx->fp64 ? beams_of<double>(ctx).size() : beams_of<float>(ctx).size();
    for (size_t b = 0; b < nb; ++b) {
      BeamDims* dp = ctx->fp64 ? beams_of<double>(ctx)[b].dims : beams_of<float>(ctx)[b].dims;
      BeamDims dh;
      CK(cudaMemcpy(&dh, dp, sizeof dh, cudaMemcpyDeviceToHost));
      ranks[b] = dh.r;
    }
  }
  return DLRA_OK;
}

dlra_status dlra_rank_log(dlra_ctx* ctx, int32_t beam_id, int32_t* log) {
  if (!ctx) return DLRA_ERR_ARG;
  size_t nb = ctx->fp64 ? beams_of<double>(ctx).size() : beams_of<float>(ctx).size();
  if (beam_id < 0 || (size_t)beam_id >= nb || !log) return fail(ctx, DLRA_ERR_ARG, "bad beam id or null log");
  dlra_status s = check_device_errors(ctx);
  if (s != DLRA_OK) return s;
  int* p = ctx->fp64 ? beams_of<double>(ctx)[beam_id].rank_log : beams_of<float>(ctx)[beam_id].rank_log;
  CK(cudaMemcpy(log, p, sizeof(int) * 2 * ctx->K, cudaMemcpyDeviceToHost));
  return DLRA_OK;
}

dlra_status dlra_get_state(dlra_ctx* ctx, int32_t beam_id, double* X, double* S, double* W, int32_t* r) {
  if (!ctx) return DLRA_ERR_ARG;
  size_t nb = ctx->fp64 ? beams_of<double>(ctx).size() : beams_of<float>(ctx).size();
  if (beam_id < 0 || (size_t)beam_id >= nb || !r) return fail(ctx, DLRA_ERR_ARG, "bad beam id or null r");
  dlra_status s = check_device_errors(ctx);
  if (s != DLRA_OK) return s;
  return ctx->fp64 ? get_state_t<double>(ctx, beam_id, X, S, W, r) : get_state_t<float>(ctx, beam_id, X, S, W, r);
}

dlra_status dlra_set_state(dlra_ctx* ctx, int32_t beam_id, const double* X, const double* S, const double* W,
                           int32_t r) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  size_t nb = ctx->fp64 ? beams_of<double>(ctx).size() : beams_of<float>(ctx).size();
  if (beam_id < 0 || (size_t)beam_id >= nb) return fail(ctx, DLRA_ERR_ARG, "bad beam id");
  if (r < 0 || r > ctx->cfg.rank_max || (r > 0 && (!X || !S || !W))) return fail(ctx, DLRA_ERR_ARG, "bad state");
  return ctx->fp64 ? set_state_t<double>(ctx, beam_id, X, S, W, r) : set_state_t<float>(ctx, beam_id, X, S, W, r);
}

dlra_status dlra_get_source(dlra_ctx* ctx, int32_t beam_id, int32_t k, double* psi, double* e_u) {
  if (!ctx) return DLRA_ERR_ARG;
  size_t nb = ctx->fp64 ? beams_of<double>(ctx).size() : beams_of<float>(ctx).size();
  if (beam_id < 0 || (size_t)beam_id >= nb || k < 0 || k >= ctx->K) return fail(ctx, DLRA_ERR_ARG, "bad beam id or bin");
  dlra_status s = check_device_errors(ctx);
  if (s != DLRA_OK) return s;
  double* ps = ctx->fp64 ? beams_of<double>(ctx)[beam_id].psi : beams_of<float>(ctx)[beam_id].psi;
  double* eu = ctx->fp64 ? beams_of<double>(ctx)[beam_id].e_u : beams_of<float>(ctx)[beam_id].e_u;
  if (psi) CK(cudaMemcpy(psi, ps + (long long)k * ctx->n, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost));
  if (e_u) CK(cudaMemcpy(e_u, eu, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost));
  return DLRA_OK;
}

dlra_status dlra_get_tables(dlra_ctx* ctx, double* A, double* absA) {
  if (!ctx) return DLRA_ERR_ARG;
  const size_t mm = (size_t)ctx->m * ctx->m;
  for (int d = 0; d < 3; ++d) {
    if (A) std::memcpy(A + d * mm, ctx->ang.A[d].data(), sizeof(double) * mm);
    if (absA) std::memcpy(absA + d * mm, ctx->ang.absA[d].data(), sizeof(double) * mm);
  }
  return DLRA_OK;
}

dlra_status dlra_get_substeps(dlra_ctx* ctx, int32_t* nsub) {
  if (!ctx || !nsub) return DLRA_ERR_ARG;
  if (!ctx->materials_set) return fail(ctx, DLRA_ERR_STATE, "no materials");
  for (int k = 0; k < ctx->K; ++k) nsub[k] = ctx->nsub[k];
  return DLRA_OK;
}

dlra_status dlra_reset(dlra_ctx* ctx, int32_t retrace) {
  if (!ctx) return DLRA_ERR_ARG;
  if (ctx->poisoned) return ctx->poisoned;
  if (!ctx->materials_set) return fail(ctx, DLRA_ERR_STATE, "no materials");
  return ctx->fp64 ? reset_t<double>(ctx, retrace) : reset_t<float>(ctx, retrace);
}

dlra_status dlra_set_profiling(dlra_ctx* ctx, int32_t enable) {
  if (!ctx) return DLRA_ERR_ARG;
  prof_collect(ctx);
  ctx->profiling = enable != 0;
  ctx->prof_ms = 0.0;
  ctx->prof_count = 0;
  return DLRA_OK;
}

dlra_status dlra_kernel_stats(dlra_ctx* ctx, double* total_ms, int64_t* launches) {
  if (!ctx || !total_ms || !launches) return DLRA_ERR_ARG;
  prof_collect(ctx);
  *total_ms = ctx->prof_ms;
  *launches = ctx->prof_count;
  return DLRA_OK;
}

dlra_status dlra_kstep(const dlra_kstep_args* args) {
  int s = check_kstep_args(args, g_kstep_msg, sizeof g_kstep_msg);
  if (s != DLRA_OK) return (dlra_status)s;
  const bool two_d = args->ny == 1 && args->dy == 0.0;
  const long long n = (long long)args->nx * args->ny * args->nz;
  const size_t bytes = kstep_scratch_bytes(n, args->r, two_d ? 2 : 3, args->stage_kernel);
  void* scratch = nullptr;
  cudaError_t e = cudaMalloc(&scratch, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    std::snprintf(g_kstep_msg, sizeof g_kstep_msg, "cudaMalloc of %zu bytes failed", bytes);
    return DLRA_ERR_OOM;
  }
  s = run_kstep(args, scratch, bytes, g_kstep_msg, sizeof g_kstep_msg);
  cudaError_t e2 = cudaStreamSynchronize((cudaStream_t)args->cuda_stream);
  cudaFree(scratch);
  if (s == DLRA_OK && e2 != cudaSuccess) {
    std::snprintf(g_kstep_msg, sizeof g_kstep_msg, "K-step failed: %s", cudaGetErrorString(e2));
    s = DLRA_ERR_CUDA;
  }
  return (dlra_status)s;
}

dlra_status dlra_stencil_gram(const dlra_stencil_gram_args* a) {
  using namespace dlra;
  if (!a) {
    set_context_free_error("null arguments");
    return DLRA_ERR_ARG;
  }
  const bool two_d = a->ny == 1 && a->dy == 0.0;
  const long long n = (long long)a->nx * a->ny * a->nz;
  if (a->nx < 1 || a->ny < 1 || a->nz < 1 || !(a->dx > 0) || !(a->dz > 0) || !(two_d || a->dy > 0) ||
      n >= (1LL << 31)) {
    set_context_free_error("bad grid");
    return DLRA_ERR_ARG;
  }
  if (a->na < 1 || a->na > 128 || a->nb < 1 || a->nb > 128 || a->lda < n || a->ldb < n || a->variant < 0 ||
      a->variant > 2) {
    set_context_free_error("need 1 <= na, nb <= 128, lda, ldb >= n and variant 0, 1 or 2");
    return DLRA_ERR_ARG;
  }
  if (!a->A || !a->B || !a->inv_rho || !a->out) {
    set_context_free_error("null device arrays");
    return DLRA_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)a->cuda_stream;
  Geo g{};
  g.nx = a->nx;
  g.ny = a->ny;
  g.nz = a->nz;
  g.nxy = (long long)a->nx * a->ny;
  g.n = n;
  g.nact = two_d ? 2 : 3;
  g.dirs[0] = 0;
  g.dirs[1] = two_d ? 2 : 1;
  g.dirs[2] = 2;
  g.inv2d[0] = 1.0 / (2.0 * a->dx);
  g.inv2d[1] = two_d ? 0.0 : 1.0 / (2.0 * a->dy);
  g.inv2d[2] = 1.0 / (2.0 * a->dz);
  const int nk = 2 * g.nact;
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    set_context_free_error("cudaMalloc of the error flag failed");
    return DLRA_ERR_OOM;
  }
  Tuning t;
  t.gs_variant = a->variant;
  TuneScope scope(&t);
  int64_t nl = 0;
  cudaMemsetAsync(err, 0, sizeof(int), st);
  cudaMemsetAsync(a->out, 0, sizeof(double) * nk * a->nb * a->na, st);
  gram_stencil<float>(st, n, a->A, a->lda, a->na, nullptr, a->B, a->ldb, a->nb, nullptr, a->inv_rho, g, a->out,
                      a->nb, a->na, nl, err);
  int flag = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(err);
  if (e != cudaSuccess) {
    char buf[200];
    std::snprintf(buf, sizeof buf, "stencil Gram failed: %s", cudaGetErrorString(e));
    set_context_free_error(buf);
    return DLRA_ERR_CUDA;
  }
  if (flag & ERR_TIMEOUT) {
    set_context_free_error("stencil Gram: a tensor-core wait ran out");
    return DLRA_ERR_TIMEOUT;
  }
  return DLRA_OK;
}

int64_t dlra_launch_count(const dlra_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* dlra_last_error(const dlra_ctx* ctx) { return ctx ? ctx->err.c_str() : g_kstep_msg; }

void dlra_destroy(dlra_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->st);
  for (auto& l : ctx->lanes) {
    if (l.s0) cudaStreamSynchronize(l.s0);
    if (l.s1) cudaStreamSynchronize(l.s1);
  }
  drop_graphs(ctx);
  if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  for (auto& l : ctx->lanes) {
    for (cudaEvent_t e : l.ev)
      if (e) cudaEventDestroy(e);
    if (l.s0) cudaStreamDestroy(l.s0);
    if (l.s1) cudaStreamDestroy(l.s1);
  }
  if (ctx->ev_step) cudaEventDestroy(ctx->ev_step);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->beams) {
    if (ctx->fp64) free_beams<double>(ctx);
    else free_beams<float>(ctx);
  }
  if (ctx->adj) {
    if (ctx->fp64) delete reinterpret_cast<AdjWork<double>*>(ctx->adj);
    else delete reinterpret_cast<AdjWork<float>*>(ctx->adj);
  }
  delete ctx;
}

}  // extern "C"
