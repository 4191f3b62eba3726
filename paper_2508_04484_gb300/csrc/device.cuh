// Device building blocks of the low-rank step: the second-order one-sided stencil
// (Sec. 3.3.2), a tiled tall-skinny product C = A B with fused operand producers
// and epilogues, and a Gram reduction C = A^T F(B) over all cells.
//
// Layouts: tall matrices (cells x columns, or moments x columns) are column-major,
// one contiguous vector per column. Small matrices are FP64 column-major.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>
#include <stdint.h>

namespace dlra {

// ---------------------------------------------------------------------------
// grid geometry and the stencils D^{+/-}_d
// ---------------------------------------------------------------------------
struct Geo {
  int nx, ny, nz;
  long long nxy, n;
  int nact;          // number of streaming directions (2 for an x-z slab, 3 otherwise)
  int dirs[3];       // active directions
  double inv2d[3];   // 1 / (2 delta_d)
};

// Value of (D^{s}_d (rho^-1 v))(cell) for stencil index k = 2*da + s, d = dirs[da]:
// s = 0: D^- = -(3 v_i - 4 v_{i-1} + v_{i-2}) / (2 delta)  (backward)
// s = 1: D^+ =  (3 v_i - 4 v_{i+1} + v_{i+2}) / (2 delta)  (forward)
// Two ghost layers of zero outside the grid.
template <typename T>
__device__ __forceinline__ T stencil_value(const T* __restrict__ col, const T* __restrict__ inv_rho,
                                           long long i, int ix, int iy, int iz, int k, const Geo& g) {
  const int da = k >> 1, s = k & 1;
  const int d = g.dirs[da];
  int c, L;
  long long st;
  if (d == 0) { c = ix; L = g.nx; st = 1; }
  else if (d == 1) { c = iy; L = g.ny; st = g.nx; }
  else { c = iz; L = g.nz; st = g.nxy; }
  const T v0 = col[i] * inv_rho[i];
  T v1 = T(0), v2 = T(0);
  if (s == 0) {
    if (c >= 1) v1 = col[i - st] * inv_rho[i - st];
    if (c >= 2) v2 = col[i - 2 * st] * inv_rho[i - 2 * st];
    return (T(-3) * v0 + T(4) * v1 - v2) * T(g.inv2d[d]);
  }
  if (c + 1 < L) v1 = col[i + st] * inv_rho[i + st];
  if (c + 2 < L) v2 = col[i + 2 * st] * inv_rho[i + 2 * st];
  return (T(3) * v0 - T(4) * v1 + v2) * T(g.inv2d[d]);
}

__device__ __forceinline__ void cell_coords(long long i, const Geo& g, int& ix, int& iy, int& iz) {
  iz = (int)(i / g.nxy);
  long long rem = i - (long long)iz * g.nxy;
  iy = (int)(rem / g.nx);
  ix = (int)(rem - (long long)iy * g.nx);
}

// Per-tile stencil tables: for the cells row0 .. row0 + TT - 1 and the 13 stencil
// points (0: centre; 1 + 4d .. 4 + 4d: -1, -2, +1, +2 along direction d), the linear
// offset of the point and rho^-1 there (offset 0 and value 0 outside the grid, so
// the ghost layers are zero without branches).
template <typename T, int TT>
__device__ void stencil_tables(int* sOff, T* sR, long long row0, long long rows, const T* __restrict__ inv_rho,
                               const Geo& g, int tid, int nt) {
  for (int e = tid; e < 13 * TT; e += nt) {
    const int pt = e / TT, t = e % TT;
    const long long r = row0 + t;
    int off = 0;
    T val = T(0);
    if (r < rows) {
      const int ri = (int)r;
      const int nxy = (int)g.nxy;
      const int iz = ri / nxy;
      const int rem = ri - iz * nxy;
      const int iy = rem / g.nx;
      const int ix = rem - iy * g.nx;
      if (pt == 0) {
        val = inv_rho[r];
      } else {
        const int d = (pt - 1) >> 2, q = (pt - 1) & 3;
        const int delta = (q == 0) ? -1 : (q == 1) ? -2 : (q == 2) ? 1 : 2;
        const int c = d == 0 ? ix : (d == 1 ? iy : iz);
        const int L = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
        const int st = d == 0 ? 1 : (d == 1 ? g.nx : nxy);
        if (c + delta >= 0 && c + delta < L) {
          off = delta * st;
          val = inv_rho[r + off];
        }
      }
    }
    sOff[e] = off;
    sR[e] = val;
  }
}

// The nk stencil values of column col at tile cell t from the tables.
template <typename T, int TT>
__device__ __forceinline__ void stencil_values(const T* __restrict__ col, const int* sOff, const T* sR, int t,
                                               const Geo& g, T* out) {
  const T v0 = col[0] * sR[t];
#pragma unroll
  for (int da = 0; da < 3; ++da) {
    if (da >= g.nact) break;
    const int d = g.dirs[da];
    const int b = 1 + 4 * d;
    const T inv = T(g.inv2d[d]);
    const T vm1 = col[sOff[b * TT + t]] * sR[b * TT + t];
    const T vm2 = col[sOff[(b + 1) * TT + t]] * sR[(b + 1) * TT + t];
    const T vp1 = col[sOff[(b + 2) * TT + t]] * sR[(b + 2) * TT + t];
    const T vp2 = col[sOff[(b + 3) * TT + t]] * sR[(b + 3) * TT + t];
    out[2 * da] = (T(-3) * v0 + T(4) * vm1 - vm2) * inv;
    out[2 * da + 1] = (T(3) * v0 - T(4) * vp1 + vp2) * inv;
  }
}

// stencil_values with the direction list fixed at compile time (x, y, z for NACT = 3; x, z for
// an x-z slab), so that no array of the Geo argument is indexed at run time
template <typename T, int TT, int NACT>
__device__ __forceinline__ void stencil_values_c(const T* __restrict__ col, const int* sOff, const T* sR, int t,
                                                 const Geo& g, T* out) {
  const T v0 = col[0] * sR[t];
#pragma unroll
  for (int da = 0; da < NACT; ++da) {
    const int d = NACT == 3 ? da : (da == 0 ? 0 : 2);
    const int b = 1 + 4 * d;
    const T inv = T(g.inv2d[d]);
    const T vm1 = col[sOff[b * TT + t]] * sR[b * TT + t];
    const T vm2 = col[sOff[(b + 1) * TT + t]] * sR[(b + 1) * TT + t];
    const T vp1 = col[sOff[(b + 2) * TT + t]] * sR[(b + 2) * TT + t];
    const T vp2 = col[sOff[(b + 3) * TT + t]] * sR[(b + 3) * TT + t];
    out[2 * da] = (T(-3) * v0 + T(4) * vm1 - vm2) * inv;
    out[2 * da + 1] = (T(3) * v0 - T(4) * vp1 + vp2) * inv;
  }
}

__device__ __forceinline__ int dev_dim(const int* p, int cap) {
  if (p == nullptr) return cap;
  int v = *p;
  return v < cap ? (v < 0 ? 0 : v) : cap;
}

// ---------------------------------------------------------------------------
// tiled product: C (rows x N) = A (rows x Q) * B (Q x N), 64-row tiles,
// BN = 4 * (blockDim.x / 16) columns per block, K-chunks of BK.
// ---------------------------------------------------------------------------
constexpr int GM_BM = 64;

// A producer: plain column-major tall matrix.
template <typename T>
struct ALoadPlain {
  static constexpr int kExtra = 0;
  const T* A;
  long long lda;
  const int* qdim;  // actual number of columns (device), nullptr = Q
  int qcap;
  __device__ void init(void*, long long, long long) const {}
  __device__ void load(T* sA, int BK, int q0, long long row0, long long rows, const void*) const {
    const int Qa = dev_dim(qdim, qcap);
    for (int e = threadIdx.x; e < BK * GM_BM; e += blockDim.x) {
      int kk = e / GM_BM, t = e % GM_BM;
      long long r = row0 + t;
      int q = q0 + kk;
      sA[kk * GM_BM + t] = (r < rows && q < Qa) ? A[(long long)q * lda + r] : T(0);
    }
  }
};

// A producer: virtual matrix of stencil values, column q = c * nk + k holds
// D_k(rho^-1 Z[:, c]); BK must be a multiple of nk. Neighbour offsets and rho^-1 of
// the tile are tabulated once per block (init).
template <typename T>
struct ALoadStencil {
  static constexpr int kExtra = 13 * GM_BM * (int)(sizeof(int) + sizeof(T));
  const T* Z;
  long long ldz;
  const T* inv_rho;
  Geo g;
  const int* cdim;  // actual number of input columns of Z
  int ccap;
  __device__ void init(void* ex, long long row0, long long rows) const {
    int* sOff = reinterpret_cast<int*>(ex);
    T* sR = reinterpret_cast<T*>(sOff + 13 * GM_BM);
    stencil_tables<T, GM_BM>(sOff, sR, row0, rows, inv_rho, g, threadIdx.x, blockDim.x);
  }
  __device__ void load(T* sA, int BK, int q0, long long row0, long long rows, const void* ex) const {
    const int* sOff = reinterpret_cast<const int*>(ex);
    const T* sR = reinterpret_cast<const T*>(sOff + 13 * GM_BM);
    const int nk = 2 * g.nact;
    const int nc = BK / nk, c0 = q0 / nk;
    const int Ca = dev_dim(cdim, ccap);
    for (int e = threadIdx.x; e < nc * GM_BM; e += blockDim.x) {
      int cc = e / GM_BM, t = e % GM_BM;
      long long r = row0 + t;
      int c = c0 + cc;
      T v[6];
      if (r < rows && c < Ca) {
        stencil_values<T, GM_BM>(Z + (long long)c * ldz + r, sOff, sR, t, g, v);
      } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = T(0);
      }
      for (int k = 0; k < nk; ++k) sA[(cc * nk + k) * GM_BM + t] = v[k];
    }
  }
};

// A producer: nk dense row-major m x m matrices side by side, A[p][k*m + q] = M_k[p][q].
template <typename T>
struct ALoadRowBlocks {
  static constexpr int kExtra = 0;
  const T* M;  // [nk][m][m]
  int m, nk;
  __device__ void init(void*, long long, long long) const {}
  __device__ void load(T* sA, int BK, int q0, long long row0, long long rows, const void*) const {
    for (int e = threadIdx.x; e < BK * GM_BM; e += blockDim.x) {
      int t = e / BK, kk = e % BK;  // consecutive threads walk q (contiguous in a row)
      long long r = row0 + t;
      int q = q0 + kk;
      int k = q / m, qq = q - k * m;
      sA[kk * GM_BM + t] = (r < rows && k < nk) ? M[((long long)k * m + r) * m + qq] : T(0);
    }
  }
};

// A producer: plain row-major matrix, A(r, q) = M[r * ld + q].
template <typename T>
struct ALoadRowMajor {
  static constexpr int kExtra = 0;
  const T* M;
  long long ld;
  int Q;
  __device__ void init(void*, long long, long long) const {}
  __device__ void load(T* sA, int BK, int q0, long long row0, long long rows, const void*) const {
    for (int e = threadIdx.x; e < BK * GM_BM; e += blockDim.x) {
      int t = e / BK, kk = e % BK;
      long long r = row0 + t;
      int q = q0 + kk;
      sA[kk * GM_BM + t] = (r < rows && q < Q) ? M[r * ld + q] : T(0);
    }
  }
};

// B producer: column-major B of element type S (converted), B(q, c) = B[c * ldb + q];
// zero for q >= qdim or c >= ndim (device dims).
template <typename T, typename S>
struct BLoadCol {
  const S* B;
  long long ldb;
  const int* qdim;
  int qcap;
  const int* ndim;
  int ncap;
  __device__ void load(T* sB, int BK, int BN, int q0, int c0) const {
    const int Qa = dev_dim(qdim, qcap), Na = dev_dim(ndim, ncap);
    for (int e = threadIdx.x; e < BK * BN; e += blockDim.x) {
      int kk = e % BK, c = e / BK;
      int q = q0 + kk, cc = c0 + c;
      sB[kk * BN + c] = (q < Qa && cc < Na) ? T(B[(long long)cc * ldb + q]) : T(0);
    }
  }
};

// B producer: row-major B (Q x N), B(q, c) = B[q * ldb + c].
template <typename T, typename S>
struct BLoadRow {
  const S* B;
  long long ldb;
  int Q, N;
  __device__ void load(T* sB, int BK, int BN, int q0, int c0) const {
    for (int e = threadIdx.x; e < BK * BN; e += blockDim.x) {
      int kk = e / BN, c = e % BN;
      int q = q0 + kk, cc = c0 + c;
      sB[kk * BN + c] = (q < Q && cc < N) ? T(B[(long long)q * ldb + cc]) : T(0);
    }
  }
};

// B producer for the m-side sum over k: B((k, q), c) = Z[(k * ncap + c) * m + q].
template <typename T>
struct BLoadKBlocks {
  const T* Z;
  int m, ncap, nk;
  __device__ void load(T* sB, int BK, int BN, int q0, int c0) const {
    for (int e = threadIdx.x; e < BK * BN; e += blockDim.x) {
      int kk = e % BK, c = e / BK;
      int q = q0 + kk, cc = c0 + c;
      int k = q / m, qq = q - k * m;
      sB[kk * BN + c] = (k < nk && cc < ncap) ? Z[((long long)k * ncap + cc) * m + qq] : T(0);
    }
  }
};

// B producer for the L-step's sum over k: B((k, a), c) = G_k[c][a] = GT[(k * RB + c) * RB + a],
// zero for a, c >= rdim (the columns beyond the rank).
template <typename T>
struct BLoadGt {
  const T* GT;
  int RB, nk;
  const int* rdim;
  __device__ void load(T* sB, int BK, int BN, int q0, int c0) const {
    const int r = dev_dim(rdim, RB);
    for (int e = threadIdx.x; e < BK * BN; e += blockDim.x) {
      int kk = e % BK, c = e / BK;
      int q = q0 + kk, cc = c0 + c;
      int k = q / RB, a = q - k * RB;
      sB[kk * BN + c] = (k < nk && a < r && cc < r) ? GT[((long long)k * RB + cc) * RB + a] : T(0);
    }
  }
};

// Epilogues. Each receives the accumulator of C(r, c) = sum_q A(r, q) B(q, c).
template <typename T>
struct EpiStore {  // C = acc (+ beta * Cin)
  T* C;
  long long ldc;
  const T* Cin;
  long long ldin;
  T alpha, beta;
  __device__ void operator()(long long r, int c, T acc) const {
    T v = alpha * acc;
    if (Cin) v += beta * Cin[(long long)c * ldin + r];
    C[(long long)c * ldc + r] = v;
  }
};

template <typename T>
struct EpiKStage {  // C = Y + beta * acc (C may alias Y)
  T* C;
  const T* Y;
  long long ld;
  T beta;
  __device__ void operator()(long long r, int c, T acc) const {
    C[(long long)c * ld + r] = Y[(long long)c * ld + r] + beta * acc;
  }
};

template <typename T>
struct EpiStoreKBlocks {  // rows r = k*m + p stored at ((k*ncap + c)*m + p)
  T* C;
  int m, ncap;
  __device__ void operator()(long long r, int c, T acc) const {
    int k = (int)(r / m);
    int p = (int)(r - (long long)k * m);
    C[((long long)k * ncap + c) * m + p] = acc;
  }
};

// Main tiled kernel.
template <typename T, int BK, class AL, class BL, class EP>
__global__ void __launch_bounds__(256) gemm_kernel(long long rows, int N, int Q, AL al, BL bl, EP ep) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);
  const int tnc = blockDim.x / 16;
  const int BN = tnc * 4;
  T* sB = sA + BK * GM_BM;
  void* ex = reinterpret_cast<void*>(sB + BK * BN);
  const int tid = threadIdx.x;
  const int tm = tid % 16, tn = tid / 16;
  const long long row0 = (long long)blockIdx.x * GM_BM;
  const int c0 = blockIdx.y * BN;
  if (AL::kExtra > 0) {
    al.init(ex, row0, rows);
    __syncthreads();
  }
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int q0 = 0; q0 < Q; q0 += BK) {
    al.load(sA, BK, q0, row0, rows, ex);
    bl.load(sB, BK, BN, q0, c0);
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk * GM_BM + tm + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk * BN + tn * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long r = row0 + tm + 16 * i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = c0 + tn * 4 + j;
      if (c < N) ep(r, c, acc[i][j]);
    }
  }
}

// ---------------------------------------------------------------------------
// Fused streaming stage of the K-step (Sec. 3.3.2-3.3.3), one thread per cell:
//   out(i, :) = y(i, :) + beta * sum_c sum_k D_k(rho^-1 z(:, c))(i) P_k[c][:]
// with the r outputs in registers, the neighbour offsets and rho^-1 of the 13
// stencil points in registers, and the stacked P (row (c*nk + k), RM columns) in
// shared memory read as broadcasts.
// ---------------------------------------------------------------------------
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ static void load(const float* p, float* v) {
    float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <>
struct Vec4<double> {
  __device__ static void load(const double* p, double* v) {
    double2 a = *reinterpret_cast<const double2*>(p);
    double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

template <typename T, int RM, int NACT>
__global__ void __launch_bounds__(128) kstage_kernel(const T* __restrict__ vin, const T* __restrict__ y,
                                                     T* __restrict__ yout, T* __restrict__ vout, long long ld,
                                                     const T* __restrict__ inv_rho, Geo g, const T* __restrict__ Pst,
                                                     const int* __restrict__ rdim, T beta, int last) {
  // vin = rho^-1 z (scaled stage input). last = 0: vout = rho^-1 (y + beta acc);
  // last = 1: yout = y + beta acc and vout = rho^-1 yout (input of the next sub-step).
  // last = 2 (transposed operator, unscaled input; Pst holds -P of the opposite sign):
  // vout = beta rho^-1 acc and yout = y + vout (y may alias yout, never vin).
  constexpr int NK = 2 * NACT;
  constexpr int NP = 1 + 4 * NACT;
  extern __shared__ __align__(16) unsigned char raw[];
  T* sP = reinterpret_cast<T*>(raw);
  const int r = dev_dim(rdim, RM);
  for (int e = threadIdx.x; e < NK * RM * r; e += blockDim.x) sP[e] = Pst[e];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int ii = (int)i, nxy = (int)g.nxy;
  const int iz = ii / nxy, rem = ii - iz * nxy;
  const int iy = rem / g.nx, ix = rem - iy * g.nx;
  // neighbour validity bits (m1, m2, p1, p2 per direction) and strides
  unsigned valid = 0;
  int stv[NACT];
#pragma unroll
  for (int da = 0; da < NACT; ++da) {
    const int d = (NACT == 3) ? da : (da == 0 ? 0 : 2);
    const int c = d == 0 ? ix : (d == 1 ? iy : iz);
    const int L = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
    stv[da] = d == 0 ? 1 : (d == 1 ? g.nx : nxy);
    valid |= (unsigned)(c >= 1) << (4 * da);
    valid |= (unsigned)(c >= 2) << (4 * da + 1);
    valid |= (unsigned)(c + 1 < L) << (4 * da + 2);
    valid |= (unsigned)(c + 2 < L) << (4 * da + 3);
  }
  T inv2[NACT];
#pragma unroll
  for (int da = 0; da < NACT; ++da) inv2[da] = T(g.inv2d[(NACT == 3) ? da : (da == 0 ? 0 : 2)]);
  // FP32: the r x r mix in packed two-lane FMAs (fma.rn.f32x2, each lane rounded as a scalar FMA),
  // half the FMA instructions of the issue-bound loop
  constexpr bool F2 = std::is_same<T, float>::value;
  T acc[RM];
  float2 acc2[F2 ? RM / 2 : 1];
#pragma unroll
  for (int c = 0; c < RM; ++c) acc[c] = T(0);
#pragma unroll
  for (int c = 0; c < (F2 ? RM / 2 : 1); ++c) acc2[c] = make_float2(0.f, 0.f);
  for (int c = 0; c < r; ++c) {
    const T* col = vin + (long long)c * ld + i;
    T v[NP];
    v[0] = col[0];
#pragma unroll
    for (int da = 0; da < NACT; ++da) {
      const int st = stv[da];
      v[1 + 4 * da] = (valid >> (4 * da)) & 1u ? col[-st] : T(0);
      v[2 + 4 * da] = (valid >> (4 * da + 1)) & 1u ? col[-2 * st] : T(0);
      v[3 + 4 * da] = (valid >> (4 * da + 2)) & 1u ? col[st] : T(0);
      v[4 + 4 * da] = (valid >> (4 * da + 3)) & 1u ? col[2 * st] : T(0);
    }
    T sv[NK];
#pragma unroll
    for (int da = 0; da < NACT; ++da) {
      sv[2 * da] = (T(-3) * v[0] + T(4) * v[1 + 4 * da] - v[2 + 4 * da]) * inv2[da];
      sv[2 * da + 1] = (T(3) * v[0] - T(4) * v[3 + 4 * da] + v[4 + 4 * da]) * inv2[da];
    }
    const T* Pc = sP + (long long)c * NK * RM;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      if constexpr (F2) {
        const float2 s2 = make_float2(sv[k], sv[k]);
#pragma unroll
        for (int cp = 0; cp < RM; cp += 4) {
          const float4 p = *reinterpret_cast<const float4*>(Pc + k * RM + cp);
          acc2[cp / 2] = __ffma2_rn(s2, make_float2(p.x, p.y), acc2[cp / 2]);
          acc2[cp / 2 + 1] = __ffma2_rn(s2, make_float2(p.z, p.w), acc2[cp / 2 + 1]);
        }
      } else {
#pragma unroll
        for (int cp = 0; cp < RM; cp += 4) {
          T p4[4];
          Vec4<T>::load(Pc + k * RM + cp, p4);
          acc[cp] += sv[k] * p4[0];
          acc[cp + 1] += sv[k] * p4[1];
          acc[cp + 2] += sv[k] * p4[2];
          acc[cp + 3] += sv[k] * p4[3];
        }
      }
    }
  }
  if constexpr (F2) {
#pragma unroll
    for (int c = 0; c < RM / 2; ++c) {
      acc[2 * c] = acc2[c].x;
      acc[2 * c + 1] = acc2[c].y;
    }
  }
  const T ir0 = inv_rho[i];
  if (last == 2) {
#pragma unroll
    for (int c = 0; c < RM; ++c) {
      const T lam = beta * ir0 * acc[c];
      vout[(long long)c * ld + i] = lam;
      yout[(long long)c * ld + i] = y[(long long)c * ld + i] + lam;
    }
  } else if (last) {
#pragma unroll
    for (int c = 0; c < RM; ++c) {
      const T yn = y[(long long)c * ld + i] + beta * acc[c];
      yout[(long long)c * ld + i] = yn;
      vout[(long long)c * ld + i] = ir0 * yn;
    }
  } else {
#pragma unroll
    for (int c = 0; c < RM; ++c) vout[(long long)c * ld + i] = ir0 * (y[(long long)c * ld + i] + beta * acc[c]);
  }
}

// The streaming stage of kstage_kernel on the FP32 path with two x-adjacent cells per thread
// (cells 2t and 2t + 1 of a row; nx even): the two cells share four of their x-neighbour loads
// and every P value read from shared memory feeds both cells' packed two-lane FMAs. Same modes
// and outputs as kstage_kernel.
template <int RM, int NACT>
__global__ void __launch_bounds__(128) kstage_pair_kernel(const float* __restrict__ vin, const float* __restrict__ y,
                                                          float* __restrict__ yout, float* __restrict__ vout,
                                                          long long ld, const float* __restrict__ inv_rho, Geo g,
                                                          const float* __restrict__ Pst,
                                                          const int* __restrict__ rdim, float beta, int last) {
  constexpr int NK = 2 * NACT;
  extern __shared__ __align__(16) unsigned char raw[];
  float* sP = reinterpret_cast<float*>(raw);
  const int r = dev_dim(rdim, RM);
  for (int e = threadIdx.x; e < NK * RM * r; e += blockDim.x) sP[e] = Pst[e];
  __syncthreads();
  const long long i = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= g.n) return;
  const int ii = (int)i, nxy = (int)g.nxy;
  const int iz = ii / nxy, rem = ii - iz * nxy;
  const int iy = rem / g.nx, ix = rem - iy * g.nx;
  // x: cells ix - 2 .. ix + 3 (offsets -2 .. 3 from cell i); y and z: -1, -2, +1, +2
  int xo[6];
  unsigned xv = 0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int c = ix - 2 + d;
    const bool ok = c >= 0 && c < g.nx;
    xo[d] = ok ? d - 2 : 0;
    xv |= ok ? (1u << d) : 0u;
  }
  int yo[4], zo[4];
  unsigned yzv = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int delta = q == 0 ? -1 : (q == 1 ? -2 : (q == 2 ? 1 : 2));
    const bool oky = NACT == 3 && iy + delta >= 0 && iy + delta < g.ny;
    const bool okz = iz + delta >= 0 && iz + delta < g.nz;
    yo[q] = oky ? delta * g.nx : 0;
    zo[q] = okz ? delta * nxy : 0;
    yzv |= (oky ? 1u << q : 0u) | (okz ? 1u << (4 + q) : 0u);
  }
  float inv2[NACT];
#pragma unroll
  for (int da = 0; da < NACT; ++da) inv2[da] = (float)g.inv2d[(NACT == 3) ? da : (da == 0 ? 0 : 2)];
  float2 acc2[2][RM / 2];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int c = 0; c < RM / 2; ++c) acc2[h][c] = make_float2(0.f, 0.f);
  for (int c = 0; c < r; ++c) {
    const float* col = vin + (long long)c * ld + i;
    float xq[6], yq[2][4], zq[2][4];
#pragma unroll
    for (int d = 0; d < 6; ++d) xq[d] = (xv >> d) & 1u ? col[xo[d]] : 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        yq[h][q] = (yzv >> q) & 1u ? col[h + yo[q]] : 0.f;
        zq[h][q] = (yzv >> (4 + q)) & 1u ? col[h + zo[q]] : 0.f;
      }
    float sv[2][NK];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float v0 = xq[2 + h];
      sv[h][0] = (-3.f * v0 + 4.f * xq[1 + h] - xq[h]) * inv2[0];
      sv[h][1] = (3.f * v0 - 4.f * xq[3 + h] + xq[4 + h]) * inv2[0];
      if (NACT == 3) {
        sv[h][2] = (-3.f * v0 + 4.f * yq[h][0] - yq[h][1]) * inv2[1];
        sv[h][3] = (3.f * v0 - 4.f * yq[h][2] + yq[h][3]) * inv2[1];
      }
      sv[h][NK - 2] = (-3.f * v0 + 4.f * zq[h][0] - zq[h][1]) * inv2[NACT - 1];
      sv[h][NK - 1] = (3.f * v0 - 4.f * zq[h][2] + zq[h][3]) * inv2[NACT - 1];
    }
    const float* Pc = sP + (long long)c * NK * RM;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const float2 s0 = make_float2(sv[0][k], sv[0][k]), s1 = make_float2(sv[1][k], sv[1][k]);
#pragma unroll
      for (int cp = 0; cp < RM; cp += 4) {
        const float4 p = *reinterpret_cast<const float4*>(Pc + k * RM + cp);
        const float2 pa = make_float2(p.x, p.y), pb = make_float2(p.z, p.w);
        acc2[0][cp / 2] = __ffma2_rn(s0, pa, acc2[0][cp / 2]);
        acc2[0][cp / 2 + 1] = __ffma2_rn(s0, pb, acc2[0][cp / 2 + 1]);
        acc2[1][cp / 2] = __ffma2_rn(s1, pa, acc2[1][cp / 2]);
        acc2[1][cp / 2 + 1] = __ffma2_rn(s1, pb, acc2[1][cp / 2 + 1]);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const long long ih = i + h;
    const float ir0 = inv_rho[ih];
#pragma unroll
    for (int c = 0; c < RM; ++c) {
      const float a = (c & 1) ? acc2[h][c / 2].y : acc2[h][c / 2].x;
      const long long e = (long long)c * ld + ih;
      if (last == 2) {
        const float lam = beta * ir0 * a;
        vout[e] = lam;
        yout[e] = y[e] + lam;
      } else if (last) {
        const float yn = y[e] + beta * a;
        yout[e] = yn;
        vout[e] = ir0 * yn;
      } else {
        vout[e] = ir0 * (y[e] + beta * a);
      }
    }
  }
}

// Cell bricks of the staged streaming stage: 256 cells per block (8 x 8 x 4 in 3-D,
// 16 x 1 x 16 in a 2-D slab) and their two-cell halo.
template <int NACT>
struct Brick {
  static constexpr int TX = NACT == 3 ? 8 : 16, TY = NACT == 3 ? 8 : 1, TZ = NACT == 3 ? 4 : 16;
  static constexpr int HX = TX + 4, HY = NACT == 3 ? TY + 4 : 1, HZ = TZ + 4;
  static constexpr int HALO = HX * HY * HZ;
  static constexpr int HPT = (HALO + 255) / 256;   // halo values staged per thread
};

// The streaming stage of kstage_kernel with the stencil inputs staged per brick: for each
// input column the block loads the brick and its halo into shared memory once (coalesced
// x-rows; the next column's values are in flight during the current column's products), and
// every thread forms its cell's six (four) stencil values from there instead of loading 13
// neighbours from global memory. Same modes and outputs as kstage_kernel.
template <typename T, int RM, int NACT>
__global__ void __launch_bounds__(256, (RM * sizeof(T) <= 96) ? 4 : 2) kstage_brick_kernel(const T* __restrict__ vin, const T* __restrict__ y,
                                                           T* __restrict__ yout, T* __restrict__ vout, long long ld,
                                                           const T* __restrict__ inv_rho, Geo g,
                                                           const T* __restrict__ Pst, const int* __restrict__ rdim,
                                                           T beta, int last) {
  using Bk = Brick<NACT>;
  constexpr int NK = 2 * NACT;
  constexpr int TX = Bk::TX, TY = Bk::TY, HX = Bk::HX, HY = Bk::HY, HALO = Bk::HALO, HPT = Bk::HPT;
  constexpr int SYH = HX, SZH = HX * HY;
  extern __shared__ __align__(16) unsigned char raw[];
  T* sP = reinterpret_cast<T*>(raw);
  T* sH = sP + NK * RM * RM;   // two halo buffers
  const int tid = threadIdx.x;
  const int r = dev_dim(rdim, RM);
  for (int e = tid; e < NK * RM * r; e += blockDim.x) sP[e] = Pst[e];
  const int bx = (g.nx + TX - 1) / TX, by = (g.ny + TY - 1) / TY;
  const int blk = blockIdx.x;
  const int x0 = (blk % bx) * TX, y0 = ((blk / bx) % by) * TY, z0 = (blk / (bx * by)) * Bk::TZ;
  const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
  const int ix = x0 + lx, iy = y0 + ly, iz = z0 + lz;
  const bool ok = ix < g.nx && iy < g.ny && iz < g.nz;
  const long long i = ((long long)iz * g.ny + iy) * g.nx + ix;
  const int hc = (lz + 2) * SZH + (NACT == 3 ? (ly + 2) * SYH : 0) + (lx + 2);
  int hcell[HPT];
#pragma unroll
  for (int u = 0; u < HPT; ++u) {
    const int h = tid + 256 * u;
    hcell[u] = -2;
    if (h < HALO) {
      const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
      const int gx = x0 + hx - 2, gy = NACT == 3 ? y0 + hy - 2 : y0, gz = z0 + hz - 2;
      hcell[u] = (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz)
                     ? (int)(((long long)gz * g.ny + gy) * g.nx + gx)
                     : -1;
    }
  }
  T inv2[NACT];
#pragma unroll
  for (int da = 0; da < NACT; ++da) inv2[da] = T(g.inv2d[(NACT == 3) ? da : (da == 0 ? 0 : 2)]);
  T acc[RM];
#pragma unroll
  for (int c = 0; c < RM; ++c) acc[c] = T(0);
  T pre[HPT];
  auto fetch = [&](int c) {
    const T* col = vin + (long long)c * ld;
#pragma unroll
    for (int u = 0; u < HPT; ++u) pre[u] = hcell[u] >= 0 ? col[hcell[u]] : T(0);
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < HPT; ++u)
      if (hcell[u] != -2) sH[buf * HALO + tid + 256 * u] = pre[u];
  };
  if (r > 0) {
    fetch(0);
    stash(0);
  }
  __syncthreads();
  for (int c = 0; c < r; ++c) {
    if (c + 1 < r) fetch(c + 1);
    const T* hv = sH + (c & 1) * HALO + hc;
    const T v0 = hv[0];
    T sv[NK];
#pragma unroll
    for (int da = 0; da < NACT; ++da) {
      const int st = NACT == 3 ? (da == 0 ? 1 : (da == 1 ? SYH : SZH)) : (da == 0 ? 1 : SZH);
      sv[2 * da] = (T(-3) * v0 + T(4) * hv[-st] - hv[-2 * st]) * inv2[da];
      sv[2 * da + 1] = (T(3) * v0 - T(4) * hv[st] + hv[2 * st]) * inv2[da];
    }
    const T* Pc = sP + (long long)c * NK * RM;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
#pragma unroll
      for (int cp = 0; cp < RM; cp += 4) {
        T p4[4];
        Vec4<T>::load(Pc + k * RM + cp, p4);
        acc[cp] += sv[k] * p4[0];
        acc[cp + 1] += sv[k] * p4[1];
        acc[cp + 2] += sv[k] * p4[2];
        acc[cp + 3] += sv[k] * p4[3];
      }
    }
    if (c + 1 < r) stash((c + 1) & 1);
    __syncthreads();
  }
  if (!ok) return;
  const T ir0 = inv_rho[i];
  if (last == 2) {
#pragma unroll
    for (int c = 0; c < RM; ++c) {
      const T lam = beta * ir0 * acc[c];
      vout[(long long)c * ld + i] = lam;
      yout[(long long)c * ld + i] = y[(long long)c * ld + i] + lam;
    }
  } else if (last) {
#pragma unroll
    for (int c = 0; c < RM; ++c) {
      const T yn = y[(long long)c * ld + i] + beta * acc[c];
      yout[(long long)c * ld + i] = yn;
      vout[(long long)c * ld + i] = ir0 * yn;
    }
  } else {
#pragma unroll
    for (int c = 0; c < RM; ++c) vout[(long long)c * ld + i] = ir0 * (y[(long long)c * ld + i] + beta * acc[c]);
  }
}

template <typename T>
struct EpiStoreScaled {  // C = acc and V = rho^-1 acc
  T* C;
  T* V;
  long long ldc;
  const T* inv_rho;
  __device__ void operator()(long long r, int c, T acc) const {
    C[(long long)c * ldc + r] = acc;
    V[(long long)c * ldc + r] = inv_rho[r] * acc;
  }
};

// ---------------------------------------------------------------------------
// Tall-skinny apply, one thread per row with the NM outputs in registers:
//   C(i, c) = alpha sum_q A(i, q) M(q, c) + beta Cin(i, c)   (c < NM, q < Q)
// A column-major (lda), M FP64 column-major (ldm) staged in shared memory as T;
// mode 1 also writes V(i, c) = inv_rho(i) C(i, c).
// ---------------------------------------------------------------------------
template <typename T, int NM>
__global__ void __launch_bounds__(128) apply_kernel(long long rows, const T* __restrict__ A, long long lda, int Q,
                                                    const int* __restrict__ qdim, const double* __restrict__ M,
                                                    long long ldm, int N, T* __restrict__ C, long long ldc,
                                                    const T* __restrict__ Cin, T alpha, T beta, T* __restrict__ V,
                                                    const T* __restrict__ inv_rho) {
  extern __shared__ __align__(16) unsigned char raw[];
  T* sM = reinterpret_cast<T*>(raw);  // Q x NM, row q contiguous
  const int Qa = dev_dim(qdim, Q);
  for (int e = threadIdx.x; e < Qa * NM; e += blockDim.x) {
    const int q = e / NM, c = e - q * NM;
    sM[e] = c < N ? T(M[(long long)c * ldm + q]) : T(0);
  }
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  // FP32: packed two-lane FMAs (fma.rn.f32x2), as in the streaming stage
  constexpr bool F2 = std::is_same<T, float>::value;
  T acc[NM];
  float2 acc2[F2 ? NM / 2 : 1];
#pragma unroll
  for (int c = 0; c < NM; ++c) acc[c] = T(0);
#pragma unroll
  for (int c = 0; c < (F2 ? NM / 2 : 1); ++c) acc2[c] = make_float2(0.f, 0.f);
  const T* a = A + i;
  // eight columns of the row loaded before they are used (eight loads in flight per thread:
  // the kernel streams n x Q values and is bound by memory latency otherwise); the sum runs
  // over q in order
  constexpr int QB = 8;
  for (int q0 = 0; q0 < Qa; q0 += QB) {
    T cv[QB];
#pragma unroll
    for (int u = 0; u < QB; ++u) cv[u] = q0 + u < Qa ? a[(long long)(q0 + u) * lda] : T(0);
#pragma unroll
    for (int u = 0; u < QB; ++u) {
      if (q0 + u >= Qa) break;
      const T cur = cv[u];
      const T* mrow = sM + (q0 + u) * NM;
      if constexpr (F2) {
        const float2 c2 = make_float2(cur, cur);
#pragma unroll
        for (int c = 0; c < NM; c += 4) {
          const float4 m = *reinterpret_cast<const float4*>(mrow + c);
          acc2[c / 2] = __ffma2_rn(c2, make_float2(m.x, m.y), acc2[c / 2]);
          acc2[c / 2 + 1] = __ffma2_rn(c2, make_float2(m.z, m.w), acc2[c / 2 + 1]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < NM; c += 4) {
          T m4[4];
          Vec4<T>::load(mrow + c, m4);
          acc[c] += cur * m4[0];
          acc[c + 1] += cur * m4[1];
          acc[c + 2] += cur * m4[2];
          acc[c + 3] += cur * m4[3];
        }
      }
    }
  }
  if constexpr (F2) {
#pragma unroll
    for (int c = 0; c < NM / 2; ++c) {
      acc[2 * c] = acc2[c].x;
      acc[2 * c + 1] = acc2[c].y;
    }
  }
  const T ir = V ? inv_rho[i] : T(0);
#pragma unroll
  for (int c = 0; c < NM; ++c) {
    if (c < N) {
      T v = alpha * acc[c];
      if (Cin) v += beta * Cin[(long long)c * ldc + i];
      C[(long long)c * ldc + i] = v;
      if (V) V[(long long)c * ldc + i] = ir * v;
    }
  }
}

// ---------------------------------------------------------------------------
// Stencil Gram G_k[a][b] = sum_i A(i, a) D_k(rho^-1 B(:, b))(i), k = 2 da + s,
// written at out[(k * ldj + b) * ldo + a]. A block takes a 64-cell chunk at a time,
// stages A and the nk stencil values of every B column in shared memory (13 loads
// per column and cell) and accumulates 4 x 8 register tiles of the (a, j = k nb + b)
// output with compensated sums across chunks.
// ---------------------------------------------------------------------------
constexpr int GS_TC = 64;

template <typename T, int NACT>
__global__ void __launch_bounds__(512) gram_stencil_kernel(long long rows, const T* __restrict__ A, long long lda, int na,
                                                           const int* adim, const T* __restrict__ B, long long ldb,
                                                           int nb, const int* bdim, const T* __restrict__ inv_rho,
                                                           Geo g, int jslice, double* __restrict__ out, int ldj,
                                                           long long ldo) {
  constexpr int NK = 2 * NACT;
  extern __shared__ __align__(16) unsigned char raw[];
  const int nj = NK * nb;
  const int naP = (na + 3) / 4 * 4;
  // row pitches padded to an odd number of 16-byte groups (fewer bank conflicts)
  const int ldA = naP + (((naP / 4) & 1) ? 0 : 4);
  const int ldS = jslice + (((jslice / 4) & 1) ? 0 : 4);
  T* sA = reinterpret_cast<T*>(raw);            // [GS_TC][ldA]
  T* sS = sA + GS_TC * ldA;                     // [GS_TC][ldS]
  int* sOff = reinterpret_cast<int*>(sS + GS_TC * ldS);  // [13][GS_TC]
  T* sR = reinterpret_cast<T*>(sOff + 13 * GS_TC);
  const int tid = threadIdx.x;
  const int tpa = naP / 4;                     // threads along a
  const int ta = tid % tpa, tj = tid / tpa;    // tile (a: 4, j: 8)
  const int j0 = blockIdx.y * jslice;
  const int jn = min(jslice, nj - j0);
  const bool owner = tj * 8 < jn;
  const int Aact = dev_dim(adim, na), Bact = dev_dim(bdim, nb);
  T acc[4][8];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = T(0);
  for (long long r0 = (long long)blockIdx.x * GS_TC; r0 < rows; r0 += (long long)gridDim.x * GS_TC) {
    stencil_tables<T, GS_TC>(sOff, sR, r0, rows, inv_rho, g, threadIdx.x, blockDim.x);
    for (int e = tid; e < GS_TC * naP; e += blockDim.x) {
      int t = e % GS_TC, a = e / GS_TC;
      long long rr = r0 + t;
      sA[t * ldA + a] = (rr < rows && a < Aact) ? A[(long long)a * lda + rr] : T(0);
    }
    __syncthreads();
    // stencil values: item (b, t) for every b whose columns j = k*nb + b fall in the slice
    for (int e = tid; e < GS_TC * nb; e += blockDim.x) {
      int t = e % GS_TC, b = e / GS_TC;
      long long rr = r0 + t;
      T sv[NK];
      if (rr < rows && b < Bact) {
        stencil_values_c<T, GS_TC, NACT>(B + (long long)b * ldb + rr, sOff, sR, t, g, sv);
      } else {
#pragma unroll
        for (int k = 0; k < NK; ++k) sv[k] = T(0);
      }
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        int jl = k * nb + b - j0;
        if (jl >= 0 && jl < jslice) sS[t * ldS + jl] = sv[k];
      }
    }
    __syncthreads();
    if (owner) {
#pragma unroll 4
      for (int t = 0; t < GS_TC; ++t) {
        T a4[4], b8[8];
        Vec4<T>::load(sA + t * ldA + ta * 4, a4);
        Vec4<T>::load(sS + t * ldS + tj * 8, b8);
        Vec4<T>::load(sS + t * ldS + tj * 8 + 4, b8 + 4);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] += a4[u] * b8[v];
      }
    }
    __syncthreads();
  }
  if (!owner) return;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int a = ta * 4 + u;
    if (a >= na) continue;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int j = j0 + tj * 8 + v;
      if (j >= nj || tj * 8 + v >= jn) continue;
      const int k = j / nb, b = j - k * nb;
      double val = (double)acc[u][v];
      if (val != 0.0) atomicAdd(out + ((long long)k * ldj + b) * ldo + a, val);
    }
  }
}

// ---------------------------------------------------------------------------
// Gram reduction: out[j * lda_out + a] += sum_rows A(row, a) F(row, j),
// 64 x 64 output tiles, 32-row chunks, FP32/FP64 per-thread accumulation with
// compensated summation across chunks, FP64 atomics at the end.
// ---------------------------------------------------------------------------
template <typename T>
struct FPlain {  // F(row, j) = B[j * ldb + row], zero for j >= jdim
  static constexpr bool kTables = false;
  __device__ void prep(int*, T*, long long, long long, int, int) const {}
  const T* B;
  long long ldb;
  const int* jdim;
  int jcap;
  __device__ T operator()(long long r, int j, int jact, int, const int*, const T*) const {
    return j < jact ? B[(long long)j * ldb + r] : T(0);
  }
  __device__ int jact() const { return dev_dim(jdim, jcap); }
};

template <typename T>
struct FDiag {  // F(row, k * nb + b) = wv[k * n + row] * B[b * ldb + row]
  static constexpr bool kTables = false;
  __device__ void prep(int*, T*, long long, long long, int, int) const {}
  const T* B;
  long long ldb;
  const T* wv;
  long long n;
  int nb;
  const int* bdim;
  int nk;
  __device__ T operator()(long long r, int j, int bact, int, const int*, const T*) const {
    int k = j / nb, b = j - k * nb;
    return (k < nk && b < bact) ? wv[(long long)k * n + r] * B[(long long)b * ldb + r] : T(0);
  }
  __device__ int jact() const { return dev_dim(bdim, nb); }
};

constexpr int GR_TC = 32;

template <typename T>
struct FStencil {  // F(row, k * nb + b) = D_k(rho^-1 B[:, b])(row), tables per row chunk
  static constexpr bool kTables = true;
  const T* B;
  long long ldb;
  const T* inv_rho;
  Geo g;
  int nb;
  const int* bdim;
  __device__ void prep(int* sOff, T* sR, long long r0, long long rows, int tid, int nt) const {
    stencil_tables<T, GR_TC>(sOff, sR, r0, rows, inv_rho, g, tid, nt);
  }
  __device__ T operator()(long long r, int j, int bact, int t, const int* sOff, const T* sR) const {
    int k = j / nb, b = j - k * nb;
    if (k >= 2 * g.nact || b >= bact) return T(0);
    const int da = k >> 1, s = k & 1;
    const int d = g.dirs[da];
    const int base = 1 + 4 * d + 2 * s;
    const T* col = B + (long long)b * ldb + r;
    const T v0 = col[0] * sR[t];
    const T v1 = col[sOff[base * GR_TC + t]] * sR[base * GR_TC + t];
    const T v2 = col[sOff[(base + 1) * GR_TC + t]] * sR[(base + 1) * GR_TC + t];
    const T inv = T(g.inv2d[d]);
    return s == 0 ? (T(-3) * v0 + T(4) * v1 - v2) * inv : (T(3) * v0 - T(4) * v1 + v2) * inv;
  }
  __device__ int jact() const { return dev_dim(bdim, nb); }
};



// Narrow Gram: out[j * ldo + a] += sum_i A(i, a) B(i, j) for at most NJ columns of B. One
// thread per row (coalesced column reads), 32 columns of A per block row (blockIdx.y), the
// partial sums reduced over the block and added with FP64 atomics. Memory-bound: A is read once.
template <typename T, int NJ>
__global__ void __launch_bounds__(256) gram_narrow_kernel(long long rows, const T* __restrict__ A, long long lda,
                                                          const int* adim, int acap, const T* __restrict__ B,
                                                          long long ldb, const int* bdim, int bcap, int ncols_j,
                                                          double* __restrict__ out, long long ldo) {
  __shared__ double red[8][32 * NJ];
  const int a0 = blockIdx.y * 32;
  const int Aact = min(dev_dim(adim, acap), acap);
  const int Bact = min(dev_dim(bdim, bcap), ncols_j);
  const int na = min(32, Aact - a0);
  T acc[32][NJ];
#pragma unroll
  for (int a = 0; a < 32; ++a)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[a][j] = T(0);
  if (na > 0) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
         i += (long long)gridDim.x * blockDim.x) {
      T f[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) f[j] = j < Bact ? B[(long long)j * ldb + i] : T(0);
#pragma unroll
      for (int a = 0; a < 32; ++a) {
        if (a < na) {
          const T v = A[(long long)(a0 + a) * lda + i];
#pragma unroll
          for (int j = 0; j < NJ; ++j) acc[a][j] += v * f[j];
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 32; ++a)
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      double v = (double)acc[a][j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][a * NJ + j] = v;
    }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * NJ; e += blockDim.x) {
    const int a = e / NJ, j = e - a * NJ;
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][e];
    if (a < na && j < ncols_j && v != 0.0) atomicAdd(out + (long long)j * ldo + a0 + a, v);
  }
}

template <typename T, class F, int TILE, int RG>
__global__ void __launch_bounds__(256) gram_kernel(long long rows, const T* __restrict__ A, long long lda,
                                                   const int* adim, int acap, int ncols_j, F f,
                                                   double* __restrict__ out, long long ldo) {
  // RG row groups per block, each with its own 32-row chunks and staging buffers;
  // their partial tiles are summed in shared memory before the FP64 atomics.
  constexpr int TPD = TILE / 4;  // threads per tile dimension, 4 x 4 outputs each
  constexpr int GT = TPD * TPD;  // threads per row group
  __shared__ T sA[RG][GR_TC][TILE + 1];
  __shared__ T sF[RG][GR_TC][TILE + 1];
  __shared__ int sOff[F::kTables ? RG * 13 * GR_TC : 1];
  __shared__ T sR[F::kTables ? RG * 13 * GR_TC : 1];
  const int g = threadIdx.x / GT, tid = threadIdx.x % GT;
  const int ta = tid % TPD, tj = tid / TPD;
  const int a0 = blockIdx.y * TILE, j0 = blockIdx.z * TILE;
  const int Aact = dev_dim(adim, acap);
  const int Jact = f.jact();
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const long long stride = (long long)gridDim.x * RG * GR_TC;
  const long long nchunk_iter = (rows + stride - 1) / stride;
  if constexpr (!F::kTables) {
    // software pipeline: the next chunk's values are loaded into registers while the
    // current chunk is multiplied out of shared memory
    constexpr int PER = GR_TC * TILE / GT;   // staged values per thread and operand
    T ra[PER], rf[PER];
    auto load = [&](long long it) {
      const long long r0 = it * stride + ((long long)blockIdx.x * RG + g) * GR_TC;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + u * GT;
        const int t = e % GR_TC, c = e / GR_TC;
        const long long r = r0 + t;
        const int a = a0 + c, j = j0 + c;
        ra[u] = (r < rows && a < Aact && a < acap) ? A[(long long)a * lda + r] : T(0);
        rf[u] = (r < rows && j < ncols_j) ? f(r, j, Jact, t, nullptr, nullptr) : T(0);
      }
    };
    if (nchunk_iter > 0) load(0);
    for (long long it = 0; it < nchunk_iter; ++it) {
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + u * GT;
        const int t = e % GR_TC, c = e / GR_TC;
        sA[g][t][c] = ra[u];
        sF[g][t][c] = rf[u];
      }
      __syncthreads();
      if (it + 1 < nchunk_iter) load(it + 1);
#pragma unroll 8
      for (int t = 0; t < GR_TC; ++t) {
        T a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = sA[g][t][ta + TPD * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = sF[g][t][tj + TPD * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
      }
      __syncthreads();
    }
  } else
  for (long long it = 0; it < nchunk_iter; ++it) {
    const long long r0 = it * stride + ((long long)blockIdx.x * RG + g) * GR_TC;
    if (F::kTables) {
      f.prep(sOff + g * 13 * GR_TC, sR + g * 13 * GR_TC, r0, rows, tid, GT);
      __syncthreads();
    }
    for (int e = tid; e < GR_TC * TILE; e += GT) {
      int t = e % GR_TC, c = e / GR_TC;
      long long r = r0 + t;
      int a = a0 + c, j = j0 + c;
      sA[g][t][c] = (r < rows && a < Aact && a < acap) ? A[(long long)a * lda + r] : T(0);
      sF[g][t][c] = (r < rows && j < ncols_j) ? f(r, j, Jact, t, sOff + g * 13 * GR_TC, sR + g * 13 * GR_TC) : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int t = 0; t < GR_TC; ++t) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[g][t][ta + TPD * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sF[g][t][tj + TPD * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  // sum the row groups' tiles through shared memory (reusing sA)
  if (RG > 1) {
    T* red = &sA[0][0][0];
    for (int gg = 1; gg < RG; ++gg) {
      if (g == gg) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) red[(i * 4 + j) * GT + tid] = acc[i][j];
      }
      __syncthreads();
      if (g == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += red[(i * 4 + j) * GT + tid];
      }
      __syncthreads();
    }
    if (g != 0) return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int a = a0 + ta + TPD * i;
    if (a >= acap) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int jj = j0 + tj + TPD * j;
      if (jj >= ncols_j) continue;
      double v = (double)acc[i][j];
      if (v != 0.0) atomicAdd(out + (long long)jj * ldo + a, v);
    }
  }
}

}  // namespace dlra
