// Device building blocks of the low-rank step: the second-order one-sided stencil
// (Sec. 3.3.2), a tiled tall-skinny product C = A B with fused operand producers
// and epilogues, and a Gram reduction C = A^T F(B) over all cells.
//
// Layouts: tall matrices (cells x columns, or moments x columns) are column-major,
// one contiguous vector per column. Small matrices are FP64 column-major.
#pragma once
#include <cuda_runtime.h>
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
  const T* A;
  long long lda;
  const int* qdim;  // actual number of columns (device), nullptr = Q
  int qcap;
  __device__ void load(T* sA, int BK, int q0, long long row0, long long rows) const {
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
// D_k(rho^-1 Z[:, c]); BK must be a multiple of nk.
template <typename T>
struct ALoadStencil {
  const T* Z;
  long long ldz;
  const T* inv_rho;
  Geo g;
  const int* cdim;  // actual number of input columns of Z
  int ccap;
  __device__ void load(T* sA, int BK, int q0, long long row0, long long rows) const {
    const int nk = 2 * g.nact;
    const int nc = BK / nk, c0 = q0 / nk;
    const int Ca = dev_dim(cdim, ccap);
    for (int e = threadIdx.x; e < nc * GM_BM; e += blockDim.x) {
      int cc = e / GM_BM, t = e % GM_BM;
      long long r = row0 + t;
      int c = c0 + cc;
      if (r < rows && c < Ca) {
        int ix, iy, iz;
        cell_coords(r, g, ix, iy, iz);
        const T* col = Z + (long long)c * ldz;
        for (int k = 0; k < nk; ++k) sA[(cc * nk + k) * GM_BM + t] = stencil_value(col, inv_rho, r, ix, iy, iz, k, g);
      } else {
        for (int k = 0; k < nk; ++k) sA[(cc * nk + k) * GM_BM + t] = T(0);
      }
    }
  }
};

// A producer: nk dense row-major m x m matrices side by side, A[p][k*m + q] = M_k[p][q].
template <typename T>
struct ALoadRowBlocks {
  const T* M;  // [nk][m][m]
  int m, nk;
  __device__ void load(T* sA, int BK, int q0, long long row0, long long rows) const {
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
  const T* M;
  long long ld;
  int Q;
  __device__ void load(T* sA, int BK, int q0, long long row0, long long rows) const {
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
  const int tid = threadIdx.x;
  const int tm = tid % 16, tn = tid / 16;
  const long long row0 = (long long)blockIdx.x * GM_BM;
  const int c0 = blockIdx.y * BN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int q0 = 0; q0 < Q; q0 += BK) {
    al.load(sA, BK, q0, row0, rows);
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
// Gram reduction: out[j * lda_out + a] += sum_rows A(row, a) F(row, j),
// 64 x 64 output tiles, 32-row chunks, FP32/FP64 per-thread accumulation with
// compensated summation across chunks, FP64 atomics at the end.
// ---------------------------------------------------------------------------
template <typename T>
struct FPlain {  // F(row, j) = B[j * ldb + row], zero for j >= jdim
  const T* B;
  long long ldb;
  const int* jdim;
  int jcap;
  __device__ T operator()(long long r, int j, int jact) const { return j < jact ? B[(long long)j * ldb + r] : T(0); }
  __device__ int jact() const { return dev_dim(jdim, jcap); }
};

template <typename T>
struct FDiag {  // F(row, k * nb + b) = wv[k * n + row] * B[b * ldb + row]
  const T* B;
  long long ldb;
  const T* wv;
  long long n;
  int nb;
  const int* bdim;
  int nk;
  __device__ T operator()(long long r, int j, int bact) const {
    int k = j / nb, b = j - k * nb;
    return (k < nk && b < bact) ? wv[(long long)k * n + r] * B[(long long)b * ldb + r] : T(0);
  }
  __device__ int jact() const { return dev_dim(bdim, nb); }
};

template <typename T>
struct FStencil {  // F(row, k * nb + b) = D_k(rho^-1 B[:, b])(row)
  const T* B;
  long long ldb;
  const T* inv_rho;
  Geo g;
  int nb;
  const int* bdim;
  __device__ T operator()(long long r, int j, int bact) const {
    int k = j / nb, b = j - k * nb;
    if (k >= 2 * g.nact || b >= bact) return T(0);
    int ix, iy, iz;
    cell_coords(r, g, ix, iy, iz);
    return stencil_value(B + (long long)b * ldb, inv_rho, r, ix, iy, iz, k, g);
  }
  __device__ int jact() const { return dev_dim(bdim, nb); }
};

constexpr int GR_TC = 32;

template <typename T, class F>
__global__ void __launch_bounds__(256) gram_kernel(long long rows, const T* __restrict__ A, long long lda,
                                                   const int* adim, int acap, int ncols_j, F f,
                                                   double* __restrict__ out, long long ldo) {
  __shared__ T sA[GR_TC][65];
  __shared__ T sF[GR_TC][65];
  const int tid = threadIdx.x;
  const int ta = tid % 16, tj = tid / 16;
  const int a0 = blockIdx.y * 64, j0 = blockIdx.z * 64;
  const int Aact = dev_dim(adim, acap);
  const int Jact = f.jact();
  T acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = T(0); cmp[i][j] = T(0); }
  for (long long r0 = (long long)blockIdx.x * GR_TC; r0 < rows; r0 += (long long)gridDim.x * GR_TC) {
    for (int e = tid; e < GR_TC * 64; e += blockDim.x) {
      int t = e % GR_TC, c = e / GR_TC;
      long long r = r0 + t;
      int a = a0 + c, j = j0 + c;
      sA[t][c] = (r < rows && a < Aact && a < acap) ? A[(long long)a * lda + r] : T(0);
      sF[t][c] = (r < rows && j < ncols_j) ? f(r, j, Jact) : T(0);
    }
    __syncthreads();
    T p[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) p[i][j] = T(0);
#pragma unroll 8
    for (int t = 0; t < GR_TC; ++t) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[t][ta + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sF[t][tj + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) p[i][j] += a[i] * b[j];
    }
    // compensated accumulation of the chunk partials
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        T y = p[i][j] - cmp[i][j];
        T s = acc[i][j] + y;
        cmp[i][j] = (s - acc[i][j]) - y;
        acc[i][j] = s;
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int a = a0 + ta + 16 * i;
    if (a >= acap) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int jj = j0 + tj + 16 * j;
      if (jj >= ncols_j) continue;
      double v = (double)acc[i][j] - (double)cmp[i][j];
      if (v != 0.0) atomicAdd(out + (long long)jj * ldo + a, v);
    }
  }
}

}  // namespace dlra
