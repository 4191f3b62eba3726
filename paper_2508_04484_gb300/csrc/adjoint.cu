// Gradient kernels of the reverse sweep: the discrete adjoint of the energy step.
//
// The loss L depends on the deposited energy e(x). The reverse sweep carries the adjoint
// state mu = dL/du as a low-rank factorisation of its own and pairs it, step by step, with
// the forward states recomputed from checkpoints. Derivatives with respect to the mixture
// (Sec. 2.1, Eq. mixXS) are collected per cell in three arrays: grad_rho = dL/d rho_s
// (rho_s = sum_i w_i rho_i s_i scales the stopping power), grad_w = the direct dL/dw_i
// (scattering and source coefficients), and the ray tracer's dL/df, dL/dtau.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"

namespace dlra {

namespace {

inline unsigned nblocks(long long cnt, int bs) { return (unsigned)((cnt + bs - 1) / bs); }

// Streaming term: for one RK4 stage the forward input z = rho_s v (v = rho_s^-1 z, in the
// forward K-step basis W_f) and the adjoint of z, lam (in the adjoint basis W_a), give
// dL/d rho_s(x) = -<v(x,:) W_f^T, lam(x,:) W_a^T> = -v(x,:) C lam(x,:)^T with C = W_f^T W_a.
template <typename T, int RM>
__global__ void __launch_bounds__(128) grad_stream_kernel(const T* __restrict__ vq, const T* __restrict__ lq, int nq,
                                                          long long n, const double* __restrict__ C, double coef,
                                                          double* __restrict__ grad_rho) {
  __shared__ T sC[RM * RM];
  for (int e = threadIdx.x; e < RM * RM; e += blockDim.x) sC[e] = T(C[e]);   // C[a + c*RM]
  __syncthreads();
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const long long ldq = n * RM;
  double acc = 0.0;
  for (int q = 0; q < nq; ++q) {
    const T* v = vq + q * ldq + x;
    const T* l = lq + q * ldq + x;
    T t[RM];
#pragma unroll
    for (int c = 0; c < RM; ++c) t[c] = T(0);
    for (int a = 0; a < RM; ++a) {
      const T va = v[(long long)a * n];
#pragma unroll
      for (int c = 0; c < RM; ++c) t[c] += va * sC[a + c * RM];
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < RM; ++c) s += t[c] * l[(long long)c * n];
    acc += (double)s;
  }
  grad_rho[x] -= coef * acc;
}

// Cl[l] = S_a (W_a[l]^T W_b[l]) S_b^T for every degree l (one block per l), where W[l] are the
// 2l+1 rows of the moments of degree l (p = l^2 .. l^2 + 2l). FP64; S column-major ld RB.
__global__ void scatter_cl_kernel(const double* __restrict__ Sa, const void* __restrict__ Wa_, const double* __restrict__ Sb,
                                  const void* __restrict__ Wb_, int fp64, int m, int RB, double* __restrict__ Cl) {
  extern __shared__ double sm[];
  double* Ml = sm;              // RB x RB, [a' + c' RB]
  double* T1 = sm + RB * RB;    // RB x RB, [a + c' RB]
  const int l = blockIdx.x;
  const int p0 = l * l, p1 = p0 + 2 * l + 1;
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
    const int ap = e % RB, cp = e / RB;
    double s = 0.0;
    for (int p = p0; p < p1 && p < m; ++p) {
      const double wa = fp64 ? static_cast<const double*>(Wa_)[(long long)ap * m + p]
                             : (double)static_cast<const float*>(Wa_)[(long long)ap * m + p];
      const double wb = fp64 ? static_cast<const double*>(Wb_)[(long long)cp * m + p]
                             : (double)static_cast<const float*>(Wb_)[(long long)cp * m + p];
      s += wa * wb;
    }
    Ml[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
    const int a = e % RB, cp = e / RB;
    double s = 0.0;
    for (int ap = 0; ap < RB; ++ap) s += Sa[(long long)ap * RB + a] * Ml[ap + cp * RB];
    T1[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
    const int a = e % RB, c = e / RB;
    double s = 0.0;
    for (int cp = 0; cp < RB; ++cp) s += T1[a + cp * RB] * Sb[(long long)cp * RB + c];
    Cl[(long long)l * RB * RB + e] = s;   // [a + c RB]
  }
}

// Scattering term: D(x, l) = sum_{p of degree l} alpha(x, p) b(x, p) = X_a(x,:) Cl[l] X_b(x,:)^T,
// with F(x, l) = sum_i wc_i(x) coef_il (wc = w / rho_s) the implicit factor u -> u / (1 - F):
// dL/dw_i(x) += beta D coef_il / rho_s and dL/d rho_s(x) -= beta D F / rho_s.
template <typename T, int RM>
__global__ void __launch_bounds__(128) grad_scatter_kernel(const T* __restrict__ Xa, const T* __restrict__ Xb,
                                                           long long n, const double* __restrict__ Cl, int N,
                                                           const double* __restrict__ coef, int M,
                                                           const T* __restrict__ wc, const double* __restrict__ rho_s,
                                                           double beta, double* __restrict__ grad_w,
                                                           double* __restrict__ grad_rho) {
  __shared__ T sC[RM * RM];
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = x < n;
  T xb[RM];
#pragma unroll
  for (int c = 0; c < RM; ++c) xb[c] = ok ? Xb[(long long)c * n + x] : T(0);
  double gr = 0.0;
  double gw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const double irs = ok ? 1.0 / rho_s[x] : 0.0;
  for (int l = 0; l <= N; ++l) {
    __syncthreads();
    for (int e = threadIdx.x; e < RM * RM; e += blockDim.x) sC[e] = T(Cl[(long long)l * RM * RM + e]);
    __syncthreads();
    if (!ok) continue;
    T D = T(0);
    for (int a = 0; a < RM; ++a) {
      T s = T(0);
#pragma unroll
      for (int c = 0; c < RM; ++c) s += sC[a + c * RM] * xb[c];
      D += Xa[(long long)a * n + x] * s;
    }
    double F = 0.0;
    for (int i = 0; i < M; ++i) F += (double)wc[(long long)i * n + x] * coef[i * (N + 1) + l];
    gr -= (double)D * F;
    for (int i = 0; i < M; ++i) {
      if (i < 8) gw[i] += (double)D * coef[i * (N + 1) + l];
      else grad_w[(long long)i * n + x] += beta * (double)D * coef[i * (N + 1) + l] * irs;
    }
  }
  if (!ok) return;
  grad_rho[x] += beta * gr * irs;
  for (int i = 0; i < M && i < 8; ++i) grad_w[(long long)i * n + x] += beta * gw[i] * irs;
}

// ysrc[i][a] = sum_c S[a][c] sum_p W[p][c] B[i][p] (one block), ld RB.
template <typename T>
__global__ void src_proj_kernel(const double* __restrict__ S, const T* __restrict__ W, const double* __restrict__ B,
                                int m, int RB, int M, double* __restrict__ ysrc) {
  extern __shared__ double sw[];   // [i * RB + c]
  for (int e = threadIdx.x; e < M * RB; e += blockDim.x) {
    const int c = e % RB, i = e / RB;
    double s = 0.0;
    for (int p = 0; p < m; ++p) s += (double)W[(long long)c * m + p] * B[(long long)i * m + p];
    sw[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < M * RB; e += blockDim.x) {
    const int a = e % RB, i = e / RB;
    double s = 0.0;
    for (int c = 0; c < RB; ++c) s += S[(long long)c * RB + a] * sw[i * RB + c];
    ysrc[e] = s;
  }
}

// Source term of one beam at step k: t_i(x) = mu(x,:) . B_i = X(x,:) ysrc_i;
// dL/dw_i(x) += beta h psi(x) t_i(x); dL/dpsi(x) = beta h sum_i w_i(x) t_i(x).
template <typename T>
__global__ void grad_source_kernel(const T* __restrict__ X, long long n, int RB, const double* __restrict__ ysrc,
                                   int M, const double* __restrict__ psi, const T* __restrict__ w, double bh,
                                   double* __restrict__ grad_w, double* __restrict__ gpsi) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  double gp = 0.0;
  const double ps = psi[x];
  for (int i = 0; i < M; ++i) {
    double t = 0.0;
    for (int a = 0; a < RB; ++a) t += (double)X[(long long)a * n + x] * ysrc[i * RB + a];
    grad_w[(long long)i * n + x] += bh * ps * t;
    gp += (double)w[(long long)i * n + x] * t;
  }
  gpsi[x] = bh * gp;
}

__global__ void grad_assemble_kernel(const double* __restrict__ grad_w, const double* __restrict__ grad_rho,
                                     const double* __restrict__ grad_f, const double* __restrict__ grad_tau,
                                     const double* __restrict__ mcoef, int M, long long n, double* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * n) return;
  const int i = (int)(e / n);
  const long long x = e - (long long)i * n;
  out[e] = grad_w[e] + mcoef[2 * i] * (grad_rho[x] + grad_f[x]) + mcoef[2 * i + 1] * grad_tau[x];
}

__global__ void dot_kernel(const double* __restrict__ g, const double* __restrict__ a, const double* __restrict__ b,
                           long long n, double* __restrict__ out) {
  double s = 0.0;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x)
    s += g[x] * (a[x] + b[x]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

// in-place transpose of nk square blocks of size n2 (block k at G + k n2 n2)
__global__ void transpose_blocks_kernel(double* __restrict__ G, int n2, int nk) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)n2 * n2;
  if (e >= per * nk) return;
  const int k = (int)(e / per);
  const int rem = (int)(e - k * per);
  const int a = rem % n2, b = rem / n2;
  if (a >= b) return;
  double* B = G + k * per;
  const double t = B[a + (long long)b * n2];
  B[a + (long long)b * n2] = B[b + (long long)a * n2];
  B[b + (long long)a * n2] = t;
}

}  // namespace

template <typename T>
void launch_grad_stream(cudaStream_t st, const T* vq, const T* lq, int nq, long long n, int RB, const double* C,
                        double coef, double* grad_rho) {
  switch (RB) {
#define GS_CASE(R) \
  case R: grad_stream_kernel<T, R><<<nblocks(n, 128), 128, 0, st>>>(vq, lq, nq, n, C, coef, grad_rho); break;
    GS_CASE(4) GS_CASE(8) GS_CASE(12) GS_CASE(16) GS_CASE(20) GS_CASE(24) GS_CASE(32) GS_CASE(40) GS_CASE(48)
    GS_CASE(64)
#undef GS_CASE
    default: break;
  }
}

void launch_scatter_cl(cudaStream_t st, const double* Sa, const void* Wa, const double* Sb, const void* Wb, int fp64,
                       int m, int N, int RB, double* Cl) {
  const size_t smem = (size_t)2 * RB * RB * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(scatter_cl_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  scatter_cl_kernel<<<N + 1, 256, smem, st>>>(Sa, Wa, Sb, Wb, fp64, m, RB, Cl);
}

template <typename T>
void launch_grad_scatter(cudaStream_t st, const T* Xa, const T* Xb, long long n, int RB, const double* Cl, int N,
                         const double* coef, int M, const T* wc, const double* rho_s, double beta, double* grad_w,
                         double* grad_rho) {
  switch (RB) {
#define GC_CASE(R)                                                                                              \
  case R:                                                                                                       \
    grad_scatter_kernel<T, R><<<nblocks(n, 128), 128, 0, st>>>(Xa, Xb, n, Cl, N, coef, M, wc, rho_s, beta,      \
                                                               grad_w, grad_rho);                              \
    break;
    GC_CASE(4) GC_CASE(8) GC_CASE(12) GC_CASE(16) GC_CASE(20) GC_CASE(24) GC_CASE(32) GC_CASE(40) GC_CASE(48)
    GC_CASE(64)
#undef GC_CASE
    default: break;
  }
}

template <typename T>
void launch_grad_source(cudaStream_t st, const T* X, const double* S, const T* W, long long n, int m, int RB,
                        const double* B, int M, const double* psi, const T* w, double bh, double* ysrc,
                        double* grad_w, double* gpsi) {
  src_proj_kernel<T><<<1, 256, (size_t)M * RB * sizeof(double), st>>>(S, W, B, m, RB, M, ysrc);
  grad_source_kernel<T><<<nblocks(n, 256), 256, 0, st>>>(X, n, RB, ysrc, M, psi, w, bh, grad_w, gpsi);
}

void launch_grad_assemble(cudaStream_t st, const double* grad_w, const double* grad_rho, const double* grad_f,
                          const double* grad_tau, const double* mcoef, int M, long long n, double* out) {
  grad_assemble_kernel<<<nblocks((long long)M * n, 256), 256, 0, st>>>(grad_w, grad_rho, grad_f, grad_tau, mcoef, M,
                                                                       n, out);
}

void launch_dot(cudaStream_t st, const double* g, const double* a, const double* b, long long n, double* out) {
  dot_kernel<<<std::min<unsigned>(nblocks(n, 256), 1024), 256, 0, st>>>(g, a, b, n, out);
}

void launch_transpose_blocks(cudaStream_t st, double* G, int n2, int nk) {
  transpose_blocks_kernel<<<nblocks((long long)n2 * n2 * nk, 256), 256, 0, st>>>(G, n2, nk);
}

template void launch_grad_stream<float>(cudaStream_t, const float*, const float*, int, long long, int, const double*,
                                        double, double*);
template void launch_grad_stream<double>(cudaStream_t, const double*, const double*, int, long long, int,
                                         const double*, double, double*);
template void launch_grad_scatter<float>(cudaStream_t, const float*, const float*, long long, int, const double*, int,
                                         const double*, int, const float*, const double*, double, double*, double*);
template void launch_grad_scatter<double>(cudaStream_t, const double*, const double*, long long, int, const double*,
                                          int, const double*, int, const double*, const double*, double, double*,
                                          double*);
template void launch_grad_source<float>(cudaStream_t, const float*, const double*, const float*, long long, int, int,
                                        const double*, int, const double*, const float*, double, double*, double*,
                                        double*);
template void launch_grad_source<double>(cudaStream_t, const double*, const double*, const double*, long long, int,
                                         int, const double*, int, const double*, const double*, double, double*,
                                         double*, double*);

}  // namespace dlra
