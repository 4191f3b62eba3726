// Small dense kernels of the low-rank step (one thread block each): the factors
// of the basis augmentation, the truncation SVD, the Galerkin S-step, the implicit
// collided L-step and its QR, the W-side augmentation and the source S assembly.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace dlra {

namespace {

template <typename T>
__device__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; sbuf holds >= 32 elements. All threads get the result.
template <typename T>
__device__ T block_sum(T v, T* sbuf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sbuf[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? sbuf[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sbuf[0] = t;
  __syncthreads();
  T r = sbuf[0];
  __syncthreads();
  return r;
}

}  // namespace

// ---------------------------------------------------------------------------
// pivoted-Cholesky factor of the projected Gram (CholeskyQR with pivoting)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) orth_factor_kernel(const double* __restrict__ G, const double* __restrict__ C1, int RBa, int qcap,
                                   double drop_tol, double* __restrict__ Mout, int* qout, int* err, int stage) {
  extern __shared__ double sh[];
  __shared__ double red[32];
  __shared__ double rdiag[128];          // 1 / L_ii
  __shared__ int s_piv, s_stop;
  __shared__ int iperm[128];             // original column -> pivoted position
  const int ldg = RBa + qcap;
  double* A = sh;                        // qcap x qcap, col-major A[j*qcap + i]
  double* Li = A + qcap * qcap;          // inverse of the lower factor
  double* Gs = Li + qcap * qcap;         // the Gram G (ldg x qcap), staged where it fits
  int* perm = reinterpret_cast<int*>(Gs + (stage ? (size_t)ldg * qcap : 0));
  const int tid = threadIdx.x, nt = blockDim.x;
  if (stage) {
    for (int e = tid; e < ldg * qcap; e += nt) Gs[e] = G[e];
    __syncthreads();
    G = Gs;
  }
  // G' = R^T R - C2^T C2 (C2 = Xa^T R is the top block)
  for (int e = tid; e < qcap * qcap; e += nt) {
    int i = e % qcap, j = e / qcap;
    double v = G[(long long)j * ldg + RBa + i];
    for (int a = 0; a < RBa; ++a) v -= G[(long long)i * ldg + a] * G[(long long)j * ldg + a];
    A[e] = v;
  }
  for (int i = tid; i < qcap; i += nt) perm[i] = i;
  double part = 0.0;
  for (int i = tid; i < qcap; i += nt) part += G[(long long)i * ldg + RBa + i];
  if (C1)
    for (int e = tid; e < RBa * qcap; e += nt) part += C1[e] * C1[e];
  const double scale2 = block_sum(part, red);
  const double thr = drop_tol * drop_tol * scale2;
  if (tid == 0) s_stop = qcap;
  __syncthreads();
  for (int j = 0; j < qcap; ++j) {
    if (tid < 32) {
      // largest remaining diagonal (first index on ties), one warp
      int p = -1;
      double best = 0.0;
      bool nan = false;
      for (int i = j + tid; i < qcap; i += 32) {
        const double d = A[i * qcap + i];
        nan = nan || d != d;
        if (p < 0 || d > best) { best = d; p = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (op >= 0 && (p < 0 || ob > best || (ob == best && op < p))) { best = ob; p = op; }
      }
      nan = __any_sync(0xffffffffu, nan);
      if (tid == 0) {
        if (!(best > thr) || nan) {
          s_stop = j;
          if (nan || best != best) atomicOr(err, ERR_NONFINITE);
        }
        s_piv = p;
      }
    }
    __syncthreads();
    if (s_stop == j) break;
    const int p = s_piv;
    if (p != j) {
      for (int k = tid; k < qcap; k += nt) {  // swap rows j, p
        double t = A[k * qcap + j];
        A[k * qcap + j] = A[k * qcap + p];
        A[k * qcap + p] = t;
      }
      __syncthreads();
      for (int k = tid; k < qcap; k += nt) {  // swap columns j, p
        double t = A[j * qcap + k];
        A[j * qcap + k] = A[p * qcap + k];
        A[p * qcap + k] = t;
      }
      if (tid == 0) {
        int t = perm[j];
        perm[j] = perm[p];
        perm[p] = t;
      }
      __syncthreads();
    }
    if (tid == 0) A[j * qcap + j] = sqrt(A[j * qcap + j]);
    __syncthreads();
    const double djj = A[j * qcap + j];
    for (int i = j + 1 + tid; i < qcap; i += nt) A[j * qcap + i] /= djj;
    __syncthreads();
    for (int e = tid; e < (qcap - j - 1) * (qcap - j - 1); e += nt) {
      int i = j + 1 + e % (qcap - j - 1), k = j + 1 + e / (qcap - j - 1);
      A[k * qcap + i] -= A[j * qcap + i] * A[j * qcap + k];
    }
    __syncthreads();
  }
  const int q = s_stop;
  for (int i = tid; i < q; i += nt) rdiag[i] = 1.0 / A[i * qcap + i];
  for (int i = tid; i < qcap; i += nt) iperm[perm[i]] = i;
  __syncthreads();
  // inverse of the lower factor L (q x q): column c solves L x = e_c, four lanes per column
  // (the sums over k split four ways and combined by shuffles)
  for (int c0 = tid >> 2; c0 < ((q + 63) / 64) * 64; c0 += nt >> 2) {
    const int c = c0, part = tid & 3;
    const bool act = c < q;
    for (int i = 0; i < q; ++i) {
      double v = 0.0;
      if (act)
        for (int k = c + part; k < i; k += 4) v -= A[k * qcap + i] * Li[c * qcap + k];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      if (act && part == 0) Li[c * qcap + i] = (i < c) ? 0.0 : (v + (i == c ? 1.0 : 0.0)) * rdiag[i];
      __syncwarp();
    }
  }
  __syncthreads();
  // T[perm[i]][c] = (L^-T)[i][c] = (L^-1)[c][i] = Li[i * qcap + c] for i < q: Mout = [-C2 T ; T]
  const int ldm = RBa + qcap;
  for (int e = tid; e < ldm * qcap; e += nt) {
    int row = e % ldm, c = e / ldm;
    double v = 0.0;
    if (c < q) {
      if (row >= RBa) {
        const int i = iperm[row - RBa];   // pivoted position of the original column
        v = i < q ? Li[i * qcap + c] : 0.0;
      } else {
        for (int i = 0; i < q; ++i) v -= G[(long long)perm[i] * ldg + row] * Li[i * qcap + c];
      }
    }
    Mout[(long long)c * ldm + row] = v;
  }
  if (tid == 0) *qout = q;
}

void launch_orth_factor(cudaStream_t st, const double* G, const double* C1, int RBa, int qcap, double drop_tol,
                        double* Mout, int* qout, int* err) {
  const size_t base = (size_t)2 * qcap * qcap * sizeof(double) + (size_t)qcap * sizeof(int) + 16;
  const size_t staged = base + (size_t)(RBa + qcap) * qcap * sizeof(double);
  const int stage = staged <= 200 * 1024 ? 1 : 0;
  const size_t smem = stage ? staged : base;
  if (smem > 48 * 1024) cudaFuncSetAttribute(orth_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  orth_factor_kernel<<<1, 256, smem, st>>>(G, C1, RBa, qcap, drop_tol, Mout, qout, err, stage);
}

// ---------------------------------------------------------------------------
// truncated SVD by one-sided (Hestenes) Jacobi with a round-robin ordering
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rr_pair(int round, int i, int n, int& a, int& b) {
  if (i == 0) a = 0;
  else a = ((i + round - 1) % (n - 1)) + 1;
  b = ((n - 1 - i + round - 1) % (n - 1)) + 1;
}

template <typename T>
__global__ void __launch_bounds__(1024) svd_trunc_kernel(const double* __restrict__ Sh, int n2, int RB, RankParams rp, int step, int event,
                                 double* __restrict__ P, double* __restrict__ Q, double* __restrict__ S,
                                 BeamDims* dims, int* rank_log, int* err, T* __restrict__ vwork) {
  extern __shared__ __align__(16) unsigned char raw[];
  T* A = reinterpret_cast<T*>(raw);
  T* V = vwork ? vwork : A + n2 * n2;   // right rotations: shared memory, or global when both do not fit
  __shared__ double sig[128];
  __shared__ int order[128];
  __shared__ T nrm[128];   // squared column norms, updated by each rotation
  __shared__ T red[32];
  __shared__ int cols[128];       // the columns that are not numerically null (plus -1 if odd)
  __shared__ unsigned s_maxrel;   // largest relative coupling |a_p . a_q| / (|a_p| |a_q|) of a sweep
  __shared__ int s_na, s_r1;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  T part = 0;
  for (int e = tid; e < n2 * n2; e += nt) {
    T v = T(Sh[e]);
    A[e] = v;
    part += v * v;
    V[e] = (e % n2 == e / n2) ? T(1) : T(0);
  }
  const T fro2 = block_sum(part, red);
  for (int j = wid; j < n2; j += nw) {
    T s2 = 0;
    for (int i = lane; i < n2; i += 32) s2 += A[j * n2 + i] * A[j * n2 + i];
    s2 = warp_sum(s2);
    if (lane == 0) nrm[j] = s2;
  }
  __syncthreads();
  const T eps = (sizeof(T) == 8) ? T(1e-14) : T(4e-6);
  // columns below this squared norm are numerically null and are not rotated
  const T null2 = fro2 * ((sizeof(T) == 8) ? T(1e-28) : T(1e-14));
  // after a sweep whose largest coupling c has c^2 below this, the next sweep (quadratic
  // convergence) would rotate by less than eps: stop
  const float stop2 = (sizeof(T) == 8) ? 1e-16f : 1e-7f;
  if (tid == 0) {
    int na = 0;
    for (int j = 0; j < n2; ++j)
      if (nrm[j] > null2) cols[na++] = j;
    if (na & 1) cols[na++] = -1;
    s_na = na;
  }
  __syncthreads();
  const int na = s_na;
  for (int sweep = 0; sweep < 60 && na >= 2; ++sweep) {
    if (tid == 0) s_maxrel = 0u;
    __syncthreads();
    // round-robin over the active columns: each round rotates na/2 disjoint pairs, one per warp
    for (int round = 0; round < na - 1; ++round) {
      for (int pi = wid; pi < na / 2; pi += nw) {
        int pp, qq;
        rr_pair(round, pi, na, pp, qq);
        const int p = cols[pp], q = cols[qq];
        if (p < 0 || q < 0) continue;
        const T al = nrm[p], be = nrm[q];
        if (al <= null2 || be <= null2) continue;
        T* ap = A + p * n2;
        T* aq = A + q * n2;
        const T x0 = lane < n2 ? ap[lane] : T(0), y0 = lane < n2 ? aq[lane] : T(0);
        const T x1 = lane + 32 < n2 ? ap[lane + 32] : T(0), y1 = lane + 32 < n2 ? aq[lane + 32] : T(0);
        T ga = x0 * y0 + x1 * y1;
        for (int i = lane + 64; i < n2; i += 32) ga += ap[i] * aq[i];
        ga = warp_sum(ga);
        const T rel = fabs(ga) / sqrt(al * be);
        if (lane == 0) atomicMax(&s_maxrel, __float_as_uint((float)rel));
        if (ga != T(0) && rel > eps) {
          T zeta = (be - al) / (T(2) * ga);
          T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          T c = T(1) / sqrt(T(1) + t * t), s = c * t;
          if (lane < n2) {
            ap[lane] = c * x0 - s * y0;
            aq[lane] = s * x0 + c * y0;
          }
          if (lane + 32 < n2) {
            ap[lane + 32] = c * x1 - s * y1;
            aq[lane + 32] = s * x1 + c * y1;
          }
          for (int i = lane + 64; i < n2; i += 32) {
            T x = ap[i], y = aq[i];
            ap[i] = c * x - s * y;
            aq[i] = s * x + c * y;
          }
          T* vp = V + p * n2;
          T* vq = V + q * n2;
          for (int i = lane; i < n2; i += 32) {
            T x = vp[i], y = vq[i];
            vp[i] = c * x - s * y;
            vq[i] = s * x + c * y;
          }
          if (lane == 0) {
            // exact norms of the rotated pair: |a_p|^2 - t ga, |a_q|^2 + t ga
            nrm[p] = al - t * ga;
            nrm[q] = be + t * ga;
          }
        }
      }
      __syncthreads();
    }
    // refresh the norms from the columns once per sweep
    for (int j = wid; j < n2; j += nw) {
      T s2 = 0;
      for (int i = lane; i < n2; i += 32) s2 += A[j * n2 + i] * A[j * n2 + i];
      s2 = warp_sum(s2);
      if (lane == 0) nrm[j] = s2;
    }
    __syncthreads();
    const float mr = __uint_as_float(s_maxrel);
    if (mr <= (float)eps || mr * mr < stop2) break;
    __syncthreads();
  }
  for (int j = wid; j < n2; j += nw) {
    T s2 = 0;
    for (int i = lane; i < n2; i += 32) s2 += A[j * n2 + i] * A[j * n2 + i];
    s2 = warp_sum(s2);
    if (lane == 0) sig[j] = sqrt((double)s2);
  }
  __syncthreads();
  for (int j = tid; j < n2; j += nt) {
    int rk = 0;
    double sj = sig[j];
    for (int i = 0; i < n2; ++i) {
      double si = sig[i];
      if (si > sj || (si == sj && i < j)) ++rk;
    }
    order[rk] = j;
  }
  __syncthreads();
  if (tid == 0) {
    double s1 = sig[order[0]];
    int r1 = 0;
    bool bad = !(s1 == s1) || isinf(s1);
    if (bad) atomicOr(err, ERR_NONFINITE);
    if (!bad && s1 > 0.0) {
      int nz = 0;
      for (int i = 0; i < n2; ++i)
        if (sig[order[i]] > rp.nz_tol * s1) ++nz;
      if (rp.mode == 2) {
        r1 = rp.schedule ? rp.schedule[2 * step + event] : 0;
        if (r1 < 0) r1 = 0;
        if (r1 > n2) r1 = n2;
      } else {
        if (rp.mode == 0) {
          r1 = rp.rank < nz ? rp.rank : nz;
        } else {
          double tot = 0.0;
          for (int i = 0; i < n2; ++i) tot += sig[i] * sig[i];
          double thr = rp.tol * sqrt(tot);
          double tail = 0.0;
          r1 = n2;
          for (int r = n2; r >= 0; --r) {  // tail(r) = sum_{i >= r} sigma_i
            if (r < n2) tail += sig[order[r]];
            if (tail <= thr) r1 = r;
            else break;
          }
          if (r1 < 1) r1 = 1;
          if (r1 > rp.rank_max) r1 = rp.rank_max;
          if (r1 > nz) r1 = nz;
        }
        int r0 = r1;
        while (r1 > 0 && r1 < n2 && sig[order[r1 - 1]] - sig[order[r1]] <= rp.cluster_tol * s1) --r1;
        if (r1 == 0) {
          r1 = r0;
          while (r1 < n2 && r1 > 0 && sig[order[r1 - 1]] - sig[order[r1]] <= rp.cluster_tol * s1) ++r1;
        }
      }
      if (r1 > RB) {
        r1 = RB;
        atomicOr(err, ERR_CAPACITY);
      }
    }
    s_r1 = r1;
    dims->r = r1;
    if (rank_log) rank_log[2 * step + event] = r1;
  }
  __syncthreads();
  const int r1 = s_r1;
  for (int e = tid; e < n2 * RB; e += nt) {
    int i = e % n2, c = e / n2;
    double pv = 0.0, qv = 0.0;
    if (c < r1) {
      int j = order[c];
      double sj = sig[j];
      pv = sj > 0.0 ? (double)A[j * n2 + i] / sj : 0.0;
      qv = (double)V[j * n2 + i];
    }
    P[(long long)c * n2 + i] = pv;
    Q[(long long)c * n2 + i] = qv;
  }
  for (int e = tid; e < RB * RB; e += nt) {
    int a = e % RB, c = e / RB;
    S[e] = (a == c && c < r1) ? sig[order[c]] : 0.0;
  }
}

template <typename T>
void launch_svd_truncate(cudaStream_t st, const double* Sh, int n2, int RB, RankParams rp, int step, int event,
                         double* P, double* Q, double* S, BeamDims* dims, int* rank_log, int* err, void* vwork) {
  const bool vg = svd_needs_vwork(n2, sizeof(T));
  size_t smem = (size_t)(vg ? 1 : 2) * n2 * n2 * sizeof(T);
  if (smem > 48 * 1024) cudaFuncSetAttribute(svd_trunc_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  svd_trunc_kernel<T><<<1, 1024, smem, st>>>(Sh, n2, RB, rp, step, event, P, Q, S, dims, rank_log, err,
                                             vg ? reinterpret_cast<T*>(vwork) : nullptr);
}
template void launch_svd_truncate<float>(cudaStream_t, const double*, int, int, RankParams, int, int, double*, double*,
                                         double*, BeamDims*, int*, int*, void*);
template void launch_svd_truncate<double>(cudaStream_t, const double*, int, int, RankParams, int, int, double*,
                                          double*, double*, BeamDims*, int*, int*, void*);

// ---------------------------------------------------------------------------
// Galerkin S-step with RK4 in Horner form
// ---------------------------------------------------------------------------
// Each thread owns an MT x MT tile of the n2 x n2 result; the products z P_k and
// G_k (z P_k) run from shared memory. The 2 nk operators are preloaded once when
// they fit, otherwise reloaded per k.
template <typename T, int MT>
__global__ void __launch_bounds__(1024) sstep_kernel(const double* __restrict__ Gh, const double* __restrict__ Ph,
                                                     int nk, const double* __restrict__ S, int RB, int n2,
                                                     const double* __restrict__ beta, int nsub, int preload,
                                                     double* __restrict__ Sh) {
  extern __shared__ __align__(16) unsigned char raw[];
  const int ne = n2 * n2;
  T* z = reinterpret_cast<T*>(raw);   // stage input, col-major
  T* tmp = z + ne;                    // z P_k
  T* ops = tmp + ne;                  // preload: [P_0..P_{nk-1}, G_0..G_{nk-1}]; else 1 slot
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nb = n2 / MT;             // tiles per dimension
  const int ti = tid % nb, tj = tid / nb;
  const bool owner = tj < nb;
  for (int e = tid; e < ne; e += nt) {
    int a = e % n2, c = e / n2;
    double y = (a < RB && c < RB) ? S[c * RB + a] : 0.0;
    Sh[e] = y;
    z[e] = T(y);
  }
  if (preload) {
    for (int e = tid; e < nk * ne; e += nt) {
      ops[e] = T(Ph[e]);
      ops[nk * ne + e] = T(Gh[e]);
    }
  }
  __syncthreads();
  for (int j = 0; j < nsub; ++j) {
    for (int s = 0; s < 4; ++s) {
      const double b = beta[4 * j + s];
      T acc[MT][MT];
#pragma unroll
      for (int u = 0; u < MT; ++u)
#pragma unroll
        for (int v = 0; v < MT; ++v) acc[u][v] = T(0);
      for (int k = 0; k < nk; ++k) {
        const T* Pk;
        const T* Gk;
        if (preload) {
          Pk = ops + (long long)k * ne;
          Gk = ops + (long long)(nk + k) * ne;
        } else {
          for (int e = tid; e < ne; e += nt) ops[e] = T(Ph[(long long)k * ne + e]);
          __syncthreads();
          Pk = ops;
          Gk = ops;
        }
        // tmp = z Pk
        if (owner) {
          T t[MT][MT];
#pragma unroll
          for (int u = 0; u < MT; ++u)
#pragma unroll
            for (int v = 0; v < MT; ++v) t[u][v] = T(0);
          for (int q = 0; q < n2; ++q) {
            T za[MT], pb[MT];
#pragma unroll
            for (int u = 0; u < MT; ++u) za[u] = z[q * n2 + ti + u * nb];
#pragma unroll
            for (int v = 0; v < MT; ++v) pb[v] = Pk[(tj + v * nb) * n2 + q];
#pragma unroll
            for (int u = 0; u < MT; ++u)
#pragma unroll
              for (int v = 0; v < MT; ++v) t[u][v] += za[u] * pb[v];
          }
#pragma unroll
          for (int u = 0; u < MT; ++u)
#pragma unroll
            for (int v = 0; v < MT; ++v) tmp[(tj + v * nb) * n2 + ti + u * nb] = t[u][v];
        }
        __syncthreads();
        if (!preload) {
          for (int e = tid; e < ne; e += nt) ops[e] = T(Gh[(long long)k * ne + e]);
          __syncthreads();
        }
        // acc += Gk tmp
        if (owner) {
          for (int q = 0; q < n2; ++q) {
            T ga[MT], tb[MT];
#pragma unroll
            for (int u = 0; u < MT; ++u) ga[u] = Gk[q * n2 + ti + u * nb];
#pragma unroll
            for (int v = 0; v < MT; ++v) tb[v] = tmp[(tj + v * nb) * n2 + q];
#pragma unroll
            for (int u = 0; u < MT; ++u)
#pragma unroll
              for (int v = 0; v < MT; ++v) acc[u][v] += ga[u] * tb[v];
          }
        }
        __syncthreads();
      }
      if (owner) {
#pragma unroll
        for (int u = 0; u < MT; ++u)
#pragma unroll
          for (int v = 0; v < MT; ++v) {
            int e = (tj + v * nb) * n2 + ti + u * nb;
            double nv = Sh[e] + b * (double)acc[u][v];
            if (s == 3) Sh[e] = nv;
            z[e] = T(nv);
          }
      }
      __syncthreads();
    }
  }
}

// The S-step on a cluster of SCL thread blocks: block c owns the output columns J_c of
// S -> sum_k G_k S P_k (Sec. 2.2, Eq. KLS). Per RK4 stage it forms U_k = z P_k(:, J_c) and
// sum_k G_k U_k for its columns, and writes its part of the next stage input z into the
// shared memory of every block of the cluster (distributed shared memory); one cluster
// barrier per stage. z is double-buffered so that a stage never overwrites the buffer the
// other blocks are still reading.
constexpr int SCL = 8;

template <typename T>
__global__ void __launch_bounds__(256) sstep_cluster_kernel(const double* __restrict__ Gh,
                                                            const double* __restrict__ Ph, int nk,
                                                            const double* __restrict__ S, int RB, int n2,
                                                            const double* __restrict__ beta, int nsub,
                                                            double* __restrict__ Sh) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int w = (n2 + SCL - 1) / SCL;                 // columns per block
  const int j0 = rank * w, jn = max(0, min(w, n2 - j0));
  const int ne = n2 * n2;
  extern __shared__ __align__(16) unsigned char raw[];
  T* G = reinterpret_cast<T*>(raw);                   // nk x n2 x n2, G_k[a][q] at (k n2 + q) n2 + a
  T* Pc = G + (size_t)nk * ne;                        // nk x n2 x w: P_k[q][j0 + j] at (k w + j) n2 + q
  T* z0 = Pc + (size_t)nk * n2 * w;                   // two stage buffers, n2 x n2 column-major
  T* z1 = z0 + ne;
  T* U = z1 + ne;                                     // nk x n2 x w
  double* y = reinterpret_cast<double*>(U + (size_t)nk * n2 * w);   // own columns of Sh, n2 x w
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < nk * ne; e += nt) G[e] = T(Gh[e]);
  for (int e = tid; e < nk * n2 * w; e += nt) {
    const int q = e % n2, kj = e / n2, j = kj % w, k = kj / w;
    Pc[e] = (j < jn) ? T(Ph[((long long)k * n2 + j0 + j) * n2 + q]) : T(0);
  }
  for (int e = tid; e < ne; e += nt) {
    const int a = e % n2, c = e / n2;
    z0[e] = T((a < RB && c < RB) ? S[c * RB + a] : 0.0);
  }
  for (int e = tid; e < n2 * w; e += nt) {
    const int a = e % n2, j = e / n2, c = j0 + j;
    y[e] = (j < jn && a < RB && c < RB) ? S[c * RB + a] : 0.0;
  }
  __syncthreads();
  int stage = 0;
  for (int js = 0; js < nsub; ++js) {
    for (int s4 = 0; s4 < 4; ++s4, ++stage) {
      const double b = beta[4 * js + s4];
      const T* z = (stage & 1) ? z1 : z0;
      T* zn = (stage & 1) ? z0 : z1;
      // U_k(:, j) = z P_k(:, j0 + j)
      for (int e = tid; e < nk * n2 * w; e += nt) {
        const int a = e % n2, kj = e / n2;
        const T* pc = Pc + (size_t)kj * n2;
        T acc = T(0);
        for (int q = 0; q < n2; ++q) acc += z[q * n2 + a] * pc[q];
        U[e] = acc;
      }
      __syncthreads();
      // out(:, j) = sum_k G_k U_k(:, j); y / z update of the own columns
      for (int e = tid; e < n2 * jn; e += nt) {
        const int a = e % n2, j = e / n2;
        T acc = T(0);
        for (int k = 0; k < nk; ++k) {
          const T* gk = G + (size_t)k * ne + a;
          const T* uk = U + ((size_t)k * w + j) * n2;
          for (int q = 0; q < n2; ++q) acc += gk[q * n2] * uk[q];
        }
        const double nv = y[e] + b * (double)acc;
        if (s4 == 3) y[e] = nv;
        const T tv = T(nv);
        const int col = j0 + j;
        for (int rk = 0; rk < SCL; ++rk) {
          T* dst = cluster.map_shared_rank(zn, rk);
          dst[col * n2 + a] = tv;
        }
      }
      cluster.sync();
    }
  }
  for (int e = tid; e < n2 * jn; e += nt) {
    const int a = e % n2, j = e / n2;
    Sh[(long long)(j0 + j) * n2 + a] = y[e];
  }
}

template <typename T>
size_t sstep_cluster_smem(int nk, int n2) {
  const int w = (n2 + SCL - 1) / SCL;
  return ((size_t)nk * n2 * n2 + 2 * (size_t)nk * n2 * w + 2 * (size_t)n2 * n2) * sizeof(T) +
         (size_t)n2 * w * sizeof(double) + 16;
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident): bar[0] counts arrivals,
// bar[1] is the generation, bar[2] an abort flag. A block that waits longer than about a second
// sets ERR_TIMEOUT and the abort flag; every later barrier of any block then returns at once,
// so the kernel finishes (with a result the host discards: the error poisons the context).
constexpr long long kBarrierSpins = 1LL << 24;

__device__ __forceinline__ void grid_barrier(unsigned* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vb = bar;
    if (vb[2] == 0u) {
      const unsigned g = vb[1];
      __threadfence();
      if (atomicAdd(&bar[0], 1u) == gridDim.x - 1u) {
        atomicExch(&bar[0], 0u);
        __threadfence();
        atomicAdd(&bar[1], 1u);
      } else {
        long long it = 0;
        while (vb[1] == g && vb[2] == 0u) {
          if (++it > kBarrierSpins) {
            atomicExch(&bar[2], 1u);
            atomicOr(err, ERR_TIMEOUT);
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
}

// The S-step over the whole grid: per RK4 stage three phases separated by grid barriers,
// each a list of 16 x 16 output tiles spread over the blocks:
//   A: U_k = z P_k            (nk tiles lists),
//   B: O_k = G_k U_k          (nk tiles lists; the sum over k is left to C),
//   C: Sh / z update with sum_k O_k (element-wise).
// Arithmetic in T (FP64 on the FP32-split path at 2r = 128, where the operators do not fit
// the shared memory of a cluster); operators read from global memory (L2-resident).
constexpr int SG_TS = 16;   // output tile
constexpr int SG_KC = 64;   // contraction chunk held in shared memory

template <typename T>
__device__ void sg_tile(int n2, const double* __restrict__ Ad, const T* __restrict__ At, long long a_ld_row,
                        long long a_ld_col, const double* __restrict__ Bd, const T* __restrict__ Bt,
                        long long b_ld_row, long long b_ld_col, int i0, int j0, T* __restrict__ out, T (*sa)[SG_KC + 1],
                        T (*sb)[SG_TS + 1]) {
  // out[(j0 + tj) * n2 + i0 + ti] = sum_q A(i0 + ti, q) B(q, j0 + tj); A(a, q) at a * a_ld_row + q * a_ld_col
  // from Ad (FP64) or At (T), B likewise
  const int tid = threadIdx.x, ti = tid % SG_TS, tj = tid / SG_TS;
  T acc = T(0);
  for (int q0 = 0; q0 < n2; q0 += SG_KC) {
    const int kc = min(SG_KC, n2 - q0);
    for (int e = tid; e < SG_TS * kc; e += blockDim.x) {
      const int a = e / kc, q = e % kc, ia = i0 + a;
      T v = T(0);
      if (ia < n2) {
        const long long o = ia * a_ld_row + (long long)(q0 + q) * a_ld_col;
        v = Ad ? T(Ad[o]) : At[o];
      }
      sa[a][q] = v;
    }
    for (int e = tid; e < kc * SG_TS; e += blockDim.x) {
      const int j = e / kc, q = e % kc, jb = j0 + j;
      T v = T(0);
      if (jb < n2) {
        const long long o = (long long)(q0 + q) * b_ld_row + jb * b_ld_col;
        v = Bd ? T(Bd[o]) : Bt[o];
      }
      sb[q][j] = v;
    }
    __syncthreads();
    if (tj < SG_TS)
      for (int q = 0; q < kc; ++q) acc += sa[ti][q] * sb[q][tj];
    __syncthreads();
  }
  if (tj < SG_TS && i0 + ti < n2 && j0 + tj < n2) out[(long long)(j0 + tj) * n2 + i0 + ti] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256) sstep_grid_kernel(const double* __restrict__ Gh, const double* __restrict__ Ph,
                                                         int nk, const double* __restrict__ S, int RB, int n2,
                                                         const double* __restrict__ beta, int nsub,
                                                         double* __restrict__ Sh, T* __restrict__ z,
                                                         T* __restrict__ U, T* __restrict__ O, unsigned* bar,
                                                         int* err) {
  __shared__ T sa[SG_TS][SG_KC + 1];
  __shared__ T sb[SG_KC][SG_TS + 1];
  const long long ne = (long long)n2 * n2;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x, gnt = (long long)gridDim.x * blockDim.x;
  for (long long e = gtid; e < ne; e += gnt) {
    const int a = (int)(e % n2), c = (int)(e / n2);
    const double y = (a < RB && c < RB) ? S[c * RB + a] : 0.0;
    Sh[e] = y;
    z[e] = T(y);
  }
  grid_barrier(bar, err);
  const int nt = (n2 + SG_TS - 1) / SG_TS;
  const int ntask = nk * nt * nt;
  for (int js = 0; js < nsub; ++js) {
    for (int s4 = 0; s4 < 4; ++s4) {
      // A: U_k(a, j) = sum_q z(a, q) P_k(q, j);  z(a, q) at q n2 + a, P_k(q, j) at (k n2 + j) n2 + q
      for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
        const int k = t / (nt * nt), ij = t % (nt * nt), i0 = (ij % nt) * SG_TS, j0 = (ij / nt) * SG_TS;
        sg_tile<T>(n2, nullptr, z, 1, n2, Ph + (long long)k * ne, nullptr, 1, n2, i0, j0, U + (long long)k * ne, sa,
                   sb);
      }
      grid_barrier(bar, err);
      // B: O_k(a, j) = sum_q G_k(a, q) U_k(q, j);  G_k(a, q) at (k n2 + q) n2 + a
      for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
        const int k = t / (nt * nt), ij = t % (nt * nt), i0 = (ij % nt) * SG_TS, j0 = (ij / nt) * SG_TS;
        sg_tile<T>(n2, Gh + (long long)k * ne, nullptr, 1, n2, nullptr, U + (long long)k * ne, 1, n2, i0, j0,
                   O + (long long)k * ne, sa, sb);
      }
      grid_barrier(bar, err);
      // C: the Horner update
      const double b = beta[4 * js + s4];
      for (long long e = gtid; e < ne; e += gnt) {
        T acc = T(0);
        for (int k = 0; k < nk; ++k) acc += O[(long long)k * ne + e];
        const double nv = Sh[e] + b * (double)acc;
        if (s4 == 3) Sh[e] = nv;
        z[e] = T(nv);
      }
      grid_barrier(bar, err);
    }
  }
}

bool sstep_needs_grid(int nk, int n2, size_t tsize) {
  return (tsize == 4 ? sstep_cluster_smem<float>(nk, n2) : sstep_cluster_smem<double>(nk, n2)) > 200 * 1024;
}

template <typename T>
void launch_sstep(cudaStream_t st, const double* Gh, const double* Ph, int nk, const double* S, int RB, int n2,
                  const double* beta, int nsub, double* Sh, const SstepWork* gw, int* err) {
  const size_t csmem = sstep_cluster_smem<T>(nk, n2);
  if (csmem > 200 * 1024 && gw && gw->grid > 0 && err) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(gw->grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, sstep_grid_kernel<T>, Gh, Ph, nk, S, RB, n2, beta, nsub, Sh,
                       reinterpret_cast<T*>(gw->z), reinterpret_cast<T*>(gw->U), reinterpret_cast<T*>(gw->O), gw->bar,
                       err);
    return;
  }
  if (csmem <= 200 * 1024) {
    if (csmem > 48 * 1024)
      cudaFuncSetAttribute(sstep_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(SCL);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = csmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = SCL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, sstep_cluster_kernel<T>, Gh, Ph, nk, S, RB, n2, beta, nsub, Sh) == cudaSuccess)
      return;
    cudaGetLastError();   // cluster launch refused: fall back to one block
  }
  const size_t ne = (size_t)n2 * n2;
  const size_t full = (2 + 2 * (size_t)nk) * ne * sizeof(T);
  const int preload = full <= 200 * 1024 ? 1 : 0;
  const size_t smem = preload ? full : 3 * ne * sizeof(T);
  if (n2 <= 64) {
    const int nb = n2 / 2;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(sstep_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    sstep_kernel<T, 2><<<1, nb * nb, smem, st>>>(Gh, Ph, nk, S, RB, n2, beta, nsub, preload, Sh);
  } else {
    const int nb = n2 / 4;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(sstep_kernel<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    sstep_kernel<T, 4><<<1, nb * nb, smem, st>>>(Gh, Ph, nk, S, RB, n2, beta, nsub, preload, Sh);
  }
}
template void launch_sstep<float>(cudaStream_t, const double*, const double*, int, const double*, int, int,
                                  const double*, int, double*, const SstepWork*, int*);
template void launch_sstep<double>(cudaStream_t, const double*, const double*, int, const double*, int, int,
                                   const double*, int, double*, const SstepWork*, int*);

// co-resident blocks of the grid-parallel S-step kernel on the current device
int sstep_grid_capacity(size_t tsize) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cudaError_t e = tsize == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sstep_grid_kernel<float>, 256, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sstep_grid_kernel<double>, 256, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * per;
}

// ---------------------------------------------------------------------------
// implicit-Euler collided L-step: one block per degree l
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) scatter_solve_kernel(const double* __restrict__ Mg, int M, const double* __restrict__ coef, int N,
                                     const double* __restrict__ S, const T* __restrict__ W, int m, int RB,
                                     T* __restrict__ L1T, int* err) {
  extern __shared__ double sh[];
  const int l = blockIdx.x;
  const int nr = 2 * l + 1, p0 = l * l;
  double* A = sh;              // RB x RB, col-major
  double* X = A + RB * RB;     // RB x nr right-hand sides / solutions
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < RB * RB; e += nt) {
    int a = e % RB, b = e / RB;
    double v = (a == b) ? 1.0 : 0.0;
    for (int i = 0; i < M; ++i) v -= coef[i * (N + 1) + l] * Mg[((long long)i * RB + b) * RB + a];
    A[e] = v;
  }
  for (int e = tid; e < RB * nr; e += nt) {
    int a = e % RB, pp = e / RB;
    double v = 0.0;
    for (int j = 0; j < RB; ++j) v += S[j * RB + a] * (double)W[(long long)j * m + p0 + pp];
    X[e] = v;
  }
  __syncthreads();
  // Cholesky A = L L^T (lower part)
  for (int j = 0; j < RB; ++j) {
    if (tid == 0) {
      double d = A[j * RB + j];
      if (!(d > 0.0)) {
        atomicOr(err, ERR_CHOLESKY);
        d = 1.0;
      }
      A[j * RB + j] = sqrt(d);
    }
    __syncthreads();
    const double djj = A[j * RB + j];
    for (int i = j + 1 + tid; i < RB; i += nt) A[j * RB + i] /= djj;
    __syncthreads();
    const int w = RB - j - 1;
    for (int e = tid; e < w * w; e += nt) {
      int i = j + 1 + e % w, k = j + 1 + e / w;
      if (k <= i) A[k * RB + i] -= A[j * RB + i] * A[j * RB + k];
    }
    __syncthreads();
  }
  // forward substitution L y = x, all right-hand sides at once
  for (int j = 0; j < RB; ++j) {
    for (int pp = tid; pp < nr; pp += nt) X[pp * RB + j] /= A[j * RB + j];
    __syncthreads();
    for (int e = tid; e < (RB - j - 1) * nr; e += nt) {
      int i = j + 1 + e % (RB - j - 1), pp = e / (RB - j - 1);
      X[pp * RB + i] -= A[j * RB + i] * X[pp * RB + j];
    }
    __syncthreads();
  }
  // backward substitution L^T x = y
  for (int j = RB - 1; j >= 0; --j) {
    for (int pp = tid; pp < nr; pp += nt) X[pp * RB + j] /= A[j * RB + j];
    __syncthreads();
    for (int e = tid; e < j * nr; e += nt) {
      int i = e % j, pp = e / j;
      X[pp * RB + i] -= A[i * RB + j] * X[pp * RB + j];
    }
    __syncthreads();
  }
  for (int e = tid; e < RB * nr; e += nt) {
    int a = e % RB, pp = e / RB;
    L1T[(long long)a * m + p0 + pp] = T(X[e]);
  }
}

template <typename T>
void launch_scatter_solve(cudaStream_t st, const double* Mg, int M, const double* coef, int N, const double* S,
                          const T* W, int m, int RB, T* L1T, int* err) {
  size_t smem = (size_t)(RB * RB + RB * (2 * N + 1)) * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(scatter_solve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  scatter_solve_kernel<T><<<N + 1, 256, smem, st>>>(Mg, M, coef, N, S, W, m, RB, L1T, err);
}
template void launch_scatter_solve<float>(cudaStream_t, const double*, int, const double*, int, const double*,
                                          const float*, int, int, float*, int*);
template void launch_scatter_solve<double>(cudaStream_t, const double*, int, const double*, int, const double*,
                                           const double*, int, int, double*, int*);

// ---------------------------------------------------------------------------
// Householder QR of L1T (m x r): L1T = Wt R, S = R^T
// ---------------------------------------------------------------------------
// CT is the arithmetic type. With gwork == nullptr (CT == T) the matrix is held in shared
// memory and Q is built in place in Wt; with gwork (2 m RB values of CT, global memory) both
// the matrix and Q live there and Q is rounded to T at the end: the FP64 QR of FP32 data, whose
// m x RB FP64 matrix does not fit in shared memory for m = 484.
template <typename T, typename CT>
__global__ void __launch_bounds__(512) qr_lt_kernel(const T* __restrict__ L1T, int m, int RB, const BeamDims* __restrict__ dims,
                             T* __restrict__ Wt, double* __restrict__ S, CT* __restrict__ gwork) {
  extern __shared__ __align__(16) unsigned char raw[];
  CT* A = gwork ? gwork : reinterpret_cast<CT*>(raw);   // m x RB col-major; reflectors below the diagonal
  __shared__ CT red[32];
  __shared__ CT rdiag[64], v0s[64], vn2[64];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  int r = dims->r;
  if (r > RB) r = RB;
  if (r > m) r = m;
  for (int e = tid; e < m * RB; e += nt) A[e] = CT(L1T[e]);
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    CT part = 0;
    for (int i = j + tid; i < m; i += nt) part += A[j * m + i] * A[j * m + i];
    CT nrm2 = block_sum(part, red);
    CT x0 = A[j * m + j];
    CT nrm = sqrt(nrm2);
    CT alpha = (x0 >= CT(0)) ? -nrm : nrm;
    CT v0 = x0 - alpha;
    CT vnorm2 = nrm2 - x0 * x0 + v0 * v0;
    __syncthreads();
    if (tid == 0) {
      rdiag[j] = (nrm2 > CT(0)) ? alpha : CT(0);
      v0s[j] = v0;
      vn2[j] = (nrm2 > CT(0)) ? vnorm2 : CT(0);
      A[j * m + j] = v0;  // reflector v = (v0, A[j+1:, j])
    }
    __syncthreads();
    if (vn2[j] > CT(0)) {
      for (int c = j + 1 + wid; c < r; c += nw) {
        CT d = 0;
        for (int i = j + lane; i < m; i += 32) d += A[j * m + i] * A[c * m + i];
        d = warp_sum(d);
        CT f = CT(2) * d / vn2[j];
        for (int i = j + lane; i < m; i += 32) A[c * m + i] -= f * A[j * m + i];
      }
    }
    __syncthreads();
  }
  // S = R^T: R[j][j] = rdiag[j], R[j][c] = A[c*m + j] for c > j
  for (int e = tid; e < RB * RB; e += nt) {
    int a = e % RB, c = e / RB;  // S[a][c] = R[c][a]
    double v = 0.0;
    if (a < r && c < r) {
      if (a == c) v = (double)rdiag[c];
      else if (a > c) v = (double)A[a * m + c];
    }
    S[e] = v;
  }
  __syncthreads();
  // Q = H_0 ... H_{r-1} applied to the first r identity columns
  CT* Q;
  if constexpr (std::is_same<CT, T>::value) Q = gwork ? gwork + (size_t)m * RB : Wt;
  else Q = (gwork ? gwork : A) + (size_t)m * RB;   // FP64 Q after the matrix (global or shared)
  for (int e = tid; e < m * RB; e += nt) {
    int i = e % m, c = e / m;
    Q[e] = (c < r && i == c) ? CT(1) : CT(0);
  }
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    if (!(vn2[j] > CT(0))) continue;
    for (int c = j + wid; c < r; c += nw) {
      CT d = 0;
      for (int i = j + lane; i < m; i += 32) d += A[j * m + i] * Q[(long long)c * m + i];
      d = warp_sum(d);
      CT f = CT(2) * d / vn2[j];
      for (int i = j + lane; i < m; i += 32) Q[(long long)c * m + i] -= f * A[j * m + i];
    }
    __syncthreads();
  }
  if (!std::is_same<CT, T>::value || gwork)
    for (int e = tid; e < m * RB; e += nt) Wt[e] = T(Q[e]);
}

template <typename T>
void launch_qr_lt(cudaStream_t st, const T* L1T, int m, int RB, const BeamDims* dims, T* Wt, double* S,
                  double* gwork) {
  if (gwork && sizeof(T) == 4) {
    // FP64 arithmetic: the matrix and Q in shared memory when both fit, else in gwork
    const size_t smem64 = (size_t)2 * m * RB * sizeof(double);
    if (smem64 <= 200 * 1024) {
      cudaFuncSetAttribute(qr_lt_kernel<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
      qr_lt_kernel<T, double><<<1, 512, smem64, st>>>(L1T, m, RB, dims, Wt, S, nullptr);
    } else {
      qr_lt_kernel<T, double><<<1, 512, 0, st>>>(L1T, m, RB, dims, Wt, S, gwork);
    }
    return;
  }
  size_t smem = (size_t)m * RB * sizeof(T);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(qr_lt_kernel<T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  qr_lt_kernel<T, T><<<1, 512, smem, st>>>(L1T, m, RB, dims, Wt, S, nullptr);
}
template void launch_qr_lt<float>(cudaStream_t, const float*, int, int, const BeamDims*, float*, double*, double*);
template void launch_qr_lt<double>(cudaStream_t, const double*, int, int, const BeamDims*, double*, double*, double*);

// ---------------------------------------------------------------------------
// W-side augmentation: pivoted Gram-Schmidt with re-orthogonalisation
// ---------------------------------------------------------------------------
// CT is the arithmetic type. With gwork == nullptr (CT == T) the residuals R and projections G
// are in shared memory and the accepted directions are written in place into Wh; with gwork
// (global memory, waug_work_size values of CT) R, G and the accepted directions U live there
// and U is rounded to T at the end (the FP64 orthogonalisation of FP32 data).
template <typename T, typename KT, typename CT>
__global__ void __launch_bounds__(512) waug_kernel(const T* __restrict__ W, int m, int RB, const KT* __restrict__ K, long long ldk, int qcap,
                            double drop_tol, T* __restrict__ Wh, BeamDims* dims, CT* __restrict__ gwork) {
  extern __shared__ __align__(16) unsigned char raw[];
  CT* R = gwork ? gwork : reinterpret_cast<CT*>(raw);   // m x qcap
  CT* G = R + (size_t)m * qcap;        // RB x qcap projections W^T R; then the r + q projections of u
  CT* U;                               // accepted new directions
  if constexpr (std::is_same<CT, T>::value)
    U = gwork ? G + (size_t)max(RB * qcap, RB + qcap) : Wh + (long long)RB * m;
  else
    U = G + (size_t)max(RB * qcap, RB + qcap);
  __shared__ CT red[32];
  __shared__ CT cn[64];
  __shared__ int used[64];
  __shared__ int s_best;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int r = dims->r < RB ? dims->r : RB;
  for (int e = tid; e < m * 2 * RB; e += nt) {
    int i = e % m, c = e / m;
    Wh[e] = (c < RB) ? W[(long long)c * m + i] : T(0);
  }
  CT part = 0;
  for (int e = tid; e < m * qcap; e += nt) {
    int i = e % m, c = e / m;
    CT v = CT(K[(long long)c * ldk + i]);
    R[e] = v;
    part += v * v;
  }
  for (int c = tid; c < qcap; c += nt) used[c] = 0;
  const CT scale2 = block_sum(part, red);
  const CT thr = CT(drop_tol * drop_tol) * scale2;
  // two passes of R -= W (W^T R) (classical Gram-Schmidt twice): all r qcap projections at
  // once over the warps, then one fused update per element
  for (int pass = 0; pass < 2; ++pass) {
    __syncthreads();
    for (int e = wid; e < r * qcap; e += nw) {
      const int a = e % r, c = e / r;
      CT d = 0;
      for (int i = lane; i < m; i += 32) d += CT(W[(long long)a * m + i]) * R[c * m + i];
      d = warp_sum(d);
      if (lane == 0) G[c * RB + a] = d;
    }
    __syncthreads();
    for (int e = tid; e < m * qcap; e += nt) {
      const int i = e % m, c = e / m;
      CT v = R[e];
      for (int a = 0; a < r; ++a) v -= G[c * RB + a] * CT(W[(long long)a * m + i]);
      R[e] = v;
    }
  }
  __syncthreads();
  int q = 0;
  for (int it = 0; it < qcap; ++it) {
    for (int c = wid; c < qcap; c += nw) {
      CT d = 0;
      for (int i = lane; i < m; i += 32) d += R[c * m + i] * R[c * m + i];
      d = warp_sum(d);
      if (lane == 0) cn[c] = used[c] ? CT(-1) : d;
    }
    __syncthreads();
    if (tid == 0) {
      int b = -1;
      CT bv = thr;
      for (int c = 0; c < qcap; ++c)
        if (cn[c] > bv) { bv = cn[c]; b = c; }
      s_best = b;
      if (b >= 0) used[b] = 1;
    }
    __syncthreads();
    const int b = s_best;
    if (b < 0) break;
    // u = R[:, b] re-orthogonalised against W and the accepted directions (one classical
    // Gram-Schmidt pass over all warps, R being orthogonal to both up to round-off already),
    // normalised
    CT* u = U + q * m;
    for (int i = tid; i < m; i += nt) u[i] = R[b * m + i];
    __syncthreads();
    for (int a = wid; a < r + q; a += nw) {
      CT d = 0;
      if (a < r)
        for (int i = lane; i < m; i += 32) d += CT(W[(long long)a * m + i]) * u[i];
      else
        for (int i = lane; i < m; i += 32) d += U[(long long)(a - r) * m + i] * u[i];
      d = warp_sum(d);
      if (lane == 0) G[a] = d;
    }
    __syncthreads();
    CT part2 = 0;
    for (int i = tid; i < m; i += nt) {
      CT x = u[i];
      for (int a = 0; a < r; ++a) x -= G[a] * CT(W[(long long)a * m + i]);
      for (int a = 0; a < q; ++a) x -= G[r + a] * U[(long long)a * m + i];
      u[i] = x;
      part2 += x * x;
    }
    const CT n2 = block_sum(part2, red);
    const CT inv = n2 > CT(0) ? CT(1) / sqrt(n2) : CT(0);
    for (int i = tid; i < m; i += nt) u[i] *= inv;
    __syncthreads();
    // remove u from the remaining columns
    for (int c = wid; c < qcap; c += nw) {
      if (used[c]) continue;
      CT d = 0;
      for (int i = lane; i < m; i += 32) d += u[i] * R[c * m + i];
      d = warp_sum(d);
      for (int i = lane; i < m; i += 32) R[c * m + i] -= d * u[i];
    }
    ++q;
    __syncthreads();
  }
  if (gwork)
    for (int e = tid; e < m * q; e += nt) Wh[(long long)RB * m + e] = T(U[e]);
  if (tid == 0) dims->qw = q;
}

template <typename T, typename KT>
void launch_waug(cudaStream_t st, const T* W, int m, int RB, const KT* K, long long ldk, int qcap, double drop_tol,
                 T* Wh, BeamDims* dims, double* gwork) {
  if (gwork && sizeof(T) == 4) {
    waug_kernel<T, KT, double><<<1, 512, 0, st>>>(W, m, RB, K, ldk, qcap, drop_tol, Wh, dims, gwork);
    return;
  }
  // R (m x qcap) and the projections (RB x qcap; >= RB + qcap for those of one direction)
  const size_t smem = ((size_t)m * qcap + (size_t)std::max(RB * qcap, RB + qcap)) * sizeof(T);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(waug_kernel<T, KT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  waug_kernel<T, KT, T><<<1, 512, smem, st>>>(W, m, RB, K, ldk, qcap, drop_tol, Wh, dims, nullptr);
}
template void launch_waug<float, float>(cudaStream_t, const float*, int, int, const float*, long long, int, double,
                                        float*, BeamDims*, double*);
template void launch_waug<float, double>(cudaStream_t, const float*, int, int, const double*, long long, int, double,
                                         float*, BeamDims*, double*);
template void launch_waug<double, double>(cudaStream_t, const double*, int, int, const double*, long long, int,
                                          double, double*, BeamDims*, double*);

// ---------------------------------------------------------------------------
// source S assembly
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) src_assemble_kernel(const double* __restrict__ S, int RB, const double* __restrict__ XA,
                                    const double* __restrict__ B, const T* __restrict__ Wh, int m, int M, int n2,
                                    double h, double* __restrict__ Sh) {
  extern __shared__ double bw[];  // M x n2: (B^T Wh)[i][c]
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < M * n2; e += nt) {
    int i = e % M, c = e / M;
    double v = 0.0;
    for (int p = 0; p < m; ++p) v += B[(long long)i * m + p] * (double)Wh[(long long)c * m + p];
    bw[e] = v;
  }
  __syncthreads();
  for (int e = tid; e < n2 * n2; e += nt) {
    int a = e % n2, c = e / n2;
    double v = (a < RB && c < RB) ? S[c * RB + a] : 0.0;
    for (int i = 0; i < M; ++i) v += h * XA[(long long)i * n2 + a] * bw[c * M + i];
    Sh[e] = v;
  }
}

template <typename T>
void launch_src_assemble(cudaStream_t st, const double* S, int RB, const double* XA, const double* B, const T* Wh,
                         int m, int M, int n2, double h, double* Sh) {
  size_t smem = (size_t)M * n2 * sizeof(double);
  src_assemble_kernel<T><<<1, 512, smem, st>>>(S, RB, XA, B, Wh, m, M, n2, h, Sh);
}
template void launch_src_assemble<float>(cudaStream_t, const double*, int, const double*, const double*, const float*,
                                         int, int, int, double, double*);
template void launch_src_assemble<double>(cudaStream_t, const double*, int, const double*, const double*,
                                          const double*, int, int, int, double, double*);

}  // namespace dlra
