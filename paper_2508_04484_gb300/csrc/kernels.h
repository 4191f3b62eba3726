// Launch wrappers of the small dense (one thread block) kernels and the ray tracer.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dlra {

// Device scalars of one low-rank state.
struct BeamDims {
  int r;     // rank of X, S, W
  int qx;    // new X-side directions of the last augmentation
  int qw;    // new W-side directions of the last augmentation
  int pad;
};

enum ErrBits { ERR_NONFINITE = 1, ERR_CHOLESKY = 2, ERR_CAPACITY = 4, ERR_TIMEOUT = 8 };

struct RankParams {
  int mode;          // 0 fixed, 1 adaptive, 2 schedule
  int rank;          // fixed rank
  int rank_max;      // capacity / adaptive maximum
  double tol;        // adaptive relative tolerance
  double nz_tol;     // numerically zero singular values (relative to sigma_1)
  double cluster_tol;
  const int* schedule;  // device [K][2] or nullptr
};

// Pivoted-Cholesky orthonormalisation factor (one block). G has ld = RBa + qcap and
// columns j < qcap holding [Xa^T R ; R^T R](:, j). C1 (RBa x qcap, ld RBa) is the
// first-pass projection used for the scale (nullptr: scale = trace of R^T R).
// Writes Mout ((RBa + qcap) x qcap, ld RBa + qcap) = [-C2 T ; T] and *qout.
void launch_orth_factor(cudaStream_t st, const double* G, const double* C1, int RBa, int qcap, double drop_tol,
                        double* Mout, int* qout, int* err);

// Truncated SVD of Sh (n2 x n2, ld n2, FP64) by one-sided Jacobi in precision T;
// writes P, Q (n2 x RB, ld n2), S (RB x RB, ld RB), dims->r, rank_log[2*step + event].
// vwork (n2 x n2 values of T, global memory): holds the right rotations when the two
// n2 x n2 matrices do not fit shared memory together (FP64 at n2 = 128); required then.
template <typename T>
void launch_svd_truncate(cudaStream_t st, const double* Sh, int n2, int RB, RankParams rp, int step, int event,
                         double* P, double* Q, double* S, BeamDims* dims, int* rank_log, int* err,
                         void* vwork = nullptr);

// true when launch_svd_truncate<T> at this size needs vwork
inline bool svd_needs_vwork(int n2, size_t tsize) { return 2 * (size_t)n2 * n2 * tsize > 200 * 1024; }

// Work space of the grid-parallel S-step (global memory, one per lane): the stage input z
// (n2 x n2), the products U_k = z P_k and the partial outputs O_k = G_k U_k (nk x n2 x n2 each),
// all in the arithmetic type; three barrier words (arrivals, generation, abort), zeroed once;
// grid = the lane's share of the co-resident blocks (cooperative launch).
struct SstepWork {
  void *z = nullptr, *U = nullptr, *O = nullptr;
  unsigned* bar = nullptr;
  int grid = 0;
};

// Galerkin S-step (Sec. 2.2, Eq. KLS) with RK4 in Horner form: Sh (n2 x n2) starts at
// [[S, 0], [0, 0]] and is advanced by nsub sub-steps with beta[4*j + 0..3];
// operator S -> sum_k Gh_k S Ph_k, Gh and Ph laid out [(k*n2 + b)*n2 + a]. On a cluster of
// eight blocks where its operators fit their shared memory; otherwise, with gw, on the whole
// grid (cooperative launch, bounded barriers that set ERR_TIMEOUT in err when they run out);
// without gw on one block.
template <typename T>
void launch_sstep(cudaStream_t st, const double* Gh, const double* Ph, int nk, const double* S, int RB, int n2,
                  const double* beta, int nsub, double* Sh, const SstepWork* gw = nullptr, int* err = nullptr);

// doubles of global work space of the grid-parallel S-step for arithmetic type of size tsize
inline size_t sstep_grid_bytes(int nk, int n2, size_t tsize) {
  return (1 + 2 * (size_t)nk) * (size_t)n2 * n2 * tsize;
}

// true when the S-step of this size needs the grid-parallel kernel (the cluster kernel's
// operators do not fit its shared memory)
bool sstep_needs_grid(int nk, int n2, size_t tsize);

// blocks of the grid-parallel S-step that fit the current device at once (0 on error)
int sstep_grid_capacity(size_t tsize);

// Implicit-Euler collided L-step (Sec. 3.3.3 step 1): per degree l solves
// (I - sum_i coef[i*(N+1)+l] Mg_i) x = S W[p,:]^T for every moment p of degree l;
// writes L1T (m x RB, ld m) in precision T. Mg_i at [(i*RB + b)*RB + a].
template <typename T>
void launch_scatter_solve(cudaStream_t st, const double* Mg, int M, const double* coef, int N, const double* S,
                          const T* W, int m, int RB, T* L1T, int* err);

// Householder QR of L1T (m x r): L1T = Wt R; writes Wt (m x RB, zero beyond r) and S = R^T.
// gwork (FP32 data only): 2 m RB doubles of global work space; the QR then runs in FP64
// arithmetic (in shared memory where the FP64 matrix and Q fit, else in gwork) and Wt is
// rounded to FP32 at the end. nullptr: arithmetic in T, shared memory.
template <typename T>
void launch_qr_lt(cudaStream_t st, const T* L1T, int m, int RB, const BeamDims* dims, T* Wt, double* S,
                  double* gwork = nullptr);

// W-side augmentation (one block): Wh = [W | orth((I - W W^T) K)], K m x qcap of type KT,
// rank-revealing with pivoted Gram-Schmidt (drop below drop_tol ||K||_F); writes dims->qw.
// gwork (FP32 data only): mside_work_doubles(m, RB) doubles of global work space; the
// orthogonalisation then runs in FP64 arithmetic and the new columns are rounded to FP32.
template <typename T, typename KT>
void launch_waug(cudaStream_t st, const T* W, int m, int RB, const KT* K, long long ldk, int qcap, double drop_tol,
                 T* Wh, BeamDims* dims, double* gwork = nullptr);

// doubles of global work space for the FP64 m-side factorisations (launch_qr_lt, launch_waug
// with qcap <= RB)
inline size_t mside_work_doubles(int m, int RB) {
  return 2 * (size_t)m * RB + (size_t)RB * RB + 2 * (size_t)RB;
}

// Source S assembly: Sh (n2 x n2) = [[S, 0], [0, 0]] + h XA (B^T Wh), XA (n2 x M, ld n2),
// B (m x M, ld m, FP64), Wh (m x n2).
template <typename T>
void launch_src_assemble(cudaStream_t st, const double* S, int RB, const double* XA, const double* B, const T* Wh,
                         int m, int M, int n2, double h, double* Sh);

// CSDA ray tracer (Sec. 3.2): rays [nray][8] = (ox, oy, oz, vx, vy, vz, E0, weight).
struct RayGeo {
  int nx, ny, nz, two_d, K;
  double dx, dy, dz, e_max, h, e_min, p, alpha, klam, volume;
};
void launch_raytrace(cudaStream_t st, const double* rays, int nray, RayGeo g, const double* f_cell,
                     const double* tau_cell, double* psi, double* e_u);

// Reverse-mode derivative of the ray tracer: for adjoint seeds gpsi (K x n) and geu (n),
// adds dL/df(x) and dL/dtau(x) (stopping factor, removal factor) to grad_f and grad_tau.
// scratch: raytrace_adjoint_scratch_bytes (the recorded voxel segments of every ray).
size_t raytrace_adjoint_scratch_bytes(int nray, RayGeo g);
void launch_raytrace_adjoint(cudaStream_t st, const double* rays, int nray, RayGeo g, const double* f_cell,
                             const double* tau_cell, const double* gpsi, const double* geu, void* scratch,
                             double* grad_f, double* grad_tau);

// Gradient kernels of the reverse sweep (adjoint.cu). Tall arrays n x RB, ld n; RB is a
// compiled rank capacity.
// grad_rho -= coef sum_q vq_q C lq_q^T row by row (nq stage pairs, stride n RB; C RB x RB).
template <typename T>
void launch_grad_stream(cudaStream_t st, const T* vq, const T* lq, int nq, long long n, int RB, const double* C,
                        double coef, double* grad_rho);
// Cl[l] = Sa (Wa[l]^T Wb[l]) Sb^T per degree l = 0..N (W of type float or double).
void launch_scatter_cl(cudaStream_t st, const double* Sa, const void* Wa, const double* Sb, const void* Wb, int fp64,
                       int m, int N, int RB, double* Cl);
// dL/dw_i and dL/d rho_s of the implicit scattering factor from D(x, l) = Xa(x,:) Cl[l] Xb(x,:)^T.
template <typename T>
void launch_grad_scatter(cudaStream_t st, const T* Xa, const T* Xb, long long n, int RB, const double* Cl, int N,
                         const double* coef, int M, const T* wc, const double* rho_s, double beta, double* grad_w,
                         double* grad_rho);
// Source term of one beam: dL/dw_i += bh psi mu.B_i and gpsi = bh sum_i w_i mu.B_i, mu = X S W^T.
template <typename T>
void launch_grad_source(cudaStream_t st, const T* X, const double* S, const T* W, long long n, int m, int RB,
                        const double* B, int M, const double* psi, const T* w, double bh, double* ysrc,
                        double* grad_w, double* gpsi);
// out[i][x] = grad_w[i][x] + mcoef[2i] (grad_rho + grad_f)[x] + mcoef[2i+1] grad_tau[x]
void launch_grad_assemble(cudaStream_t st, const double* grad_w, const double* grad_rho, const double* grad_f,
                          const double* grad_tau, const double* mcoef, int M, long long n, double* out);
// *out += sum_x g[x] (a[x] + b[x])
void launch_dot(cudaStream_t st, const double* g, const double* a, const double* b, long long n, double* out);
// transpose each of nk column-major n2 x n2 blocks in place
void launch_transpose_blocks(cudaStream_t st, double* G, int n2, int nk);

// Stencil Gram on the tensor cores (FP32): out[(k ldj + b) ldo + a] += sum_i A(i, a)
// D_k(rho^-1 B(:, b))(i) for a < dim(adim, na), b < dim(bdim, nb); out accumulates (FP64
// atomics). Needs na <= 128 and rows < 2^31 (gram_stencil_tc_supported). A wait that runs out
// sets ERR_TIMEOUT in *err and leaves out without this launch's terms.
struct Geo;
bool gram_stencil_tc_supported(int na, long long rows);
void launch_gram_stencil_tc(cudaStream_t st, long long rows, const float* A, long long lda, int na, const int* adim,
                            const float* B, long long ldb, int nb, const int* bdim, const float* inv_rho,
                            const Geo& g, double* out, int ldj, long long ldo, int waves_x2, int* err);

// The same Gram with A == B on a 3-D grid, its inputs staged by TMA in a window that slides
// along each stencil's axis and the stencil operand written into tensor memory (gram_win.cu).
// Needs na == nb <= 128, adim == bdim, nx and lda multiples of 4, 16-byte aligned A and
// inv_rho; returns false (nothing launched) otherwise.
bool launch_gram_stencil_win(cudaStream_t st, long long rows, const float* A, long long lda, int na,
                             const int* adim, const float* B, long long ldb, int nb, const int* bdim,
                             const float* inv_rho, const Geo& g, double* out, int ldj, long long ldo, int* err);
// Tall-skinny Gram on the tensor cores (gram_tt.cu): out[j ldo + a] += sum_t A(t, a) F(t, j) for
// a < dim(adim, acap), j < ncols, with F(t, j) = B(t, j) (nbw == 0, j < dim(jdim, jcap)) or
// F(t, k nbw + b) = wv[k rows + t] B(t, b) (k < nk, b < dim(jdim, jcap)). Needs acap <= 128,
// rows < 2^31, lda, ldb multiples of 4 and 16-byte aligned bases (and nbw <= 64, nk <= 8 for
// the weighted form); returns false (nothing launched) otherwise. A wait that runs out sets
// ERR_TIMEOUT in *err and leaves out without this launch's terms.
bool launch_gram_tt(cudaStream_t st, long long rows, const float* A, long long lda, const int* adim, int acap,
                    const float* B, long long ldb, const int* jdim, int jcap, int ncols, const float* wv, int nbw,
                    int nk, double* out, long long ldo, int* err);
// cuTensorMapEncodeTiled from the driver (nullptr where it cannot be had)
PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn();

// Work-space bytes of one stand-alone K-step (see dlra_kstep) and the step itself on
// caller-provided device work space of at least that many bytes.
size_t kstep_scratch_bytes(long long n, int r, int nact, int stage_kernel);
int run_kstep(const void* args, void* scratch, size_t scratch_bytes, char* msg, int msg_len);

}  // namespace dlra
