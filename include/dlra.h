/*
 * dlra.h -- C ABI of the GB300 low-rank collided-proton transport library.
 *
 * The library advances the collided proton flux of arXiv 2508.04484 in energy
 * (pseudo-time t = E_max - E, Sec. 3.3) as a rank-r factorisation
 * u = X S W^T (Sec. 2.2) of its real spherical-harmonic moments (Sec. 3.3.1) on a
 * uniform voxel grid (Sec. 3.3.2). One energy step is the Lie split of Sec. 3.3.3:
 * streaming by the augmented BUG integrator with RK4 time updates, collided
 * self-scattering by an implicit-Euler L-step, and the first-collision source of
 * a CSDA ray tracer (Sec. 3.2) by augmented BUG K/L/S steps with explicit Euler.
 *
 * Units: cm, MeV, g/cm^3. Each beam is solved at unit weight (one source proton)
 * and enters the dose times its weight; 2-D slabs (ny == 1, dy == 0) are per unit
 * length in y.
 *
 * Conventions for every entry point:
 *  - All functions return a dlra_status; no exception crosses the ABI.
 *  - Host pointers are read or written during the call only; the caller keeps
 *    ownership. "on_device" arguments say a pointer is device memory of the
 *    context's GPU; device pointers must be ordered with the context's stream.
 *  - Matrices are dense; "column-major" means element (i, j) of an R x C matrix
 *    is at [j * R + i].
 *  - After DLRA_ERR_CUDA, DLRA_ERR_NONFINITE or DLRA_ERR_TIMEOUT the context is
 *    poisoned: every later call returns the same status until dlra_destroy.
 *  - A context is used by one host thread at a time; contexts are independent.
 *  - dlra_last_error gives a one-line description of the last failure.
 */
#ifndef DLRA_H
#define DLRA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dlra_ctx dlra_ctx;

typedef enum {
  DLRA_OK = 0,
  DLRA_ERR_ARG = 1,       /* invalid argument (size, pointer, value)          */
  DLRA_ERR_STATE = 2,     /* call out of order (e.g. dlra_step before a beam) */
  DLRA_ERR_CUDA = 3,      /* a CUDA runtime call or kernel failed             */
  DLRA_ERR_OOM = 4,       /* device allocation failed                         */
  DLRA_ERR_NONFINITE = 5, /* the low-rank state became non-finite             */
  DLRA_ERR_RANK = 6,      /* rank bookkeeping failed (capacity exceeded)      */
  DLRA_ERR_TIMEOUT = 7    /* a bounded device-side wait gave up               */
} dlra_status;

enum { DLRA_FOKKER_PLANCK = 0, DLRA_BOLTZMANN = 1 };
enum { DLRA_RANK_FIXED = 0, DLRA_RANK_ADAPTIVE = 1, DLRA_RANK_SCHEDULE = 2 };
enum { DLRA_FP64 = 0, DLRA_FP32_MIXED = 1, DLRA_FP32_SPLIT = 2 };

/* Problem configuration (Sec. 3.3, Sec. 4).
 *  nx, ny, nz, dx, dy, dz : voxel grid, cell index (k*ny + j)*nx + i (Sec. 3.3.2).
 *                           ny == 1 && dy == 0 selects a 2-D x-z slab (no y streaming).
 *  sh_degree              : N, m = (N+1)^2 moments (Sec. 3.3.1); 1 <= N <= 31.
 *  collision              : DLRA_FOKKER_PLANCK or DLRA_BOLTZMANN (Sec. 2.1).
 *  transport_correction   : 1 = extended transport correction of the Boltzmann
 *                           moments, sigma_l - sigma_{N+1} (Sec. 3.3.1); 2 = the same
 *                           and, for Fokker-Planck, the delta-function corrected
 *                           moments of Landesman and Morel (Sec. 3.3.1): G_l =
 *                           (xi_1/2) [(N+1)(N+2) - l(l+1)], Sigma_t = G_0 (the uncollided
 *                           beam is then removed into the collided source); 0 = none.
 *  rank_mode, rank,       : truncation (Sec. 2.2). FIXED keeps min(rank, numerical rank);
 *  rank_max, trunc_tol      ADAPTIVE keeps the smallest r with sum_{i>r} sigma_i <=
 *                           trunc_tol * ||sigma||_2 clamped to [1, rank_max]; SCHEDULE
 *                           replays rank_schedule. rank_max (<= 64) is the capacity.
 *  rank_schedule          : SCHEDULE only; host array [n_energy_steps][2] of ranks after
 *                           the streaming and the source truncation (-1 = none), copied
 *                           by dlra_init.
 *  e_max, e_min,          : uniform energy grid E_k = e_max - k dE (Sec. 3.3).
 *  n_energy_steps
 *  cfl_max                : streaming RK4 sub-steps per energy step are
 *                           ceil(dE sum_d lam_max/delta_d / (min_x S(x,E_k) cfl_max)).
 *  precision              : DLRA_FP64, or DLRA_FP32_MIXED (FP32 n-side data and
 *                           arithmetic, FP64 reductions, factorisations and S), or
 *                           DLRA_FP32_SPLIT (as DLRA_FP32_MIXED with the 2r x 2r
 *                           truncation SVD, the Galerkin S-step, the Householder QR of
 *                           the collided L-step and the W-side augmentation in FP64
 *                           arithmetic; W is stored in FP32).
 *  bk_p, bk_alpha         : Bragg-Kleeman water stopping power S_w(E) = E^(1-p)/(p alpha).
 *  t100                   : water scattering power at 100 MeV, T_w(E) = t100 (100/E)^2.
 *  max_concurrent_beams   : beams advanced concurrently (one work space and stream pair
 *                           each; 0 = 8, 1 = one beam after the other).
 *  cuda_stream            : borrowed cudaStream_t; every call orders its work after what
 *                           is already enqueued on it. NULL = legacy default stream.
 */
typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;
  int32_t sh_degree;
  int32_t collision;
  int32_t transport_correction;
  int32_t rank_mode, rank, rank_max;
  double trunc_tol;
  const int32_t* rank_schedule;
  double e_max, e_min;
  int32_t n_energy_steps;
  double cfl_max;
  int32_t precision;
  double bk_p, bk_alpha, t100;
  int32_t max_concurrent_beams;
  void* cuda_stream;
} dlra_config;

/* Base material of the mixture (Sec. 2.1, Eq. mixXS): density and ratios to water
 * of the mass stopping power and mass scattering power, and the screening
 * parameter eta of its screened-Rutherford kernel C/(1 - mu + 2 eta)^2. */
typedef struct {
  double density, sp_ratio, scatter_ratio, screening;
} dlra_material;

/* Pencil beam (Sec. 4): mean energy and Gaussian energy spread (MeV), a point on
 * its axis and its direction, Gaussian spot sigma (cm) perpendicular to it, weight. */
typedef struct {
  double energy, energy_sigma;
  double pos[3], dir[3];
  double spot_sigma, weight;
} dlra_beam;

/* Create a context: validates cfg, builds the angular tables (A_x, A_y, A_z and
 * |A_d|, Sec. 3.3.1-3.3.2) and allocates the low-rank state at capacity rank_max.
 * *out receives the context; nothing is launched yet. */
dlra_status dlra_init(const dlra_config* cfg, dlra_ctx** out);

/* Set the mixture (Sec. 2.1): n_mat base materials and weights w [n_mat][n] (cell
 * order of Sec. 3.3.2), w_m(x) >= 0 summing to 1 per cell. w may be host or device
 * memory (w_on_device); it is copied. Computes the per-step physics tables and the
 * streaming sub-step counts. Must precede dlra_add_beam. May be called again with the
 * same n_mat (new materials and weights): every beam is then retraced and rewound to
 * E_max as by dlra_reset(ctx, 1). */
dlra_status dlra_set_materials(dlra_ctx* ctx, int32_t n_mat, const dlra_material* mats,
                               const double* w, int32_t w_on_device);

/* Add a beam (independent low-rank state per beam): runs the CSDA ray tracer on
 * the GPU (Sec. 3.2) for the bin-averaged uncollided fluence of every energy bin
 * and the uncollided energy deposit. *beam_id receives its index. Must precede
 * the first dlra_step. */
dlra_status dlra_add_beam(dlra_ctx* ctx, const dlra_beam* beam, int32_t* beam_id);

/* Advance every beam by n_steps energy steps (Sec. 3.3.3), enqueued on the
 * context's stream; returns after enqueueing unless an error is already latched.
 * Fails with DLRA_ERR_STATE past the last energy step. */
dlra_status dlra_step(dlra_ctx* ctx, int32_t n_steps);

/* Dose e(x) = weighted sum over beams of collided + uncollided deposited energy [MeV/cm^3]
 * (per_mass = 1: divided by the density of the mixture, MeV/g). out [n] doubles,
 * host or device memory. The collided part accumulates dE sqrt(4 pi) u_0(x) after
 * every energy step. Synchronises the stream when out is a host pointer. */
dlra_status dlra_dose(dlra_ctx* ctx, double* out, int32_t out_on_device, int32_t per_mass);

/* Energy steps done so far (*step) and current rank of each beam (ranks[n_beams],
 * may be NULL). Synchronises the stream. */
dlra_status dlra_query(dlra_ctx* ctx, int32_t* step, int32_t* ranks);

/* Ranks chosen by every truncation so far for one beam: log [n_energy_steps][2]
 * (after streaming, after the source; -1 = no truncation). Synchronises. */
dlra_status dlra_rank_log(dlra_ctx* ctx, int32_t beam_id, int32_t* log);

/* Copy one beam's factors to host doubles: X [n][r] column-major n x r, S r x r
 * column-major, W m x r column-major, *r the rank. Buffers must hold rank_max
 * columns. Synchronises. */
dlra_status dlra_get_state(dlra_ctx* ctx, int32_t beam_id, double* X, double* S, double* W, int32_t* r);

/* Replace one beam's factors (host doubles, same layout as dlra_get_state;
 * X and W must have orthonormal columns, 0 <= r <= rank_max). */
dlra_status dlra_set_state(dlra_ctx* ctx, int32_t beam_id, const double* X, const double* S,
                           const double* W, int32_t r);

/* Copy the ray tracer's output of one beam to the host: the bin-averaged
 * uncollided fluence of energy bin k (psi [n], 1/(cm^2 MeV)) and the uncollided
 * deposit (e_u [n], MeV/cm^3); either pointer may be NULL. Synchronises. */
dlra_status dlra_get_source(dlra_ctx* ctx, int32_t beam_id, int32_t k, double* psi, double* e_u);

/* Copy the angular tables to the host, m x m row-major each: A [3][m][m] and
 * absA [3][m][m] = |A_d| = V_d |Lambda_d| V_d^T. Either pointer may be NULL. */
dlra_status dlra_get_tables(dlra_ctx* ctx, double* A, double* absA);

/* Number of RK4 sub-steps of the streaming update of each energy step,
 * nsub [n_energy_steps]. Available after dlra_set_materials. */
dlra_status dlra_get_substeps(dlra_ctx* ctx, int32_t* nsub);

/* Rewind to E_max for a new solve with the same phantom and beams: zeroes every
 * low-rank state, dose and rank log; retrace = 1 reruns the ray tracer of every
 * beam into its existing buffers. Enqueued on the context's stream; allocates nothing. */
dlra_status dlra_reset(dlra_ctx* ctx, int32_t retrace);

/* Set the weight of one beam (>= 0): the dose is sum_b weight_b e_b with e_b the
 * beam's deposit at unit weight, so a new weight takes effect at the next dlra_dose
 * without stepping again. */
dlra_status dlra_set_beam_weight(dlra_ctx* ctx, int32_t beam_id, double weight);

/* Prepare the reverse sweep (dlra_backward): from the next dlra_step on, every
 * beam's low-rank state is copied on the device at the start of energy steps 0,
 * I, 2I, ... (I = checkpoint_interval >= 1; 0 switches it off). Must be called at
 * step 0 (after dlra_init or dlra_reset). Memory: ceil(K/I) states per beam. */
dlra_status dlra_enable_adjoint(dlra_ctx* ctx, int32_t checkpoint_interval);

/* Gradient of a loss L(e) of the dose e(x) (MeV/cm^3, the quantity of dlra_dose with
 * per_mass = 0) after the energy steps run so far, by the discrete adjoint of those
 * steps (the paper states only the forward method). Input dL_de [n] (host or device,
 * in_on_device). Outputs, either may be NULL:
 *   dL_dweight [n_beams] (host): dL/d weight_b = <dL/de, e_b> (exact; e_b at unit weight);
 *   dL_dw [n_mat][n] (host or device, out_on_device): dL/dw_m(x) through the stopping
 *     power S(x, E) = sum_m w_m S_m(E) in streaming and collisions, the scattering and
 *     first-collision coefficients (Sec. 2.1, Eq. mixXS) and the ray tracer (Sec. 3.2).
 * The adjoint state is a low-rank factorisation advanced by the same BUG steps with
 * the transposed operators (its rank control: the forward's, adaptive when the forward
 * replays a schedule); forward states are recomputed from the checkpoints of
 * dlra_enable_adjoint, one segment at a time (see dlra_set_adjoint_store). Requires
 * dlra_enable_adjoint before the first step (else DLRA_ERR_STATE). Synchronises. The
 * forward state is unchanged. */
dlra_status dlra_backward(dlra_ctx* ctx, const double* dL_de, int32_t in_on_device, double* dL_dweight,
                          double* dL_dw, int32_t out_on_device);

/* Memory/time trade of dlra_backward's segment replay. keep = 1 (default): while replaying a
 * segment of I energy steps, keep each step's streaming-stage inputs (4 n_sub buffers of
 * n x capacity) and post-collision state, so the reverse steps reuse them; taken only when
 * they fit in a third of the free device memory, else as keep = 0. keep = 0: store only the
 * start state of each step and recompute the forward step during the reverse sweep. Same
 * results either way up to the summation order of the FP64 atomic reductions. */
dlra_status dlra_set_adjoint_store(dlra_ctx* ctx, int32_t keep);

/* Autotuner: times the launch variants of the heavy cell-side kernels on this context's work
 * space (filled with synthetic values at full rank capacity; the streaming stages one launch at
 * a time after a 256 MB write, i.e. with a cold L2 as inside a solve; allocates those 256 MB
 * for the duration of the call) and keeps the fastest: the
 * streaming stage per cell with FMA, on the tensor cores (FP32 path) or per brick with FMA and
 * staged stencil inputs; the grid of the Gram reductions (608 / 1216 / 2432 / 4864 target
 * blocks) and of the stencil Grams (0.5 / 1 / 2 waves of the FMA kernel, and the tensor-core
 * kernel) and of the truncation apply (FMA or tensor cores). Needs materials and a beam;
 * synchronises; drops captured graphs. report (optional, 31 doubles): ms of the per-cell and tensor-core stages, of the four Gram grids, of the three
 * stencil-Gram grids, the chosen stage variant (0 .. 13 as dlra_set_stage_kernel), Gram block
 * target, stencil-Gram waves x 2, ms of the brick stage, ms of the tensor-core stencil Gram,
 * the chosen stencil-Gram kernel (0 FMA, 1 tensor cores), ms of the cell-pair stage, ms of
 * the TMA-staged tensor-core stages with 128- and 256-cell bricks, of its persistent form and
 * of its form with A in tensor memory, ms of the truncation apply with FMA and on the tensor
 * cores, the chosen apply kernel (0 FMA, 1 tensor cores), ms of the cluster form of the stage,
 * ms of the windowed stencil Gram, ms of the three-tile form of the stage, ms of the Gram
 * reduction on the tensor cores, ms of the eight-column form of the stage, ms of its form with
 * eight formation warps, ms of its form with five boxes and an FP32 B image, ms of that form
 * with the split B image (-1 where not applicable). */
dlra_status dlra_autotune(dlra_ctx* ctx, double* report);

/* Streaming-stage kernel: 0 one thread per cell loading its 13 stencil neighbours (default),
 * 1 the tensor-core kernel of dlra_set_tensor_cores (FP32 path; the FMA kernel on FP64),
 * 2 one block per 256-cell brick with the stencil inputs staged in shared memory, 3 two
 * x-adjacent cells per thread with packed FP32x2 FMAs (FP32 path with nx even; else variant 0),
 * 4 / 5 the r x r mix on the tensor cores (tcgen05.mma kind::tf32 with high/low TF32 splits,
 * FP32 accuracy) with each chunk of four input columns of a 128- / 256-cell brick and its
 * two-cell halo staged by one TMA copy (FP32 path, 3-D, nx and the cell count multiples of 4,
 * rank capacity >= 32; else variant 0), 6 the 128-cell form as one persistent block per SM
 * that streams its bricks' chunks through a four-deep TMA ring and drains one brick's TMEM
 * accumulator while the next brick accumulates in a second one, 7 the 128-cell form with the
 * A operand (the stencil values) written to tensor memory (tcgen05.st) and read from there by
 * the products, leaving shared memory to the halo and B, 8 variant 7 on clusters of two CTAs
 * owning y-adjacent bricks: one multicast TMA copy loads the pair's common halo box and one
 * multicast bulk copy the chunk's B image into both CTAs (variant 7 where the cluster launch is
 * refused), 9 variant 7 on bricks of three 128-cell tiles stacked along z (8 x 4 x 12 cells, one
 * block per SM) sharing one halo box and one B image per chunk, 10 variant 7 on chunks of eight
 * input columns (half the chunks per brick), 11 variant 7 with eight formation warps, two per
 * TMEM lane quarter, each forming the stencil values of two of the chunk's four columns, 12
 * variant 11 staging each chunk as five TMA boxes (the brick with its x halo and its four y and z
 * faces: half the values of the halo box, the stencil being a cross) and its B operand as one
 * FP32 image that the formation warps split into TF32 parts in shared memory, 13 variant 12
 * with the B image of TF32 high and low parts copied as it is (no split in shared memory). Same
 * results up to rounding; dlra_autotune picks among them. */
dlra_status dlra_set_stage_kernel(dlra_ctx* ctx, int32_t variant);

/* Kernel of the cell-side tall-skinny Grams (the augmentation's projections X^T K and the
 * Grams of its pivoted CholeskyQR2 passes, Sec. 2.2; the material Grams X^T diag(w_k) X of the
 * collided scattering step, Sec. 3.3.1): 0 FMA with FP64 sums across blocks (default), 1 on the
 * tensor cores (FP32 path, at least 65,536 cells and 8 columns, at most 128 columns on the
 * X side: 32-row chunks loaded by TMA, TF32 high/low splits, tcgen05.mma kind::tf32, sums
 * restarted every 8 chunks and added up in FP32 with round-to-nearest, FP64 across blocks; the
 * FMA kernel otherwise), 2 as 1 at any cell count. Same results up to rounding; dlra_autotune
 * picks between 0 and 1. */
dlra_status dlra_set_gram_kernel(dlra_ctx* ctx, int32_t variant);

/* Kernel of the cell-side tall-skinny products (the augmentation's projections and the
 * truncation's X = X^ P, Sec. 2.2): 0 one thread per cell with FMA (default), 1 on the tensor
 * cores (FP32 path, at least 65,536 cells and 16 output columns: each 128-cell tile of A loaded
 * by TMA, split into TF32 high and low parts into tensor memory, tcgen05.mma kind::tf32 with
 * FP32 accumulation; the FMA kernel otherwise), 2 as 1 at any cell count. Same results up to
 * rounding; dlra_autotune picks between 0 and 1. */
dlra_status dlra_set_apply_kernel(dlra_ctx* ctx, int32_t variant);

/* Stencil-Gram kernel (the Galerkin blocks X^T D_k rho^-1 X of the L-step and S-step):
 * 0 FMA (default), 1 on the tensor cores (FP32-mixed path only: tcgen05.mma kind::tf32 with
 * high/low TF32 splits of both operands, FP32 accumulation in tensor memory, FP64 sums across
 * blocks; the FMA kernel on FP64 or for more than 128 columns), 2 on the tensor cores with the
 * inputs staged by TMA in a window that slides along each stencil's axis and the stencil
 * operand in tensor memory (FP32-mixed path, 3-D grids, the same basis on both sides: the
 * L-step and S-step Grams; kernel 1 otherwise); its tensor-core sums restart every 8 chunks of
 * 32 cells and are added up in FP32 with round-to-nearest (the tensor core's own FP32
 * accumulation rounds toward zero, which leaves kernel 1's long sums up to ~5e-4 low at 2M
 * cells). Same results up to rounding; dlra_autotune picks among them. */
dlra_status dlra_set_stencil_gram_kernel(dlra_ctx* ctx, int32_t variant);

/* enable = 1: on the FP32-mixed path, the streaming stage runs on the fifth-generation tensor
 * cores (tcgen05.mma kind::tf32 with the operands split into high and low TF32 parts, FP32
 * accuracy; accumulators in tensor memory) instead of FP32 FMA. Measured slower than the FMA
 * kernel on the 64^3, rank-20 workload (the stage is bound by its stencil loads, not by the
 * r x r products), so it is off by default. No effect on the FP64 path. */
dlra_status dlra_set_tensor_cores(dlra_ctx* ctx, int32_t enable);

/* enable = 1: dlra_step captures the work of its n energy steps into a CUDA graph the
 * first time it runs from a given step with a given set of active beams, and replays the
 * graph afterwards (ranks live on the device, so the launch sequence depends on nothing
 * else); repeated solves after dlra_reset then cost one graph launch each. Graphs are
 * dropped when materials, beams or the checkpoint interval change, and bypassed while
 * profiling. A capture the driver rejects falls back to direct launches and switches the
 * option off. enable = 0 drops every graph. */
dlra_status dlra_set_graphs(dlra_ctx* ctx, int32_t enable);

/* Per-kernel timing with CUDA events on the context's stream. enable = 1 records an
 * event pair around every launch of the fused streaming-stage kernel (the K-step
 * RK4 stage: stencil + r x r mix) until disabled; dlra_kernel_stats synchronises and
 * returns the summed time in ms and the number of timed launches since enabling. */
dlra_status dlra_set_profiling(dlra_ctx* ctx, int32_t enable);
dlra_status dlra_kernel_stats(dlra_ctx* ctx, double* total_ms, int64_t* launches);

/* Arguments of the stand-alone streaming K-step (no context needed). All arrays are
 * FP32 device memory of the current device, ordered with cuda_stream:
 *   K0 (in), K1 (out) : n x r column-major, n = nx ny nz; K1 must not alias K0.
 *   inv_rho           : n values 1/rho_s(x), where S(x, E) = rho_s(x) S_w(E).
 *   P                 : nk matrices r x r, column-major, P_k at P + k r r, nk = 4 for an
 *                       x-z slab (ny == 1, dy == 0) and 6 otherwise; k = 2 da + s pairs the
 *                       stencil D^-_d (s = 0) with W^T A^+_d W and D^+_d (s = 1) with
 *                       W^T A^-_d W, d running over the streaming directions x, (y,) z.
 *   e0, de, n_sub     : energy at the start of the step, energy step, RK4 sub-steps.
 *   bk_p, bk_alpha    : water stopping power S_w(E) = E^(1-p)/(p alpha).
 * 1 <= r <= 64. */
typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;
  int32_t r;
  double e0, de;
  int32_t n_sub;
  double bk_p, bk_alpha;
  const float* K0;
  float* K1;
  const float* inv_rho;
  const float* P;
  void* cuda_stream;
  int32_t stage_kernel; /* streaming-stage kernel, 0 .. 13 as dlra_set_stage_kernel (0: per-cell FMA) */
} dlra_kstep_args;

/* The K-step of the streaming update (Sec. 2.2, Eq. KLS first line, with F_S of
 * Sec. 3.3.2 and RK4 time updates, Sec. 3.3.3): integrates
 * K' = S_w(E(t))^-1 sum_k D_k(rho_s^-1 K) P_k from K(t_k) = K0 over one energy step
 * with n_sub RK4 sub-steps, K1 = K(t_k + de), with the streaming-stage kernel
 * stage_kernel (the tensor-core kernels 4 .. 13 on 3-D grids with nx and n multiples of 4
 * and rank capacity >= 32, the per-cell FMA kernel otherwise). Allocates its work space
 * (3 n x r, the packed P and, for kernels 4 .. 13, the B images) with cudaMalloc and frees
 * it before returning; synchronises cuda_stream. */
dlra_status dlra_kstep(const dlra_kstep_args* args);

/* The same K-step as dlra_kstep for callers that cannot allocate device memory
 * (the paper has no counterpart; this is a library-usage variant). Its work space
 * is a static device array of 32 MiB held by every GPU that loads the library
 * until the process exits; problems whose work space exceeds it are rejected with
 * DLRA_ERR_ARG and a message naming both sizes. The work space is 3 n rcap +
 * 2 nact rcap^2 FP32 words (nact = 2 on an x-z slab, 3 in 3-D; rcap = r rounded
 * up to 4, 8, ..., 24, 32, 40, 48 or 64) plus up to 256 bytes of alignment per
 * buffer and one rank word, and with stage_kernel 4 .. 13 on a 3-D grid the B images of
 * the tensor-core stages (2 x 6 rcap x round16(rcap) FP32 words). The first call on each device looks up the array's
 * device address with that device current and keeps it for the process; make
 * that first call before any stream capture. A cudaDeviceReset (or any other
 * teardown of the device's primary context) unloads the array, so the entry
 * point must not be called on that device afterwards in the same process. Every call uses the whole array and
 * writes all of it that it reads (nothing needs to start at zero); calls that
 * overlap on the GPU (different streams, threads or processes sharing a context)
 * race on it. Enqueued on cuda_stream without synchronising; calls no cudaMalloc
 * or cudaFree. */
dlra_status dlra_kstep_noalloc(const dlra_kstep_args* args);

/* Arguments of the stand-alone stencil Gram (no context needed). Device memory of the current
 * device, ordered with cuda_stream:
 *   A  : FP32, n x na column-major with leading dimension lda >= n, n = nx ny nz;
 *   B  : FP32, n x nb column-major with leading dimension ldb >= n;
 *   inv_rho : FP32, n values 1/rho_s(x);
 *   out: FP64, nk nb na values, G_k[a][b] at out[(k nb + b) na + a]; overwritten.
 * nk and k = 2 da + s as for dlra_kstep_args.P; 1 <= na, nb <= 128. variant: 0 FMA kernel,
 * 1 tensor-core kernel, 2 windowed tensor-core kernel where A and B are the same array (as
 * dlra_set_stencil_gram_kernel). */
typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;
  int32_t na, nb;
  const float* A;
  int64_t lda;
  const float* B;
  int64_t ldb;
  const float* inv_rho;
  double* out;
  int32_t variant;
  void* cuda_stream;
} dlra_stencil_gram_args;

/* The Galerkin blocks of the streaming operator between two cell bases (Sec. 3.3.2, the
 * X^T D X terms of the L-step and S-step with the one-sided second-order stencils of Eq.
 * (D+-) and two ghost layers of zeros): G_k[a][b] = sum_i A(i, a) D_k(rho_s^-1 B(:, b))(i),
 * summed in FP32 within a block and in FP64 across blocks. Allocates a 4-byte error flag;
 * synchronises cuda_stream. DLRA_ERR_TIMEOUT if a tensor-core wait ran out (out is then
 * incomplete); errors read with dlra_last_error(NULL). */
dlra_status dlra_stencil_gram(const dlra_stencil_gram_args* args);

/* Arguments of the straggling tables (host only, no context, no device memory). */
typedef struct {
  double e_min, e_max;    /* energy interval of the discretisation, MeV (0 < e_min < e_max) */
  int32_t n_elem;         /* equal energy elements (the paper uses 128), 1 .. 65536 */
  double bk_p, bk_alpha;  /* water stopping power S_w(E) = E^(1-p) / (p alpha) */
  double t100;            /* removal reference Sigma_t / tau = t100 (100 / E)^2 / 2 */
  int32_t straggling;     /* 0: T = 0 (the CSDA limit) */
} dlra_straggling_args;

/* The operators of the uncollided transport along a ray with energy straggling (Sec. 3.2:
 * d psi/dz + Sigma_t psi = d(S* psi)/dE + (1/2) d/dE (T d psi/dE), S* = S + T'/2), discretised
 * in energy by discontinuous Galerkin with the Legendre polynomials P_0..P_2 of each element, a
 * Lax-Friedrichs flux for slowing down and SIPG for straggling (penalty 18 kappa / Delta, no
 * diffusive flux through the ends), for water (S_w above; T_w = T_Bohr (1 + 4 I/(3 m_e v^2)
 * ln(2 m_e v^2 / I)), I = 75 eV) and a unit material factor. Host outputs, caller-allocated:
 *   mass [3 n_elem]           diagonal of the mass matrix (Delta / (2 j + 1));
 *   adv, sipg, rem [n_elem][3][3][3]  block-tridiagonal operators: block (e, b) couples the
 *     dofs i of element e (rows) with the dofs j of element e - 1 + b (b = 0, 1, 2; blocks
 *     outside the interval are zero); adv is the slowing-down term int d(S* psi)/dE v,
 *     sipg the SIPG form of kappa = T/2, rem the removal int sigma_ref psi v.
 * A ray segment with stopping factor f and removal factor tau advances by
 * M dc/dz = -(-f adv + f sipg + tau rem) c. Errors: DLRA_ERR_ARG (read with
 * dlra_last_error(NULL)). */
dlra_status dlra_straggling_tables(const dlra_straggling_args* args, double* mass, double* adv, double* sipg,
                                   double* rem);

/* Arguments of the stand-alone straggling ray trace (no context). Device memory of the current
 * device, ordered with cuda_stream:
 *   f_cell [n]  stopping factor rho_s(x) (S(x, E) = f S_w(E)); T(x, E) = f T_w(E);
 *   tau_cell [n] removal factor (Sigma_t(x, E) = tau t100 (100/E)^2 / 2, the ray tracer's model);
 *   psi [n_bins][n] (out) bin-averaged uncollided fluence of a unit-weight beam per energy bin
 *     [E_{k+1}, E_k], E_k = e_max - k (e_max - e_min) / n_bins, and voxel (1/(cm^2 MeV));
 *   e_u [n] (out) energy lost to slowing down per volume (MeV/cm^3).
 * Grid as for dlra_kstep_args; the energy interval is discretised by n_elem DG elements (the
 * paper: 128) and the depth by Crank-Nicolson steps of at most h_max cm (the paper: 0.01);
 * straggling = 0 gives the CSDA limit. Beam: spot grid of pitch min(delta)/4 within 3.5
 * spot_sigma with Gaussian weights, initial energy distribution a Gaussian of energy_sigma
 * (a delta for 0) projected on the DG space. n_elem >= 1 with at most 8 energy bins
 * overlapping one element; at most 1e6 Crank-Nicolson steps on one ray (the sum over its voxel
 * segments of ceil(length / h_max)), else DLRA_ERR_ARG before any launch. */
typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;
  double e_min, e_max;
  int32_t n_bins, n_elem;
  double h_max;
  double bk_p, bk_alpha, t100;
  int32_t straggling;
  double energy, energy_sigma, spot_sigma;
  double pos[3], dir[3];
  const double* f_cell;
  const double* tau_cell;
  double* psi;
  double* e_u;
  void* cuda_stream;
} dlra_straggling_trace_args;

/* The uncollided transport of one beam with energy straggling (Sec. 3.2: energy DG with a
 * Lax-Friedrichs slowing-down flux and SIPG straggling, Crank-Nicolson in depth), one device
 * thread per ray marching the block-tridiagonal system with FP64 Thomas elimination.
 * Overwrites psi and e_u; allocates its tables and work space (3 G x 4 + 18 G doubles per ray)
 * and frees them; synchronises cuda_stream. Errors: DLRA_ERR_ARG, DLRA_ERR_OOM, DLRA_ERR_CUDA
 * (dlra_last_error(NULL)); a failed host-to-device copy returns DLRA_ERR_CUDA before the
 * launch. */
dlra_status dlra_straggling_trace(const dlra_straggling_trace_args* args);

/* enable = 1: the uncollided fluence and deposit of every beam come from the energy-DG tracer
 * with straggling (Sec. 3.2; the computation of dlra_straggling_trace: n_elem P2 elements in
 * energy, Crank-Nicolson steps of at most h_max cm, straggling = 0 for its CSDA limit) instead
 * of the CSDA ray tracer, for the beams added afterwards and at every dlra_reset with a retrace
 * (call dlra_reset(ctx, 1) to re-trace beams added before). Synchronises each trace. The
 * reverse sweep is not available with this source (DLRA_ERR_STATE). */
dlra_status dlra_set_straggling(dlra_ctx* ctx, int32_t enable, int32_t n_elem, double h_max, int32_t straggling);

/* enable = 1: the beams of this context share one low-rank state (the paper's multi-beam
 * solve, Sec. 4.3), instead of one state per beam. Each energy step streams and scatters
 * the joint state once and adds the first-collision sources of all beams that have one,
 * each beam's rank-M factor (M materials) scaled by its weight, stacked into one source of
 * rank M x (beams) (at most the rank capacity; DLRA_ERR_ARG at the next dlra_step otherwise).
 * The collided deposit is the joint state's (weights included); the uncollided deposits
 * enter times their beam's weight. dlra_rank_log(ctx, 0, ...) gives the joint state's ranks;
 * dlra_set_beam_weight changes a beam's weight for the next solve (the source uses it).
 * Direct launches only (dlra_set_graphs has no effect); no reverse sweep. Call before the
 * first step; DLRA_ERR_STATE otherwise. */
dlra_status dlra_set_joint(dlra_ctx* ctx, int32_t enable);

/* Kernel launches issued by this context so far (for launch accounting). */
int64_t dlra_launch_count(const dlra_ctx* ctx);

/* One-line description of the last error of this context (never NULL); with
 * ctx == NULL, the last error of a context-free call on this host thread. */
const char* dlra_last_error(const dlra_ctx* ctx);

/* Release every resource of the context (NULL is ignored). */
void dlra_destroy(dlra_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DLRA_H */
