/* gbdmrg test and timing hooks: the steps gbd_solve runs, exposed one by one
 * so that each can be compared with an independent CPU implementation and
 * timed on its own.  Same conventions as gbdmrg.h (status codes, host
 * buffers, no exceptions).
 *
 * MPS exchange format ("canonical blocks").  Bond k (0..n) is a list of
 * sectors (N_alpha, N_beta, dim) of the left block (sites < k), sorted by
 * (N_alpha, N_beta); `sectors` holds the triples of all bonds back to back
 * and n_sectors[k] their counts.  Site i stores, for every sector q_l of
 * bond i in order and every local state s = 0..3 ([0, alpha, beta,
 * alpha+beta]) with q_r = q_l + s present in bond i+1, one row-major
 * dim(q_l) x dim(q_r) block; `data` holds all sites back to back.
 *
 * Two-site vector format for bond pair (k, k+1): for every sector q_l of bond
 * k in order, s1 = 0..3, s2 = 0..3 with q_r = q_l + s1 + s2 present in bond
 * k+2, one row-major dim(q_l) x dim(q_r) block.
 */
#ifndef GBDMRG_TEST_H
#define GBDMRG_TEST_H

#include "gbdmrg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double sigma_flops;     /* algorithmic flops of all sigma builds (2mnk per block product) */
  double sigma_ms;        /* device time of the sigma builds (CUDA events on the engine stream) */
  double env_flops, env_ms;
  double enlarge_ms;      /* host wall time forming the enlarged operators */
  double davidson_ms, truncate_ms, step_ms;
  int64_t n_sigma, n_steps, kernel_launches, h2d_bytes, d2h_bytes;
  double max_discarded_weight;
  double sigma_flops_exec;   /* flops executed by the tensor-core tiles (with padding) */
  double tc_ms, tc_flops;    /* tensor-core sigma builds only: device time, algorithmic flops */
  int64_t n_sigma_tc;
  int64_t tier_iterations[3];   /* Davidson iterations in the BF16/TF32 tier, the TF32x3 tier, FP64 */
  double max_final_residual;    /* largest ||r|| at the end of a step's Davidson solve */
  double sum_final_residual;    /* sum of those over the steps */
  int64_t graph_launches;       /* sigma builds replayed from a captured CUDA graph */
  int64_t autotune_trials;      /* tensor-core plans built and timed by the tile-shape autotuner */
  double tc_gemm_ms;            /* device time of the tc_gemm_kernel launches alone (CUDA events) */
  double tc_bytes;              /* algorithmic HBM bytes of the tensor-core sigma builds */
  double tc_flops_by_type[4];   /* algorithmic flops of those builds with BF16, TF32, TF32x3, BF16x3 operands */
  double tc_gemm_ms_by_type[4]; /* tc_gemm_kernel device time of those builds */
  double tc_build_ms;           /* host wall time building tensor-core plans, autotuning included */
  double tc_build_phase_ms[5];  /* of which: layouts and groups, panels, tile lists, upload, tensor maps */
  double enlarge_host_ms;       /* host part of enlarge_ms (sub-block lists, before the device axpy) */
  double diag_ms;               /* H_eff diagonal (wall) */
  double truncate_rho_ms, truncate_eig_ms;   /* decimation: density matrices to the host; eigensolves */
  double env_wall_ms;           /* environment updates, wall time incl. plan upload (env_ms: kernels only) */
  double tc_stage_alg_bytes[2]; /* tc_bytes split by stage: A (Renl, psi, Y^T write), B (Y^T read, Lenl, sigma) */
  double tc_stage_box_bytes[4]; /* bytes the TMA boxes request from L2: stage A (A box, B box), stage B (A, B) */
  double tc_stage_dense_bytes[4]; /* the valid rows x K of those boxes, without row, K or box-width padding */
  double tc_gemm_ms_by_stage[2];  /* tc_gemm_ms split into stage A and stage B */
  int64_t davidson_iterations;    /* outer Davidson iterations (all tiers) */
  int64_t inner_matvecs;          /* sigma builds inside inner-PCG corrections (in n_sigma too) */
  int64_t n_solves;               /* Davidson solves (one per two-site step) */
  int64_t n_solves_above_tol;     /* of which ended with ||r|| >= the step's tolerance */
  double sweep_max_residual;      /* largest final ||r|| of the current or last sweep */
  double enlarge_dev_ms;          /* device time of the block-axpy launches forming the enlarged operators */
  double enlarge_bytes;           /* their algorithmic bytes: 8 (terms + 1) per output element */
  double rdm_ms;                  /* wall time of the last gbd_rdms (or RDMs of a solve) */
  double rdm_env_bytes;           /* peak device bytes of its operator-string environments */
  double h2d_wait_ms;             /* host time waiting for a region of the pinned staging ring */
} gbd_stats;

/* Sigma launch sequences replayed as CUDA graphs (1, the default) or
 * launched kernel by kernel (0); results are identical either way. */
int gbd_set_graphs(gbd_ctx *ctx, int32_t enable);

/* Tile shape of the tensor-core sigma: 0 (default) = autotuned per shape
 * class; 64, 128 or 256 = that largest N tile for both stages.  The shape
 * never changes the arithmetic (same products, same summation order). */
int gbd_set_tc_tile(gbd_ctx *ctx, int32_t ncap);

/* Per-bond adaptive bond dimension for the following solves on this
 * context (the paper's dynamically adapted per-bond bond dimension): each
 * decimation keeps the fewest states whose discarded weight is at most
 * max_discarded.  It never splits a near-degenerate cluster, keeps at least
 * m_min, and keeps at most the schedule's bond dimension of that sweep.
 * max_discarded = 0 (the default) is the fixed bond dimension.  The choice
 * is made on the host; the device path is that of any smaller bond. */
int gbd_set_adaptive_bond_dim(gbd_ctx *ctx, double max_discarded, int32_t m_min);

/* Order in which the persistent tensor-core CTAs take the stage-B tiles of
 * the sigma (output sector q, 128-row block m0 of E_R(q), split-K chunk,
 * N tile n0 of E_L(q)): 0 by (q, m0, chunk, n0), 1 (default) by
 * (q, chunk, m0, n0), 2 by (q, chunk, n0, m0).  Tiles running at the same
 * time share operand boxes through L2 in different ways; every tile
 * computes the same products in the same order, so the result is
 * identical for all three. */
int gbd_set_tc_order(gbd_ctx *ctx, int32_t order);
/* Tile order of stage A (Y^T = Renl stack x psi^T): 0 (default) most
 * expensive tile first; 1 the N tiles of each 128-row block of the Renl
 * stack adjacent (blocks most expensive first), so that they share its A
 * boxes through L2.  Results are identical for both. */
int gbd_set_tc_order_a(gbd_ctx *ctx, int32_t order);
/* Stage B of the tensor-core sigma per output sector q: with E_L(q) of at
 * least min_rows rows (default 160), one product per s_out section of E_L(q)
 * over the Y^T sections that section reads (its Lenl panel holds that
 * section's rows only), else one product over all of E_L(q) (its panel has
 * the zero rows of the sections a Y^T section does not reach).  0 splits
 * every sector, a large value none.  The sums differ only in their split-K
 * grouping. */
int gbd_set_tc_sout_split(gbd_ctx *ctx, int32_t min_rows);

/* Preconditioner of the following Davidson solves (GBD_PRECOND_DIAG or
 * GBD_PRECOND_LEARNED; the latter needs weights in the context). */
int gbd_set_preconditioner(gbd_ctx *ctx, int32_t preconditioner);

/* Operands of the accurate Davidson tier of reduced-precision schedules:
 * 3 = TF32x3 (default), 4 = BF16x3 (the codes of gbd_apply_heff_prec). */
int gbd_set_accurate_tier(gbd_ctx *ctx, int32_t prec);

/* Stopping rule of the accurate (TF32x3 / BF16x3) Davidson tier: a plateau
 * (||r|| not cut by 30 % over 3 iterations) ends it once ||r|| is below
 * floor_mult x u x max(1, |theta|), u being the tier's measured relative
 * sigma error (default floor_mult 1); hard_stag > 0 also ends a
 * reduced-precision tier after hard_stag iterations without a 30 % cut at
 * any level (default 8; 0: off).  GBD_ERR_ARG for floor_mult <= 0 or
 * hard_stag < 0. */
int gbd_set_tier_stop(gbd_ctx *ctx, double floor_mult, int32_t hard_stag);

/* Environment updates of the sweep steps of reduced-precision schedules:
 * prec 0 = FP64 (the default), 3 = on the tensor cores with TF32x3 operands,
 * 4 = BF16x3 (FP32 accumulation in chunks of at most 512 of K, summed in
 * FP64).  Environments built outside the steps (initial state, saved
 * state, installed MPS) and those the reported energy uses are FP64.
 * GBD_ERR_ARG for another prec. */
int gbd_set_env_precision(gbd_ctx *ctx, int32_t prec);

/* Environment updates compute one channel of each certified
 * Hermitian-conjugate pair and fill the other with its transpose times the
 * pair's sign (enable = 1, the default), or compute every channel
 * (enable = 0).  Certification (at gbd_setup, from the MPO's W tensors):
 * L[d] = sign L[c]^T holds for every MPS because W's column d equals the
 * transposed, conjugate-relabelled column c times sign, inductively from
 * bond 0 (right environments: W's rows, from bond n).  GBD_ERR_ARG for
 * another enable. */
int gbd_set_env_conjugates(gbd_ctx *ctx, int32_t enable);
/* The certified pairs of one bond (side 0 = left environments, 1 = right):
 * partner[c] = the conjugate channel (c for a self-conjugate or zero
 * channel, -1 when none is certified), sign[c] its sign; count = channels
 * of the bond (buffers of cap entries, either may be NULL).
 * GBD_ERR_STATE before gbd_setup. */
int gbd_env_conjugates(gbd_ctx *ctx, int32_t side, int32_t bond, int32_t *partner, int32_t *sign, int32_t cap,
                       int32_t *count);

/* Reduced-precision schedules solve steps whose two-site state has fewer
 * than n elements (chain ends) in FP64: there the tensor-core plan costs
 * more than it saves.  Default 4096; 0 = always the tensor-core tiers. */
int gbd_set_tc_min_two_site(gbd_ctx *ctx, int64_t n);

/* One Davidson solve at the current centre k (environments k and k+2
 * valid, as after gbd_init_state for k = 0 or after steps up to k-1) in
 * schedule precision `precision` (GBD_FP64/TF32/BF16) with at most
 * `fp64_refine` FP64 iterations and residual tolerance `tol`, without
 * decimation or environment update.  theta = its Ritz value, e64 = the FP64
 * Rayleigh quotient <x|H|x>/<x|x> of the resulting vector, r64 = the FP64
 * residual norm ||Hx - e64 x|| / ||x||.  Isolates the effect of the matvec
 * precision on one step. */
int gbd_probe_step(gbd_ctx *ctx, int32_t k, int32_t precision, int32_t fp64_refine, double tol, double *theta,
                   double *e64, double *r64);

/* Keep a device copy of the current MPS, whose centre must be at bond
 * (0,1) (after gbd_init_state, gbd_set_mps with center 0 or a full sweep);
 * a later save replaces it.  gbd_restore_state puts the copy back (the copy
 * stays) and rebuilds the environments, so that several sweeps can start
 * from the same state.  GBD_ERR_STATE without an MPS / without a copy. */
int gbd_save_state(gbd_ctx *ctx);
int gbd_restore_state(gbd_ctx *ctx);
/* Bond dimension M (>= 1) and Davidson tolerance tol (> 0) of schedule
 * entry `sweep` for the following gbd_run_sweep calls. */
int gbd_set_sweep_schedule(gbd_ctx *ctx, int32_t sweep, int32_t M, double tol);

/* Validate the problem and schedule, build the MPO; no MPS yet. */
int gbd_setup(gbd_ctx *ctx, const gbd_problem *problem, const gbd_schedule *schedule);
/* Change the matvec precision (and FP64 refinement limit) of the current
 * state for the following sweeps. */
int gbd_set_precision(gbd_ctx *ctx, int32_t precision, int32_t fp64_refine);
/* Seeded initial MPS (right-canonical) and all right environments. */
int gbd_init_state(gbd_ctx *ctx);
/* One full sweep with the schedule's entry `sweep`; energy = last Ritz value. */
int gbd_run_sweep(gbd_ctx *ctx, int32_t sweep, double *energy);
/* <psi|H|psi>/<psi|psi> + e_core of the current MPS (evaluated at bond (0,1)). */
int gbd_final_energy(gbd_ctx *ctx, double *energy);
/* Sector triples of one bond; count = number of sectors (cap in triples). */
int gbd_get_bond(gbd_ctx *ctx, int32_t bond, int32_t *triples, int32_t cap, int32_t *count);
/* Install an MPS in canonical blocks.  Sites < center must be left-
 * orthonormal and sites > center+1 right-orthonormal; left environments up
 * to bond `center` and right environments from bond center+2 are built. */
int gbd_set_mps(gbd_ctx *ctx, const int32_t *n_sectors, const int32_t *sectors, const double *data,
                int32_t center);
/* Length of the two-site vector at (k, k+1). */
int gbd_two_site_size(gbd_ctx *ctx, int32_t k, int64_t *size);
/* out = H_eff in (two-site format); diag (may be NULL) = diagonal of H_eff. */
int gbd_apply_heff(gbd_ctx *ctx, int32_t k, const double *in, double *out, double *diag);
/* out = H_eff in through the tensor-core sigma: prec 1 TF32, 2 BF16,
 * 3 TF32x3, 4 BF16x3 (0 = the FP64 path, same as gbd_apply_heff). */
int gbd_apply_heff_prec(gbd_ctx *ctx, int32_t k, int32_t prec, const double *in, double *out);
/* One two-site step at (k, k+1): Davidson from the current two-site state,
 * decimation to at most M states and the environment update.  dir 0 = left
 * to right, 1 = right to left.  kept: the kept weights sigma^2 in descending
 * order (cap entries, count in *nkept). */
int gbd_run_step(gbd_ctx *ctx, int32_t k, int32_t dir, int32_t M, double tol, double *energy,
                 double *discarded, double *kept, int32_t cap, int32_t *nkept);
/* One- and two-particle RDMs of the current MPS (conventions of
 * gbd_result); rdm1 [n^2], rdm2 [n^4] or NULL.  Contracted through the MPS
 * (operator-string environments, cost polynomial in n and M; device FP64
 * environments of at most a few GB at n = 20, M = 1024). */
int gbd_rdms(gbd_ctx *ctx, double *rdm1, double *rdm2);
/* The same RDMs from the determinant expansion of the MPS (an independent
 * route for cross-checks); GBD_ERR_ARG above 4e8 determinants. */
int gbd_rdms_ci(gbd_ctx *ctx, double *rdm1, double *rdm2);
/* One- and two-orbital reduced density matrices of the current MPS (the
 * inputs of gbd_orbital_entropies): rho1 [n][4][4] in the local basis |0>,
 * |alpha>, |beta>, |alpha beta> = c+_alpha^x c+_beta^y |vac> (index x + 2y);
 * rho2 [n(n-1)/2][16][16] for the pairs (i < j) in lexicographic order, pair
 * index x_i + 4 x_j with the modes of i before those of j.  Either may be
 * NULL.  Contracted through the MPS, like gbd_rdms: entries that connect
 * different particle numbers are exactly zero and not computed. */
int gbd_orbital_rdms(gbd_ctx *ctx, double *rho1, double *rho2);
/* The same from the determinant expansion (GBD_ERR_ARG above 4e8
 * determinants), for cross-checks. */
int gbd_orbital_rdms_ci(gbd_ctx *ctx, double *rho1, double *rho2);
/* MPO channel keys of one bond (kind<<40 | nops<<32 | code0<<16 | code1). */
int gbd_mpo_labels(gbd_ctx *ctx, int32_t bond, uint64_t *keys, int32_t cap, int32_t *count);
/* One environment block (side 0 = left, 1 = right) for (channel, sector index). */
int gbd_env_block(gbd_ctx *ctx, int32_t side, int32_t bond, int32_t channel, int32_t sector, double *out,
                  int64_t cap, int32_t *rows, int32_t *cols);
int gbd_get_stats(const gbd_ctx *ctx, gbd_stats *stats);
/* Counters summed over the workers of the last gbd_solve_batched call. */
int gbd_get_batch_stats(const gbd_ctx *ctx, gbd_stats *s);
/* Counter-based initial-MPS entry (splitmix64; the same definition as the
 * synthetic-input generator), for checking that both agree. */
double gbd_mps_init_value(uint64_t seed, int32_t site, int32_t na, int32_t nb, int32_t s, int32_t row,
                          int32_t col);

/* Davidson overlap reduction out[j] = V_j . x for j < k, V_j = V + j*stride.
 * V and x are device pointers (n doubles each, stride >= n); out is a host
 * array of k doubles.  Partial sums go to scratch memory allocated on the
 * context's stream; 1 <= k <= 32. */
int gbd_multi_dot(gbd_ctx *ctx, const double *V, int64_t stride, int32_t k, const double *x, int64_t n,
                  double *out);
/* gbd_multi_dot without any allocation, for callers that cannot call
 * cudaMalloc (their memory comes from an arena they own, or allocation is
 * not allowed where they call from).  The paper has no counterpart: this is
 * an interface of this library only.  Inputs V (k vectors at V + j*stride, n
 * doubles each) and x, and the output out[k], are device pointers on
 * `device`; the work is enqueued on `stream` (a cudaStream_t, NULL = the
 * default stream) and this call returns without waiting for it.
 * Partial sums live in a fixed device array of 32 x 608 doubles (152 KB per
 * GPU, kept until the process exits) shared by every call: two calls that
 * overlap on the GPU race on it, so order them on one stream or synchronise
 * in between.  Every partial the reduction reads is written earlier in the
 * same call, so nothing needs clearing.  The first call on a device looks up
 * that device's copy of the array (cudaGetSymbolAddress with the device
 * current); make that first call before any stream capture.
 * Returns GBD_ERR_ARG for NULL pointers, k < 1, k > 32 (the array's limit),
 * n < 0 or stride < n; GBD_ERR_CUDA if a CUDA call fails, or without
 * launching anything if a CUDA error from earlier work is already pending on
 * the calling thread (that error is left in place).  n = 0 gives zeros.  No cudaMalloc,
 * cudaFree or allocating library routine is called. */
int gbd_multi_dot_noalloc(int32_t device, const double *V, int64_t stride, int32_t k, const double *x, int64_t n,
                          double *out, void *stream);
/* Self-test of the tensor-core grouped GEMM (tcgen05 + TMA): nterms random
 * products of M x K by K x N in precision prec (0 BF16, 1 TF32, 2 TF32x3)
 * accumulated in TMEM, against an FP64 host product of the operands as
 * stored (BF16/TF32) or of the FP64 originals (TF32x3).  Returns the largest
 * absolute error and the largest |reference| element. */
int gbd_tc_selftest(int32_t device, int32_t prec, int32_t M, int32_t N, int32_t K, int32_t nterms, uint64_t seed,
                    double *max_err, double *max_ref);
/* One Davidson correction on the device, as the solver computes it: from
 * the Ritz vector x (|x| = 1), sx = H x and theta, r = sx - theta x and
 * t = the correction of kind GBD_PRECOND_DIAG (Jacobi) or GBD_PRECOND_OLSEN
 * (see gbdmrg.h).  Host arrays of length n >= 1; returns |r|^2.
 * GBD_ERR_ARG for NULL pointers, n < 1 or another kind. */
int gbd_correction_selftest(int32_t device, int32_t kind, int64_t n, const double *x, const double *sx,
                            const double *diag, double theta, double *r_out, double *t_out, double *rr);
/* The inner-PCG Davidson correction (GBD_PRECOND_PCG) as the solver computes
 * it, at the current centre k (environments k and k+2 valid): the FP64 sigma
 * of that step, its own H_eff diagonal, at most 4 PCG steps with relative
 * tolerance 0.1, stopped by the first direction of non-positive curvature.
 * x (unit norm), r and the output t are host arrays in the two-site vector
 * format (length from gbd_two_site_size); matvecs = sigma builds it made.
 * GBD_ERR_ARG for NULL pointers; GBD_ERR_STATE without valid environments. */
int gbd_pcg_selftest(gbd_ctx *ctx, int32_t k, const double *x, const double *r, double theta, double *t,
                     int64_t *matvecs);
/* Dense throughput of the tensor-core grouped GEMM (the roof the sigma's
 * tensor view is compared with): one M x N x K product in precision prec
 * (0 BF16, 1 TF32, 2 TF32x3, 3 BF16x3) on 128 x 256 tiles, timed with CUDA
 * events over `reps` launches after one warm-up.  tflops = 2 M N K per
 * launch / time; ms_per_launch the average launch.  M a multiple of 128, N
 * of 256, K of 64.  Device memory: (M + N) K x 2 (split types) element
 * panels plus M N doubles. */
int gbd_tc_rate(int32_t device, int32_t prec, int32_t M, int32_t N, int32_t K, int32_t reps, double *tflops,
                double *ms_per_launch);
/* Self-test of the tensor-core executor of grouped GEMM plans (the path of
 * gbd_set_env_precision): an M x N output summing nterms products of K
 * columns (flags: 1 = A transposed, 2 = B transposed; alternating signs) and
 * a smaller second output, on random operands, run on the tensor cores
 * (prec 3 TF32x3, 4 BF16x3) and by the FP64 grouped GEMM.  Returns max
 * |difference| and max |FP64 result|. */
int gbd_gemm_tc_selftest(gbd_ctx *ctx, int32_t M, int32_t N, int32_t K, int32_t nterms, int32_t flags, int32_t prec,
                         uint64_t seed, double *max_err, double *max_ref);
/* Failure detection without a fault: one bounded mbarrier wait (the helper
 * every role of the tensor-core kernel uses).  arrive = 0: nothing completes
 * the barrier, the wait runs out after its poll limit (2^22 polls, a few
 * seconds) and
 * returns with *err_flag = 1, *waited_ok = 0; arrive = 1: *err_flag = 0,
 * *waited_ok = 1. */
int gbd_wait_selftest(int32_t device, int32_t arrive, int32_t *err_flag, int32_t *waited_ok);
/* Preconditioner network pieces for gradient checks: install FP32 weights
 * (kept FP16 on the device for inference); loss sum w (g-y)^2 / sum w +
 * lam mean(g^2) and its gradient over n feature rows X [n*8] with targets y
 * and weights w (FP32 device arithmetic, FP64 reduction; params [1281] =
 * W1 (128x8), b1, w2, b2); the fused preconditioner
 * t = -r/(d-theta)(1+clip(g,-0.9,4)) on host vectors (iteration counter
 * `iter` enters the features). */
int gbd_set_precond_weights(gbd_ctx *ctx, const float *params);
int gbd_mlp_loss_grad(gbd_ctx *ctx, const float *X, const float *y, const float *w, int64_t n, const float *params,
                      double lam, double *loss, double *grad);
int gbd_mlp_precond(gbd_ctx *ctx, const double *r, const double *d, double theta, double iter, int64_t n, double *t);
/* Davidson iteration count and learned-preconditioner fallbacks so far. */
int gbd_davidson_counts(gbd_ctx *ctx, int64_t *iterations, int64_t *fallbacks, int64_t *samples);
/* ---- host-only pieces of the planner (no GPU needed) ---- */
/* The decimation's host eigensolver (Householder + implicit QL): A [n*n]
 * symmetric row-major; w [n] ascending; Z [n*n] with column j = eigenvector j. */
int gbd_host_sym_eig(int32_t n, const double *A, double *w, double *Z);
/* Initial bond dimensions of the seeded MPS for n orbitals, (N_alpha,
 * N_beta) electrons and bond dimension M; n_sectors [n+1], triples [3 cap]. */
int gbd_host_initial_dims(int32_t n, int32_t n_alpha, int32_t n_beta, int32_t M, int32_t *n_sectors,
                          int32_t *triples, int32_t cap);
/* Decimation rule on `count` weights lam (= sigma^2) with sector keys
 * (64 N_alpha + N_beta) and in-sector ranks j: indices of the kept weights
 * in kept order, their number, and the total weight.  max_discarded > 0
 * turns on the per-bond adaptive bond dimension (see
 * gbd_set_adaptive_bond_dim); 0 is the fixed-M rule.  GBD_ERR_ARG for
 * max_discarded < 0 or m_min < 1. */
int gbd_host_select(int32_t count, const double *lam, const int32_t *key, const int32_t *j, int32_t M,
                    double cutoff, double tie, double max_discarded, int32_t m_min, int32_t *kept_index,
                    int32_t *nkept, double *total);
/* MPO bond dimensions [n+1]; if dense != NULL (n <= 5) also the full
 * 4^n x 4^n matrix of the contracted MPO in the product basis
 * |s_0 ... s_{n-1}> (site 0 most significant). */
int gbd_host_mpo(int32_t n, const double *h, int32_t n_chol, const double *chol, int32_t k_switch,
                 int32_t *bond_dims, double *dense);
/* The certified Hermitian-conjugate channel pairs of the MPO of (h, chol)
 * at one bond, as gbd_env_conjugates reports them for a context (side 0 =
 * left environments, 1 = right); host only.  GBD_ERR_ARG for bad sizes or a
 * buffer smaller than the bond's channel count. */
int gbd_host_mpo_conjugates(int32_t n, const double *h, int32_t n_chol, const double *chol, int32_t k_switch,
                            int32_t side, int32_t bond, int32_t *partner, int32_t *sign, int32_t cap,
                            int32_t *count);

#ifdef __cplusplus
}
#endif
#endif
