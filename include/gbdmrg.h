/* gbdmrg -- two-site DMRG sweep engine for GB300 (sm_103a), C ABI.
 *
 * The library takes active-space integrals (the one-electron matrix and the
 * Cholesky factors of the two-electron integrals) to a converged
 * matrix-product state and returns its energy and one-/two-particle reduced
 * density matrices.  That is the role of the DMRG node in the paper's
 * pipeline (Sec. "Contraction-DAG transpose", the paragraph introducing the
 * DMRG node, and Sec. "The DMRG-QD-NEVPT2 energy").  Inside, every two-site step solves the
 * effective Hamiltonian matrix-free against the MPO with Davidson and
 * decimates the enlarged bond by SVD (Fig. 2, Sec. "Cholesky decomposition
 * for the wavefunction"); all contractions run in this library's CUDA
 * kernels on one GPU.
 *
 * Conventions for every entry point:
 *   - return GBD_OK (0) on success, a negative GBD_ERR_* code otherwise;
 *     gbd_last_error(ctx) then holds a one-line reason.  No C++ exception
 *     crosses this boundary.
 *   - input arrays are host memory, read during the call, copied and never
 *     retained; outputs are written into caller-owned host buffers.
 *   - a context owns its device memory and CUDA stream; it is not thread
 *     safe (use one context per host thread).
 */
#ifndef GBDMRG_H
#define GBDMRG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBD_OK 0
#define GBD_ERR_ARG (-1)      /* invalid argument (sizes, symmetry, NaN) */
#define GBD_ERR_OOM (-2)      /* device allocation failed */
#define GBD_ERR_CUDA (-3)     /* a CUDA call failed */
#define GBD_ERR_NOCONV (-4)   /* no converged or well-defined result (Davidson, eigensolver,
                                 too few roots of the target spin, degenerate ordering) */
#define GBD_ERR_TIMEOUT (-5)  /* a bounded device wait ran out */
#define GBD_ERR_STATE (-6)    /* call order violated (e.g. sweep before prepare) */

/* precision of the Davidson matvecs (sigma build).  GBD_TF32 / GBD_BF16:
 * tensor-core tiers -- the named precision while ||r|| is large, then TF32x3
 * (split TF32 hi/lo, FP32 accumulation) -- then optional FP64 refinement.
 * Environments, H_eff diagonal, Davidson orthogonalisation, Rayleigh-Ritz,
 * decimation and the final energy are FP64 in every mode. */
#define GBD_FP64 0
#define GBD_TF32 1
#define GBD_BF16 2

/* Davidson correction t from the Ritz pair (theta, x) and residual r, with
 * den = d - theta kept at least 1e-8 from zero (d: H_eff diagonal).  The
 * paper names a run-time-selectable family: Jacobi, deflation-aware
 * diagonal, Olsen, and shift-and-invert inner PCG with an indefiniteness
 * guard (Sec. "Computational details").  None changes the converged energy.
 *   GBD_PRECOND_DIAG    Jacobi: t = -r / den
 *   GBD_PRECOND_LEARNED diagonal step scaled by a trained network (below)
 *   GBD_PRECOND_OLSEN   t = -(r - eps x) / den, eps = (x.r/den)/(x.x/den): x.t = 0
 *   GBD_PRECOND_PCG     t from at most 4 preconditioned CG steps on
 *                       (1 - xx^T)(H_eff - theta)(1 - xx^T) t = -r, t orthogonal to x
 *                       (preconditioner: the Olsen-projected den), stopping at
 *                       |residual| < 0.1 |r| or at a direction of non-positive
 *                       curvature; each step costs one extra sigma build.
 * The deflation-aware diagonal belongs to deflated excited-state solves: in
 * gbd_solve_states every member above sees den + penalty * sum_j phi_j^2
 * as its diagonal. */
#define GBD_PRECOND_DIAG 0
#define GBD_PRECOND_LEARNED 1
#define GBD_PRECOND_OLSEN 2
#define GBD_PRECOND_PCG 3

typedef struct gbd_ctx gbd_ctx;

/* Active-space problem (Sec. "The DMRG-QD-NEVPT2 energy"):
 *   H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps)
 *   (pq|rs) = sum_Q chol[Q,p,q] chol[Q,r,s]   (Cholesky-factorised ERIs)
 * h:    [n_orb * n_orb] row-major, symmetric to 1e-12, finite.
 * chol: [n_chol * n_orb * n_orb] row-major, each slice symmetric.
 * n_elec in [0, 2 n_orb]; n_elec and two_sz have equal parity;
 * |two_sz| <= min(n_elec, 2 n_orb - n_elec).  2 <= n_orb <= 32.
 * e_core is added to every returned energy. */
typedef struct {
  int32_t n_orb, n_elec, two_sz, n_chol;
  const double *h;
  const double *chol;
  double e_core;
} gbd_problem;

/* Sweep schedule.  One sweep = left-to-right over the bonds (0,1)..(n-2,n-1)
 * then right-to-left back, 2(n-1) two-site steps.
 * bond_dim[s], davidson_tol[s]: bond dimension M and the tolerance on the
 * residual norm ||H psi - theta psi|| of the normalised Ritz vector, per
 * sweep s.  svd_cutoff: discarded-weight floor on sigma^2 (0 -> 1e-12).
 * seed: seeds the counter-based initial MPS. */
typedef struct {
  int32_t n_sweeps;
  const int32_t *bond_dim;
  const double *davidson_tol;
  int32_t davidson_max_iter;      /* per two-site step (0 -> 100) */
  int32_t davidson_max_subspace;  /* restart size limit (0 -> 24) */
  int32_t precision;              /* GBD_FP64 | GBD_TF32 | GBD_BF16 */
  int32_t preconditioner;         /* GBD_PRECOND_DIAG | _LEARNED | _OLSEN | _PCG */
  uint64_t seed;
  double svd_cutoff;
  int32_t fp64_refine;            /* GBD_TF32/GBD_BF16: at most this many FP64
                                     Davidson iterations after the tensor-core
                                     tiers when ||r|| is still above tol (0 = none) */
} gbd_schedule;

/* Results.  sweep_energies: [n_sweeps] caller-owned (may be NULL); rdm1
 * [n^2] and rdm2 [n^4] caller-owned or NULL (skipped).  RDM conventions:
 * rdm1[p,q] = sum_s <a+_ps a_qs>, rdm2[p,q,r,s] = sum_st <a+_ps a+_rt a_st a_qs>,
 * so E = sum h rdm1 + 1/2 sum (pq|rs) rdm2 + e_core. */
typedef struct {
  double energy;
  double *sweep_energies;
  double *rdm1;
  double *rdm2;
  double max_discarded_weight;
  int64_t n_matvec;
  int32_t status;
} gbd_result;

/* Create a context on CUDA device `device_ordinal`. */
int gbd_create(gbd_ctx **ctx, int device_ordinal);
/* Release all device memory and the stream of a context (NULL is a no-op). */
void gbd_destroy(gbd_ctx *ctx);
/* Reason for the last failure on this context ("" if none). */
const char *gbd_last_error(const gbd_ctx *ctx);

/* Full solve: validate, build the MPO, initial MPS and environments on the
 * device, run the schedule, then energy and RDMs.  Host<->device traffic is
 * the inputs once and the results once. */
int gbd_solve(gbd_ctx *ctx, const gbd_problem *problem, const gbd_schedule *schedule,
              gbd_result *result);

/* Excited states by penalty deflation (Sec. "Excited states: dual-penalty
 * deflation and NACMEs").  Roots are solved one after another, each from
 * its own seeded initial MPS (seed + attempt), with every earlier root kept
 * on the device and added to H_eff of every two-site step as
 * penalty * |phi_j><phi_j|.  Here phi_j is that root projected onto the
 * current two-site basis through overlap environments, and the Davidson
 * diagonal gains penalty * phi_j^2 (the deflation-aware diagonal).
 * penalty (Ha, > 0) must exceed the gap between the wanted roots and the
 * ones below them.
 *
 * Root selection by <S^2>: each converged root gets
 * <S^2> = -1/2 sum_pq rdm2[p,q,q,p] - N^2/4 + N from its 2-RDM.  When
 * target_s2 >= 0, a root with |<S^2> - target_s2| >= 0.1 is not reported
 * but stays deflated (an M_s = 0 triplet, say, when singlets are wanted).
 * At most n_states + max_extra roots are solved.  The dual penalty of the
 * paper (lambda S_z^2 + mu (N - N_el)^2) is zero in the (N_alpha, N_beta)
 * sector this solver is blocked by, so it is not applied.
 *
 * results[0 .. *n_found-1] are filled as by gbd_solve: energy = <H> of the
 * root without the penalty; sweep energies are the Ritz values with it.
 * s2[i] is the root's <S^2>.  Returns GBD_OK when n_states roots were
 * found, else GBD_ERR_NOCONV with the roots found so far in place. */
int gbd_solve_states(gbd_ctx *ctx, const gbd_problem *problem, const gbd_schedule *schedule, int32_t n_states,
                     double penalty, double target_s2, int32_t max_extra, gbd_result *results, double *s2,
                     int32_t *n_found);

/* Fiedler ordering of the orbitals (Sec. "Cholesky decomposition for the
 * wavefunction", ingredient (ii): the lattice is ordered by mutual
 * information).  W: [n*n] symmetric, non-negative couplings between
 * orbitals (diagonal ignored), e.g. a mutual-information matrix, supplied
 * by the caller; this library does not compute two-orbital density
 * matrices.  order[k] = the original orbital to place at site k: the
 * eigenvector f of the second-smallest eigenvalue of the Laplacian
 * diag(W 1) - W, ascending (equal values by index), in the direction that
 * starts at the smaller index.  Permute the integrals before a solve:
 * h'[a][b] = h[order[a]][order[b]], likewise each Cholesky slice.  Host
 * only.  GBD_ERR_ARG for an asymmetric, negative or non-finite W;
 * GBD_ERR_NOCONV when that eigenvalue is degenerate or the graph is
 * disconnected. */
int gbd_host_fiedler_order(int32_t n, const double *W, int32_t *order);

/* Spin-summed three-particle RDM of the state the last gbd_solve (or
 * gbd_init_state / sweeps / gbd_set_mps) on this context left, one of the
 * densities the paper forms on the device (Sec. "Computational details"):
 *   rdm3[((((p n + q) n + r) n + s) n + t) n + u]
 *     = sum_{sigma,tau,upsilon} <a+_p sigma a+_r tau a+_t upsilon a_u upsilon a_s tau a_q sigma>
 * (the index convention of gbd_result.rdm2 extended by one pair), n^6
 * doubles, caller-owned.  Computed in FP64 from the determinant expansion of
 * the MPS; it needs 2 n^2 vectors of the determinant length on the device,
 * so it is refused (GBD_ERR_ARG) above 64 GB of them (CAS(12,12): 2 GB).
 * GBD_ERR_STATE without a state. */
int gbd_rdm3(gbd_ctx *ctx, double *rdm3);

/* Orbital entropies and mutual information of the same state (the paper
 * orders the lattice by the mutual information, Sec. "Cholesky
 * decomposition for the wavefunction", ingredient (ii)):
 * s1[i] = -tr rho_i ln rho_i of the one-orbital RDM, mi[i n + j] = s_i + s_j
 * - s_ij with s_ij the entropy of the two-orbital RDM (0 on the diagonal;
 * values below 0 from rounding are set to 0).  The RDMs are fermionic partial
 * traces of the determinant expansion (up to 4e8 determinants).  s1 or mi
 * may be NULL.  GBD_ERR_STATE without a state. */
int gbd_orbital_entropies(gbd_ctx *ctx, double *s1, double *mi);

/* Orbital order by mutual information: a preliminary solve of `problem`
 * with `schedule` (typically a small bond dimension and a few sweeps), the
 * mutual information of its state (gbd_orbital_entropies), and the Fiedler
 * order of that coupling (gbd_host_fiedler_order): order[k] = the orbital to
 * place at site k; mi [n*n] (may be NULL) receives the coupling.  The caller
 * permutes h and the Cholesky slices and solves again.  Errors as for
 * gbd_solve and gbd_host_fiedler_order. */
int gbd_mi_order(gbd_ctx *ctx, const gbd_problem *problem, const gbd_schedule *schedule, int32_t *order,
                 double *mi);

/* Many independent active spaces in one call (the paper solves one active
 * space per call; batching is this library's addition).  problems[i] is
 * solved with schedules[i] into results[i] (caller-owned, as for
 * gbd_solve), i = 0..n-1.  Every problem and schedule is validated before
 * any work starts: on a bad one nothing runs, no result is touched, and
 * GBD_ERR_ARG names its index.  The problems are then handed, most expensive first (n_orb x
 * M^3 x sweeps), to a pool of host worker threads, each with its own
 * engine, CUDA stream and device memory, so that the kernels of different
 * problems run concurrently on the device.  Results do not depend on the
 * number of workers or on the order of completion.  A problem that fails
 * at run time sets results[i].status to its error code; the others still
 * run, and the call returns the code of the failed problem with the
 * lowest index (its message in gbd_last_error).  Learned preconditioning
 * uses the weights this context holds. */
int gbd_solve_batched(gbd_ctx *ctx, int32_t n, const gbd_problem *problems, const gbd_schedule *schedules,
                      gbd_result *results);
/* Worker threads of gbd_solve_batched: 0 (default) = min(n, 16, host
 * hardware threads); otherwise at most `workers`. */
int gbd_set_batch_workers(gbd_ctx *ctx, int32_t workers);

/* Splitting a set of independent active spaces over several GPUs (one
 * process per GPU; the paper runs on one device, so this is the library's
 * own addition).  gbd_host_batch_costs writes the estimated cost of each
 * problem, n_orb x M_max^3 x n_sweeps (the order gbd_solve_batched hands
 * problems out in).  gbd_host_partition assigns n problems with costs
 * cost[i] >= 0 to `ranks` ranks by longest-processing-time-first greedy:
 * problems in descending cost (equal costs by index), each to the rank with
 * the smallest load so far (equal loads: the lowest rank).  owner[i] = the
 * rank of problem i; load[r] (may be NULL) = the summed cost of rank r.  The
 * result is a deterministic function of the costs, so every rank computes
 * the same partition without communication.  Host only, no GPU needed.
 * GBD_ERR_ARG for n < 0, ranks < 1, NULL arrays with n > 0, or a negative
 * or non-finite cost. */
int gbd_host_batch_costs(int32_t n, const gbd_problem *problems, const gbd_schedule *schedules, double *cost);
int gbd_host_partition(int32_t n, const double *cost, int32_t ranks, int32_t *owner, double *load);

/* Learned Davidson preconditioner (not in the paper, which names Jacobi,
 * deflation-aware diagonal, Olsen and shift-and-invert members of a
 * run-time-selectable family, Sec. "Computational details"; the reading used
 * here): a pointwise two-layer MLP (8 features -> 128 ReLU -> 1, FP16
 * weights, FP32 math) rescales the Jacobi step, t_i = -r_i/(d_i-theta)(1+g_i).
 * With schedule.preconditioner = GBD_PRECOND_LEARNED a context uses the
 * weights it holds; a Davidson solve falls back to the diagonal when ||r||
 * stops dropping for three iterations or a correction is not finite, so the
 * converged energy never depends on the network. */
/* Solve each problem with the diagonal preconditioner while recording
 * residual samples (2048 positions per Davidson iteration) and, once each
 * step converges, the targets; then train the network on the device
 * (full-batch Adam, `epochs` steps, learning rate lr).  final_loss may be
 * NULL.  The context keeps the trained weights. */
int gbd_train_precond(gbd_ctx *ctx, int32_t n_problems, const gbd_problem *problems,
                      const gbd_schedule *schedules, int32_t epochs, double lr, double *final_loss);
/* Store / load the network weights (file: "GBDMLP1\n", F, H, FP32 weights). */
int gbd_save_precond(gbd_ctx *ctx, const char *path);
int gbd_load_precond(gbd_ctx *ctx, const char *path);

#ifdef __cplusplus
}
#endif
#endif
