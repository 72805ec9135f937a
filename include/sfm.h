/*
 * libsfm - S-fraction multiscale finite-volume wave propagation on one GPU.
 *
 * C ABI of the GB300 (sm_103a) library.  The method is Druskin, Mamonov and
 * Zaslavsky, "S-fraction multiscale finite-volume method for spectrally
 * accurate wave propagation": the domain is split into box subdomains, each
 * subdomain's fine-grid operator is reduced offline to a reduced-order model
 * (ROM) in matrix S-fraction form (Algorithm 1 stage 1, Eqs. 5-13), and the
 * ROMs are stepped together with explicit leapfrog, coupled through the
 * m-dimensional face data of shared subdomain faces at every step
 * (Algorithm 1 stage 2, Eqs. 17-19).
 *
 * Conventions used by every call
 * -------------------------------
 *  - Every call returns an int status: SFM_OK (0) or a negative SFM_ERR_*.
 *    sfm_last_error() describes the last failure on a handle.
 *  - A handle owns all device memory it allocates; nothing is shared
 *    between handles.  Calls on one handle must not run concurrently.
 *  - Array arguments are host memory, row-major, owned by the caller, and
 *    read or written only during the call (never retained), unless the call
 *    says otherwise.
 *  - Subdomains are numbered 0..nsub-1.  Faces of a subdomain are numbered
 *    0..5 = -x, +x, -y, +y, -z, +z.  A subdomain's block width is
 *    b = sum over its 6 faces of the face mode counts m_f; its state has k
 *    levels U_1..U_k, each in R^b; level 1 is split into the 6 face blocks
 *    in face order.
 *  - Sign convention: with the paper's u_tt = A u (A <= 0) we use L = -A;
 *    all S-fraction coefficients are symmetric positive (semi)definite.
 */
#ifndef SFM_H
#define SFM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfm_handle sfm_handle;

enum sfm_status {
    SFM_OK = 0,
    SFM_ERR_ARG = -1,        /* invalid argument or size                      */
    SFM_ERR_CUDA = -2,       /* a CUDA runtime call failed                    */
    SFM_ERR_NOT_SPD = -3,    /* a coefficient block is not positive definite  */
    SFM_ERR_BREAKDOWN = -4,  /* rank-deficient block in the block Krylov step */
    SFM_ERR_UNSTABLE = -5,   /* non-finite traces (time step above the CFL)   */
    SFM_ERR_TIMEOUT = -6,    /* a device-wide barrier timed out               */
    SFM_ERR_NOMEM = -7,      /* device allocation failed                      */
    SFM_ERR_STATE = -8       /* call made before the data it needs was set    */
};

enum sfm_precision {
    SFM_FP64 = 0,            /* FP64 coefficients, state and sums              */
    SFM_FP32 = 1,            /* FP32 coefficients, state and sums              */
    SFM_FP32X2 = 2,          /* two-float numbers (hi + lo FP32, ~48-bit
                                significand) with compensated FP32 arithmetic */
    SFM_FP32F = 3,           /* FP32 state and sums; each S-fraction block
                                applied through its FP32 Cholesky factor,
                                Gamma = L L^T (factored in FP64 on the GPU),
                                which keeps it positive semi-definite under
                                rounding                                       */
    SFM_TF32X3 = 4,          /* multi-shot panels: shots stepped 16 at a time,
                                every factor product L (L^T X) on the tensor
                                cores with TF32 inputs split into head and
                                tail words (3 products, FP32 accumulation);
                                FP32 factors and state                         */
    SFM_TF32 = 5,            /* as SFM_TF32X3 with single-word TF32 inputs
                                (11 significant bits; deep ROMs diverge)       */
    SFM_BF16 = 6,            /* not built: sfm_run returns SFM_ERR_ARG (BF16's
                                8-bit significand is coarser than TF32's)      */
    SFM_FP32FX2 = 7,         /* SFM_FP32F's FP32 Cholesky factors (the same
                                coefficient bytes) with the state, the vectors
                                of each product and its sums in SFM_FP32X2's
                                two-float form: the factors' rounding is the
                                only FP32 rounding                             */
    SFM_FP32X2P = 8          /* multi-shot panels as SFM_TF32X3 (shots 16 at a
                                time, each S-fraction block read once for the
                                16), with SFM_FP32X2's two-float blocks, state
                                and face data and compensated products on the
                                CUDA cores: SFM_FP32X2's accuracy for deep
                                ROMs that no FP32-coefficient mode steps
                                within 1e-3                                    */
};

/* flags for sfm_run */
#define SFM_DEVICE_PTR 1     /* wavelet/traces are device pointers            */
#define SFM_ENERGY 2         /* evaluate the discrete energy at the start and
                                the end of the run (sfm_run_report)            */

/* Report of the last sfm_run on a handle (sfm_run_report). */
typedef struct sfm_run_info {
    int precision;           /* precision of the run, -1 before the first one  */
    int nsteps, nshots;
    int launches;            /* device kernels launched by the call            */
    double kernel_ms;        /* device time of the stepping kernel alone       */
    double total_ms;         /* the whole call, host wall clock                */
    int status;              /* the call's return code                         */
    int unstable_step;       /* time step at which the instability sentinel
                                stopped the run, -1 if it did not              */
    int energy;              /* 1 if energies were evaluated (SFM_ENERGY)       */
} sfm_run_info;

/* Create a handle bound to CUDA device `device`.  *h receives the handle.
 * Errors: SFM_ERR_ARG (h NULL, bad device), SFM_ERR_CUDA. */
int sfm_create(sfm_handle** h, int device);

/* Free the handle and all device memory it owns.  NULL is accepted. */
int sfm_destroy(sfm_handle* h);

/* Static text describing the last error on h (or a global error when h is
 * NULL).  Valid until the next call on the same handle. */
const char* sfm_last_error(const sfm_handle* h);

/* Make every later call on h enqueue its work on `stream` (a cudaStream_t
 * of h's device, owned by the caller and never destroyed by the library);
 * NULL goes back to a stream the handle owns.  Waits for the handle's
 * previous stream first. */
int sfm_set_stream(sfm_handle* h, void* stream);

/*
 * Subdomain topology (the split of section "Introduction" and the faces
 * B^{ab} of section "Stage 1").
 *   nsub          number of subdomains
 *   k_sub[nsub]   number of S-fraction levels k of each subdomain (>= 1)
 *   m_face[nsub*6] modes on each face of each subdomain (>= 0); both sides
 *                 of a shared face must give the same count
 *   nbr[nsub*6]   neighbour across each face, -1 for an outer face
 *                 (homogeneous Neumann); must be symmetric: if nbr[s][f] = t
 *                 then nbr[t][f^1] = s.
 * Limits of the stepping kernels: m <= 32 on a face, block width
 * b_s = sum of the six face counts in 1..192, k_s * b_s <= 16384.  Blocks
 * wider than 64 (the paper's 25 modes per face give b = 150) step in
 * SFM_FP64, SFM_FP32X2 and SFM_FP32 and build with sfm_build_roms; the
 * factored and panel modes, the energy report (SFM_ENERGY), sfm_cut_depth,
 * the surrogate calls and sfm_run_static return SFM_ERR_ARG for them.
 * Resets coefficients, sources and receivers.
 * Errors: SFM_ERR_ARG for inconsistent topology or sizes beyond the limits.
 */
int sfm_set_topology(sfm_handle* h, int nsub, const int* k_sub, const int* m_face,
                     const int* nbr);

/*
 * S-fraction coefficients Gamma_j and Gammahat_j, j = 1..k (Eq. 13; used by
 * Eqs. 12, 18, 19).  For each subdomain s in order: k_s blocks Gamma_1..
 * Gamma_k, then k_s blocks Gammahat_1..Gammahat_k, each b_s x b_s row-major
 * FP64 (symmetric).  `count` is the total number of doubles.  Gammahat_1
 * must be block diagonal over the faces (its face blocks define the face
 * coupling H_f = (sum over the sides of a face of [Gammahat_1]_f^{-1})^{-1}
 * of Eq. 18, computed on the device in FP64).
 * Errors: SFM_ERR_ARG (count mismatch), SFM_ERR_STATE (no topology),
 * SFM_ERR_NOT_SPD (a face block of Gammahat_1 failed its Cholesky).
 */
int sfm_set_coeffs(sfm_handle* h, const double* coeffs, size_t count);

/* Copy the FP64 coefficients currently held (same layout as sfm_set_coeffs)
 * into `coeffs` (capacity `count` doubles); *needed receives the size. */
int sfm_get_coeffs(sfm_handle* h, double* coeffs, size_t count, size_t* needed);

/*
 * Projected point sources (Algorithm 1 step 1.4 / Eq. 16): the force of shot
 * q acts on level j of subdomain s as Gammahat_j p_j f_q(t).  Given as
 * npairs (shot, subdomain) pairs; pair i has rows[off_i .. off_i + k_s*b_s)
 * (levels 1..k, each b_s long), with off_i the running sum of the previous
 * pairs' k*b.  A (shot, subdomain) pair may appear at most once.
 */
int sfm_set_sources(sfm_handle* h, int nshots, int npairs, const int* pair_shot,
                    const int* pair_sub, const double* rows);

/*
 * Projected receivers: receiver r reads d_r = sum over its pairs of
 * sum_j rho_j^T U_j (Eq. 16 inverted).  Layout as sfm_set_sources.
 */
int sfm_set_receivers(sfm_handle* h, int nrec, int npairs, const int* pair_rec,
                      const int* pair_sub, const double* rows);

/*
 * Initial state of the coupled stepping (Algorithm 1 step 1.4 for initial
 * conditions; Stage 2 starts from U_j|t=0 and dU_j/dt|t=0): per (shot,
 * subdomain) pair a row block u0_rows[k_s][b_s] of U_j(0) and, unless
 * v0_rows is NULL (zero velocity), one of dU_j/dt(0), both FP64, pairs
 * concatenated in the order given; pairs not listed start at rest.  For a
 * nodal field u the rows are U_j = G_j [Qh^T V^T M^{1/2} u]_j (Eq. 16).
 * sfm_run then starts with U^0 and the increment
 *     delta^0 = dt V^0 - dt^2/2 a_hom(U^0)
 * (the second-order Taylor start; a_hom: the right-hand side of Eqs.
 * 18-19 without the source, evaluated in FP64 on the GPU).  nshots must
 * equal the sources' shot count at sfm_run.  npairs = 0 clears the initial
 * state.  Host arrays, copied.  Errors: SFM_ERR_ARG, SFM_ERR_STATE (no
 * topology).  sfm_run_static always starts from rest.
 */
int sfm_set_initial(sfm_handle* h, int nshots, int npairs, const int* pair_shot,
                    const int* pair_sub, const double* u0_rows, const double* v0_rows);

/*
 * Coupled leapfrog time stepping (Algorithm 1 stage 2): from rest (or from
 * the state of sfm_set_initial), for
 * n = 0..nsteps-1 the right-hand sides of Eqs. 18-19 (with the source term
 * f_q(t_n)) are evaluated at t_n = n*dt and
 *     delta^{n+1} = delta^n + dt^2 a^n,  U^{n+1} = U^n + delta^{n+1}.
 *   precision      SFM_FP64, SFM_FP32, SFM_FP32X2, SFM_FP32F or SFM_FP32FX2
 *                  (one kernel over every shot), SFM_TF32X3, SFM_TF32 or
 *                  SFM_FP32X2P (the multi-shot panels); the factored
 *                  modes first factor every block used (SFM_ERR_NOT_SPD if
 *                  one is not positive definite in FP64)
 *   wavelet        [nshots][nsteps] FP64 samples f_q(t_n)
 *   traces         [nshots][nrec][nsteps+1] FP64 output, d_r(t_n), n=0..nsteps
 *   flags          SFM_DEVICE_PTR: wavelet and traces are device pointers
 *   kernel_ms      if not NULL, receives the device time of the persistent
 *                  stepping kernel alone (CUDA events around its launch)
 * All shots are stepped in one launch.  One persistent cooperative kernel
 * runs every step; the only cross-block dependency per step is one
 * device-wide barrier between the face-data publication (step 2.1, with
 * 2.2) and the face update (step 2.3).
 * Errors: SFM_ERR_STATE (missing data), SFM_ERR_TIMEOUT (barrier timed out),
 * SFM_ERR_UNSTABLE (non-finite traces), SFM_ERR_NOT_SPD, SFM_ERR_CUDA.
 */
int sfm_run(sfm_handle* h, int precision, double dt, int nsteps, const double* wavelet,
            double* traces, int flags, double* kernel_ms);

/*
 * Report of the last sfm_run (Stage 2's leapfrog and its conserved energy).
 * info receives the run's precision, size, launches, timings, status and the
 * sentinel's step: every step checks each updated face-block entry, and a
 * non-finite value or one beyond 1e30 sets SFM_ERR_UNSTABLE and stops the
 * persistent kernel at its next device-wide barrier, so a run above the CFL
 * limit ends within a few steps of its blow-up instead of after nsteps.
 * With SFM_ENERGY the run evaluated, in FP64 on the device, the discrete
 * energy of the assembled leapfrog (Eqs. 17-19 as one system MM U'' = -KK U)
 *     E^{n+1/2} = 1/2 (delta/dt)^T MM (delta/dt) + 1/2 (U^{n+1})^T KK U^n,
 * delta = U^{n+1} - U^n, once for the starting state (n = -1: U^0 and
 * delta^0) and once for the final one (n = N - 1); without a source term it
 * is conserved.  energy[0 .. nshots-1] receives the start values and
 * energy[nshots .. 2 nshots-1] the end values (capacity >= 2 nshots; NULL
 * skips them).  Errors: SFM_ERR_ARG.
 */
int sfm_run_report(const sfm_handle* h, sfm_run_info* info, double* energy, int capacity);

/*
 * Largest eigenvalue of the coupled ROM system's MM^{-1} KK and the leapfrog
 * limit dt_cfl = 2/sqrt(lambda_max): `iters` power iterations with the FP64
 * stepping operator, reporting the Rayleigh quotient q^T KK q / q^T MM q in
 * the MM inner product (a lower bound that converges quadratically).
 * Either output may be NULL.
 */
int sfm_cfl_dt(sfm_handle* h, int iters, double* lambda_max, double* dt_cfl);

/*
 * Shape search for the stepping kernel of `precision` on this handle (no
 * counterpart in the paper, whose method fixes no launch shape).  Each
 * candidate block shape - consumer warps in {2,4,6,8} times
 * coefficient ring stages in {2,3,4,6,8,12,16}, those whose shared memory
 * fits (for SFM_FP32F only stage counts that are multiples of the warps;
 * for the panel modes
 * 16-shot groups per task in {1, 2, 4, 8} times stages in {2, 3, 4, 6, 8}) -
 * steps the coupled system `nsteps` steps from rest with a zero source
 * twice (a state from sfm_set_initial or sfm_restore is left aside for
 * the probes and kept for the next sfm_run); the
 * fastest (step kernel alone, CUDA events) becomes the shape of later
 * sfm_run calls in that precision.  Results do not depend on the shape:
 * every shape sums in the same order.  Outputs: the chosen consumer warps,
 * ring stages and microseconds per time step; any may be NULL.  Needs
 * coefficients, sources and receivers.  Errors: as sfm_run.
 */
int sfm_autotune(sfm_handle* h, int precision, int nsteps, int* ncw, int* nstage,
                 double* us_per_step);

/*
 * Checkpoint of the stepping state: U^N and the increment delta^N =
 * U^N - U^{N-1} left by the last successful sfm_run (N its nsteps), for all
 * its shots, converted to FP64, in a self-describing blob (native byte
 * order, 8-byte aligned buffer): 8 int64 words {magic, version, nshots,
 * nstate, nsub, topology fingerprint, N, precision} followed by U^N and
 * delta^N, nshots * nstate doubles each, in the state layout (per shot,
 * per subdomain, levels 1..k of b numbers).  *bytes: on entry the capacity
 * of buf, on return the size needed; buf NULL only asks for the size.
 * sfm_autotune and sfm_set_topology discard the state.  Errors:
 * SFM_ERR_STATE (no state), SFM_ERR_ARG (capacity too small).
 *
 * Restore: the next sfm_run (and every later one, until sfm_set_initial or
 * sfm_set_topology) starts from that U^0 and delta^0 instead of from rest,
 * so an N-step run, its checkpoint, and an M-step run from the restored
 * state with the wavelet samples N..N+M-1 give the traces of one N+M-step
 * run (sample 0 of the second run repeats sample N of the first).  The
 * handle's topology must match the checkpoint's and its source shot count
 * must equal the checkpoint's at sfm_run.  Host buffer, copied.  Errors:
 * SFM_ERR_ARG (not a checkpoint, other topology, size mismatch),
 * SFM_ERR_STATE (no topology).
 */
int sfm_checkpoint(sfm_handle* h, void* buf, size_t* bytes);
int sfm_restore(sfm_handle* h, const void* buf, size_t bytes);

/*
 * ---------------------------------------------------------------------------
 * Offline stage on the GPU (Algorithm 1 stage 1, FP64)
 * ---------------------------------------------------------------------------
 * Fine operator (the paper leaves it generic, Eq. 1; this library reads it
 * as vertex-centred finite volumes for u_tt = c^2 Laplacian u): each cell of
 * side h adds h/4 to the conductance of its 12 edges and h^3/(8 c^2) to the
 * lumped mass of its 8 corners; subdomain boundaries are natural (Neumann).
 * Face basis (section "Stage 1"): m cosine modes per face on the OPEN face
 * (face nodes on no subdomain edge, so different faces never overlap),
 * cos(pi p (s-1/2)/n_s) cos(pi q (t-1/2)/n_t) times h^2, modes by ascending
 * p^2+q^2, then q, then p; a shared face carries min(m_a, m_b) modes.
 */

/* Velocity model c[nz][ny][nx] (m/s, cell-centred, FP64) on cells of side
 * hgrid and the subdomain cuts per axis (node indices, cuts[0] = 0,
 * cuts[n] = n, at least 2 cells per subdomain).  Subdomain (ix,iy,iz) is
 * numbered ix + ncx*(iy + ncy*iz).  Errors: SFM_ERR_ARG. */
int sfm_set_model(sfm_handle* h, int nx, int ny, int nz, double hgrid, const double* c,
                  int ncx, const int* xcuts, int ncy, const int* ycuts, int ncz,
                  const int* zcuts);

typedef struct sfm_build_report {
    double seconds;            /* wall time of the build                        */
    int cg_iterations_max;     /* most CG iterations of one block solve          */
    double cg_residual_max;    /* worst final relative residual of the solves    */
    double krylov_min_ratio;   /* smallest min/max diag of a Krylov block's R    */
    int nclasses;              /* subdomain shape classes built as batches       */
    int nregularized;          /* blocks projected on the semi-definite cone
                                  (deep levels singular at FP64 rounding level)  */
} sfm_build_report;

/*
 * Build every subdomain's ROM and its S-fraction coefficients (Alg. 1 steps
 * 1.1-1.3): V = orth[F, (L+sigma)^{-1}F, ..., (L+sigma)^{-(k-1)}F] (the
 * rational block Krylov space of Eq. 6 with one repeated shift sigma > 0 and
 * F itself as the first block, each solve a Jacobi-preconditioned CG to the
 * relative residual cg_tol, block Gram-Schmidt twice), L~ = V^T L V,
 * F~ = V^T F (Eq. 5), block Lanczos on (L~, F~) with full
 * reorthogonalisation (Eq. 8) and the recursion of Eq. 13.  Every finished
 * block is test-factored in FP64; one with a non-positive pivot (a deep
 * level whose smallest eigenvalues sit at the rounding level, some of them
 * rounded below zero) is replaced by its projection on the positive
 * semi-definite cone (negative eigenvalues set to 0; counted in
 * rep->nregularized).  Sets the
 * topology and coefficients exactly as sfm_set_topology + sfm_set_coeffs
 * would.  m_sub[nsub], k_sub[nsub]: modes per face and levels per subdomain.
 * Errors: SFM_ERR_STATE (no model), SFM_ERR_ARG (block width above 64 or
 * more modes than open-face nodes), SFM_ERR_BREAKDOWN (a rank-deficient
 * block or a CG that did not converge), SFM_ERR_NOT_SPD, SFM_ERR_NOMEM.
 */
int sfm_build_roms(sfm_handle* h, const int* m_sub, const int* k_sub, double sigma,
                   double cg_tol, sfm_build_report* rep);

/* The same build with distinct finite shifts (Eq. 6's rational Krylov
 * family): block j+1 of the subspace is (L + shifts[j-1])^{-1} applied to
 * block j, j = 1..k_s-1, so the subspace holds F and (L + sigma_j)^{-1} F
 * for every shift and the ROM interpolates the NtD map and its derivative
 * at each of them.  shifts[nshifts] > 0, nshifts >= max k - 1; a subdomain
 * with k_s levels uses the first k_s - 1.  Equal shifts give sfm_build_roms.
 * Errors: as sfm_build_roms. */
int sfm_build_roms_shifts(sfm_handle* h, const int* m_sub, const int* k_sub, const double* shifts,
                          int nshifts, double cg_tol, sfm_build_report* rep);

/* Algorithm 1 step 1.4 for point forces: a normalised Gaussian of the given
 * width (cut at 3 widths) around each point xyz[nshots][3] (metres); a node
 * shared by several subdomains gives each the share M^a/M of its force.
 * Projects with the bases of the last sfm_build_roms and sets the sources as
 * sfm_set_sources would.  Errors: SFM_ERR_STATE (nothing built). */
int sfm_project_sources(sfm_handle* h, int nshots, const double* xyz, double width);

/* Receivers reading the trilinear interpolation of nodal u at xyz[nrec][3],
 * the value at a shared node being the mass-weighted mean over its copies.
 * Sets the receivers as sfm_set_receivers would. */
int sfm_project_receivers(sfm_handle* h, int nrec, const double* xyz);

/* Release the offline builder's per-subdomain bases (Krylov V, Lanczos
 * basis, masses); the coefficients, sources and receivers already set stay.
 * Projecting new points afterwards needs a new sfm_build_roms. */
int sfm_free_build(sfm_handle* h);

/*
 * Usable depth of each subdomain's S-fraction (an extension of the offline
 * stage; the paper's ROMs are three levels deep).  Deep levels of an
 * accurate ROM at a small shift run past FP64's dynamic range: their
 * Gamma_j, Gammahat_j (Eq. 13) have eigenvalues at the rounding level and
 * the fraction's stability limit falls far below the Galerkin ROM's.  The
 * usable depth of subdomain s is the number of leading levels before the
 * first level j whose Gammahat_j, or Gamma_j for j < k_s (Gamma_k is
 * semidefinite by construction), has lambda_min <= tau * lambda_max; at
 * least one level is kept.
 *
 * sfm_usable_depths is the decision alone, on the host (no device work):
 *   range[nsub][2*kmax][2]  (lambda_min, lambda_max) of the blocks of each
 *                           subdomain in the sfm_set_coeffs order (Gamma_1..k
 *                           then Gammahat_1..k); entries past 2 k_s unused
 *   depth[nsub]             out
 * Errors: SFM_ERR_ARG (tau outside [0, 1), k_s outside 1..kmax).
 *
 * sfm_cut_depth computes the ranges of the coefficients held (FP64 cyclic
 * Jacobi on the device), decides the depths with sfm_usable_depths and,
 * when a level goes, keeps levels 1..d_s of every subdomain: coefficients,
 * source, receiver and initial rows (their first d_s levels), set again as
 * sfm_set_topology, sfm_set_coeffs, sfm_set_sources, sfm_set_receivers and
 * sfm_set_initial would; the cut fraction is terminated with U_{d+1} = 0
 * like the full one (Eq. 12).  It releases the offline bases as
 * sfm_free_build does (they describe the uncut fraction), so project the
 * sources and receivers first.  depth_out (depth_cap >= nsub entries, the
 * kept depths) and nlevels_cut (levels removed in all) may be NULL.
 * Errors: SFM_ERR_ARG, SFM_ERR_STATE (no
 * coefficients), SFM_ERR_CUDA, SFM_ERR_NOMEM; after an error past the
 * decision the handle's ROM data are undefined and must be set again.
 */
int sfm_usable_depths(int nsub, const int* k_sub, int kmax, const double* range, double tau,
                      int* depth);
int sfm_cut_depth(sfm_handle* h, double tau, int* depth_out, int depth_cap, int* nlevels_cut);

/*
 * sfm_run_static - the FP64 coupled stepping of sfm_run without allocating
 * any device memory.  (Not a step of the paper's method, which has no
 * counterpart to it: it serves callers of this library that cannot allocate
 * device memory at the time they step, e.g. an application or framework
 * that owns the whole GPU through its own allocator and treats further
 * cudaMalloc calls as errors, or a latency-critical loop that must not pay
 * for the device-wide synchronisation of cudaMalloc/cudaFree.)
 *
 * All inputs and outputs belong to the caller.  Host arrays: k_sub, m_face,
 * nbr (as sfm_set_topology), src_shot/src_sub and rec_id/rec_sub (as
 * sfm_set_sources/sfm_set_receivers).  Device arrays on `device`: coeffs
 * (the sfm_set_coeffs layout, FP64), src_rows and rec_rows (the
 * sfm_set_sources/sfm_set_receivers row layouts, FP64), wavelet
 * [nshots][nsteps] and the output traces [nshots][nrec][nsteps+1] (FP64).
 * Work is enqueued on `stream` (a cudaStream_t, NULL for the legacy default
 * stream) and the call returns when it is done.
 *
 * Scratch memory: one static device array of 64 MiB per GPU, held until
 * the process exits.  It is reserved when the library's device code is
 * loaded on that GPU; with lazy module loading (the CUDA runtime's default)
 * that is the first call on the device, so make one warm-up call before
 * another allocator takes the GPU's memory (a first call that finds no room
 * returns SFM_ERR_CUDA), and before any stream capture.  Every call looks
 * up the array's device address (cudaGetSymbolAddress) with `device`
 * current.  A problem whose layout tables, tile-packed coefficients, state
 * and partial receiver sums need more than 64 MiB returns SFM_ERR_ARG
 * (sfm_last_error(NULL) gives the size needed) before touching the device.
 * Every call shares the one array and re-initialises what must start at
 * zero, so calls that overlap on the GPU (two streams, two host threads)
 * race and must be serialised by the caller.  No cudaMalloc, cudaFree or
 * allocating library routine is called.  The caller's current device is
 * the same on return.
 * Errors: SFM_ERR_ARG, SFM_ERR_CUDA (also an out-of-memory error on the
 * first call on a device), SFM_ERR_TIMEOUT, SFM_ERR_NOT_SPD (checked before
 * any stepping work), SFM_ERR_UNSTABLE, reported through
 * sfm_last_error(NULL).
 */
int sfm_run_static(int device, void* stream, int nsub, const int* k_sub, const int* m_face,
                   const int* nbr, const double* coeffs, int nshots, int nsrc_pairs,
                   const int* src_shot, const int* src_sub, const double* src_rows, int nrec,
                   int nrec_pairs, const int* rec_id, const int* rec_sub, const double* rec_rows,
                   double dt, int nsteps, const double* wavelet, double* traces);

/*
 * ---------------------------------------------------------------------------
 * Learned surrogate of the offline stage (an extension of Algorithm 1 stage
 * 1, Eqs. 5-13: when the velocity changes between inversion iterations, a
 * network maps a subdomain's velocity block to its S-fraction coefficients)
 * ---------------------------------------------------------------------------
 * Network: input log(c / 2500 m/s) on an n^3 block of cells; three 3x3x3
 * convolutions of stride 2 and zero padding 1 with c1, c2, c3 channels and
 * ReLU; a dense layer of `hidden` units with ReLU; a dense layer to a code
 * z of `code` numbers.  Parameters in the order c1 weights [c1][1][3][3][3],
 * c1 biases, c2 weights [c2][c1][3][3][3], c2 biases, c3 weights, c3 biases,
 * W1 [hidden][c3 * m^3] (m = the block side after three stride-2 layers;
 * features flattened channel-major, then z, y, x), b1, W2 [code][hidden],
 * b2.  Training is FP32 (loss: mean over the batch of the mean squared code
 * error; Adam); inference FP32 or BF16 (BF16 weights and convolution
 * activations, FP32 accumulation).  Device arrays are on the network's
 * device; velocities are FP32 [batch][n][n][n] (z, y, x), codes FP32
 * [batch][code].  Errors are reported through sfm_net_last_error.
 */
typedef struct sfm_net sfm_net;

/* Create a network with seeded He-style initial weights (biases zero).
 * Errors: SFM_ERR_ARG (sizes), SFM_ERR_CUDA, SFM_ERR_NOMEM. */
int sfm_net_create(sfm_net** net, int device, int n, int c1, int c2, int c3, int hidden, int code,
                   unsigned long long seed);
int sfm_net_destroy(sfm_net* net);
const char* sfm_net_last_error(const sfm_net* net);

/* All parameters as one FP32 host array in the order above: set = 0 copies
 * them out, set = 1 replaces them (and resets the Adam moments).  *count
 * receives the parameter count; host NULL only asks for it. */
int sfm_net_params(sfm_net* net, float* host, size_t capacity, size_t* count, int set);

/* Loss of a batch of B blocks c (device) against target codes zt (device),
 * and the gradient of every parameter by the backward pass, kept for
 * sfm_net_adam; grad_host (host, parameter count) may be NULL. */
int sfm_net_grad(sfm_net* net, const float* c, const float* zt, int B, float* loss, float* grad_host);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradient. */
int sfm_net_adam(sfm_net* net, float lr);

/* Codes z (device [B][code]) of B blocks c (device); bf16 selects the BF16
 * inference pass. */
int sfm_net_forward(sfm_net* net, const float* c, int B, float* z, int bf16);

/*
 * Decoder of the surrogate (FP64, fixed once fitted, not trained).  A set of
 * S-fraction coefficients of width b and k >= 2 levels is 2k blocks b x b in
 * the sfm_set_coeffs order (Gamma_1..k, Gammahat_1..k); its raw vector is,
 * for the blocks Gamma_2..Gamma_k then Gammahat_2..Gammahat_k, the strictly
 * lower entries of U row by row followed by log of the pivots, where the
 * Cholesky factor of the block is L = U diag(pivots), U unit lower
 * triangular: nraw = 2 (k-1) (b(b-1)/2 + b) numbers per set.  Every raw
 * vector decodes to positive definite blocks L L^T, and a raw error moves a
 * pivot by a relative factor.  Level 1 is not encoded: it has closed forms
 * (Gammahat_1 = F^T F, Gamma_1 = Gammahat_1^{-1} F^T L F Gammahat_1^{-1}).
 *
 * sfm_raw_encode: raw vectors [count][nraw] (device) of count coefficient
 *   sets (device); a pivot at or below 1e-14 of the block's largest
 *   diagonal entry (a level semi-definite to rounding) is floored there.
 * sfm_net_fit_decoder: the decoder of the network for (b, k): mu = the mean
 *   of N raw targets [N][nraw] (device) and P [nraw][code], an orthonormal
 *   basis of their leading principal subspace by randomized subspace
 *   iteration (Halko, Martinsson and Tropp) with `iters` power passes and
 *   Cholesky-QR orthonormalisation, each column then scaled by the RMS of
 *   its coordinate over the targets (so codes are of order one and
 *   mu + P z is unchanged); codes (device FP32 [N][code], may be NULL)
 *   receive the targets' codes (least-squares coordinates in that basis).
 *   N >= code.
 * sfm_net_decode: coefficient sets (device FP64, B sets) of B codes (device
 *   FP32): levels 2..k written from mu + P z, level 1 left untouched.
 * sfm_ntd_error: err[i][l] = |S_a - S_r|_F / |S_r|_F of two families of
 *   count coefficient sets (device) at nlam complex lambda (host
 *   [nlam][re, im]), S the S-fraction's transfer function (Eq. 15) by its
 *   continued fraction Y_k = lambda Gammahat_k^{-1} + Gamma_k,
 *   Y_j = lambda Gammahat_j^{-1} + (Gamma_j^{-1} + Y_{j+1}^{-1})^{-1},
 *   S = Y_1^{-1}, in FP64 complex arithmetic on the device; err is host
 *   [count][nlam].
 * Errors: SFM_ERR_ARG, SFM_ERR_STATE (no decoder), SFM_ERR_BREAKDOWN
 * (rank-deficient targets), SFM_ERR_CUDA, SFM_ERR_NOMEM; through
 * sfm_net_last_error or, without a network, sfm_last_error(NULL).
 */
int sfm_raw_encode(int device, int count, int b, int k, const double* coef, double* raw);
int sfm_net_fit_decoder(sfm_net* net, int b, int k, const double* raw, int N, int iters,
                        unsigned long long seed, float* codes);
int sfm_net_decode(sfm_net* net, const float* z, int B, double* coef);
int sfm_ntd_error(int device, int count, int b, int k, const double* coef_a, const double* coef_r,
                  int nlam, const double* lam, double* err);

/*
 * Offline stage with the surrogate (replacing Algorithm 1 steps 1.1-1.3 for
 * the subdomains the network can serve, with the exact build as fallback).
 * A subdomain is served when it is a cube of the network's n cells, has the
 * decoder's k levels and m = b/6 modes on all six faces (its neighbours'
 * m included), and exact[s] is 0 (exact may be NULL).  For the served
 * subdomains, in batches on the device: level 1 from its closed forms
 * (Gammahat_1 = F^T F, Gamma_1 = Gammahat_1^{-1} F^T L F Gammahat_1^{-1}),
 * levels 2..k from the network (BF16 inference) and its decoder, and one
 * block solve W = (L + sigma)^{-1} F (CG to cg_tol), which gives the exact
 * S(sigma) = F^T W and S'(sigma) = -W^T W; a subdomain whose decoded
 * S-fraction misses either by more than nt_tol (relative Frobenius; its
 * derivative by a central difference) falls back to the exact build, which
 * then runs for the
 * fallbacks and every subdomain not served (as sfm_build_roms would, with
 * the same m_sub, k_sub, sigma and cg_tol).  Coefficients of served
 * subdomains carry no Krylov basis: sources and receivers must not touch
 * them (mark their subdomains exact), else sfm_project_* returns
 * SFM_ERR_STATE.  rep (may be NULL) reports the exact build; srep (may be
 * NULL) the surrogate pass.  Errors: as sfm_build_roms, and SFM_ERR_STATE
 * (the network has no decoder).
 */
typedef struct sfm_surrogate_report {
    int eligible;                 /* subdomains the network served             */
    int accepted;                 /* ... whose S(sigma) passed nt_tol          */
    int fallback;                 /* ... rebuilt exactly                       */
    double sigma_err_median;      /* median of the larger relative error of
                                     S(sigma) and S'(sigma), served            */
    double sigma_err_max_accepted;
    double seconds_surrogate;     /* wall time of the surrogate pass           */
    double seconds_exact;         /* wall time of the exact build that followed */
} sfm_surrogate_report;

int sfm_build_roms_surrogate(sfm_handle* h, sfm_net* net, const int* m_sub, const int* k_sub,
                             double sigma, double cg_tol, double nt_tol, const int* exact,
                             sfm_surrogate_report* srep, sfm_build_report* rep);

/*
 * The stepping kernel's work partition (host logic only, no device work; no
 * counterpart in the paper): the (unit, level) sequence of nunits units,
 * unit u having k_sub[u % nsub] levels, cut into contiguous pieces for
 * `grid` blocks so that the blocks' estimated costs are even; a unit is
 * never cut at level 1.  Outputs: ptr[grid+1] (the pieces of block c are
 * ptr[c] .. ptr[c+1]-1) and pieces[3*i .. 3*i+2] = (unit, j0, j1), levels
 * j0 .. j1-1.  *npieces receives the number of pieces; SFM_ERR_ARG if it
 * exceeds max_pieces (nothing written to pieces) or an argument is bad.
 */
int sfm_plan_pieces(int nunits, int nsub, const int* k_sub, int grid, int* ptr, int* pieces,
                    int max_pieces, int* npieces);

/* Number of device kernels launched by the last sfm_run. */
int sfm_last_launches(const sfm_handle* h, int* launches);

/*
 * Test hooks for the failure-detection paths (no fault, every wait bounded):
 *   key 1: device-wide barrier time limit in nanoseconds (default 2e9);
 *   key 2: index of a block that skips its barrier arrivals (-1 = none), so
 *          that every block's bounded wait runs out and sfm_run returns
 *          SFM_ERR_TIMEOUT with the context still usable;
 *   key 3: consumer warps per stepping block (1..8), all precisions;
 *   key 4: coefficient ring stages per stepping block (2..16), all
 *          precisions (keys 3 and 4 override sfm_autotune's choice; for
 *          SFM_FP32F the stages are rounded up to a multiple of the warps).
 * Errors: SFM_ERR_ARG for an unknown key or a value out of range.
 */
int sfm_debug_set(sfm_handle* h, int key, long long value);

/*
 * Read-bandwidth probe (no counterpart in the paper; the measured roof for a
 * kernel whose working set stays in L2).  On `device`, allocates a buffer of
 * `bytes` (rounded down to 16), zeroes it, reads it once to bring it into
 * L2, then times one launch that reads it `repeats` times with 16-byte loads
 * cached in L2 only (CUDA events); *gbs receives bytes * repeats / time in
 * GB/s.  A buffer larger than L2 measures HBM instead.  The buffer is freed
 * before return and the caller's current device is restored.
 * Errors: SFM_ERR_ARG (bytes < 16, repeats < 1, NULL gbs), SFM_ERR_CUDA
 * (device, allocation or launch; message in sfm_last_error(NULL)).
 */
int sfm_probe_read_gbs(int device, size_t bytes, int repeats, double* gbs);

#ifdef __cplusplus
}
#endif

#endif /* SFM_H */
