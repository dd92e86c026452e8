/*
 * iobm.h -- C ABI of the GB300 IOBM transport solver.
 *
 * The library solves, for every incident electrode channel and energy, the
 * complex-symmetric real-space finite-difference equations of the improved
 * overbridging boundary-matching (IOBM) method,
 *
 *     [E - H_T - H~] Psi = b                                   (Eq. 7)
 *
 * on a transition region of N_x x N_y x (N_z+2) grid points (Eqs. 1-4),
 * laterally periodic, between two identical semi-infinite jellium electrodes
 * whose self-energy is diagonal in the lateral Fourier basis (Eqs. 8, 18-2,
 * 19) and is applied through lateral 2D FFTs.  The solver is a
 * preconditioned conjugate-orthogonal CG (the "CG method for a
 * non-Hermitian matrix" of Sec. II, valid since the matrix equals its
 * transpose) with the truncated-Laplacian-Green preconditioner of Eq. 10.
 * The solved waves are projected onto the electrode channels (Eq. 6) to
 * give transmission, reflection and the Landauer conductance (Sec. III).
 *
 * Units: Hartree atomic units (energies in Ha, lengths in bohr); the
 * electrode potential is the zero of energy; the lateral Bloch vector is 0
 * unless iobm_set_bloch sets another.
 * Conductance is returned in units of G_0 = 2 e^2 / h.
 *
 * Layouts: grid functions are [z][y][x] with x fastest (z = plane index
 * 0 .. N_z+1).  Complex vectors are interleaved (re, im) pairs of double
 * (IOBM_ELEM_C64) or float (IOBM_ELEM_C32).  A batch of vectors is [rhs][z][y][x].
 *
 * Ownership: the caller owns every input buffer; the library copies what it
 * keeps during iobm_create.  The handle owns its persistent device tables
 * (allocated with cudaMalloc in iobm_create, freed in iobm_destroy).  Solve
 * workspace is caller-provided device memory (iobm_workspace_size /
 * iobm_set_workspace); when none is set the handle allocates and owns it.
 * Every device operation is ordered on the CUDA stream given at create.
 *
 * Errors: every int-returning call returns IOBM_OK (0) or one of the
 * IOBM_E_* codes; iobm_last_error(handle) then holds a one-line message.
 * A right-hand side that does not converge does not fail the call: its
 * status is reported per RHS in iobm_report.
 */
#ifndef IOBM_H
#define IOBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define IOBM_OK               0
#define IOBM_E_ARG            1  /* invalid argument (sizes, pointers, options)          */
#define IOBM_E_THRESHOLD      2  /* E within 1e-9 Ha of a channel threshold (v -> 0)      */
#define IOBM_E_PROJ_BOUNDARY  3  /* a projector touches the N_f outermost planes          */
#define IOBM_E_NOCONV         4  /* per-RHS: iteration limit reached                      */
#define IOBM_E_BREAKDOWN      5  /* per-RHS: COCG breakdown (r^T z or p^T A p vanished)   */
#define IOBM_E_TIMEOUT        6  /* a bounded device wait gave up (see iobm_set_wait_limit):
                                    the kernel drained its own copies and returned, the
                                    call's results are invalid, the context stays usable   */
#define IOBM_E_CUDA           7  /* CUDA runtime error                                    */
#define IOBM_E_STATE          8  /* call out of order (e.g. transmission before solve)    */
#define IOBM_E_UNSUPPORTED    9  /* size outside what the library supports (see message)*/

/* precision of the solver */
#define IOBM_FP64   0  /* plain FP64: vectors, stencil, Krylov recurrences in FP64     */
#define IOBM_MIXED  1  /* complex FP32 Krylov inner iterations, FP64 residual
                          replacement (iterative refinement) and FP64 projection   */

/* element type of vectors passed to iobm_apply / iobm_apply_precond */
#define IOBM_ELEM_C64   0  /* complex double, interleaved */
#define IOBM_ELEM_C32   1  /* complex float, interleaved  */
#define IOBM_ELEM_C64_DF 2 /* complex double data, stencil in double-float arithmetic (FP32
                              pairs, about 47 significant bits): what the mixed solver's FP64
                              residual uses; iobm_apply only */

typedef struct iobm_handle iobm_handle;

/* Transition-region grid (Sec. II).  nz counts the planes z_0 .. z_{N_z+1}
 * (nz = N_z + 2).  nf is the FD half-width N_f of Eq. 1 (1 .. 4); the
 * self-energy then acts on the nf outermost planes at each end.  x and y
 * are periodic with period nx*hx and ny*hy.  nx and ny may only contain
 * the prime factors 2, 3 and 5 (lateral FFT radices).  Planes of at most
 * 4096 points are transformed in one CTA's shared memory; larger planes
 * (nx <= 256 and ny <= 256) by two passes through global memory. */
typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    int nf;
} iobm_grid;

/* Kleinman-Bylander projectors in CSR form (norm-conserving pseudopotential
 * of Sec. III): projector p has support idx[row_ptr[p] .. row_ptr[p+1]) with
 * values val[...] (linear grid index (z*ny + y)*nx + x, each index once per
 * projector) and coupling E_p = coupling[p] in Ha.  The nonlocal operator is
 * sum_p E_p |p><p| with <p|psi> = hx*hy*hz * sum_r p(r) psi(r).  nproj may
 * be 0 (all pointers may then be NULL). */
typedef struct {
    int nproj;
    const int64_t* row_ptr;
    const int32_t* idx;
    const double* val;
    const double* coupling;
} iobm_projectors;

/* Preconditioners (iobm_options.use_precond) */
#define IOBM_PRECOND_NONE     0
#define IOBM_PRECOND_EQ10     1  /* truncated Laplacian Green's function of Eq. 10           */
#define IOBM_PRECOND_FOURIER  2  /* (E - T - H~)^{-1}: the potential-free Green's function,
                                    diagonal in the lateral Fourier basis (Eq. 19) and
                                    banded in z; applied with lateral FFTs (default)       */
#define IOBM_PRECOND_EQ10_FOURIER 3  /* Eq. 10 applied in the lateral Fourier basis: plane
                                    FFT, per-mode tridiagonal multiply in z, inverse FFT;
                                    the same operator as IOBM_PRECOND_EQ10 up to rounding  */

/* How each COCG iteration forms q = A p (iobm_options.op_form).  With the
 * free-propagator preconditioner M = (E - T - H~)^{-1} the operator splits as
 * A = M^{-1} - W, W = V_loc + V_NL the potential terms of H_T (Eqs. 2-4), and as the
 * iteration has z = M r in hand, A z = r - W z; the new direction p = z + beta p'
 * then gives q = A p = (r - W z) + beta q' with no stencil or self-energy
 * application (the same iterates in exact arithmetic; the FP64 residual checks
 * still apply the full operator).  IOBM_OP_AUTO takes this form whenever
 * use_precond is IOBM_PRECOND_FOURIER and the explicit form otherwise;
 * IOBM_OP_EXPLICIT always applies the stencil, self-energy and projectors. */
#define IOBM_OP_AUTO      0
#define IOBM_OP_EXPLICIT  1

/* How the end-plane self-energy term of Eq. 7 is applied (iobm_options.sigma_form).
 * IOBM_SIGMA_FFT (default): diagonal per lateral mode after the lateral FFT of
 * Eq. 19, O(N_xy log N_xy) per plane.  IOBM_SIGMA_DENSE: the dense N_f N_xy square
 * matrix of each energy, kept in device memory (FP32 and FP64 copies) and multiplied
 * directly, O((N_f N_xy)^2) per RHS: the solver (b) of Sec. III, an ablation of the
 * transform (the same operator up to rounding).  Dense matrices above 64 GB per
 * handle, a nonzero Bloch vector and batched solves return IOBM_E_UNSUPPORTED. */
#define IOBM_SIGMA_FFT    0
#define IOBM_SIGMA_DENSE  1

/* Solver options.  use_precond: one of IOBM_PRECOND_*.  alpha: parameter of
 * Eq. 10 (C_0 = 1, C_1 = exp(-alpha)) for IOBM_PRECOND_EQ10(_FOURIER).  tol: stop when
 * ||b - A psi||_2 / ||b||_2 <= tol, the residual evaluated in FP64.
 * max_iter: Krylov iteration limit per RHS.  refine_delta: in IOBM_MIXED the
 * FP64 residual replaces the FP32 recurrence residual whenever the latter has
 * fallen by this factor since the last replacement (0 < delta < 1).
 * chunk: iterations per captured CUDA graph between convergence checks.
 * max_iter_mixed: in IOBM_MIXED, FP32 iteration limit per RHS; an RHS that
 * stops there (or breaks down) without converging is continued with FP64
 * iterations from its FP64 iterate, up to max_iter more (precision escalation:
 * once cond(A) times the FP32 rounding unit is no longer small, the FP32 inner
 * iteration stops making progress while FP64 still converges).
 * op_form: IOBM_OP_AUTO or IOBM_OP_EXPLICIT (above).
 * fp64_modes: in IOBM_MIXED with IOBM_PRECOND_FOURIER, the number of lateral modes
 * per energy nearest their channel threshold (smallest |E - eps_perp|) whose
 * preconditioner z-sweeps run in double-float arithmetic with FP64 factors inside the
 * FP32 iterations: their banded z-systems are the worst conditioned, and FP32 sweeps
 * there cost iterations; 0 sweeps every mode in FP32; -1 (default) takes
 * max(16, N_xy / 128) (16 up to 48 x 48 planes, 128 at 128 x 128, where the larger
 * plane has more modes near threshold).
 * sigma_form: IOBM_SIGMA_FFT or IOBM_SIGMA_DENSE (above). */
typedef struct {
    double alpha;
    int use_precond;
    double tol;
    int max_iter;
    int precision;
    double refine_delta;
    int chunk;
    int max_iter_mixed;
    int op_form;
    int fp64_modes;
    int sigma_form;
} iobm_options;

/* Per right-hand-side report, in solve order (energy-major, then incident
 * channel in the canonical open-channel order). */
typedef struct {
    int energy_index;
    int channel;        /* index into the open channels of that energy      */
    int side;           /* 0: incident from the left, 1: from the right      */
    int status;         /* IOBM_OK, IOBM_E_NOCONV or IOBM_E_BREAKDOWN         */
    int iterations;     /* Krylov iterations                                  */
    int replacements;   /* FP64 residual replacements                         */
    double residual;    /* final ||b - A psi|| / ||b|| in FP64                */
} iobm_report;

/* Fill opts with the defaults: alpha 1.8, use_precond IOBM_PRECOND_FOURIER, tol 1e-8,
 * max_iter 20000, precision IOBM_MIXED, refine_delta 0.01, chunk 32,
 * max_iter_mixed 1000, op_form IOBM_OP_AUTO, fp64_modes -1 (automatic), sigma_form
 * IOBM_SIGMA_FFT. */
void iobm_default_options(iobm_options* opts);

/* Create a solver for one junction: the truncated Hamiltonian H_T of the
 * transition region (Eqs. 1-4: FD kinetic operator, local potential V_loc and
 * the nonlocal Kleinman-Bylander term of the norm-conserving pseudopotentials
 * of Sec. III) between two jellium electrodes (Sec. II).  V_loc: host
 * [nz][ny][nx] local potential (Ha), copied.  proj: KB projectors (host arrays, copied; NULL
 * for none).  rs: Wigner-Seitz radius of the jellium electrodes (bohr); it
 * only sets iobm_fermi_energy.  opts: NULL for defaults.  cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).  Errors: IOBM_E_ARG for bad
 * sizes / non-finite V, IOBM_E_PROJ_BOUNDARY if a projector reaches the nf
 * outermost planes, IOBM_E_UNSUPPORTED for lateral sizes whose FFT does not
 * fit the library's kernels, IOBM_E_CUDA.  On an error *out may still receive a handle
 * (so that iobm_last_error can explain it); pass it to iobm_destroy. */
int iobm_create(const iobm_grid* grid, const double* V_loc, const iobm_projectors* proj,
                double rs, const iobm_options* opts, void* cuda_stream, iobm_handle** out);

void iobm_destroy(iobm_handle* h);

/* Create n junction handles in one call, as iobm_create for each j with
 * grids[j], V[j], projs[j] (projs may be NULL: no projectors anywhere; an entry
 * with nproj = 0 means none for that junction), rs[j] and the shared options
 * and stream; out[0..n) receives the handles (destroy each with iobm_destroy).
 * On an error no handle is left: those created are destroyed, out[] is NULL,
 * and the return value is the failing junction's status. */
int iobm_create_batch(int n, const iobm_grid* grids, const double* const* V,
                      const iobm_projectors* projs, const double* rs, const iobm_options* opts,
                      void* cuda_stream, iobm_handle** out);

const char* iobm_status_string(int status);
const char* iobm_last_error(const iobm_handle* h);

/* Jellium Fermi energy (9 pi / 4)^(2/3) / (2 rs^2) of the handle's electrodes. */
double iobm_fermi_energy(const iobm_handle* h);

/* Number of open (propagating, right-going) electrode channels at energy E,
 * and optionally their lateral indices (nu_x, nu_y) pairs and group
 * velocities in the canonical order (nu_y major, then nu_x, each from
 * -N/2 upward).  nu and vel may be NULL; otherwise they hold room for
 * max_out channels.  Eqs. 8.5-9 generalised to N_f (Appendix). */
int iobm_open_channels(iobm_handle* h, double E, int* n_open, int max_out, int* nu, double* vel);

/* Number of internal right-hand sides iobm_solve will run for these
 * arguments.  An incident wave exp(i G.r) with G != 0 would make the
 * unconjugated COCG form b^T P b vanish, so the solver runs the real lateral
 * profiles cos(G.r) and sin(G.r) of each +-G channel pair and recombines them
 * (two internal RHS per pair, one for a self-conjugate G). */
/* The per-energy mode tables built for the count are kept in the handle and
 * taken over by the next iobm_solve if it has the same energies (bit-identical
 * values, same order), which then skips rebuilding them; a count, solve or
 * gradient with other energies discards them.  The tables depend on the
 * lateral grid, N_f and E only, never on the potential. */
int iobm_solve_rhs_count(iobm_handle* h, const double* E, int nE, const int* channels, int nch,
                         int* n_internal);

/* Workspace: bytes of device memory a solve of nrhs internal right-hand sides needs
 * at the handle's precision, and attach caller memory (256-byte aligned,
 * kept by the handle until replaced or destroyed; the caller must keep it
 * alive).  Passing NULL detaches it. */
int iobm_workspace_size(iobm_handle* h, int nrhs, size_t* bytes);
int iobm_set_workspace(iobm_handle* h, void* dev_ptr, size_t bytes);

/* Solve Eq. 7 for every energy E[0..nE) and incident channel.  channels:
 * NULL = every open channel of each energy; otherwise nch indices into each
 * energy's open-channel list (indices beyond that list are skipped).
 * side: 0 left-incident (Eq. 7 as printed), 1 right-incident.  All RHS are
 * solved together in one batched launch sequence.  The solution vectors stay
 * in the workspace for iobm_transmission / iobm_solution.  Returns IOBM_OK
 * when the batch ran (check iobm_report for per-RHS convergence). */
int iobm_solve(iobm_handle* h, const double* E, int nE, const int* channels, int nch, int side);

/* Solve several junctions together (not in the paper, which treats one incident
 * wave of one junction at a time).  handles[j] (from iobm_create, all on the
 * current device, distinct, each with its own workspace: attached or owned) is
 * solved at energies E[j][0..nE[j]) for every open incident channel from `side`.
 * Each junction's tables, RHS and solver start run on its handle's stream; then
 * ONE CUDA graph launch runs all junctions concurrently: a conditional WHILE node
 * per junction repeats that junction's chunk of COCG iterations (with its FP64
 * residual replacements) on the device until every one of its RHS has stopped or
 * its iteration limit is reached; then each junction's final FP64 residual and
 * channel projections run.  Results are read per handle (iobm_transmission,
 * iobm_solution).  Per RHS the arithmetic is that of iobm_solve on the handle
 * alone.  Returns IOBM_OK or the first error (the failing handle reports it in
 * iobm_last_error); per-iteration kernel profiling is not collected here. */
int iobm_solve_batch(int n, iobm_handle* const* handles, const double* const* E, const int* nE,
                     int side);

/* Stencil tiling autotuner: times the fused COCG stencil (p = z + beta p_old,
 * A p, p^T A p) on nrhs RHS of this handle's grid for z-chunks of 16, 32 and 64
 * planes per CTA and, in the mixed solver, for the FP32 row kernels (variants 0, 1,
 * 3, 4 of iobm_set_tiling), keeps the fastest for the handle's later solves
 * and returns it in *zchunk / *variant (either may be NULL).  Binds the workspace
 * for nrhs RHS (the attached one must be large enough).  The choice changes only
 * the order of the partial sums of the dot products. */
int iobm_autotune(iobm_handle* h, int nrhs, int* zchunk, int* variant);

/* Set the stencil tiling explicitly: zchunk >= 16 z-planes per CTA; variant 0 =
 * the fastest kernel for the shape, 1 = the register-pipelined row kernel, 3 = the
 * bulk-copy row kernel with one row per thread, 4 = the bulk-copy kernel whose operand
 * planes k - N_f .. k + N_f sit in a shared-memory ring (one thread per point of a
 * 16-row tile; N_f 1 or 4, ny a multiple of 16) (FP32 rows of 12 .. 64 points; 0 takes
 * the bulk-copy kernel with several rows per thread where the shape allows). */
int iobm_set_tiling(iobm_handle* h, int zchunk, int variant);

/* Average device time (ms, CUDA events on the handle's stream) of one launch of the
 * fused COCG operator kernel of the explicit operator form -- p = z + beta p_old,
 * q = (E - T - V) p with the FD stencil of Eqs. 1-4, and the p^T q partials -- on
 * nrhs RHS of this grid with every RHS active and the handle's tiling, after one
 * warm-up launch; reps timed launches.  Binds the workspace for nrhs RHS (an attached
 * one must be large enough) and overwrites it: the last solve's results are gone.
 * A kernel-timing aid (the roofline of the stencil at full load). */
int iobm_time_operator(iobm_handle* h, int nrhs, int reps, double* ms_per_launch);

/* Eigenchannel transmissions of energy index e of the last solve (Sec. IV,
 * Table II: the eigenvalues of T^dagger T, T the transmission matrix): with
 * t~_oc = t_oc sqrt(v_o / v_c) the flux-normalised amplitudes (out o, in c) of
 * the FP64 solutions, tau[0..n) are the eigenvalues of t~^dagger t~ in
 * descending order; they lie in [0, 1] and sum to G of that energy.  Needs
 * every open incident channel of the energy in the last solve (IOBM_E_STATE
 * otherwise).  *n_out = number of open channels; tau may be NULL to query it,
 * else it holds max_out >= n values.  Host computation (cyclic Jacobi). */
int iobm_eigenchannels(iobm_handle* h, int e, double* tau, int max_out, int* n_out);

/* Number of incident channels (user-visible RHS) of the last solve. */
int iobm_num_rhs(const iobm_handle* h);

/* Largest open-channel count over the energies of the last solve (the
 * smallest max_open iobm_transmission accepts); 0 before any solve. */
int iobm_max_open(const iobm_handle* h);

/* Transmission/reflection of the last solve (Eq. 6, Landauer-Buttiker of
 * Sec. III).  T, R: host [rhs][max_open] with T[rhs][o] = |t_o|^2 v_o / v_in
 * for out-channel o of that RHS's energy (zero past its n_open); pass NULL to
 * skip.  G: host [nE], conductance in G_0 summed over the solved incident
 * channels of each energy.  nopen: host [nE] (may be NULL).  reports: host
 * [nrhs] (may be NULL).  max_open: row stride of T and R. */
int iobm_transmission(iobm_handle* h, double* T, double* R, int max_open, double* G,
                      int* nopen, iobm_report* reports);

/* Copy the FP64 solution of RHS `rhs` of the last solve ([z][y][x] complex
 * double) to dst (host or device). */
int iobm_solution(iobm_handle* h, int rhs, void* dst, int dst_is_device);

/* dG/dV(r) (G_0 per Ha) at energy E for left-incident waves.  Not in the
 * paper: it differentiates the Landauer sum of Sec. III through Eq. 7 with
 * dA/dV(r) = -e_r e_r^T, using A = A^T (Eq. 8 is symmetric in l <-> l' at a
 * zero lateral Bloch vector).  Takes the energy itself rather than an index
 * into an earlier solve, so it needs no prior iobm_solve.  It solves the
 * n_open forward waves and the n_open adjoint waves A lambda_o = w_o (same
 * operator, A = A^T) in one batch, then accumulates
 * dG/dV(r) = sum_{o,i} 2 (v_o/v_i) Re[conj(t_oi) lambda_o(r) psi_i(r)] in FP64.
 * dGdV: [nz][ny][nx] double, host or device.  G_out (may be NULL): the
 * conductance of the same solve. */
int iobm_grad_V(iobm_handle* h, double E, double* dGdV, int dst_is_device, double* G_out);

/* y = (E - H_T - H~) x for nrhs vectors (Eqs. 1-4, 7-2, 8 via FFT),
 * x and y device buffers [nrhs][nz][ny][nx] of element type `elem`
 * (IOBM_ELEM_C64 computes in FP64, IOBM_ELEM_C32 in FP32, IOBM_ELEM_C64_DF
 * the stencil in double-float arithmetic on FP64 data, the self-energy and KB
 * terms in FP64).  Uses the workspace for the projector scratch. */
int iobm_apply(iobm_handle* h, double E, int elem, const void* x, void* y, int nrhs);

/* y = P x with the handle's preconditioner at energy E: Eq. 10 (six face
 * neighbours, C_0 = 1, C_1 = exp(-alpha), zero beyond the end planes; E is
 * then unused) or the lateral-Fourier free propagator (E - T - H~)^{-1}.
 * Same buffer conventions as iobm_apply. */
int iobm_apply_precond(iobm_handle* h, double E, int elem, const void* x, void* y, int nrhs);

/* Replace the local potential V_loc ([nz][ny][nx], Ha; host or device
 * memory) of an existing handle, e.g. between the forward passes of a
 * gradient-based optimisation.  Eqs. 2-4: V enters H_T on every plane. */
int iobm_set_potential(iobm_handle* h, const double* V_loc, int src_is_device);

/* Lateral Bloch vector kappa = (kappa_x, kappa_y) (1/bohr) of the later solves,
 * gradients and operator applications of this handle (Eq. 8: every lateral mode
 * becomes G_nu + kappa and the wave picks up exp(i kappa L) across a lateral
 * period); (0, 0), the default, is the periodic problem.
 *
 * At kappa != 0 the matrix of Eq. 7 is no longer complex symmetric: A(kappa)^T =
 * A(-kappa).  The library then solves in the gauge phi = exp(-i kappa.r) psi (where
 * the lateral FFTs, the self-energy and preconditioner tables at G_nu + kappa and
 * the channel projections keep their periodic form; the FD couplings and the
 * projectors carry the phases) by preconditioned Bi-CG, whose shadow sequence
 * solves the transposed system: iobm_solve pairs every incident channel nu at kappa
 * with the channel -nu at -kappa incident from the same side (the time-reversed
 * partner) and returns both.  After such a solve, energy slot e in [0, nE) of
 * iobm_transmission (G, nopen, iobm_report.energy_index) is E[e] at +kappa and slot
 * nE + e is E[e] at -kappa; iobm_num_rhs counts the channels of both, the -kappa
 * ones after the +kappa ones in the same order, each with its channel index in the
 * open list at -kappa.  iobm_grad_V pairs each forward wave with the adjoint wave
 * of the same channel (lambda_o = A(kappa)^{-T} w_o).  iobm_solution returns psi
 * (the gauge undone).  iobm_apply applies the operator at +kappa to phi (the
 * gauge representation) in FP64 only (IOBM_ELEM_C64; IOBM_ELEM_C64_DF is computed
 * as IOBM_ELEM_C64); iobm_apply_precond applies (E - T - H~)^{-1} at +kappa.
 * Requires use_precond = IOBM_PRECOND_FOURIER and op_form = IOBM_OP_AUTO
 * (IOBM_E_UNSUPPORTED otherwise); iobm_solve_batch refuses handles with kappa != 0.
 * IOBM_E_ARG for a non-finite kappa. */
int iobm_set_bloch(iobm_handle* h, double kappa_x, double kappa_y);

/* Host-only set-up (needs no GPU and no handle): the electrode channel data
 * at energy E for a lateral grid, as used by the solver.  n_open: number of
 * open channels.  nu [max_out][2], vel [max_out], lam [max_out][2] (the
 * propagating right-going root, re/im), btilde [max_out][nf][2] (incident
 * source coefficients per depth, Eq. 7 generalised to N_f planes), mrow
 * [max_out][nf][2] (t = sum_d mrow[d] psi~(depth d)), sigma
 * [ny][nx][nf][nf][2] (Sigma~ per lateral FFT bin, Eqs. 17, 18-2); any of
 * them may be NULL.  Returns IOBM_E_THRESHOLD near a channel edge. */
int iobm_channels_host(const iobm_grid* grid, double E, int* n_open, int max_out, int* nu,
                       double* vel, double* lam, double* btilde, double* mrow, double* sigma);

/* The same tables at a lateral Bloch vector (kappa_x, kappa_y) (1/bohr): every lateral
 * mode becomes G_nu + kappa (Eq. 8), the wave picking up exp(i kappa L) across a lateral
 * period.  iobm_channels_host is this call at kappa = 0 (the solver takes kappa from
 * iobm_set_bloch).  IOBM_E_ARG for a non-finite kappa. */
int iobm_channels_host_bloch(const iobm_grid* grid, double kappa_x, double kappa_y, double E,
                             int* n_open, int max_out, int* nu, double* vel, double* lam,
                             double* btilde, double* mrow, double* sigma);

/* CUDA-event timing of one kernel of every COCG iteration inside the captured
 * iteration graphs; resets the counters.  enable: 0 off; 1 the operator kernel
 * (the fused stencil p = z + beta p_old, q = (E - T - V) p with the p^T q
 * partials, or in the implicit operator form the pass p = z + beta p_old,
 * q = (r - V z) + beta q_old); 2 the update x += alpha p, r -= alpha q with the
 * forward plane FFTs; 3 the z-sweeps; 4 the inverse plane FFTs with the r^T z
 * and |r|^2 partials (2-4: Fourier preconditioners with planes of at most 4096
 * points).  IOBM_E_ARG for other values.  The FP64 residual replacements run as
 * conditional graph nodes, whose kernels kernel profilers cannot list; with
 * IOBM_GRAPH_CONDITIONALS=0 in the environment when a handle is created they are
 * captured as plain masked launches instead (bit-identical results). */
int iobm_profile(iobm_handle* h, int enable);

/* Limit of the bounded device waits of this handle's kernels (the bulk-copy
 * stencil waits on its staged copies): cycles = 0 restores the default of
 * about one second of SM clock.  A wait that reaches the limit gives up: its
 * CTA waits (with the default limit) for its own copies still in flight and
 * returns, and the call reports IOBM_E_TIMEOUT.  inject_stall = 1 makes every
 * CTA of that kernel also wait once on a barrier that no copy completes, so
 * that the give-up path runs (for tests of the error path; 0 = off).  Applies
 * to later calls; the bulk-copy kernel serves FP32 operators and the Eq. 10
 * preconditioner on rows of 12, 16, 24, 32, 48 or 64 points. */
int iobm_set_wait_limit(iobm_handle* h, long long cycles, int inject_stall);

/* Accumulated device time (ms) and count of the timed launches since
 * iobm_profile(h, enable > 0). */
int iobm_kernel_stats(const iobm_handle* h, double* kernel_ms, long long* kernel_launches);

/* Allocation-free form of the Eq. 10 preconditioner with its COCG dot
 * products, for callers that cannot allocate device memory: for instance an
 * application whose memory pool owns the whole GPU, a latency-critical loop
 * that cannot afford the implicit synchronisation of cudaMalloc/cudaFree, or
 * code running while a stream is being captured into a CUDA graph.  The paper
 * has no counterpart; it is the same operation as iobm_apply_precond with
 * IOBM_PRECOND_EQ10 in FP64, plus the sums the solver forms from it.
 *
 * Needs no handle.  r and z: device [nrhs][nz][ny][nx] complex double
 * (interleaved); z = P r with C_0 = 1, C_1 = exp(-alpha), six face neighbours,
 * laterally periodic, zero beyond the end planes.  rho: device [nrhs][2]
 * receives r^T z (unconjugated, re/im); rr: device [nrhs] receives |r|^2.
 * Everything is enqueued on cuda_stream (a cudaStream_t, NULL = legacy
 * default stream); the call does not synchronise.
 *
 * r and z must not overlap (z = P r reads neighbours of r that other blocks
 * may already have written to z): overlapping ranges return IOBM_E_ARG.
 *
 * The per-block partial sums live in a fixed device array compiled into the
 * library (1.5 MiB per GPU, held by every GPU that loads the library until the
 * process exits): at most 65536 partial slots, where one RHS uses at most
 * ceil(nx/32) * ceil(ny/8) * ceil(nz/32) slots, and nrhs <= 65535 (the RHS
 * index is a grid dimension); larger requests return IOBM_E_UNSUPPORTED.
 * A call made while cuda_stream is not being captured looks up that array's
 * device address (cudaGetSymbolAddress) with the device current; a call during
 * stream capture uses the address found by the last such call, so make at
 * least one call on the device before capturing a stream (and again after a
 * cudaDeviceReset, which invalidates it).  Every call shares the array and
 * overwrites every slot it reads, so calls need no clearing, but calls that
 * overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Calls no cudaMalloc, cudaFree or allocating
 * library routine.  Errors: IOBM_E_ARG, IOBM_E_UNSUPPORTED, IOBM_E_CUDA. */
int iobm_precond_dots_noalloc(const iobm_grid* grid, double alpha, const void* r, void* z,
                              int nrhs, double* rho, double* rr, void* cuda_stream);

/* Device-side time (ms) of the last iobm_solve's iteration phase, measured
 * with CUDA events on the handle's stream, and the number of kernel launches
 * it issued. */
int iobm_last_solve_stats(const iobm_handle* h, double* ms, long long* launches,
                          long long* iterations_total);

#ifdef __cplusplus
}
#endif

#endif /* IOBM_H */
