/*
 * dda.h - C ABI of the GB300 preconditioned discrete dipole approximation.
 *
 * The library solves the voxelised volume-integral-equation system of
 * Groth, Polimeridis & White, "Preconditioning the discrete dipole
 * approximation" (arXiv 1903.09802):
 *
 *     (alpha^{-1} - dx^3 G) c = E_inc                       (Section 2.2)
 *
 * with G the block-Toeplitz Toeplitz-block (BTTB) matrix of the dyadic Green
 * function sampled on a uniform l x m x n voxel box (Algorithm 1), applied
 * with a zero-padded 3-D FFT; the multilevel (Chan-Olkin) circulant
 * preconditioner P = alpha_tilde^{-1} I - dx^3 C (Section 3, eq. 20) with
 * the circulant taken on all three levels, or on two as in the paper
 * (dda_precond2_*); and restarted GMRES or BiCG-Stab (Section 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every device buffer is allocated and owned by the caller.  A plan keeps
 *   pointers into the caller's workspace and never allocates device memory.
 * - Box fields are complex, layout [rhs][component 0..2][z][y][x], x fastest.
 *   Precision DDA_C128 means interleaved double (re, im); DDA_C64 means
 *   interleaved float.  Air voxels (material 0) belong to the box; their rows
 *   of the box matrix are alpha_tilde^{-1} c (decoupled), so with a zero
 *   right-hand side on air their unknowns solve to zero and the scatterer's
 *   unknowns are those of the paper's system (eq. 8: air carries no
 *   polarization).
 * - Unknowns are the paper's c (eq. 9); dipole moments are p = dx^3 c.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).  Calls
 *   are stream-ordered and asynchronous unless they return host results
 *   (dda_solve stats, dda_cross_sections, dda_autotune's timings), which
 *   synchronise that stream.
 * - Errors come back as dda_status_t; arguments are checked before any
 *   launch; a failing call leaves outputs unspecified.  dda_last_error()
 *   returns a thread-local description of the last failure.  No entry point
 *   aborts the process or throws across the ABI.
 * - One plan must not be used from two host threads at once.
 */
#ifndef DDA_H_
#define DDA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DDA_OK = 0,
  DDA_ERR_INVALID_ARG = 1,
  DDA_ERR_UNSUPPORTED_SIZE = 2,
  DDA_ERR_WORKSPACE = 3,
  DDA_ERR_CUDA = 4,
  DDA_ERR_NOT_CONVERGED = 5,
  DDA_ERR_BREAKDOWN = 6,
  DDA_ERR_SINGULAR_PRECOND = 7,
  DDA_ERR_NAN = 8,
  DDA_ERR_TIMEOUT = 9,
  DDA_ERR_NO_PRECOND = 10
} dda_status_t;

typedef enum { DDA_C128 = 0, DDA_C64 = 1 } dda_precision_t;

/* Bits of dda_plan_desc_t.precisions: which spectra the plan stores. */
#define DDA_PLAN_C128 1
#define DDA_PLAN_C64 2

typedef struct dda_plan_s* dda_plan_t;

typedef struct {
  int32_t l, m, n;       /* box edges along x, y, z, 1..512: powers of two, or
                            even 7-smooth numbers (2^a 3^b 5^c 7^d, a >= 1) taken
                            by mixed-radix transforms: all of them up to 208,
                            above that those whose transform tiles fit (see
                            dda_plan_create)                                    */
  double dx;             /* voxel edge Delta (length unit of the caller)        */
  double k;              /* wavenumber in the same unit                          */
  int32_t n_materials;   /* K >= 1 materials; voxel material 0 is air           */
  int32_t max_rhs;       /* largest right-hand-side batch used with this plan   */
  int32_t krylov_m;      /* GMRES restart length to reserve (0: no solver)      */
  int32_t precisions;    /* DDA_PLAN_C128 | DDA_PLAN_C64                         */
  int32_t precond2;      /* reserve the 2-level preconditioner: 1 with z as its
                            Toeplitz (dense) level as in the paper, 2 with x, 3 with
                            y (Section 5's alternative for long prisms).  Storage:
                            (l'/2+1)(m'/2+1)(3n')^2 complex64 values for the box
                            relabelled so that the Toeplitz level is z' (the other
                            frequency pairs follow by parity), plus build scratch */
  int32_t circulant;     /* circulant of the preconditioners (Section 3): 0 T. Chan's
                            optimal one (eq. 13), 1 Strang's (central diagonals kept;
                            at p = L/2 of an even level the mean of t_{L/2}, t_{-L/2}) */
  int32_t voxel_eps;     /* 1: reserve a permittivity per voxel (dda_set_voxel_eps):
                            (16 + max_rhs * 40) bytes per voxel                      */
  int32_t rhs_chunk;     /* right-hand sides the FFT scratch holds (0: max_rhs); larger
                            batches pass through the transforms in chunks of it, so a
                            batch of many waves needs scratch for rhs_chunk only      */
  int32_t krylov_c64;    /* 1: the Krylov basis and step vectors are reserved in
                            complex64 (solves with inner_prec = DDA_C64 only), half
                            the memory of the complex128 reservation                  */
  int32_t sstep;         /* block size s of the s-step GMRES (method 2) to reserve: 0
                            none, 2..8 (at most krylov_m): s more Krylov vectors per
                            right-hand side, the unrotated Hessenberg matrix, shifts  */
} dda_plan_desc_t;

/* Plane wave E_inc = pol * exp(i k dir . r), r measured from the box centre.
 * dir and pol are unit vectors with dir . pol = 0 (checked to 1e-9). */
typedef struct {
  double dir[3];
  double pol[3];
} dda_incidence_t;

typedef struct {
  double tol;            /* stop when ||b - A x||_2 / ||b||_2 <= tol (FP64 residual)  */
  int32_t max_iters;     /* cap on inner GMRES iterations per right-hand side          */
  int32_t restart;       /* GMRES(m) restart length, 1 <= restart <= plan krylov_m;
                            BiCG-Stab: iterations per refinement cycle (any >= 1)     */
  int32_t precond;       /* 0: none; 3: three-level circulant (dda_precond_build first);
                            2: the paper's 2-level circulant (dda_precond2_build first) */
  int32_t inner_prec;    /* DDA_C128: complex128 cycles (FP64 Gram-Schmidt, Givens and
                            preconditioner; the matvec in double-float arithmetic, see
                            dda_matvec); DDA_C64: complex64 cycles inside FP64
                            iterative refinement                                      */
  double inner_tol;      /* a cycle ends early once its residual estimate falls below
                            inner_tol times the cycle's starting residual (0: only tol) */
  double reorth_eta;     /* second Gram-Schmidt pass when ||w_after|| < reorth_eta *
                            ||w_before|| (0: never, > 1: always; 1/sqrt(2) is the classical
                            choice of Daniel, Gragg, Kaufman & Stewart)                      */
  int32_t method;        /* 0: GMRES(restart); 1: BiCG-Stab (van der Vorst), the paper's
                            second solver (Section 4), restart = iterations per
                            refinement cycle; the plan needs krylov_m >= 7;
                            2: s-step GMRES(restart) with the plan's s (desc.sstep,
                            restart a multiple of s): the same GMRES iterates computed
                            in blocks of s Newton-basis vectors (Bai, Hu & Reichel
                            1994) whose shifts are the Leja-ordered Ritz values of
                            the solve's first cycle (plain Arnoldi); each block is
                            orthogonalised by block classical Gram-Schmidt twice and
                            a Cholesky QR, reading the basis four times per s
                            columns instead of twice or more per column; iterations
                            count columns, the last block of a cycle may compute up
                            to s - 1 products beyond the converged column           */
  int32_t history_cap;   /* entries of h_history per right-hand side (0: none)        */
  int64_t timeout_ns;    /* time limit of the solve on the device's global timer
                            (0: none); checked after every inner iteration and at
                            every restart: right-hand sides not converged by then
                            stop with DDA_ERR_TIMEOUT, x holding the last cycle's
                            iterate                                                   */
  double* h_history;     /* host [nrhs][history_cap] or NULL: relative residual after
                            each inner iteration (entry i after i iterations; GMRES's
                            estimate |g_{j+1}|/||b||, BiCG-Stab's ||r||/||b||, the
                            true FP64 residual at every restart, entry 0 = the
                            initial one): the convergence history of Section 4's
                            figures.  dda_solve_many needs NULL                      */
} dda_solve_opts_t;

typedef struct {
  int32_t iters;         /* inner GMRES iterations (matvecs with A P^{-1})             */
  int32_t cycles;        /* restart cycles = FP64 residual evaluations after the first */
  int32_t converged;     /* 1 when the FP64 relative residual reached tol              */
  int32_t status;        /* dda_status_t of this right-hand side                       */
  double rel_resid;      /* final ||b - A x|| / ||b|| evaluated in complex128          */
  int32_t reorth;        /* Arnoldi steps that needed a second Gram-Schmidt pass       */
  int32_t history_len;   /* entries written to this RHS's row of h_history             */
  int32_t graph;         /* 1: the solve ran as one CUDA graph launch (below)          */
  float ms;              /* wall time of the dda_solve call, milliseconds              */
} dda_rhs_stats_t;

/* Bytes of device workspace a plan with this description needs (0 when the
 * description is invalid; dda_last_error() says why).  The workspace holds
 * the kernel spectrum and the circulant spectrum (compressed to one octant by
 * the parity of each Green-function component), the FFT scratch for max_rhs
 * right-hand sides and, when krylov_m > 0, the Krylov basis and GMRES state. */
size_t dda_workspace_size(const dda_plan_desc_t* desc);

/* Build a plan: evaluates the Green function at every signed voxel offset
 * (Algorithm 1, extended to negative offsets), embeds it in a (2l, 2m, 2n)
 * circulant whose wrap index is zero, transforms it by FFT and stores the
 * spectrum of each of the six unique blocks (Section 2.2).
 *   d_mat   device uint8 [n][m][l] material index per voxel, 0 = air, 1..K.
 *           The pointer is kept by the plan and must stay valid.
 *   h_eps   host double[2*K]: (re, im) relative permittivity of materials 1..K
 *           (eps = m^2, Section 2.1).  Copied.
 *   d_work  device workspace of at least dda_workspace_size(desc) bytes,
 *           256-byte aligned, owned by the caller, kept by the plan.
 * Errors: DDA_ERR_INVALID_ARG, DDA_ERR_UNSUPPORTED_SIZE (edge above 512,
 * neither a power of two nor an even 7-smooth number, a mixed-radix edge e
 * whose three-component tile of length e or 2e needs more than 256 threads
 * (3 c L / 8 with c the least power of two making 3 c L a multiple of 8:
 * 210, 250, 270, 294, 350, 360, 378, 384, 392, 400, 420, 432, 448, 450, 480,
 * 486, 490, 500, 504), or lcm(2l, 2m, 2n) above 2^20), DDA_ERR_WORKSPACE (too
 * small / misaligned), DDA_ERR_CUDA. */
dda_status_t dda_plan_create(dda_plan_t* out, const dda_plan_desc_t* desc, const uint8_t* d_mat,
                             const double* h_eps, void* d_work, size_t work_bytes, void* stream);

/* Set the incident waves of the next calls (nrhs <= max_rhs).  Computes, in
 * FP64 on the host, the LDR polarizability of every material for every
 * right-hand side (Section 2.1; S = sum_j (d_j e_j)^2 depends on the wave)
 * and alpha_tilde, the polarizability of the most frequent non-air material
 * (Section 3.1, eq. 20), and uploads them on `stream`. */
dda_status_t dda_set_incidence(dda_plan_t plan, int32_t nrhs, const dda_incidence_t* h_inc,
                               void* stream);

/* A complex permittivity for every voxel (Section 2.1 defines alpha from a
 * voxel's eps = m^2; nothing in the method requires it to be one value per
 * material): d_eps is device complex128 [n][m][l] (re, im pairs), copied.
 * Voxels of material 0 stay air and their entries are ignored; every other
 * voxel's alpha^{-1} (CM + LDR, per right-hand side) comes from its own eps
 * in the matvec, the cross sections and dda_ext_gradient.  alpha_tilde (air
 * rows, preconditioners) stays that of the material table (dda_plan_create's
 * h_eps).  Needs a plan made with desc.voxel_eps = 1; may be called before or
 * after dda_set_incidence (the per-voxel polarizabilities are re-tabulated
 * on the device for the current incidences).  NULL turns the table off. */
dda_status_t dda_set_voxel_eps(dda_plan_t plan, const void* d_eps, void* stream);

/* d_b[rhs] = E_inc on scatterer voxels, 0 on air; complex128 box fields. */
dda_status_t dda_incident_field(dda_plan_t plan, int32_t nrhs, void* d_b, void* stream);

/* y = A x for nrhs box fields in precision prec (the plan must hold it):
 *   scatterer rows: alpha_j^{-1} x_j - dx^3 sum_{i scatterer, i != j} g(r_j - r_i) x_i
 *   air rows:       alpha_tilde^{-1} x_j
 * G is applied by the zero-padded FFT convolution (Section 1, Section 2.2).
 * DDA_C128 fields are converted to double-float values (pairs of floats,
 * about 48 significant bits) and transformed in that arithmetic on the FP32
 * units, then converted back (relative error well below 1e-10 of the FP64
 * result); DDA_C64 computes in FP32.  d_x and d_y must not overlap. */
dda_status_t dda_matvec(dda_plan_t plan, int32_t prec, int32_t nrhs, const void* d_x, void* d_y,
                        void* stream);

/* Build the 3-level circulant: T. Chan's optimal circulant (eq. 13; Strang's
 * with desc.circulant = 1) applied on the x, y and z levels of each of the
 * six blocks, then its 3-D DFT (Section 3).  Independent of the incident
 * wave. */
dda_status_t dda_precond_build(dda_plan_t plan, void* stream);

/* z = M o P^{-1} (M o v), P = alpha_tilde^{-1} I - dx^3 C, M the scatterer
 * mask: the unknowns live on scatterer voxels (eq. 8) and P is the matrix of
 * the box filled with the scatterer's material (Section 1), so v is extended
 * by zeros over air, P^{-1} applied on the box, and air entries of z zeroed.
 * P^{-1}: 3-D FFT of each component, the 3x3 symbol
 * Lambda(w) = alpha_tilde^{-1} I - dx^3 Chat(w) solved per frequency, inverse
 * FFT.  v and z may be the same buffer. */
dda_status_t dda_precond_apply(dda_plan_t plan, int32_t prec, int32_t nrhs, const void* d_v,
                               void* d_z, void* stream);

/* dda_precond_apply for callers that cannot allocate device memory during
 * the call: real-time or embedded hosts whose device memory is fixed at
 * start-up, frameworks that own every byte of the device through their own
 * pool and forbid allocations from outside it.  The paper has no counterpart; this is a
 * deployment variant.  Same arguments and result as dda_precond_apply, but
 * the transform's scratch (nrhs * 3 * l*m*n complex values) lives in a
 * 32 MiB array compiled into the library instead of the plan's workspace;
 * larger requests return DDA_ERR_WORKSPACE.  Every GPU on which a plan is
 * created holds that array until the process exits: dda_plan_create loads
 * it into the current context (with lazy module loading that is when its
 * memory is reserved), so make the plan while allocation is still allowed.
 * Each call looks the array's device address up again with the plan's device
 * current (a host-side lookup that allocates nothing), so a context reset
 * leaves no stale address; plans made before a reset are invalid anyway.
 * All calls share the one array, and it keeps the last call's contents
 * (each call overwrites everything it reads): calls that overlap on the GPU,
 * on any streams, race and give wrong results.  Uses the plan's launch
 * schedule like dda_precond_apply.  Allocates nothing.  Power-of-two boxes
 * only (DDA_ERR_UNSUPPORTED_SIZE otherwise): the FP64 mixed-radix kernels
 * carry a local stack frame whose first launch may make the driver enlarge
 * the context's local-memory reservation. */
dda_status_t dda_precond_apply_noalloc(dda_plan_t plan, int32_t prec, int32_t nrhs,
                                       const void* d_v, void* d_z, void* stream);

/* The paper's 2-level circulant preconditioner (Section 3, eqs. 17-19; the
 * block inversion of Section 3.1): T. Chan's circulant (eq. 13) on the x and
 * y levels, the z level kept Toeplitz, so after a 2-D DFT every frequency
 * pair (wx, wy) carries a dense 3n x 3n block alpha_tilde^{-1} I -
 * dx^3 Chat2(wx, wy), inverted on the GPU (Gauss-Jordan with partial
 * pivoting, complex64) and stored.  With desc.precond2 = 2 (3) the Toeplitz
 * level is x (y) instead: the same construction on the box relabelled by the
 * rotation (x', y', z') = (y, z, x) ((z, x, y)), fields relabelled on the way
 * in and out of the apply.  alpha_tilde is that of the first right-hand side
 * of the current incidence (call after dda_set_incidence; the blocks serve
 * the whole batch).  Needs a plan with desc.precond2 >= 1.
 * DDA_ERR_SINGULAR_PRECOND if a block is singular. */
dda_status_t dda_precond2_build(dda_plan_t plan, void* stream);

/* z = M o P2^{-1}(M o v) (restricted to the scatterer as dda_precond_apply):
 * masked 2-D FFT, dense block times the (component, z) vector of every
 * frequency pair, inverse FFT.  v and z may be the same buffer. */
dda_status_t dda_precond2_apply(dda_plan_t plan, int32_t prec, int32_t nrhs, const void* d_v,
                                void* d_z, void* stream);

/* In-place unnormalised 3-D DFT (inverse: sign +, scaled by 1/(l m n)) of
 * nbatch complex l x m x n arrays [batch][z][y][x].  Same kernels as the
 * preconditioner's transforms; exposed for testing and reuse. */
dda_status_t dda_fft3d(dda_plan_t plan, int32_t prec, int32_t nbatch, void* d_data,
                       int32_t inverse, void* stream);

/* Solve A x = b for nrhs right-hand sides (the incidence of dda_set_incidence).
 *   d_b   complex128 box fields, or NULL for the plane waves (then written
 *         nowhere: the library forms b in its workspace).
 *   d_x   complex128 box fields: initial guess in, solution out.
 *   h_stats host array of nrhs records (may be NULL).
 * Right-preconditioned restarted GMRES: Arnoldi with classical Gram-Schmidt
 * and a second pass whenever the first left less than reorth_eta of ||w||
 * (selective reorthogonalisation); dots and norms summed in FP64 across
 * threads (complex64 vectors: FP32 products with compensated FP32 per-thread
 * sums); Givens rotations and the small least-squares solve in FP64 on the
 * device.  Every restart recomputes
 * the residual b - A x in complex128; with inner_prec = DDA_C64 the Krylov
 * basis, matvecs and preconditioner run in complex64 (FP64 iterative
 * refinement).  The loop's decisions (restart, convergence, iteration cap,
 * time limit) are taken on the device; with the plan's schedule field graph
 * = 1 (the default) the whole loop is one CUDA graph launch (see
 * dda_schedule_t), captured on the first solve with given arguments and
 * reused by later ones with the same arguments, device pointers included.
 * Returns DDA_ERR_NOT_CONVERGED if any right-hand side missed tol within
 * max_iters (x then holds the last iterate), DDA_ERR_TIMEOUT if the time
 * limit stopped one, DDA_ERR_BREAKDOWN if a restart cycle ended without a
 * single iteration (BiCG-Stab breaking down at its first step: the next
 * cycle would repeat it, so that right-hand side stops; the loop always
 * ends), DDA_ERR_NAN on a non-finite residual, DDA_ERR_NO_PRECOND
 * if precond = 3 was asked before dda_precond_build.  Synchronises
 * `stream`. */
dda_status_t dda_solve(dda_plan_t plan, int32_t nrhs, const void* d_b, void* d_x,
                       const dda_solve_opts_t* opts, dda_rhs_stats_t* h_stats, void* stream);

/* Newton shifts of the s-step GMRES (method 2) from Arnoldi Hessenberg
 * matrices, as the solver computes them after its first cycle: for each
 * right-hand side r, the eigenvalues of the leading k x k block of
 * d_hraw[r] (device complex128 [(m+1) x m], column-major: entry (i, j) at
 * j*(m+1) + i; upper Hessenberg), k = min(d_jlen[r], 4 s, 32), by shifted QR
 * iterations, and the first s of them in Leja order (Reichel, BIT 30 (1990)
 * 332: the one of largest modulus, then each next maximising the product of
 * its distances to those taken) into d_theta[r] (device complex128 [8];
 * entries past min(s, k) are zero).  d_jlen: device int32 [nrhs].  Queued on
 * `stream`, no synchronisation.  DDA_ERR_INVALID_ARG on NULL or m < 1,
 * nrhs < 1, s outside 1..8.  A test hook of the solver. */
dda_status_t dda_ritz_shifts(const void* d_hraw, int32_t m, const int32_t* d_jlen, int32_t nrhs,
                             int32_t s, void* d_theta, void* stream);

/* Several independent systems solved concurrently: plan i's system (arguments
 * as dda_solve's, arrays of length nplans; d_b may be NULL or hold NULL
 * entries for the incident field, h_stats may be NULL or hold NULL entries)
 * with the shared options *opts.  One host thread per plan drives its solve
 * loop on streams[i], so the short kernels of small systems (an uneven batch
 * of prisms) overlap on the GPU; every result equals that of the same
 * dda_solve call alone.  Plans must be distinct and so must the non-NULL
 * streams (NULL entries use the default stream and serialise).  Returns when
 * every solve has ended: DDA_OK, or the first failing status in plan order
 * (dda_last_error names the plan).  Not part of the paper: a batching form of
 * its solve (Section 4). */
dda_status_t dda_solve_many(int32_t nplans, const dda_plan_t* plans, const int32_t* nrhs,
                            const void* const* d_b, void* const* d_x,
                            const dda_solve_opts_t* opts, dda_rhs_stats_t* const* h_stats,
                            void* const* streams);

/* Cross sections of the solutions d_c (complex128 box fields) for the
 * incidence set by dda_set_incidence; h_out[3*r + {0,1,2}] = C_ext, C_abs,
 * C_sca of right-hand side r.  The paper prints no formula; these are the
 * standard DDA expressions (Draine & Flatau) with p = dx^3 c, |E_inc| = 1:
 *   C_ext = 4 pi k sum Im(conj(E_inc) . p)
 *   C_abs = 4 pi k sum (-Im(1/alpha_DF) - 2k^3/3) |p|^2,  alpha_DF = dx^3 alpha
 *   C_sca = 4 pi k [Im(p^H G p) + (2/3) k^3 |p|^2]   (G p by one complex128 FFT matvec;
 *           equals 4 pi k p^H Im(G) p because G is complex symmetric)
 * Synchronises `stream`. */
dda_status_t dda_cross_sections(dda_plan_t plan, int32_t nrhs, const void* d_c, double* h_out,
                                void* stream);

/* Kernel timing (tracing).  While enabled, the library brackets each
 * launch of the operator's FFT passes and of the Gram-Schmidt kernels with
 * CUDA events on the launching stream.  dda_profile_read synchronises those
 * events and returns, per kernel class, the summed milliseconds and the
 * launch count: index 0..4 matvec passes (x forward, y forward, z with the
 * spectrum multiply, y inverse, x inverse with the diagonal), 5..9 the
 * preconditioner's passes in the same order, 10 Gram-Schmidt dots,
 * 11 Gram-Schmidt update (first pass only), 12 the 2-level
 * preconditioner's block pass (its FFT passes count as 5, 6, 8, 9), 13..17
 * the matvec passes and 18..22 the preconditioner passes of complex128
 * launches (0..9 count complex64 launches only); n entries are written
 * (n <= 23); reset != 0 zeroes the sums.  h_bytes (may be NULL) receives the
 * summed algorithmic bytes of the timed launches: per right-hand side and
 * with F = one three-component box field (3 l m n values), matvec passes 3F
 * (+mask), 6F, 8F (+ the kernel spectrum once), 6F, 4F (+mask);
 * preconditioner passes 2F each (+mask, + the circulant spectrum once for
 * the middle one); Gram-Schmidt dots (j+2)F, update (j+3)F at Arnoldi step
 * j.  Events add a few microseconds per launch. */
dda_status_t dda_profile_enable(dda_plan_t plan, int32_t on);
dda_status_t dda_profile_read(dda_plan_t plan, double* h_ms, int64_t* h_count, double* h_bytes,
                              int32_t n, int32_t reset);

/* Right-hand side of the adjoint problem: d_b[rhs] = conj(E_inc) on scatterer
 * voxels, 0 on air (complex128).  The DDA matrix is complex symmetric
 * (A = A^T, Section 2.2), so the adjoint of the extinction functional is the
 * solve A lambda = conj(E_inc) with the same plan, preconditioner and
 * solver (dda_solve with d_b = this field). */
dda_status_t dda_adjoint_rhs(dda_plan_t plan, int32_t nrhs, void* d_b, void* stream);

/* Gradient of C_ext with respect to every voxel's permittivity, from the
 * solution c (A c = E_inc) and the adjoint solution lambda (A lambda =
 * conj(E_inc)), both complex128 box fields.  Perturbing eps_j changes only
 * alpha_j^{-1} (Section 2.1), so with g_j = (lambda_j . c_j) d(alpha_j^{-1})/
 * d(eps_j) (unconjugated over the 3 components) and
 * d(alpha^{-1})/d(eps) = -4 pi/(eps-1)^2 + (b2 + b3 S)(k dx)^2:
 *   d_grad[rhs][0][z][y][x] = dC_ext/dRe(eps) = -4 pi k dx^3 Im(g),
 *   d_grad[rhs][1][z][y][x] = dC_ext/dIm(eps) = -4 pi k dx^3 Re(g),
 * zero on air (device doubles, 2 * l*m*n per right-hand side). */
dda_status_t dda_ext_gradient(dda_plan_t plan, int32_t nrhs, const void* d_c,
                              const void* d_lambda, double* d_grad, void* stream);

/* Launch schedule of a plan: choices that change how the operator's kernels
 * are launched, never what they compute (every schedule gives the same
 * results up to rounding order).
 *   rr_z: 1 = the complex64 matvec's z pass at transform lengths 64 and 128
 *         keeps the last forward and first inverse butterflies in registers
 *         (the 3x3 spectrum multiply between them); 0 = the all-shared-memory
 *         z kernel.  Other lengths and complex128 ignore it.
 *   pdl:  1 = kernels are launched with programmatic dependent launch (the
 *         next kernel's blocks become resident while the previous one drains);
 *         0 = ordinary stream-ordered launches.
 *   z_occ: 1 = the register-resident z pass of 256-thread tiles (lengths 128
 *         and 256) is compiled with registers bounded so that three blocks share
 *         an SM (more warps in flight); 0 = the compiler's own register count.
 *   graph: 1 = dda_solve captures its whole loop once into a CUDA graph whose
 *         conditional nodes (a WHILE over restart cycles, an IF per cycle, a
 *         WHILE over the cycle's steps) take their conditions from the device
 *         (convergence, iteration cap, time limit), so a solve is one graph
 *         launch with no host round trip; the graph is kept and reused while
 *         the solve's arguments stay the same.  0 = the host drives the loop
 *         and polls the device's decisions.  Kernel timing
 *         (dda_profile_enable) always uses the host-driven loop.
 * A new plan starts with {1, 0, 1, 1} (programmatic dependent launch
 * measured slower on the 64^3 solves).  The environment variables DDA_RR_FFT3C=0,
 * DDA_PDL=0 and DDA_SOLVE_GRAPH=0 force the plain forms whatever the schedule.
 * The schedule applies to dda_matvec, dda_precond_apply, dda_precond2_apply
 * and dda_solve (hence dda_solve_many) of that plan, in the calling thread.
 * Not in the paper. */
typedef struct {
  int32_t rr_z;
  int32_t pdl;
  int32_t graph;
  int32_t z_occ;
} dda_schedule_t;

/* Set or read a plan's schedule (no GPU work).  Fields must be 0 or 1;
 * DDA_ERR_INVALID_ARG otherwise or on NULL. */
dda_status_t dda_schedule_set(dda_plan_t plan, const dda_schedule_t* sched);
dda_status_t dda_schedule_get(dda_plan_t plan, dda_schedule_t* out);

/* What dda_autotune measured. */
typedef struct {
  dda_schedule_t chosen;     /* the schedule now set on the plan */
  int32_t cached;            /* 1: taken from the process-wide table, nothing timed */
  int32_t ncand;             /* schedules timed (0 when cached) */
  dda_schedule_t cand[8];    /* the schedules timed, in order (graph as set) */
  float ms_per_matvec[8];    /* their mean CUDA-event time per matvec call */
} dda_tune_report_t;

/* Autotuner: choose the plan's schedule by timing the matvec.  Each of the
 * eight schedules (rr_z x pdl x z_occ) runs 2 untimed then `reps` timed dda_matvec calls
 * (precision prec, nrhs right-hand sides, input d_x, output d_y: caller-owned
 * device fields of that precision, box layout as dda_matvec's, not
 * overlapping; d_y is overwritten) bracketed by CUDA events on `stream`; the
 * fastest is set on the plan and recorded in a process-wide table keyed on
 * (device, l, m, n, prec, nrhs).  A later call with the same key takes the
 * recorded schedule without timing unless flags bit 0 (re-measure) is set.
 * h_report (host, may be NULL) receives the measurements.  reps in 1..1000.
 * Synchronises `stream`; errors as dda_matvec's (the plan's schedule is then
 * left as it was).  Not in the paper. */
dda_status_t dda_autotune(dda_plan_t plan, int32_t prec, int32_t nrhs, const void* d_x,
                          void* d_y, int32_t reps, int32_t flags, dda_tune_report_t* h_report,
                          void* stream);

/* Release the host-side plan object (device memory stays the caller's). */
void dda_plan_destroy(dda_plan_t plan);

/* Thread-local text of the last error ("" if none). */
const char* dda_last_error(void);

/* Number of CUDA kernels the library has launched in this process so far. */
int64_t dda_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* DDA_H_ */
