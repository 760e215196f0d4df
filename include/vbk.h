/*
 * vbk.h - C ABI of the GB300 library for vibronic dynamics in the electron continuum.
 *
 * The library solves, for many energies at once, the complex-symmetric linear system
 *     (E - H_ef) Psi = Phi                                      (arXiv:2307.13483, Eq. Ax=b)
 * with H_ef = H_0 + U + F(E - H_0) (Sec. II.A, Eq. H_ef) in the harmonic-oscillator product
 * basis (Sec. II.D), by preconditioned Krylov methods (Sec. III: restarted GMRES and COCG with
 * block-diagonal preconditioners), and evaluates the T-matrix, cross sections (Eqs. Td, crs,
 * crs2), the 2D electron energy-loss spectrum (Eq. 2Dsp) and adjoint gradients of a
 * cross-section loss.
 *
 * Conventions for every call:
 *  - Energies are in eV.  All floating-point data crossing the ABI are IEEE double; complex
 *    data are interleaved (re, im) doubles ("complex128").
 *  - Vectors over the discretised space use the compound index alpha = (d, n_1, ..., n_M)
 *    with the state index d slowest and the last mode fastest (C order); N = n_states *
 *    prod_m n_basis[m] is the number of unknowns.
 *  - Pointers named *_dev are device pointers owned by the caller; other pointers are host
 *    pointers owned by the caller.  The library never frees caller memory.  Models are owned
 *    by the library and released with vbk_free_model.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work is enqueued on
 *    it; calls that return host results (vbk_stats, gradients on the host) synchronise it.
 *    One model handle must not be used from two host threads at the same time.
 *  - Every call returns a status (VBK_OK = 0 on success).  No C++ exception crosses the
 *    ABI.  On an error the output buffers are unspecified and vbk_last_error() returns a
 *    message for the calling thread.
 */
#ifndef VBK_H
#define VBK_H

#ifdef __cplusplus
extern "C" {
#endif

#define VBK_MAX_MODES 4
#define VBK_MAX_STATES 4
#define VBK_MAX_CHANNELS 8
#define VBK_MAX_CTERMS 32

/* Return codes of the API calls. */
#define VBK_OK 0
#define VBK_ERR_INVALID_ARG 1   /* a size, index or parameter is out of range          */
#define VBK_ERR_OOM 2           /* device or host allocation failed                    */
#define VBK_ERR_CUDA 3          /* a CUDA runtime call or kernel launch failed          */
#define VBK_ERR_NOT_CONVERGED 4 /* at least one system did not reach the tolerance      */
#define VBK_ERR_UNSUPPORTED 5   /* the model uses a feature this build does not support */
#define VBK_ERR_NO_DEVICE 6     /* no CUDA device is visible                            */

/* Per-system outcome (vbk_stats.status). */
#define VBK_SYS_CONVERGED 0 /* ||Phi - A psi|| / ||Phi|| <= tol (refinement residual, VBK_MIXED) */
#define VBK_SYS_MAX_ITER 1  /* iteration or refinement cap reached                             */
#define VBK_SYS_BREAKDOWN 2 /* COCG bilinear form p^T A p or r^T z vanished (Sec. III.A)       */
#define VBK_SYS_NAN 3       /* a non-finite value appeared                                     */
#define VBK_SYS_PIVOT 4     /* a zero pivot in the LDL^T factor of a preconditioner block      */
#define VBK_SYS_ZERO_RHS 5  /* Phi = 0 (closed incident channel); psi = 0 is returned          */

/* One polynomial term of the direct vibronic coupling U (Sec. II.A, Eq. H_d; Eq. U):
 * coef * T in the block (d, dp) of U with T = prod_m O_m, where O_m = q_m^pow[m], or, for a
 * mode with raise[m] or lower[m] nonzero (then pow[m] = 0), the ladder monomial
 * (a_m^+)^raise[m] a_m^lower[m] (normal order).  q_m is the dimensionless normal coordinate with
 * <n|q|n+1> = sqrt((n+1)/2) (Sec. III), a_m|n> = sqrt(n)|n-1>; powers and monomials are products
 * of the truncated matrices.  Only d <= dp is given: a term with d < dp adds coef T^T to block
 * (dp, d), and one with d = dp adds the symmetric part coef (T + T^T)/2 (T itself when every
 * O_m is a power of q), so U is real symmetric.  State energies E_d are terms with all powers
 * zero.  Ladder monomials serve a two-dimensional mode written in circular oscillator quanta
 * n_+-, the polar eigenfunctions |v, l> of the 2D isotropic oscillator with v = n_+ + n_-,
 * l = n_+ - n_- (Sec. III.C, CO2 model): there q_x +- i q_y = a_-+ + a_+-^+ have real matrix
 * elements.  raise[m], lower[m], pow[m] are each 0..8. */
typedef struct {
    int d, dp;
    double coef;
    int pow[VBK_MAX_MODES];
    int raise[VBK_MAX_MODES];
    int lower[VBK_MAX_MODES];
} vbk_term;

/* Coupling of discrete state d to partial wave mu (Sec. II.B): width
 * Gamma(eps) = a * eps^(l + 1/2) * exp(-b * eps), f = sqrt(Gamma / 2 pi) >= 0.  Without
 * polynomial terms (vbk_cterm) the coupling is independent of q and the channel adds the level
 * shift F[Gamma/2pi](E - E_nu) (Eq. IntF) to the diagonal of its state.  A state couples to a
 * partial wave at most once. */
typedef struct {
    int d, mu;
    double a, b;
    int l;
} vbk_channel;

/* One term of the coupling polynomial P_c(q) of channel c, making the coupling q-dependent
 * and separable, V^mu_{d eps}(q) = f_d^mu(eps) P_c(q) (Sec. II.C): coef * prod_m q_m^pow[m],
 * powers as in vbk_term (products of truncated matrices).  A channel without terms has
 * P_c = 1.  A partial wave whose channels carry terms, or that couples to two or more states,
 * contributes the non-local operator F_dd' = sum_mu P_c F[f_c f_c'](E - H_0) P_c' over the
 * ordered pairs (c, c') of its channels (Eq. FE, from Eq. F_gen), with
 * f_c f_c' = (sqrt(a_c a_c') / 2 pi) eps^(l + 1/2) exp(-(b_c + b_c') eps / 2); the channels
 * of such a wave must share l.  Phi^{v mu} then carries f_c(eps) P_c(q)|v> (Sec. II.D). */
typedef struct {
    int channel;
    double coef;
    int pow[VBK_MAX_MODES];
} vbk_cterm;

/* Model: states, harmonic modes (Eq. H0harm: omega[m], basis n = 0..n_basis[m]-1),
 * polynomial U and continuum channels.  Arrays are copied by vbk_build_model. */
typedef struct {
    int n_states;                  /* 1..VBK_MAX_STATES           */
    int n_modes;                   /* 1..VBK_MAX_MODES            */
    int n_basis[VBK_MAX_MODES];    /* >= 1 each                   */
    double omega[VBK_MAX_MODES];   /* > 0 each                    */
    int n_terms;
    const vbk_term* terms;         /* host, [n_terms]             */
    int n_channels;                /* 1..VBK_MAX_CHANNELS         */
    const vbk_channel* channels;   /* host, [n_channels]          */
    int n_cterms;                  /* 0..VBK_MAX_CTERMS (0: every coupling independent of q) */
    const vbk_cterm* cterms;       /* host, [n_cterms], or NULL when n_cterms = 0            */
} vbk_model_desc;

typedef struct vbk_model vbk_model;

/* Krylov methods (Sec. III.A). */
#define VBK_GMRES 0 /* restarted GMRES(m), right-preconditioned, CGS2 Arnoldi, FP64 Givens LSQ */
#define VBK_COCG 1  /* preconditioned COCG with the bilinear form a^T b                        */

/* Arithmetic of the Krylov iterations. */
#define VBK_FP64 0  /* complex FP64 throughout                                                  */
#define VBK_MIXED 1 /* complex FP32 Krylov iterations inside iterative refinement.  The
                       refinement residual b - A x and the solution x are kept in FP64, except
                       on the resident path (VBK_COCG with the point preconditioner and
                       opts.resident = 1, when a system fits one SM's shared memory): there
                       x, the diagonal of A and the residual are double-float numbers
                       (unevaluated sums hi + lo of two FP32 values: ~48-bit significands,
                       FP32 exponent range) formed on the FP32 pipes, and ||r||^2 is summed
                       in FP32 within a warp and in FP64 across warps (relative error
                       ~1e-7 of the norm, i.e. of the stopping threshold, not of r).  psi is
                       returned in FP64 (hi + lo, exact).  The GMRES Hessenberg least-squares
                       problem is FP64 in every case.                                         */

/* Block-diagonal preconditioner (Sec. III.B), given by the indices its blocks SPAN:
 * bit 0 = the discrete-state index d, bit (1 + m) = mode m.  The paper names preconditioners
 * by the indices held FIXED: for two modes (g = mode 0, u = mode 1),
 *   M^{gu} = span d          = 0x1   (2x2 blocks)
 *   M^{g}  = span d and u    = 0x5   (2 N_u blocks)
 *   M^{u}  = span d and g    = 0x3
 *   M^{d}  = span g and u    = 0x6
 *   M^{dg} = span u = 0x4,  M^{du} = span g = 0x2.
 * 0 = point Jacobi.  VBK_PRECOND_NONE disables preconditioning.  Blocks are factored as
 * B = L D L^T (complex symmetric, no pivoting) once per energy before iterating. */
#define VBK_PRECOND_NONE (-1)

typedef struct {
    int method;        /* VBK_GMRES or VBK_COCG                                            */
    int precision;     /* VBK_FP64 or VBK_MIXED                                            */
    int precond_span;  /* see above                                                        */
    int restart;       /* GMRES restart length m (1..256); one restart cycle per refinement */
    int max_iter;      /* cap on Krylov iterations per system, summed over refinements     */
    int max_refine;    /* cap on refinement steps per system                               */
    double tol;        /* stop when ||Phi - A psi||_2 / ||Phi||_2 <= tol (true residual)    */
    double inner_tol;  /* relative tolerance of each inner solve (COCG; GMRES stops a cycle
                          early when its residual estimate reaches it)                      */
    int check_every;   /* iterations between host convergence checks (>= 1)                */
    int timing;        /* 1: record per-kernel CUDA-event timings (see vbk_kernel_timings);
                          the Krylov loop then launches kernels directly instead of as graphs */
    int autotune;      /* 1: on the first solve of a model, time the matvec kernel variants on
                          the batch and keep the fastest (per precision) for later calls       */
    int resident;      /* FP32 COCG with the point preconditioner (or none), when a system's
                          p and q (2 N * 8 bytes + tables) fit one thread block's shared memory:
                          1 = the whole refinement of each system (double-float residual, checks,
                          inner solves, FP64 output) in one thread block, all systems in one
                          launch; 2 = each inner solve in one thread block, the refinement steps
                          between launches; 3 = as 1 but one cluster of n_states thread blocks
                          per system (one block per discrete state, every FP32 vector on chip;
                          falls back to 2 where it does not fit); 0 = grid-wide kernels     */
    int inner_max_iter; /* VBK_MIXED COCG: iterations of one FP32 inner solve before it ends
                          and the refinement residual restarts it (complex-FP32 COCG can stagnate
                          short of inner_tol on hard systems); 0 = no cap                    */
    int matvec_variant; /* -1: the autotuned (or default) kernel variant of the batched matvec on
                          the grid-wide paths; 0 .. VBK_MATVEC_NVARIANTS - 1: that variant (see
                          vbk_matvec) for the Krylov operator and the FP64 residual, wherever it
                          is valid for their precision; VBK_ERR_INVALID_ARG if it is valid for
                          neither.  Not used by the one-block-per-system paths (resident 1..3)  */
} vbk_opts;

/* Fills `o` with defaults: GMRES, VBK_MIXED, Jacobi, restart 64, max_iter 20000,
 * max_refine 40, tol 1e-8, inner_tol 1e-5, check_every 8, timing 0, autotune 1, resident 1,
 * inner_max_iter 2000, matvec_variant -1. */
void vbk_default_opts(vbk_opts* o);

typedef struct {
    int status;          /* VBK_SYS_*                                                    */
    int iterations;      /* Krylov iterations (matrix-vector products in the inner loop) */
    int refinements;     /* refinement residual evaluations after the first              */
    double rel_residual; /* final ||Phi - A psi|| / ||Phi|| of the refinement residual: FP64,
                            or double-float on the resident VBK_MIXED path (see VBK_MIXED)  */
} vbk_stats;

/* Builds a model from the description (Sec. II; tables of Sec. III: oscillator matrix
 * elements and their truncated powers are precomputed once).  *out receives a handle.
 * Errors: VBK_ERR_INVALID_ARG for out-of-range sizes/indices, non-finite or non-positive
 * omega, b <= 0, a < 0, l < 0, a state coupled twice to one partial wave, channels of a
 * q-dependent partial wave with different l, a coupling term naming no channel;
 * VBK_ERR_UNSUPPORTED when the q-dependent couplings need more than 64 polynomial points in
 * all; VBK_ERR_NO_DEVICE, VBK_ERR_OOM, VBK_ERR_CUDA. */
int vbk_build_model(const vbk_model_desc* desc, vbk_model** out);

/* Releases the model and its device tables.  NULL is ignored. */
void vbk_free_model(vbk_model* model);

/* Number of unknowns N and of partial waves n_mu (= 1 + the largest mu of a channel). */
int vbk_model_size(const vbk_model* model, int* n_unknowns, int* n_partial_waves);

/* Solves (E - H_ef) psi = Phi^{v_i mu} (Eq. Ax=b; Phi of Sec. II.D) for every incident
 * energy eps_i[e] (host, [n_eps], > 0), every initial state vi[i] (host, [n_vi][n_modes]
 * multi-indices) and every partial wave mu = 0..n_mu-1, with total energy
 * E = eps_i + E_{v_i} (Eq. Econserv).
 *   psi_dev : device complex128 [n_eps][n_vi][n_mu][N], written.
 *   stats   : host [n_eps * n_vi * n_mu] in the same order, or NULL.
 * Returns VBK_ERR_NOT_CONVERGED if any system ended with a status other than CONVERGED or
 * ZERO_RHS (psi then holds the last iterate).  With VBK_MIXED COCG, a system whose FP32 inner
 * iterations stop helping (a refinement step lowers the refinement residual by less than 10%, or a
 * non-finite value or a breakdown appears) is solved again in FP64 from psi = 0, and its stats
 * add both runs.  Synchronises `stream`. */
int vbk_solve(vbk_model* model, int n_eps, const double* eps_i, int n_vi, const int* vi,
              const vbk_opts* opts, void* psi_dev, vbk_stats* stats, void* stream);

/* Cross sections sigma_{vf <- vi}(eps_i) = 2 pi^3 / eps_i * sum_{mu_i, mu_f} |T|^2 with
 * T_{mu_f vf <- mu_i vi} = <Phi^{vf mu_f} | Psi^{vi mu_i}> (Eqs. Td, crs, crs2), from the
 * solutions of vbk_solve with the same (n_eps, eps_i, n_vi, vi).  Energies in eV, sigma raw
 * (eV units, no conversion to a_0^2).
 *   vf        : host [n_vf][n_modes] final multi-indices; closed channels give sigma = 0.
 *   sigma_dev : device double [n_eps][n_vi][n_vf], written.
 *   t_dev     : device complex128 [n_eps][n_vi][n_mu(i)][n_vf][n_mu(f)] or NULL.
 * Asynchronous on `stream`. */
int vbk_cross_sections(vbk_model* model, int n_eps, const double* eps_i, int n_vi, const int* vi,
                       const void* psi_dev, int n_vf, const int* vf, double* sigma_dev,
                       void* t_dev, void* stream);

/* 2D electron energy-loss spectrum S(eps_i, de) = sum_f sigma_f(eps_i) rho(de - (E_vf - E_vi))
 * (Eq. 2Dsp) with rho a unit-area Gaussian of full width at half maximum `fwhm` (eV).
 *   sigma_dev : device double [n_eps][n_vi][n_vf] from vbk_cross_sections.
 *   de        : host [n_de] energy-loss grid.   S_dev : device double [n_eps][n_vi][n_de].
 * Asynchronous on `stream`. */
int vbk_eels(vbk_model* model, int n_eps, int n_vi, const int* vi, int n_vf, const int* vf,
             const double* sigma_dev, int n_de, const double* de, double fwhm, double* S_dev,
             void* stream);

/* Gradient of a loss L(sigma) with respect to model parameters by the adjoint method.
 * Given dL/dsigma (device double [n_eps][n_vi][n_vf]) and the forward solutions psi_dev of
 * vbk_solve, it solves A lambda = sum_{f, mu_f} w_f Phi^{vf mu_f} per forward system with the
 * same operator (A = A^T, Sec. II.D) and contracts
 *   dL/dtheta = Re sum [ sum_f w_f dPhi_f^T psi + lambda^T dPhi_i - lambda^T (dA/dtheta) psi ],
 *   w_f = dL/dsigma * 2 pi^3/eps_i * 2 conj(T_f).
 * theta_ids (host [n_theta]): k < n_terms is the coefficient of term k; n_terms + 2c and
 * n_terms + 2c + 1 are a and b of channel c; n_terms + 2 n_channels + t is the coefficient of
 * coupling term t (vbk_cterm, in the order given; Sec. II.C).  For q-dependent partial waves
 * the derivatives run through the non-local level shift of Eq. FE (pair transforms
 * F[f_c f_c'] depend on a_c through sqrt(a_c a_c') and on b_c through (b_c + b_c') / 2) and
 * through Phi = f_c P_c |v>.
 *   grad      : host double [n_theta], written (a host buffer: the ~20 numbers are reduced
 *               on the device and copied back, since callers use them on the host, e.g. in
 *               an optimiser or a torch.autograd backward that builds a CPU tensor).
 *   stats     : host [n_eps * n_vi * n_mu] adjoint solve outcomes, or NULL.
 * Synchronises `stream`. */
int vbk_solve_adjoint(vbk_model* model, int n_eps, const double* eps_i, int n_vi, const int* vi,
                      const vbk_opts* opts, const void* psi_dev, int n_vf, const int* vf,
                      const double* dL_dsigma_dev, int n_theta, const int* theta_ids,
                      double* grad, vbk_stats* stats, void* stream);

/* Number of matvec kernel variants vbk_matvec accepts (0 .. VBK_MATVEC_NVARIANTS - 1). */
#define VBK_MATVEC_NVARIANTS 20

/* y = A(E_k) x for a batch: the matrix-free operator of Sec. III (diagonal energy and
 * level-shift factors plus the q-polynomial stencils; with q-dependent couplings also the
 * non-local level shift of Eq. FE, applied as two stencil passes through the coupling
 * polynomials with the pair transforms tabulated per energy; only variant 8 (or -1) then).
 *   E       : host [n_E] total energies.   n_vec : vectors per energy.
 *   x_dev, y_dev : device complex128 [n_E][n_vec][N].
 *   precision: VBK_FP64 computes in FP64; VBK_MIXED rounds x and the operator to FP32,
 *   computes in FP32 and widens y.
 *   variant : kernel variant, -1 = the model's autotuned choice; 0..3 = register-blocked
 *   kernel with (systems, elements) per thread (1,4), (2,4), (4,2), (2,2); 4..7 = shared-
 *   memory-windowed kernel with (1,4), (2,4), (4,2), (8,1); 8, 9 = direct kernel with 1 or 4
 *   systems per thread; 10, 11 = one or two systems per thread block with x in shared memory
 *   (VBK_MIXED only); 12..15 = every state of a tile per thread block, x windows staged
 *   asynchronously, coefficients from shared memory, (systems per block, elements per thread)
 *   = (2,4), (2,2), (4,2), (1,4); 16..19 = persistent streaming kernel: a producer warp per
 *   thread block brings the x windows and diagonal rows of tiles of (systems, rows of the first
 *   mode) into a ring of shared-memory stages by bulk asynchronous copies while the other warps
 *   compute, (systems per tile, row groups, rows per tile, stages) = (4,4,8,2), (4,2,4,2),
 *   (2,2,8,3), (2,4,16,2); offered when n_states * N_nu / n_basis[0] <= 640, every term involves at
 *   most two modes and, in VBK_MIXED, N_nu / n_basis[0] is even.  VBK_ERR_INVALID_ARG if the
 *   variant does not fit this model and precision.  Asynchronous on `stream`. */
int vbk_matvec(vbk_model* model, int n_E, const double* E, int n_vec, const void* x_dev,
               void* y_dev, int precision, int variant, void* stream);

/* y = A(E_k) x in FP64 without allocating device memory (the paper has no counterpart: this
 * is a service of the library).  For callers that cannot allocate when they apply the
 * operator, e.g. a process whose device memory another framework's allocator has already
 * reserved, or a real-time loop that allows no allocation after start-up.  Same operator,
 * shapes and result as vbk_matvec with VBK_FP64; the model must have been built before.
 * Scratch (energies, system map, diagonal tables) lives in a fixed 8 MiB device array inside
 * the library, held by every GPU that loads the library until the process exits:
 *   n_E * N * 16 + n_E * 8 + n_E * n_vec * 4 bytes (each part rounded up to 256) <= 8 MiB,
 *   and n_E * n_vec <= 4096; larger requests return VBK_ERR_INVALID_ARG with a message.
 * The first call on a device looks up the array's device address (set-up); make that first
 * call before any stream capture.  All calls share the array: calls that overlap on the GPU
 * (other streams, other host threads) race.  Synchronises `stream`.  No cudaMalloc, cudaFree
 * or allocating library routine is called.  Models with q-dependent couplings (vbk_cterm, or a
 * partial wave coupled to several states) need per-call tables of the non-local level shift
 * that the array does not hold: VBK_ERR_UNSUPPORTED. */
int vbk_matvec_noalloc(vbk_model* model, int n_E, const double* E, int n_vec, const void* x_dev,
                       void* y_dev, void* stream);

/* z = B^-1 r with B the block-diagonal preconditioner `precond_span` of A(E_k) (Sec. III.B),
 * factored as L D L^T; its blocks include the entries of the non-local level shift (Eq. FE)
 * that fall inside them.  Shapes as in vbk_matvec.  Asynchronous on `stream`.  A zero pivot
 * gives VBK_ERR_NOT_CONVERGED (and synchronises). */
int vbk_precond_apply(vbk_model* model, int n_E, const double* E, int n_vec, int precond_span,
                      const void* r_dev, void* z_dev, int precision, void* stream);

/* Per-kernel timings of the last vbk_solve / vbk_solve_adjoint run with opts.timing = 1:
 * up to `cap` entries of (name, launches, total milliseconds measured with CUDA events on
 * the launch stream).  Returns the number of entries available. */
int vbk_kernel_timings(const vbk_model* model, int cap, const char** names, int* launches,
                       double* total_ms);

/* on = 1: each later vbk_matvec / vbk_precond_apply call on this model records per-kernel
 * CUDA-event timings of its own launches (replacing those of the previous call or solve; read
 * them with vbk_kernel_timings) and synchronises `stream`; on = 0 (the default) turns it off.
 * The paper has no counterpart: this serves measurement of the operator kernels alone. */
int vbk_set_op_timing(vbk_model* model, int on);

/* Test hook for the bounded waits of the streaming matvec (variants 16..19; the paper has no
 * counterpart).  The next launch of such a variant holds the first copies of every thread
 * block back by `ms` milliseconds (0 .. 10000; later launches are not affected).  With a delay
 * past the kernels' wait limit (1 s) the computing warps stop waiting instead of waiting
 * without end: the launch completes, a device flag records it, its output is not valid, and
 * the call that reads the flag (vbk_solve, or vbk_matvec with vbk_set_op_timing on) returns
 * VBK_ERR_CUDA with a message.  The CUDA context stays usable.  VBK_ERR_INVALID_ARG for a delay
 * out of range. */
int vbk_debug_stream_delay(int ms);

/* Matvec kernel variant the autotuner chose for this model in `precision` (VBK_MIXED: the FP32
 * Krylov operator, VBK_FP64: the FP64 residual), or -1 if it has not run yet. */
int vbk_matvec_variant(const vbk_model* model, int precision);

/* Number of kernel launches issued by the last vbk_solve / vbk_solve_adjoint call. */
long long vbk_last_launch_count(const vbk_model* model);

/* The level-shift factor F[Gamma/2pi](eps) of one channel (Eq. IntF with the width
 * Gamma(eps) = a eps^(l+1/2) exp(-b eps) of Sec. II.B), evaluated on the host with the same
 * closed form the device tables use.  Writes Re F and Im F = -Gamma/2.  Needs no GPU. */
int vbk_level_shift(double eps, double a, double b, int l, double* re, double* im);

/* The same level-shift factor evaluated in double-float arithmetic (unevaluated sums of two
 * floats, ~2^-47 relative per operation), the way the FP32 refinement path builds its energy
 * tables on the GPU (GB300 runs FP32 far faster than FP64); host evaluation of the identical
 * code, for checking it against vbk_level_shift.  Needs no GPU. */
int vbk_level_shift_df(double eps, double a, double b, int l, double* re, double* im);

/* Human-readable text of a return code (VBK_OK, VBK_ERR_*). */
const char* vbk_status_str(int code);

/* Human-readable text of a per-system status (VBK_SYS_*). */
const char* vbk_sys_status_str(int status);

/* Message of the last error on the calling thread (empty string if none). */
const char* vbk_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VBK_H */
