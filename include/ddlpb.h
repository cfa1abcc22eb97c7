/*
 * ddlpb.h -- C ABI of the GB300 (sm_103a) ddLPB energy + analytical force library.
 *
 * The method: Jha, Nottoli, Mikhalev, Quan, Stamm, "Linear scaling computation
 * of forces for the domain-decomposition linear Poisson-Boltzmann method"
 * (arXiv:2203.00552).  A solute is a union of M atom-centred balls
 * (Sec. 1; van der Waals radii, or solvent-accessible radii = vdW + 1.4 A)
 * carrying point charges (Eq. rho_definition).  Each ball carries real
 * spherical-harmonic expansions up to degree lmax of the reaction potential
 * psi_r and the extended potential psi_e (Sec. 2.2), sampled on a Lebedev grid.
 * The library assembles and solves the block system L X = g (Eq. AXg), the
 * adjoint system L* X_adj = Q (Eqs. adjoint_system, AstarXg), and returns the
 * solvation energy (Eq. energy_computation) and forces (Eq. force_lpb).
 *
 * Units: atomic units throughout.  Positions and radii in Bohr, charges in e,
 * kappa in 1/Bohr, energies in Hartree, forces in Hartree/Bohr.  The solute
 * permittivity eps_1 is 1 (Sec. 4).
 *
 * Memory: every pointer argument names memory that the caller owns; the
 * library copies inputs during the call and never keeps a caller pointer.
 * Functions whose name ends in _device take CUDA device pointers (on the device
 * that was current at ddlpb_setup); all others take host pointers.  The
 * context owns all device memory it allocates and frees it in ddlpb_free.
 * Every call runs on the CUDA stream given in ddlpb_options.cuda_stream (NULL:
 * the legacy default stream) and returns only after its results are
 * available to the caller.  Device memory is allocated and freed stream-ordered
 * on that stream, so contexts on different streams (driven from different host
 * threads) run concurrently.
 *
 * Errors: every call returns a ddlpb_status and never aborts the process.  On
 * error, ddlpb_last_error(ctx) returns a message (for a failed setup the
 * message is available through ddlpb_last_setup_error()).  A context whose
 * call returned DDLPB_ECUDA must be freed.
 */
#ifndef DDLPB_H
#define DDLPB_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DDLPB_API __attribute__((visibility("default")))
#else
#define DDLPB_API
#endif

typedef struct ddlpb_ctx ddlpb_ctx;

typedef enum { DDLPB_VDW = 0, DDLPB_SAS = 1 } ddlpb_surface;

typedef enum {
    DDLPB_OK = 0,
    DDLPB_EINVAL = 1,    /* invalid argument (size, radius, lmax vs grid, NaN ...) */
    DDLPB_ENOMEM = 2,    /* device allocation failed */
    DDLPB_ENOTCONV = 3,  /* outer solve did not reach tol within max_iter */
    DDLPB_ECUDA = 4,     /* CUDA runtime error; the context must be freed */
    DDLPB_EORDER = 5     /* call order violated (e.g. forces before adjoint) */
} ddlpb_status;

typedef enum { DDLPB_FP64 = 0, DDLPB_MIXED = 1 } ddlpb_precision;

typedef struct {
    double eta;          /* width of the smooth switch chi_eta (Eq. regular_char_function); default 0.1 */
    double tol;          /* relative residual ||g - L X|| / ||g|| of both solves; default 1e-8 */
    int max_iter;        /* cap on outer (FP64) Krylov iterations; default 500 */
    int gmres_restart;   /* Krylov basis size before restart, 1..2000; default 150 (the preconditioned
                            spectrum is real but spread, so short restarts stagnate) */
    int precision;       /* ddlpb_precision; default DDLPB_FP64 */
    int fmm_order;       /* 0: direct summation of the dense coupling; p in [lmax + 1, 21]: its far field
                            by the fast multipole method of the Appendix with expansions of order p
                            (binary tree over the Morton-ordered spheres, single-sphere leaves,
                            near pairs summed directly); default 0 */
    void* cuda_stream;   /* cudaStream_t the context launches on; NULL = legacy default stream */
    double precond_tol;  /* relative tolerance of the inner A/B solves that apply the L_AB
                            preconditioner of Sec. 4 inside flexible GMRES; default 1e-3;
                            1.0 switches the preconditioner off (plain restarted GMRES) */
    int kernel_timing;   /* 1: record CUDA events around every launch of the hot kernels (read
                            with ddlpb_kernel_time); 2: also around every other group of
                            launches (Krylov vector work, projections, forces, setup); default 0 */
    int precond_coupling; /* nonzero: the preconditioner also holds the coupling C1/C2 between
                            each sphere and its neighbours (sources j in N_i and i itself);
                            0: L_AB = diag(A, B) only, as in Sec. 4; default 0 (with an
                            iterative inner solve the near coupling slows convergence down) */
    int precond_fp16;    /* nonzero: in the mixed-precision form, the inner A/B solves of the
                            preconditioner stream an FP16 copy of the stored A/B basis (FP32
                            arithmetic; an inexact preconditioner is allowed in flexible GMRES);
                            0: they use the FP32 basis; no effect in the FP64 form; default 1 */
    double fmm_theta;    /* admissibility of the FMM: a target node A and source node B interact by
                            M2L when Rt_A + Rs_B < fmm_theta |c_A - c_B|; in (0, 1); default 0.4
                            (the far-field error falls steeply with it: at order 16 on a
                            1000-sphere SAS globule, lmax 8, the energy error against direct
                            summation is 9e-5 at 0.5, 5e-8 at 0.4, 1.5e-10 at 0.3) */
} ddlpb_options;

typedef struct {
    int n_atoms;
    int lmax;
    int n_lebedev;
    long long n_neighbour_pairs;   /* sum_i |N_i| (Sec. 2.2) */
    long long n_hits;              /* (i, n, j) with omega_ij^eta(x_i^n) > 0: nonzeros of A/B rows */
    long long n_external;          /* grid points with chi_i^eta(x_i^n) > 0 */
    int solve_iterations;          /* Krylov iterations of the last primal solve */
    int adjoint_iterations;        /* Krylov iterations of the last adjoint solve */
    double solve_residual;         /* final FP64 relative residual of the primal solve */
    double adjoint_residual;       /* final FP64 relative residual of the adjoint solve */
    int refinement_steps;          /* FP64 refinement steps of the last solve (mixed precision) */
    int inner_iterations;          /* inner A/B Krylov iterations of the last solve (preconditioner) */
    int n_sources;                 /* spheres with at least one external point (sources of the coupling) */
    long long kernel_launches;     /* CUDA kernels this context has launched since setup began */
    long long fmm_nodes;           /* FMM tree nodes (0 without the FMM) */
    long long fmm_m2l;             /* M2L translations of one FMM pass */
    long long fmm_near_pairs;      /* (target sphere, source sphere) pairs summed directly */
    double fmm_m2l_flops;          /* arithmetic of the M2L translations of one pass (rotations with the
                                      J table and the coaxial products, 2 flops per multiply-add) */
} ddlpb_info;

/* Fill *opt with the defaults listed above. */
DDLPB_API void ddlpb_default_options(ddlpb_options* opt);

/*
 * Build the discrete problem of Sec. 2.2 for one solute and compute the
 * right-hand side g = [G0 + F0; F0] (Eqs. definition_of_G_0, definition_of_F_0).
 *   n         number of atoms M >= 1
 *   centres   n*3 doubles, x y z of atom k at 3k..3k+2 (Bohr)
 *   radii     n doubles (Bohr), > 0; surface == DDLPB_SAS adds the 1.4 A probe (Sec. 4)
 *   charges   n doubles (e)
 *   eps_solvent  relative permittivity of the solvent eps_2 > 1
 *   kappa     Debye-Hueckel screening constant (1/Bohr), > 0
 *   lmax      maximum degree of the expansions, 0 <= lmax <= 16
 *   n_lebedev number of Lebedev points; one of 6, 14, 26, 38, 50, 74, 86, 110,
 *             146, 170, 194, 230, 266, 302, 350, 434, 590, 770, with an exact
 *             degree >= 2*lmax (so that the projections of Sec. 2.2 are exact)
 *   opt       NULL for the defaults
 *   out       receives the new context (NULL on error)
 * Errors: DDLPB_EINVAL (bad sizes, NaN/Inf, coincident centres, radius <= 0,
 * unsupported grid), DDLPB_ENOMEM, DDLPB_ECUDA.
 */
DDLPB_API ddlpb_status ddlpb_setup(int n, const double* centres, const double* radii, const double* charges,
                         double eps_solvent, double kappa, int lmax, int n_lebedev,
                         ddlpb_surface surface, const ddlpb_options* opt, ddlpb_ctx** out);

/* Same as ddlpb_setup with centres, radii and charges in device memory. */
DDLPB_API ddlpb_status ddlpb_setup_device(int n, const double* centres, const double* radii, const double* charges,
                                double eps_solvent, double kappa, int lmax, int n_lebedev,
                                ddlpb_surface surface, const ddlpb_options* opt, ddlpb_ctx** out);

/* Solve L X = g (Eq. AXg) to the FP64 relative residual opt.tol, by flexible GMRES
 * right-preconditioned with L_AB = diag(A, B) (Sec. 4; the inner A and B solves are
 * GMRES on the sparse blocks).  In the mixed precision mode the Krylov solve runs in
 * FP32 inside FP64 iterative refinement.  Warm-starts from the previous solution of
 * this context if there is one.  DDLPB_ENOTCONV if max_iter is reached (X then holds
 * the last iterate). */
DDLPB_API ddlpb_status ddlpb_solve(ddlpb_ctx* ctx);

/* Solve L* X_adj = Q (Eqs. adjoint_system, AstarXg), Q_{j00} = q_j Y_00.  Requires
 * a successful ddlpb_solve (else DDLPB_EORDER). */
DDLPB_API ddlpb_status ddlpb_adjoint(ddlpb_ctx* ctx);

/* E_s = 1/2 <X, Q> (Eq. energy_computation), Hartree, written to *e (host).
 * Requires ddlpb_solve. */
DDLPB_API ddlpb_status ddlpb_energy(ddlpb_ctx* ctx, double* e);

/* Forces F_k = -dE_s/dx_k (Eq. force_lpb with the derivatives of Sec. 3.1),
 * n*3 doubles in the layout of centres.  Requires ddlpb_adjoint (else
 * DDLPB_EORDER).  f is host memory (ddlpb_forces) or device memory
 * (ddlpb_forces_device). */
DDLPB_API ddlpb_status ddlpb_forces(ddlpb_ctx* ctx, double* f);
DDLPB_API ddlpb_status ddlpb_forces_device(ddlpb_ctx* ctx, double* f);

/* Energy into device memory (one double). */
DDLPB_API ddlpb_status ddlpb_energy_device(ddlpb_ctx* ctx, double* e);

/*
 * Operator access (device pointers, vectors of 2*n*(lmax+1)^2 doubles laid out
 * as [X_r ; X_e], each block sphere-major with the (l, m) index l*l + l + m).
 *   op = 0: y = L x        (Eq. AXg)
 *   op = 1: y = L* x       (Eq. AstarXg)
 *   op = 2: y = [A x_r ; B x_e]                   (Eqs. definition_of_A/B_matrix)
 *   op = 3: y = [A^T x_r ; B^T x_e]
 *   op = 4: y = [C1 x_r + C2 x_e ; same]          (Eqs. definition_of_C1/C2_matrix)
 *   op = 5: y = [C1^T (x_r + x_e) ; C2^T (x_r + x_e)]
 *   op = 8..13: the same operators in the FP32 arithmetic of the mixed-precision
 *            form (inputs rounded to FP32, outputs widened to FP64)
 *   op = 16, 17: ops 2 and 3 as the preconditioner of the mixed-precision form applies
 *            them (FP16 stored basis, FP32 arithmetic; see precond_fp16)
 * Errors: DDLPB_EINVAL for any other op.
 */
DDLPB_API ddlpb_status ddlpb_apply_device(ddlpb_ctx* ctx, int op, const double* x, double* y);

/* Copy g (op 0), X (op 1) or X_adj (op 2) into device memory y (same layout as above). */
DDLPB_API ddlpb_status ddlpb_get_vector_device(ddlpb_ctx* ctx, int which, double* y);

/* Launch count and summed device time (ms, CUDA events on the context's stream) of
 * one hot kernel since the last reset, when the context was created with
 * kernel_timing set.  name is one of ab_apply_f32, ab_apply_f64, ab_transpose_f32,
 * ab_transpose_f64, yukawa_pot_f32, yukawa_pot_f64, yukawa_adj_f32, yukawa_adj_f64;
 * an unknown or unused name gives 0 launches.  Synchronises the stream. */
DDLPB_API ddlpb_status ddlpb_kernel_time(ddlpb_ctx* ctx, const char* name, long long* launches, double* ms);

/* Reset the kernel timers. */
DDLPB_API ddlpb_status ddlpb_kernel_time_reset(ddlpb_ctx* ctx);

/* Initial guess for the next solve: which = 1 sets X (for ddlpb_solve), which = 2 sets
 * X_adj (for ddlpb_adjoint); x is device memory in the layout above.  Used to warm-start a
 * geometry close to an earlier one with that one's solutions (the reuse of the previous
 * iterate that Sec. 4 makes inside its solver, carried across geometries).  Resets the
 * call-order state: ddlpb_solve (and ddlpb_adjoint) must run again.  DDLPB_EINVAL for
 * another which. */
DDLPB_API ddlpb_status ddlpb_set_vector_device(ddlpb_ctx* ctx, int which, const double* x);

/* Counters and solver statistics. */
DDLPB_API ddlpb_status ddlpb_get_info(const ddlpb_ctx* ctx, ddlpb_info* info);

/* Message of the last error of ctx ("" if none). */
DDLPB_API const char* ddlpb_last_error(const ddlpb_ctx* ctx);

/* Message of the last failed ddlpb_setup/ddlpb_setup_device of this thread. */
DDLPB_API const char* ddlpb_last_setup_error(void);

/*
 * Energy without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need the
 * energy (an engine whose own allocator owns all device memory, or an MD driver that
 * already holds the solution vector X and hands the library only that).
 *   n        number of atoms, 1 <= n <= 1048576 (the size of the library's static
 *            scratch: 4097 doubles); larger n returns DDLPB_EINVAL
 *   lmax     degree of the expansions of X, 0 <= lmax <= 16
 *   charges  device pointer, n doubles
 *   X        device pointer to the solution [X_r ; X_e] in the layout of
 *            ddlpb_get_vector_device (only the X_r block is read)
 *   e        receives E_s = 1/2 sum_j q_j Y_00 X_r[j, 00] (Hartree); host or device memory
 *   cuda_stream  stream to run on (NULL: legacy default stream); the call synchronises
 *            this stream and returns after the result is in *e, so it cannot be used
 *            inside a stream capture or a host callback
 * The scratch is a fixed device array shared by every call in the process; it keeps
 * the last call's contents, so calls that overlap on the GPU (other threads, other
 * streams) race and must be serialised by the caller.  The first call on each device
 * looks up the array's device address (with that device current) and keeps it for the
 * life of the process (the device's primary context must not be reset in between).
 * Nothing is allocated: no cudaMalloc, no cudaFree.
 * Errors: DDLPB_EINVAL (NULL pointer, n or lmax out of range, device index above 63),
 * DDLPB_ECUDA; the message is in ddlpb_noalloc_last_error().
 */
DDLPB_API ddlpb_status ddlpb_energy_noalloc(int n, int lmax, const double* charges, const double* X, double* e,
                                            void* cuda_stream);

/* Message of the last failed ddlpb_energy_noalloc of this thread ("" if none). */
DDLPB_API const char* ddlpb_noalloc_last_error(void);

/* Free every device allocation of ctx (NULL is allowed). */
DDLPB_API void ddlpb_free(ddlpb_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DDLPB_H */
