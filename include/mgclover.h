/*
 * mgclover.h -- C ABI of a GB300 (sm_103a) multigrid solver for the
 * even-odd preconditioned Wilson-clover Dirac equation
 *
 *     [D(U) + m] psi = eta                 (Osborn et al., Lattice 2010, Eq. 1)
 *
 * solved by flexible GCR on the reduced even-odd system, preconditioned by a
 * recursive adaptive-multigrid K-cycle whose coarse operator is the Galerkin
 * projection R D_p P of the full even-odd preconditioned operator
 * (section "Red-black preconditioning"; section "Implementation").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status: MG_OK (0) or a negative MG_ERR_*.
 *   No C++ exception crosses this boundary.  mg_strerror() names a status.
 * - A context owns all of its internal device memory (gauge and clover
 *   fields, null vectors, prolongators, coarse links, Krylov spaces).  It is
 *   bound to one CUDA device and one stream, is single-stream and is not
 *   thread-safe.  Calls return after the stream has drained (the results are
 *   visible to the caller on any stream).
 * - Caller buffers are plain pointers.  `where` says whether they are host
 *   (MG_HOST) or device (MG_DEVICE) memory; the library never keeps them.
 * - Lattice dims are {Lx, Ly, Lz, Lt}; all four must be even (even-odd
 *   preconditioning) and x is the fastest index.
 * - Fine vectors (spinors): complex128, layout [rhs][t][z][y][x][spin 4][colour 3].
 * - Gauge field: complex128, layout [t][z][y][x][mu 4][a 3][b 3], mu = x,y,z,t;
 *   U_mu(x) is the link from x to x+mu.
 * - Coarse vectors of level l >= 1: complex128, layout
 *   [rhs][t_c][z_c][y_c][x_c][chirality 2][Nv_{l-1}].
 * - Gamma matrices: DeGrand-Rossi chiral basis, gamma_5 = diag(1,1,-1,-1);
 *   chirality of a spin index is spin/2.  Fermion boundary conditions are
 *   periodic in x, y, z and antiperiodic in t; the gauge field is periodic.
 * - The operator (the paper does not write it out; this is the reading used):
 *     D psi(x) = A(x) psi(x)
 *              - 1/2 sum_mu [(1-gamma_mu) U_mu(x) psi(x+mu) + (1+gamma_mu) U_mu(x-mu)^dag psi(x-mu)]
 *     A(x) = (4 + m0) + csw (i/4) sum_{mu != nu} sigma_{mu nu} F_{mu nu}(x),
 *   sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], F = (Q - Q^dag)/8 made traceless,
 *   Q the sum of the four plaquette leaves.  D_ee = A_e, D_oo = A_o.
 * - Working precision is internal: FP64 for the outer GCR, FP32 for the
 *   multigrid preconditioner, FP32/FP16/BF16 storage for prolongators and
 *   coarse links (mg_params.storage; 16-bit values carry one FP32 scale per
 *   (block, chirality) tile of P and per (site, direction) tile of the links;
 *   X, X^{-1} and all vectors stay FP32, accumulation is FP32).  The ABI
 *   always exchanges complex128.
 */
#ifndef MGCLOVER_H
#define MGCLOVER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MG_API __attribute__((visibility("default")))
#else
#define MG_API
#endif

#define MG_MAX_LEVELS 4

enum mg_status {
  MG_OK = 0,
  MG_ERR_ARG = -1,             /* null pointer, bad enum, nrhs < 1, tol <= 0 ...      */
  MG_ERR_DIMS = -2,            /* odd extent, block not dividing a lattice extent,   */
                               /* even-odd requested on a level with an odd extent   */
  MG_ERR_NV = -3,              /* Nv < 1, Nv too large for the block, Nv unsupported */
  MG_ERR_STATE = -4,           /* call order: e.g. solve before gauge/mass/setup      */
  MG_ERR_GS_BREAKDOWN = -5,    /* null vectors locally linearly dependent in a block */
  MG_ERR_SINGULAR_CLOVER = -6, /* a clover block (or coarse X) is numerically singular */
  MG_ERR_NOT_CONVERGED = -7,   /* psi holds the best iterate; info has its residual  */
  MG_ERR_NAN = -8,             /* NaN/Inf in an input or in a Krylov scalar           */
  MG_ERR_CUDA = -9,            /* a CUDA runtime call failed                          */
  MG_ERR_ALLOC = -10           /* device or pinned host allocation failed             */
};

enum mg_where { MG_HOST = 0, MG_DEVICE = 1 };

/* Operators for mg_apply.  `level` selects the lattice (0 = fine). */
enum mg_op {
  MG_OP_D = 0,          /* full D (fine) or D_hat (coarse), whole lattice                 */
  MG_OP_DP = 1,         /* D_p = D diag(M)^{-1} = 1 + H M^{-1}, whole lattice              */
  MG_OP_DR = 2,         /* D_r = 1 - H_eo M_o^{-1} H_oe M_e^{-1}; reads the even sites of  */
                        /* `in`, writes even sites of `out` and zeros its odd sites        */
  MG_OP_BR = 3,         /* b_r = b_e - H_eo M_o^{-1} b_o (odd sites of out set to zero)    */
  MG_OP_M = 4,          /* site-local M (clover A on the fine level, X on coarse levels)    */
  MG_OP_MINV = 5,       /* M^{-1}                                                          */
  MG_OP_HOP = 6,        /* hopping term H alone                                            */
  MG_OP_R = 7,          /* restriction R = P^dag: level l vector -> level l+1 vector       */
  MG_OP_P = 8,          /* prolongation P: level l+1 vector -> level l vector              */
  MG_OP_CYCLE = 9,      /* one multigrid cycle K_l (the preconditioner of D_r on level l): */
                        /* reads the even sites of `in`, writes z_e ~ D_r^{-1} r_e to the  */
                        /* even sites of `out` and zeros its odd sites (FP32 arithmetic)   */
  MG_OP_DR_DAG = 10     /* D_r^dag = gamma_5 M_e^{-1} D_r M_e gamma_5, fine level only (the */
                        /* operator of CGNR); even sites as MG_OP_DR                        */
};

enum mg_prec { MG_FP64 = 0, MG_FP32 = 1 };
enum mg_storage { MG_STORE_FP32 = 0, MG_STORE_FP16 = 1, MG_STORE_BF16 = 2 };
/* Solvers of the reduced system D_r y_e = b_r (section "Results" compares
 * multigrid with the Krylov solvers in use):
 *   MG_MODE_MG           multigrid-preconditioned FGCR (FP64 outer, FP32 cycle)
 *   MG_MODE_EO_GCR       plain FP64 GCR(restart_fine)
 *   MG_MODE_BICGSTAB     FP64 BiCGStab
 *   MG_MODE_CGNR         FP64 CG on D_r^dag D_r y = D_r^dag b_r
 *   MG_MODE_BICGSTAB_MP  mixed precision by iterative refinement: FP64
 *                        residual, FP32 BiCGStab reducing it by 1e-4 per step
 * All stop on the FP64 true residual of the full system (mg_solve). */
enum mg_mode {
  MG_MODE_MG = 0,
  MG_MODE_EO_GCR = 1,
  MG_MODE_BICGSTAB = 2,
  MG_MODE_CGNR = 3,
  MG_MODE_BICGSTAB_MP = 4
};
enum mg_coarse_op { MG_COARSE_DP = 0, MG_COARSE_D = 1 };
/* Output of mg_force. */
enum mg_force_kind {
  MG_FORCE_SU3 = 0,        /* su(3) force sum_a F^a T_a (traceless Hermitian), T_a = lambda_a / 2     */
  MG_FORCE_WIRTINGER = 1,  /* unconstrained gradient dL/dRe U + i dL/dIm U of every complex link entry */
  MG_FORCE_FP32 = 16       /* flag, or-ed with a kind: compute in FP32 (FP32 gauge copy, vectors and  */
                           /* arithmetic; the result is still written as complex128)                  */
};

/* Multigrid parameters (section "Implementation"; section "Setup procedure").
 * Arrays are indexed by the level they map FROM: block[l], nv[l] build P_l
 * from level l to level l+1. */
typedef struct {
  int levels;                     /* total levels including the fine one (1..MG_MAX_LEVELS)      */
  int block[MG_MAX_LEVELS][4];    /* aggregation block {bx,by,bz,bt} of P_l                      */
  int nv[MG_MAX_LEVELS];          /* null vectors of P_l, 1..32 (coarse dof per site = 2*nv[l])  */
  int setup_iters;                /* inverse-iteration passes per null vector (cap)              */
  int setup_inner;                /* GCR iterations on D_p per pass                              */
  double setup_rq_tol;            /* stop a vector when |dRQ| < setup_rq_tol * RQ                */
  int nu_pre, nu_post;            /* minimal-residual smoothing steps on D_r                     */
  double tol_coarse;              /* relative residual target of every coarse GCR (paper: ~0.1) */
  int maxit_coarse;               /* iteration cap of every coarse GCR                           */
  int restart_coarse;             /* GCR restart length on coarse levels                         */
  int restart_fine;               /* GCR restart length of the outer solver                      */
  int maxit_fine;                 /* outer iteration cap                                         */
  int storage;                    /* mg_storage of prolongators and coarse links                 */
  int coarse_op;                  /* mg_coarse_op: Galerkin projection of D_p (paper) or of D    */
  uint64_t seed;                  /* Philox4x32-10 key of the setup's random start vectors       */
  int rhs_block;                  /* mg_solve (MG mode): right-hand sides solved together in      */
                                  /* lock-step, 1..16 (1: one after another)                      */
  int cuda_graphs;                /* 1: replay the 2-level cycle of a single-rhs solve as a        */
                                  /* captured CUDA graph (0: launch its kernels one by one)        */
  int coarse_impl;                /* coarsest-level persistent GCR: 0 chosen by timing on the      */
                                  /* first solve; 1 single-system kernel, 2 batched kernel,        */
                                  /* 3 links streamed through shared memory (even-odd levels),     */
                                  /* 4 tensor cores (even-odd levels, FP16 storage, Nc a multiple  */
                                  /* of 8 up to 64; also the batched cycle's solves); an           */
                                  /* implementation that does not apply falls back to 1            */
  int outer_prec;                 /* MG mode: precision of the outer FGCR's product D_r z inside a */
                                  /* restart cycle -- MG_FP32 (the FP32 D_r of the FP32 cycle      */
                                  /* output, widened to FP64 for the FP64 orthogonalisation and    */
                                  /* update) or MG_FP64; the true residual at every restart and    */
                                  /* the final check are FP64 either way                           */
  int level_timing;               /* 1: time every level's work with CUDA events into              */
                                  /* mg_solve_info.level_ms (the cycle graph is not used then;     */
                                  /* events add a few microseconds per coarse solve); 0: off       */
} mg_params;

typedef struct {
  double setup_ms;                          /* wall time of mg_setup                          */
  int vectors[MG_MAX_LEVELS];               /* null vectors built per transfer                */
  int passes[MG_MAX_LEVELS];                /* inverse-iteration passes summed over vectors   */
  double rq_last[MG_MAX_LEVELS];            /* Rayleigh quotient of the last vector found     */
  int coarse_sites[MG_MAX_LEVELS];          /* sites of the coarse lattice of each transfer   */
} mg_setup_info;

typedef struct {
  int outer_iterations;                     /* outer GCR iterations (summed over rhs)         */
  int restarts;                             /* outer restarts (true-residual recomputations)  */
  long long coarse_iterations[MG_MAX_LEVELS]; /* GCR iterations run on each coarse level    */
  double true_residual;                     /* max over rhs of ||eta - D psi|| / ||eta||      */
  double solve_ms;                          /* wall time of the call                          */
  long long dslash_launches;                /* fine hopping-term launches in the call         */
  long long kernel_launches;                /* all library kernel launches in the call        */
  double level_ms[MG_MAX_LEVELS];           /* with mg_params.level_timing: GPU ms inside the */
                                            /* level-0 cycles (the whole preconditioner) and  */
                                            /* inside the level-l coarse solves (l >= 1, each */
                                            /* including the levels below it); else 0         */
} mg_solve_info;

/* Kernels for mg_benchmark_kernel. */
enum mg_kernel {
  MG_KERNEL_DSLASH_CLOVER = 0,  /* fused hop + clover-inverse epilogue (t_o = A_o^{-1} H_oe s_e) */
  MG_KERNEL_DSLASH_XPAY = 1,    /* fused hop + axpy epilogue (y_e - H_eo t_o)                    */
  MG_KERNEL_DR = 2,             /* a whole D_r application (clover apply + the two kernels above) */
  MG_KERNEL_COARSE_DR = 3,      /* a whole coarse D_hat_r application on level 1 (needs setup)   */
  MG_KERNEL_RESTRICT = 4,       /* R = P^dag from the fine even sites to level 1 (needs setup)   */
  MG_KERNEL_PROLONG = 5         /* P from level 1 onto the fine even sites (needs setup)         */
};

/* Name of a status code (static string). */
MG_API const char* mg_strerror(int status);

/* Detail of the last failed call on this thread (empty after a success).
 * Valid until the next call on the same thread. */
MG_API const char* mg_last_error(void);

/* Fill `p` with the defaults: 2 levels, 4^4 blocks, Nv = 24, 20 passes of 8
 * GCR iterations, RQ tolerance 0.05, nu_post = 4, coarse tolerance 0.1,
 * coarse restart 32 / cap 50, outer restart 16 / cap 500, FP32 storage,
 * Galerkin projection of D_p, seed 3, rhs_block 16, cuda_graphs 1, coarse_impl 0,
 * outer_prec MG_FP32, level_timing 0.  Errors: MG_ERR_ARG (p NULL). */
MG_API int mg_default_params(mg_params* p);

/* Create a context for a lattice of `dims` on CUDA device `device`; kernels
 * run on `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 * Errors: MG_ERR_ARG, MG_ERR_DIMS (an extent is odd or < 2), MG_ERR_CUDA. */
MG_API int mg_create(void** ctx_out, const int dims[4], int device, void* cuda_stream);

/* Release the context and all device memory it owns.  NULL is a no-op.
 * Errors: MG_ERR_CUDA (a failed release; the context is gone either way). */
MG_API int mg_destroy(void* ctx);

/* Copy in the gauge field (layout above; host or device memory as `where`
 * says, read once, not kept).  Invalidates the clover field and any multigrid
 * setup.  Errors: MG_ERR_ARG (NULL context or field, bad `where`),
 * MG_ERR_CUDA. */
MG_API int mg_load_gauge(void* ctx, const void* U, int where);

/* Set the clover coefficient csw and the bare mass m0 and build A and A^{-1}
 * in FP64 (plus the FP32 copies the preconditioner uses) from the loaded
 * gauge field.  Invalidates the multigrid setup.  Errors: MG_ERR_STATE (no
 * gauge), MG_ERR_SINGULAR_CLOVER (a 6x6 chiral block has a pivot below
 * 1e-12 of its largest entry). */
MG_API int mg_set_clover(void* ctx, double csw, double m0);

/* The anisotropic Wilson-clover operator (section "Results": the lattices
 * are anisotropic clover lattices; the paper gives no formula, so this is a
 * stated reading).  Every hop in direction mu is scaled by the weight w[mu]
 * (x, y, z, t), the diagonal mass term becomes w[0]+w[1]+w[2]+w[3] + m0 in
 * place of 4 + m0, and the clover coefficient is csw_t on the three planes
 * that contain t and csw_s on the three spatial planes.  At w = (1,1,1,1)
 * and csw_t = csw_s the operator is the isotropic one of mg_set_clover, bit
 * for bit (mg_set_clover calls this).  The solver, the setup, the
 * multigrid hierarchy (built by Galerkin projection of this operator) and
 * mg_force (the weighted hops and per-plane coefficients differentiated)
 * all use the result.  `w` is host memory, four doubles, copied.  Errors:
 * MG_ERR_ARG (w NULL, a weight not finite or not > 0, csw or m0 not
 * finite), MG_ERR_STATE (no gauge), MG_ERR_SINGULAR_CLOVER. */
MG_API int mg_set_clover_aniso(void* ctx, const double w[4], double csw_s, double csw_t, double m0);

/* Set multigrid parameters (copied).  Invalidates the setup (and any
 * injected null vectors) when a field the setup depends on changes: levels,
 * block, nv, setup_iters, setup_inner, setup_rq_tol, restart_coarse, storage,
 * coarse_op or seed; the other fields take effect at the next solve.  Errors:
 * MG_ERR_ARG, MG_ERR_DIMS (a block does not divide its lattice, or a level
 * below the coarsest has an odd extent), MG_ERR_NV. */
MG_API int mg_set_params(void* ctx, const mg_params* p);

/* Copy out the context's current parameters (the defaults until
 * mg_set_params or mg_load_setup set them).  Errors: MG_ERR_ARG. */
MG_API int mg_get_params(void* ctx, mg_params* p);

/* Run the setup ("Setup procedure"): for every transfer l, find nv[l]
 * near-null vectors of level l's D_p by inverse iteration (unless injected by
 * mg_set_null_vectors), split them by chirality, block-orthonormalise them
 * into P_l, and build the Galerkin coarse links and their site inverses.
 * `info` may be NULL.  Errors: MG_ERR_STATE, MG_ERR_GS_BREAKDOWN,
 * MG_ERR_SINGULAR_CLOVER (a coarse X block), MG_ERR_CUDA. */
MG_API int mg_setup(void* ctx, mg_setup_info* info);

/* Inject (set) or read (get) the nv raw null vectors of transfer `level`:
 * complex128 [k][level-l lattice vector layout].  Injected vectors replace
 * the inverse iteration of that level at the next mg_setup (used by tests
 * and to reuse a setup).  get returns the vectors of the last setup.  `V`
 * is host or device memory as `where` says, copied.  Errors: MG_ERR_ARG (V
 * NULL, bad `where`, `level` not a transfer: 0 <= level < levels - 1),
 * MG_ERR_NV (nv is not nv[level] of the parameters), MG_ERR_STATE (get: no
 * setup yet), MG_ERR_CUDA. */
MG_API int mg_set_null_vectors(void* ctx, int level, const void* V, int nv, int where);
MG_API int mg_get_null_vectors(void* ctx, int level, void* V, int nv, int where);

/* Setup reuse.  The paper keeps the null vectors and coarse operators of a
 * setup for later use; here the raw null vectors of every transfer are the
 * saved state, and P and the coarse operators are rebuilt from them (block
 * Gram-Schmidt and Galerkin links: no inverse iteration) for the current
 * gauge field, clover and mass.
 *   mg_save_setup:  writes the multigrid parameters, csw, m0 and the null
 *                   vectors (complex128) of the current setup to `path`.
 *   mg_load_setup:  reads such a file for a context with the same lattice
 *                   (gauge field and clover already set), applies its
 *                   parameters and rebuilds the hierarchy; `info` (may be
 *                   NULL) as mg_setup, setup_ms being the whole call.
 *   mg_update_mass: sets a new bare mass (same csw) and rebuilds the
 *                   hierarchy from the current null vectors -- setup reuse
 *                   across masses.
 * Errors: MG_ERR_ARG (unreadable or foreign file), MG_ERR_DIMS (another
 * lattice), MG_ERR_STATE (no setup / no clover), MG_ERR_GS_BREAKDOWN,
 * MG_ERR_SINGULAR_CLOVER, MG_ERR_CUDA. */
MG_API int mg_save_setup(void* ctx, const char* path);
MG_API int mg_load_setup(void* ctx, const char* path, mg_setup_info* info);
MG_API int mg_update_mass(void* ctx, double m0, mg_setup_info* info);

/* Adaptive refinement of a setup -- the adaptive idea the paper plans for the
 * clover case (section "Setup procedure"), with the current multigrid solver
 * as the approximate inverse: `passes` times, and for each of the `transfers`
 * finest transfers (0: all), from the finest down, take each of its null
 * vectors through `relax` steps of inverse subspace iteration on its level,
 * v_k <- M v_k (M ~ D_p^{-1}: the even-odd reduction of the level and one of
 * its cycles), Gram-Schmidt against v_0 .. v_{k-1} and normalised; then
 * rebuild P and the coarse operators, the transfers below that level being
 * set up afresh (inverse iteration, as mg_setup) on the refined coarse
 * operator.  `info` (may be NULL) as mg_setup, setup_ms being the whole call.
 * Errors: MG_ERR_ARG (passes or relax < 1, transfers < 0), MG_ERR_STATE,
 * MG_ERR_DIMS (a relaxed coarse level with an odd extent),
 * MG_ERR_GS_BREAKDOWN (a vector lost in the iteration or in a block),
 * MG_ERR_CUDA. */
MG_API int mg_adapt_setup(void* ctx, int passes, int relax, int transfers, mg_setup_info* info);

/* Read the coarse operator of level `level` (1 .. levels-1) after mg_setup,
 * as the solver applies it: the Galerkin links of section "Implementation"
 * (D_hat v(x) = X(x) v(x) + sum_d Y_d(x) v(x + d), d < 4: from x + mu,
 * d >= 4: from x - mu), dequantised from their storage format (FP16/BF16
 * values times their per-tile scale) to complex128.  Layouts (nc = 2 Nv of
 * the transfer into the level, sites lexicographic as in coarse vectors):
 * Y [t_c][z_c][y_c][x_c][d 8][row nc][col nc], X [t_c][z_c][y_c][x_c][row nc][col nc].
 * Buffers are owned by the caller.  Errors: MG_ERR_ARG, MG_ERR_STATE,
 * MG_ERR_CUDA. */
MG_API int mg_get_coarse_links(void* ctx, int level, void* Y, void* X, int where);

/* Solve D psi = eta for nrhs right-hand sides (layout above) to
 * ||eta - D psi|| / ||eta|| <= tol, in MG_MODE_MG (multigrid-preconditioned
 * FGCR; needs mg_setup) or one of the unpreconditioned modes of enum mg_mode
 * (maxit_fine caps the iterations of every mode; an iteration applies D_r
 * once in GCR, twice in BiCGStab, D_r and D_r^dag in CGNR, and is one inner
 * FP32 BiCGStab iteration in the mixed-precision mode, whose refinement steps
 * are counted in info->restarts).  In
 * MG mode groups of up to mg_params.rhs_block right-hand sides are solved
 * together: one FGCR per right-hand side, run in lock-step so that every
 * iteration applies D_r to all of them in one multi-RHS launch and the
 * multigrid cycle to all of them at once (all coarsest-level solves in one
 * persistent launch); each right-hand side keeps its own Krylov space and
 * convergence test, so the results match separate solves to the tolerance.
 * info->outer_iterations sums the iterations of every right-hand side.  `info`
 * may be NULL.  Errors: MG_ERR_STATE, MG_ERR_ARG, MG_ERR_NAN,
 * MG_ERR_NOT_CONVERGED (psi holds the best iterate), MG_ERR_CUDA. */
MG_API int mg_solve(void* ctx, void* psi, const void* eta, int nrhs, double tol, int mode, int where,
             mg_solve_info* info);

/* Solve several lattices together: context i (its own lattice, gauge field,
 * clover and multigrid setup; all contexts on one device) solves
 * D_i psi[i] = eta[i] for nrhs[i] right-hand sides (fine-vector layout of its
 * lattice) to tolerance tol, by multigrid-preconditioned FGCR, one per
 * right-hand side, run in lock-step: each iteration applies the fine
 * operators of every context to all of its right-hand sides in multi-RHS
 * launches, and puts the coarsest-level solves of all right-hand sides of all
 * 2-level contexts into shared persistent launches (up to 16 systems and 8
 * lattices each; contexts whose hierarchy is deeper, or whose coarse storage,
 * restart or cap differ from the first's, solve their own).  Right-hand sides
 * are taken in context order in groups of at most the first context's
 * rhs_block (a context's right-hand sides are not split when they fit in a
 * fresh group).
 * The contexts need the same restart_fine.  `where` applies to every buffer;
 * infos (may be NULL) receives one mg_solve_info per context, solve_ms and
 * kernel_launches being those of the whole call.  An extension of the paper's
 * repeated solves "for varying sources and gauge fields".  Errors: MG_ERR_ARG
 * (a context twice, different devices, ...), MG_ERR_STATE, MG_ERR_NAN,
 * MG_ERR_NOT_CONVERGED, MG_ERR_CUDA. */
MG_API int mg_solve_batch(void* const* ctxs, int nctx, void* const* psi, const void* const* eta, const int* nrhs,
                          double tol, int where, mg_solve_info* infos);

/* Solve the adjoint system D^dag psi = eta with the same solver and
 * multigrid, through gamma_5-hermiticity D^dag = gamma_5 D gamma_5:
 * psi = gamma_5 D^{-1} (gamma_5 eta).  This is the backward solve of a
 * differentiated solve (the paper has no gradient; it solves D only).
 * Arguments, layouts, tolerance (on ||eta - D^dag psi|| / ||eta||, equal to
 * the residual of the gamma_5-rotated system) and errors as mg_solve; eta is
 * not modified. */
MG_API int mg_solve_dagger(void* ctx, void* psi, const void* eta, int nrhs, double tol, int mode, int where,
                           mg_solve_info* info);

/* Gauge-link derivative of f(U) = -Re <lambda, D(U) psi> for fixed fine
 * vectors lambda and psi (complex128, fine-vector layout, one right-hand
 * side each; `where` says host or device for all three buffers).  With
 * psi = D^{-1} eta and lambda = D^{-dag} chi (mg_solve_dagger) it is the
 * derivative of L = Re <chi, D^{-1} eta> with respect to the gauge field --
 * an extension: the paper does not differentiate the solve.  Both the hopping
 * term and the clover term (through its plaquette leaves, with the csw of the
 * last mg_set_clover, or the hopping weights and per-plane coefficients of
 * the last mg_set_clover_aniso) are differentiated, in FP64 -- or in FP32 when `kind`
 * carries the MG_FORCE_FP32 flag (FP32 gauge copy, vectors and arithmetic).
 *   MG_FORCE_SU3:       F_mu(x) = sum_a F^a T_a with F^a = df/d omega^a for
 *                       U_mu(x) -> exp(i omega^a T_a) U_mu(x), T_a = lambda_a/2;
 *   MG_FORCE_WIRTINGER: g_mu(x) with df = Re sum tr(g^dag dU) for any complex
 *                       dU (the gradient convention of torch for complex
 *                       tensors).
 * `F` has the gauge-field layout [t][z][y][x][mu][3][3] complex128 and is
 * owned by the caller.  Errors: MG_ERR_ARG, MG_ERR_STATE (no clover),
 * MG_ERR_CUDA. */
MG_API int mg_force(void* ctx, void* F, const void* lambda, const void* psi, int kind, int where);

/* Apply operator `op` (enum mg_op) of level `level` to nrhs vectors of that
 * level (for MG_OP_R the output is a level+1 vector, for MG_OP_P the input
 * is).  `prec` selects FP64 or FP32 arithmetic on the fine level; coarse
 * levels compute in FP32 from their storage format.  Coarse levels and R/P
 * need mg_setup.  Errors: MG_ERR_ARG, MG_ERR_STATE, MG_ERR_DIMS (MG_OP_DR or
 * MG_OP_BR on a level with an odd extent), MG_ERR_CUDA. */
MG_API int mg_apply(void* ctx, int op, int level, void* out, const void* in, int nrhs, int prec, int where);

/* Allocation-free variant of mg_apply for the fine level.  The paper has no
 * counterpart: it exists for callers that cannot call cudaMalloc -- code whose
 * device memory is owned by another allocator (a framework's caching
 * allocator or a fixed pool) and latency-critical loops that cannot afford
 * the implicit device synchronisation of cudaMalloc/cudaFree.  mg_apply
 * allocates staging buffers and temporaries on every call; this entry point
 * allocates nothing.
 *
 * Applies op (MG_OP_D, MG_OP_DP, MG_OP_DR, MG_OP_BR, MG_OP_M, MG_OP_MINV or
 * MG_OP_HOP) of the fine level to ONE vector: `in` and `out` are DEVICE
 * pointers to complex128 fine vectors in the layout above (owned by the
 * caller, not kept); `prec` is MG_FP64 or MG_FP32.  Results equal mg_apply's.
 *
 * Its scratch is one file-scope device array of 9 MiB (16384 sites x 576
 * bytes), which every GPU that loads the library holds until the process
 * exits.  Lattices above 16384 sites are rejected with MG_ERR_DIMS.  The
 * first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents (the parts that must start at zero are cleared by each
 * call), so calls that overlap on the GPU -- other streams, other threads,
 * other contexts on the same device -- race: serialise them.  Runs on the
 * context's stream and returns after it has drained.  Errors: MG_ERR_ARG,
 * MG_ERR_STATE (no clover), MG_ERR_DIMS (too large), MG_ERR_CUDA. */
MG_API int mg_apply_noalloc(void* ctx, int op, void* out, const void* in, int prec);

/* Time one hot kernel in isolation on the context's resident fields (needs
 * gauge and clover; MG_KERNEL_COARSE_DR needs setup): `warmup` untimed
 * launches, then `iters` back-to-back launches bracketed by CUDA events on
 * the context stream.  Returns the average milliseconds per launch and the
 * algorithmic bytes one launch must move (every input field read once and
 * the output written once, as counted for the roofline):
 *   DSLASH_CLOVER: Vh * (8 links * 18 + 24 spinor + 72 clover + 24 out) reals,
 *   DSLASH_XPAY:   Vh * (8 * 18 + 24 + 24 x + 24 out) reals,
 *   DR:            the sum of its three kernels,
 *   COARSE_DR:     Vc/2 * (18 Nc^2 link/inverse entries + 7 Nc vector entries) complex,
 *   RESTRICT, PROLONG: the P rows of the even fine sites (Vh * 12 * Nv entries
 *                  of the storage format: 8 bytes FP32, 4 bytes FP16/BF16) + the
 *                  even half of the fine vector (24 Vh floats) + the coarse
 *                  vector (Vc * 2 Nv complex FP32).
 * The transfers always run in FP32 (`prec` is ignored for them); the other
 * `prec` selects FP64 or FP32 for the fine kernels.  Errors: MG_ERR_ARG,
 * MG_ERR_STATE, MG_ERR_CUDA. */
MG_API int mg_benchmark_kernel(void* ctx, int kernel, int prec, int warmup, int iters, double* avg_ms,
                               double* bytes_per_launch);

/* mg_benchmark_kernel for nrhs right-hand sides per launch (fine kernels:
 * the multi-RHS forms with their autotuned CTA size; nrhs = 1 is
 * mg_benchmark_kernel).  Algorithmic bytes count links and clover once per
 * site and spinors once per (site, rhs):
 *   DSLASH_CLOVER: Vh * (144 + 72 + 48 nrhs) reals,
 *   DSLASH_XPAY:   Vh * (144 + 72 nrhs) reals,
 *   DR:            Vh * (432 + 168 nrhs) reals,
 *   RESTRICT, PROLONG: the P rows once + nrhs times both vectors.
 * Errors as mg_benchmark_kernel; MG_KERNEL_COARSE_DR takes nrhs = 1 only. */
MG_API int mg_benchmark_kernel_nrhs(void* ctx, int kernel, int prec, int nrhs, int warmup, int iters, double* avg_ms,
                                    double* bytes_per_launch);

/* Measures the CUDA-core FMA throughput of `device` in precision `prec`
 * (MG_FP64 or MG_FP32) with CUDA events: 8 independent FMA chains per thread,
 * 8 blocks of 256 threads per SM, 2 flops per FMA.  The roofline
 * denominator of the kernels bound by FP64 (or FP32) arithmetic rather than
 * by memory; not part of the paper's method.  *tflops receives TFLOP/s.
 * Errors: MG_ERR_ARG, MG_ERR_CUDA. */
MG_API int mg_benchmark_fma(int device, int prec, double* tflops);

/* Times `iters` solves of the coarsest level's system (after `warmup`
 * untimed ones) for a fixed Philox right-hand side: the persistent
 * coarsest-level GCR with its even-odd reconstruction, as the multigrid cycle
 * runs it (section "Implementation": unpreconditioned GCR on the coarsest
 * lattice to the relative tolerance tol_coarse), with the implementation
 * mg_params.coarse_impl selects or the autotuner picked.  CUDA events on the
 * context's stream.  Outputs: *avg_ms per solve, *iterations_per_solve (GCR
 * iterations), *bytes_per_solve = the coarse links one application of the
 * reduced operator reads (half x 8 Nc^2 complex, folded links in FP32 and
 * Y in the storage format) times the applications per solve (iterations +
 * 1.5 for b_r and the closing true residual; odd-extent coarsest levels:
 * the 9 Nc^2 complex FP32 links per site, iterations + 1).  Needs mg_setup.
 * Errors: MG_ERR_ARG, MG_ERR_STATE, MG_ERR_CUDA (also when a bounded wait
 * inside the persistent kernel ran out of time). */
MG_API int mg_benchmark_coarse_solve(void* ctx, int warmup, int iters, double* avg_ms, double* bytes_per_solve,
                                     double* iterations_per_solve);

/* Floors of one coarsest-level GCR iteration (section "Implementation":
 * unpreconditioned GCR on the coarsest lattice; needs setup and an even-odd
 * coarsest level), on the grid of the streamed solver (coarse_impl 3), timed
 * with CUDA events on the context stream: *barrier_us = one time-bounded grid
 * barrier of a cooperative kernel that does nothing else (3000 in a row; a
 * GCR iteration passes three), *stream_us = moving the links one iteration
 * reads -- the folded odd-site links A (FP32) and the even-site Y (storage
 * format), *stream_bytes in total -- from L2 to shared memory by per-warp
 * double-buffered bulk copies without arithmetic (20 repetitions), *grid =
 * the CTAs used.  Errors: MG_ERR_ARG, MG_ERR_STATE (no setup, or no even-odd
 * coarsest level), MG_ERR_CUDA (also when a bounded wait ran out of time). */
MG_API int mg_benchmark_coarse_floor(void* ctx, double* barrier_us, double* stream_us, double* stream_bytes,
                                     int* grid);

/* Lattice size of level `level` after setup (dims_out[4] = {Lx,Ly,Lz,Lt})
 * and its dof per site (12 on the fine level, 2*nv[level-1] on coarse ones).
 * Computed from the parameters, so it also answers before mg_setup.
 * Errors: MG_ERR_ARG (NULL outputs, level outside 0 .. levels - 1). */
MG_API int mg_level_info(void* ctx, int level, int dims_out[4], int* ndof_out);

#ifdef __cplusplus
}
#endif
#endif /* MGCLOVER_H */
