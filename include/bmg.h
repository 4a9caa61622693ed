/*
 * bmg.h -- C ABI of the GB300 structured black-box multigrid solver.
 *
 * The library solves the discrete diffusion problem that the paper obtains
 * by pulling -div(kappa grad u) = f back through a map onto the structured
 * computational grid (Sec. 2, eq. "weak_computational"; Sec. 2.1, effective
 * coefficient D_c = J_T (D o T^-1) J_T^T |J_T^-1|), with the structured
 * multigrid of Sec. 2.2: factor-two coarsening, operator-induced
 * interpolation, Galerkin coarse operators and a V-cycle, here wrapped in
 * preconditioned conjugate gradients.  The setup/solve split follows the
 * paper's "Setup phase" (assemble A_c or take it as given, set up the
 * multigrid) and "Solution phase".
 *
 * Grids: n = 2^k + 1 nodes per side (k >= 1) on [0,1]^d, d = 2 or 3.
 * Node (i,j[,k]) has index i + n*(j + n*k) (i fastest); cell (ci,cj[,ck])
 * (lower corner) has index ci + (n-1)*(cj + (n-1)*ck).  All nodes on the
 * boundary carry zero Dirichlet data: they are not unknowns, their entries
 * are ignored on input and written as 0 on output.  DoF = (n-2)^d.
 *
 * Memory and streams.  The library allocates no device memory: the caller
 * queries bmg_workspace_bytes, allocates one device buffer (e.g. a torch
 * tensor) and attaches it with bmg_attach together with a CUDA stream; all
 * work is ordered on that stream.  Array arguments are caller-owned and
 * must stay alive for the call.  Unless a call says otherwise, array
 * arguments are device pointers on the context's device; bmg_solve and
 * bmg_vcycle also accept host pointers (pageable or pinned), which they
 * stage through the workspace (the copies are part of the call).
 *
 * Errors.  Every call returns a bmg_status and never aborts or traps.
 * Device-side checks (folded map, setup breakdown, CG breakdown) set a
 * device error word that the call reads back before returning.  After an
 * error the context stays valid; the data it holds may not be.
 */
#ifndef BMG_H
#define BMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bmg_ctx bmg_ctx;   /* opaque; created and destroyed by the library */

typedef enum {
    BMG_OK = 0,
    BMG_ERR_ARG = 1,               /* invalid argument (null pointer, bad option) */
    BMG_ERR_SHAPE = 2,             /* n is not 2^k+1 or dim not in {2,3} */
    BMG_ERR_DEVICE = 3,            /* a CUDA runtime call failed */
    BMG_ERR_WORKSPACE = 4,         /* no workspace attached or too small */
    BMG_ERR_MAP_FOLDED = 5,        /* det J <= 0 at a quadrature point */
    BMG_ERR_SETUP_BREAKDOWN = 6,   /* zero collapsed denominator / non-positive diagonal */
    BMG_ERR_NOT_SPD = 7,           /* CG breakdown: p^T A p <= 0 */
    BMG_ERR_NOT_CONVERGED = 8,     /* maxit reached before tol */
    BMG_ERR_TIMEOUT = 9,           /* a bounded device wait expired */
    BMG_ERR_STATE = 10             /* call out of order (e.g. solve before setup) */
} bmg_status;

enum {
    BMG_PREC_FP64 = 0,             /* V-cycle in FP64 */
    BMG_PREC_FP32 = 1              /* V-cycle in FP32; outer CG, residuals, dots
                                      and the coarsest solve stay FP64 */
};

enum {
    BMG_OUTER_CG = 0,              /* beta = r_{k+1}.z_{k+1} / r_k.z_k */
    BMG_OUTER_FLEXIBLE_CG = 1,     /* beta = r_{k+1}.(z_{k+1}-z_k) / r_k.z_k */
    BMG_OUTER_REFINEMENT = 2       /* iterative refinement (needs BMG_PREC_FP32):
                                      FP64 residual r = b - A x, an inner FP32
                                      flexible CG on A d = r preconditioned by the
                                      FP32 V-cycle, x += d in FP64; repeated until
                                      the FP64 residual meets tol */
};

enum {
    BMG_FLAG_UNFUSED = 1,          /* V-cycle from separate per-colour, residual,
                                      restriction and prolongation kernels instead
                                      of the streaming fused kernels (2-D) or the
                                      half-sweep smoother kernels, one launch per
                                      colour parity of k (3-D) */
    BMG_FLAG_NO_GRAPHS = 2         /* launch every kernel of an iteration directly
                                      instead of replaying a CUDA graph of the
                                      iteration (graphs are also bypassed while
                                      profiling is on) */
};

typedef struct {
    int dim;          /* 2 or 3 */
    int n;            /* nodes per side, 2^k + 1, k >= 1 */
    int precision;    /* BMG_PREC_FP64 or BMG_PREC_FP32 */
    int outer;        /* BMG_OUTER_CG, BMG_OUTER_FLEXIBLE_CG or BMG_OUTER_REFINEMENT */
    int flags;        /* BMG_FLAG_* bits, 0 by default */
    int max_rhs;      /* 1 (default) to 4: on a 2-D context with BMG_PREC_FP32,
                         BMG_OUTER_REFINEMENT, the streaming kernels and n >= 65,
                         values above 1 reserve workspace for solving up to 4
                         right-hand sides together (bmg_solve with nrhs > 1:
                         one stencil read per sweep for all of them); other
                         contexts ignore it */
} bmg_opts;

typedef struct {
    int iterations;               /* PCG iterations done (inner ones for refinement) */
    int levels;                   /* multigrid levels (finest .. 3 nodes per side) */
    double relres;                /* recursive ||r_k|| / ||b|| at exit */
    double true_relres;           /* ||b - A x|| / ||b|| at exit, FP64 */
    double rho;                   /* (||r_k|| / ||r_0||)^(1/k) */
    double grid_complexity;       /* sum_l N_l / N_0 (Sec. 4) */
    double operator_complexity;   /* sum_l stored_l / stored_0 (symmetric storage) */
    int status;                   /* bmg_status of the solve */
    int refinements;              /* FP64 residual evaluations after the first
                                     (BMG_OUTER_REFINEMENT), else 0 */
} bmg_info;

/* Defaults: dim 2, precision FP64, outer CG (flexible CG when FP32). */
void bmg_default_opts(bmg_opts* opts);

/* Creates a context (host memory only).  Fails with BMG_ERR_SHAPE for
   invalid n/dim.  *ctx is NULL on failure. */
bmg_status bmg_create(const bmg_opts* opts, bmg_ctx** ctx);

/* Bytes of device workspace the context needs (256-byte aligned start). */
bmg_status bmg_workspace_bytes(const bmg_ctx* ctx, size_t* bytes);

/* Attaches a caller-owned device workspace of at least bmg_workspace_bytes
   and the cudaStream_t (as void*; NULL = legacy default stream) all later
   calls are ordered on.  The device current at this call becomes the
   context's device.  The workspace must outlive the context's use. */
bmg_status bmg_attach(bmg_ctx* ctx, void* workspace, size_t bytes, void* stream);

/* Assembles the finest-grid operator A_c (Sec. 2.1, "Setup phase" step 2):
   Q1 elements, 2^d-point Gauss rule per cell, isoparametric map from the
   nodal coordinates, per-cell coefficient kappa, effective coefficient
   kappa det J J^-1 J^-T at each Gauss point; couplings to boundary nodes
   dropped.  coords: device, d planes of n^d doubles (x plane, y plane[,
   z plane]); kappa: device, (n-1)^d doubles.  Errors: BMG_ERR_MAP_FOLDED. */
bmg_status bmg_assemble(bmg_ctx* ctx, const double* coords, const double* kappa);

/* As bmg_assemble with an SPD diffusion tensor per cell instead of a scalar
   (the general coefficient of Sec. 2, Eq. pde): the effective coefficient
   at each Gauss point is det J J^-1 D J^-T (Sec. 2.1).  D: device, the
   upper triangle of each cell's tensor as planes of (n-1)^d doubles,
   D11, D12, D22 in 2-D and D11, D12, D13, D22, D23, D33 in 3-D (cells in
   the order of kappa).  Errors: BMG_ERR_MAP_FOLDED.  An indefinite D is not
   detected here; it shows up in bmg_setup or bmg_solve.  bmg_adjoint_grad
   (a gradient with respect to a scalar kappa) returns BMG_ERR_STATE on such
   a context. */
bmg_status bmg_assemble_tensor(bmg_ctx* ctx, const double* coords, const double* D);

/* Non-zero Dirichlet data (the lift term of Sec. 2, Eq. weak_computational):
   out_i = -sum over boundary nodes j of A_ij g_j for every interior node i,
   the couplings that bmg_assemble drops, from the same map and scalar
   coefficient; out is zero on the boundary.  The solution with boundary
   values g and right-hand side f is then x = A^-1 (f + out) in the interior
   (bmg_solve) and g on the boundary.  coords, kappa: as bmg_assemble; g,
   out: device, n^d doubles, i fastest (interior values of g are ignored).
   Does not change the context's operator.  Errors: BMG_ERR_MAP_FOLDED. */
bmg_status bmg_boundary_rhs(bmg_ctx* ctx, const double* coords, const double* kappa, const double* g,
                            double* out);

/* Sets the finest operator directly, the alternative Sec. 2.2 allows to
   assembling it from the coefficient.  stencil: device, n^d rows of 3^d
   doubles, entry (dx+1)+3(dy+1)[+9(dz+1)] = A[node, node+offset]; the
   operator must be symmetric with zero couplings to boundary nodes (only
   the lower half of each row is read). */
bmg_status bmg_set_stencil(bmg_ctx* ctx, const double* stencil);

/* Builds the multigrid hierarchy ("Setup phase" step 3): operator-induced
   interpolation from each level's stencil, Galerkin coarse operators
   P^T A P, FP32 copies when precision is FP32.  Errors:
   BMG_ERR_SETUP_BREAKDOWN, BMG_ERR_STATE (no operator yet). */
bmg_status bmg_setup(bmg_ctx* ctx);

/* One V(1,1)-cycle from a zero initial guess: z = M r ("Solution phase"
   step 3).  r, z: n^d doubles, host or device.  Boundary entries of r are
   ignored; z is 0 on the boundary. */
bmg_status bmg_vcycle(bmg_ctx* ctx, const double* r, double* z);

/* Preconditioned CG, M = one V-cycle, until ||r_k|| <= tol ||b|| for the
   recursive and then the true residual (when only the recursive one
   passes, r is replaced by the true residual and CG continues), or maxit
   iterations.  tol <= 0 runs exactly maxit iterations.  nrhs >= 1
   right-hand sides with the same operator (the solution phase of Sec. 2.2
   applied to each): b, x: nrhs consecutive vectors of n^d doubles, host or
   device; x holds the initial guesses on entry and the iterates on exit
   (also on BMG_ERR_NOT_CONVERGED).  info: NULL or nrhs entries.  With
   nrhs > 1 on a context created with max_rhs >= 2 (and eligible, see
   bmg_opts), groups of up to max_rhs right-hand sides are solved together
   (the lockstep refinement of bmg_batch_solve, tol > 0 required); otherwise
   the right-hand sides are solved one after the other.  Returns the first
   non-OK status. */
bmg_status bmg_solve(bmg_ctx* ctx, int nrhs, const double* b, double* x, double tol, int maxit,
                     bmg_info* info);

/* Solves count independent problems, nrhs right-hand sides each, to a
   relative FP64 residual of tol (> 0), running them concurrently: every
   context must have been set up with BMG_OUTER_REFINEMENT and should be
   attached to a stream of its own (contexts sharing a stream serialise).
   A host-side scheduler keeps every problem's refinement loop in flight
   (iteration graphs, asynchronous residual checks, event polling) instead
   of waiting on one problem at a time.  b[p*nrhs + r], x[p*nrhs + r]:
   problem p's r-th right-hand side / initial guess and solution, n_p^d
   doubles on the host or the device.  infos: count*nrhs entries or NULL.
   The right-hand sides of one problem are solved one after the other with
   its hierarchy.  Returns the first non-OK status of any solve. */
bmg_status bmg_solve_many(bmg_ctx* const* ctxs, int count, int nrhs, const double* const* b, double* const* x,
                          double tol, int maxit, bmg_info* infos);

/* ---------------------------------------------------------------------
   Batched solve: many independent problems, up to 4 right-hand sides each,
   with one stencil read per sweep for all right-hand sides of a problem
   (the problem-and-right-hand-side batching of the solution phase of
   Sec. 2.2, step 3, applied to every problem of a set).

   Every context must be a 2-D context with precision BMG_PREC_FP32, outer
   BMG_OUTER_REFINEMENT, the streaming kernels (no BMG_FLAG_UNFUSED), n >= 65,
   attached on one device and set up (bmg_setup); the batch keeps pointers
   into their hierarchies, so they must outlive it and must not be set up
   again.  Each solve runs, for all problems and right-hand sides together
   (lockstep), the refinement mode of bmg_solve: FP64 residual, inner FP32
   flexible CG preconditioned by one FP32 V(1,1)-cycle per right-hand side,
   updates into the FP64 iterate, until every system's FP64 residual meets
   tol.  The V-cycle runs per size class: the levels of all problems with
   the same n are stored together (copied from the contexts at attach) and
   processed by one persistent launch that walks the class's work-list of
   (problem, level, tile) items; the levels n <= 33 of every problem run in
   one launch, one CTA per problem.  One inner iteration of the whole batch
   is one CUDA graph (unless flags has BMG_FLAG_NO_GRAPHS).  Between two
   FP64 residuals every active system takes the number of inner iterations
   the single-problem refinement would give it, or fewer: it stops as soon
   as its r.z (the recursive residual in the V-cycle's norm) has fallen by
   the square of the reduction that run aims at.  It then freezes until the
   run of the slowest one ends; converged systems stop updating, and a
   problem whose systems are all frozen is skipped by the batch's kernels.
   Right-hand sides of a problem are
   interleaved in the batch's own storage (the caller's arrays keep their
   n x n layout). */
typedef struct bmg_batch bmg_batch;   /* opaque */

/* Creates a batch over count set-up contexts (host memory only).
   Errors: BMG_ERR_ARG (a context not eligible, see above, or on another
   device), BMG_ERR_STATE (a context not set up). */
bmg_status bmg_batch_create(int count, bmg_ctx* const* ctxs, int flags, bmg_batch** batch);

/* Device workspace the batch needs (256-byte aligned base). */
bmg_status bmg_batch_workspace_bytes(const bmg_batch* batch, size_t* bytes);

/* Attaches the workspace and the stream the batch's work is ordered on,
   copies the FP32 levels of every context into the size-class storage and
   chooses tile shapes from the kernels' occupancy.  The device must be the
   contexts' and current.  Errors: BMG_ERR_WORKSPACE, BMG_ERR_ARG,
   BMG_ERR_DEVICE. */
bmg_status bmg_batch_attach(bmg_batch* batch, void* workspace, size_t bytes, void* stream);

/* Solves problem p's nrhs (1..4) right-hand sides b[p*nrhs + r] with initial
   guesses and solutions x[p*nrhs + r] (n_p x n_p doubles each, host or
   device; boundary entries ignored on input and 0 on output) to a relative
   FP64 residual of tol (> 0), at most maxit inner iterations per system.
   infos: count*nrhs entries or NULL (iterations = inner iterations of that
   system, true_relres = its final FP64 residual).  Returns the first
   non-OK status (BMG_ERR_NOT_CONVERGED, BMG_ERR_NOT_SPD, BMG_ERR_TIMEOUT). */
bmg_status bmg_batch_solve(bmg_batch* batch, int nrhs, const double* const* b, double* const* x, double tol,
                           int maxit, bmg_info* infos);

/* Size classes (the fused levels by decreasing n, then the tails' first
   level, n = 33); tile shape of class cls: n, strip width wc (16 or 32
   coarse columns), hc coarse rows per item, and its member count (the tail
   class reports wc = hc = 0). */
int bmg_batch_classes(const bmg_batch* batch);
bmg_status bmg_batch_get_tiles(const bmg_batch* batch, int cls, int* n, int* wc, int* hc, int* members);
bmg_status bmg_batch_set_tiles(bmg_batch* batch, int cls, int wc, int hc);

/* Autotuner: times each class's down and up kernels over all its members
   for every strip width and the modelled, half and twice the rows (best of
   reps after a warm-up run) and keeps the fastest; *ms (may be NULL): the
   sum of the chosen times. */
bmg_status bmg_batch_autotune(bmg_batch* batch, int reps, double* ms);

/* Kernel launches the batch has issued (graph replays count their kernels). */
long long bmg_batch_launch_count(const bmg_batch* batch);

void bmg_batch_destroy(bmg_batch* batch);

/* Adjoint gradient with respect to the per-cell coefficient for a loss
   L(u) of the solution u = A^-1 b: solves A lambda = dL/du with the same
   hierarchy (A is symmetric) and evaluates, per cell e,
   dLdkappa[e] = -lambda_e^T K_e^0 u_e, K_e^0 the element matrix at
   kappa = 1.  (dL/db = lambda.)  nrhs >= 1 independent losses with the same
   operator (their adjoint solves go through bmg_solve with nrhs, so they
   share the stencil reads as bmg_solve describes): u, dLdu, lambda: nrhs
   consecutive vectors of n^d doubles (device); dLdkappa: nrhs consecutive
   arrays of (n-1)^d doubles (device); coords: the coordinates given to
   bmg_assemble (device); info: NULL or nrhs entries.  Needs a context built
   by bmg_assemble. */
bmg_status bmg_adjoint_grad(bmg_ctx* ctx, int nrhs, const double* coords, const double* u,
                            const double* dLdu, double* lambda, double* dLdkappa,
                            double tol, int maxit, bmg_info* info);

/* The per-cell contraction of bmg_adjoint_grad alone, for an adjoint
   lambda the caller has already solved for (e.g. with bmg_solve_many over a
   batch of problems): dLdkappa[e] = -lambda_e^T K_e^0 u_e, the derivative
   of lambda^T A(kappa) u in kappa_e, A linear in each cell's coefficient
   (Sec. 2, the assembly of Eq. pde by elements).  Arguments, layout and
   requirements as for bmg_adjoint_grad; runs on the context's stream and
   returns BMG_ERR_MAP_FOLDED if a Jacobian determinant is not positive. */
bmg_status bmg_adjoint_cells(bmg_ctx* ctx, const double* coords, const double* u,
                             const double* lambda, double* dLdkappa);

/* Hierarchy queries (for diagnostics and parity checks). */
int bmg_levels(const bmg_ctx* ctx);
int bmg_level_n(const bmg_ctx* ctx, int level);

/* Copies level `level`'s operator into out (device, n_l^d rows of 3^d
   doubles, the full stencil as in bmg_set_stencil). */
bmg_status bmg_get_stencil(bmg_ctx* ctx, int level, double* out);

/* Copies the interpolation from level level+1 to level `level` into out
   (device, n_l^d rows of 2^d doubles): entry s = sx + 2 sy [+ 4 sz] of
   fine node (i,j[,k]) is its weight to coarse node
   (i>>1 + sx, j>>1 + sy[, k>>1 + sz]); weights to boundary coarse nodes
   and rows of boundary fine nodes are 0. */
bmg_status bmg_get_interp(bmg_ctx* ctx, int level, double* out);

/* Kernel classes timed by the profiler (finest level only). */
enum {
    BMG_PROF_SMOOTH = 0,          /* Gauss-Seidel sweeps */
    BMG_PROF_RESIDUAL = 1,        /* residual r = f - A x */
    BMG_PROF_RESTRICT = 2,        /* b_c = P^T r */
    BMG_PROF_PROLONG = 3,         /* x += P x_c */
    BMG_PROF_SPMV = 4,            /* q = A p with p.q (outer CG) */
    BMG_PROF_UPDATE = 5,          /* x += alpha p, r -= alpha q, r.r */
    BMG_PROF_VDOWN = 6,           /* fused pre-smooth + residual + restriction */
    BMG_PROF_VUP = 7,             /* fused prolongation + post-smooth */
    BMG_PROF_KINDS = 8
};

/* Starts (enable=1, clearing earlier records) or stops (enable=0) timing:
   while on, every launch of a profiled class on the finest level is
   bracketed by CUDA events recorded on the context's stream, and the
   library adds that launch's algorithmic bytes (the compulsory HBM
   traffic of its data: each stencil, vector and interpolation value read
   or written once). */
bmg_status bmg_profile(bmg_ctx* ctx, int enable);

/* Reads the accumulated device time (ms), launch count and algorithmic
   bytes of one class (synchronises the stream). */
bmg_status bmg_profile_read(bmg_ctx* ctx, int kind, double* ms, long long* launches, double* bytes);

/* Tile shape of the streaming 2-D V-cycle kernels on level `level` (the
   kernels that go from level to level+1 and back): wc coarse columns per
   CTA, common to both kernels, and the coarse rows per CTA of the down
   kernel (hc) and of the up kernel (hc_up).  set: wc a multiple of 8 in
   [8, 64], hc and hc_up positive multiples of the rows per step (2);
   BMG_ERR_ARG otherwise or when the context does not use the streaming
   kernels. */
bmg_status bmg_get_tiles(const bmg_ctx* ctx, int level, int* wc, int* hc, int* hc_up);
bmg_status bmg_set_tiles(bmg_ctx* ctx, int level, int wc, int hc, int hc_up);

/* Autotuner: after bmg_setup, times candidate tile shapes of every level on
   the device (the level's down and up kernels, best of reps runs each) and
   keeps the fastest width and, for that width, each kernel's fastest row
   count; *ms (may be NULL) receives the sum of the chosen times.  The
   choice can be read back with bmg_get_tiles and cached by the caller. */
bmg_status bmg_autotune(bmg_ctx* ctx, int reps, double* ms);

/* Kernel launches the context has issued since creation (all kinds). */
long long bmg_launch_count(const bmg_ctx* ctx);

void bmg_destroy(bmg_ctx* ctx);
const char* bmg_status_str(bmg_status status);

/* Allocation-free assembly.  The paper has no counterpart: this entry point
   serves callers that may not allocate (another allocator owns the device
   memory, a hard memory cap, or a path where an allocation is not allowed).
   It computes the same operator as bmg_assemble followed by
   bmg_get_stencil(level 0) but needs no context and no workspace, and it makes
   no allocating call: its working storage (a device error word and the
   half-plane operator) is a static device array of BMG_NOALLOC_SCRATCH_BYTES
   per device.
   dim: 2 or 3.  n: nodes per side, any n >= 3, as long as
   256 + P * ld * n^(dim-1) * 8 bytes fit that array, with P = 5 (2-D) or 14
   (3-D) and ld = n rounded up to a multiple of 32; that is n <= 640 in 2-D
   and n <= 48 in 3-D.  A larger n returns BMG_ERR_SHAPE before any device
   work.  coords, kappa: as for bmg_assemble.  stencil: device, n^dim rows of
   3^dim doubles, written as bmg_get_stencil writes them.  All three on the
   calling thread's current device.  stream: a cudaStream_t, or NULL for the
   legacy default stream; the call returns when its work on the stream is
   done.
   Set-up: the first call on a device looks up the static array's device
   address (cudaGetSymbolAddress) with that device current; make that first
   call before any stream capture begins on the device.  Concurrency: calls
   that overlap in time on one device (other threads or streams) share the
   array and race; serialise them.
   Errors: BMG_ERR_SHAPE, BMG_ERR_ARG (null or non-device pointer),
   BMG_ERR_MAP_FOLDED, BMG_ERR_DEVICE. */
#define BMG_NOALLOC_SCRATCH_BYTES (16u << 20)
bmg_status bmg_assemble_noalloc(int dim, int n, const double* coords, const double* kappa, double* stencil,
                                void* stream);

/* ---------------------------------------------------------------------
   Auxiliary-space two-grid method (Sec. 2.2 "Setup phase" and "Solution
   phase", Sec. 2.3, Sec. 2.4): the structured solve above is the coarse
   level of a two-grid method for the P1 system A_p u_p = f_p on a
   triangulation of the physical domain.  One cycle:
     u_p <- u_p + omega D^-1 (f_p - A_p u_p)        (relaxation S: damped Jacobi)
     r_c  = P^T (f_p - A_p u_p)                     (restriction, Sec. 2.3)
     e_c  = V-cycle of the coarse context on r_c    (BoxMG on A_c)
     u_p <- u_p + gamma P e_c                       (prolongation, Sec. 2.4 scaling)
     u_p <- u_p + omega D^-1 (f_p - A_p u_p)
   with P = M_p^-1 C (Sec. 2.3): M_p the P1 mass matrix, C the coupled mass
   C_ij = integral over the computational domain of (phi_p^i o T^-1) phi_c^j
   |det J_T^-1| (Eq. coupled_mass_comp).  C is accumulated over (triangle,
   cell) pairs: each mapped triangle (vertices mapped by T, straight edges
   in computational space) is clipped to each computational cell it
   overlaps and the pair's 3 x 4 block is integrated exactly over the
   intersection; |det J| is that of the coarse context's Q1 map.  M_p^-1 is
   applied with `mass_steps` CG iterations from zero (the paper uses 2), or
   with the lumped mass (one third of the area around each vertex) when
   mass_steps is 0.  Dirichlet vertices and the computational boundary are
   eliminated.  All values are FP64. */
typedef struct bmg_aux bmg_aux;   /* opaque */

typedef struct {
    double omega;      /* Jacobi weight of S (default 2/3) */
    int mass_steps;    /* CG iterations for M_p^-1 (>= 1), or 0 for the lumped mass (default 0) */
    double gamma;      /* coarse-grid scaling (default 1) */
    int krylov;        /* 0: the paper's stationary iteration of cycles (default); 1: flexible CG
                          with one cycle from a zero guess as the preconditioner.  With the
                          lumped mass and an FP32 coarse context, that preconditioning cycle
                          runs its physical level in FP32 too (A_p products in difference
                          form with FP64 row sums); the CG itself stays FP64 */
} bmg_aux_opts;

void bmg_aux_default_opts(bmg_aux_opts* opts);

/* Builds the host-side structure of the method: interior numbering, the
   sparsity of A_p, M_p and C, the (triangle, cell) pairs and the
   deterministic summation lists.  coarse: a 2-D context on which bmg_setup
   has run; it must outlive the aux object, whose solves use its stream,
   its V-cycle and its Krylov buffers.  Host arrays, copied: xy (nv x 2
   physical vertex coordinates), st (nv x 2, their images T(xy) in the
   computational square [0,1]^2), dirichlet (nv bytes, nonzero =
   eliminated), tri (ntri x 3 vertex indices, counter-clockwise in both
   spaces).  opts may be NULL (defaults).
   Errors: BMG_ERR_ARG (null pointer, vertex index out of range, opts out of
   range), BMG_ERR_SHAPE (coarse not 2-D, a count too large for 32-bit
   indices), BMG_ERR_STATE (coarse not set up). */
bmg_status bmg_aux_create(bmg_ctx* coarse, int nv, const double* xy, const double* st,
                          const unsigned char* dirichlet, int ntri, const int* tri,
                          const bmg_aux_opts* opts, bmg_aux** aux);

/* Device workspace the object needs (bytes, 256-byte aligned base). */
bmg_status bmg_aux_workspace_bytes(const bmg_aux* aux, size_t* bytes);

/* Attaches the workspace and computes A_p, M_p (per-triangle coefficient
   kappa: device, ntri doubles) and C (coords: device, the coarse grid's
   2 x n x n nodal coordinates as given to bmg_assemble) on the device, on
   the coarse context's stream.  Errors: BMG_ERR_WORKSPACE, BMG_ERR_ARG,
   BMG_ERR_MAP_FOLDED (a triangle of non-positive physical area),
   BMG_ERR_DEVICE. */
bmg_status bmg_aux_setup(bmg_aux* aux, void* workspace, size_t bytes, const double* kappa, const double* coords);

/* Stationary two-grid iteration (or flexible CG, opts.krylov = 1) until
   ||f - A_p u|| <= tol ||f|| over the interior vertices, or maxit cycles
   (CG iterations).  With flexible CG the reported residual is the true one
   of the returned iterate, which can sit slightly above the recursive one
   that stopped the loop.  f, u: device, nv doubles (all
   vertices); u holds the initial guess on entry and the iterate on exit,
   with its Dirichlet entries set to zero; f's Dirichlet entries are
   ignored.  info (may be NULL): cycles in `iterations`, the relative
   residual in `relres` and `true_relres`.  Errors: BMG_ERR_NOT_CONVERGED
   (u still holds the last iterate), BMG_ERR_STATE (no setup). */
bmg_status bmg_aux_solve(bmg_aux* aux, const double* f, double* u, double tol, int maxit, bmg_info* info);

bmg_status bmg_aux_set_gamma(bmg_aux* aux, double gamma);

/* Coarse-grid scaling gamma (Sec. 2.4, Eqs. cgc_scaling_1 and gen_eigvalue):
   the mean of the Ritz values of k steps of generalized Lanczos on the
   pencil (P^T A_p P, A_c), i.e. on A_c^-1 P^T A_p P in the A_c inner
   product, with the solver's own P and P^T.  The start vector is
   A_c^-1 y0 (y0: device, the coarse grid's n x n layout, boundary
   ignored).  The recurrence carries the dual vectors A_c q_j, so each step
   costs one P^T A_p P product and one solve with the coarse context (to
   relative residual tol; the context's Krylov buffers are overwritten).
   The mean of the Ritz values is the mean of the Lanczos alpha_j (the
   trace of the tridiagonal matrix over its order).  Outputs (host):
   gamma; alpha (k doubles), beta (k-1 doubles) and steps (the number of
   alphas written: fewer than k if the Krylov space became invariant), each
   may be NULL.  Does not change the aux object's gamma (bmg_aux_set_gamma
   does).  Errors: BMG_ERR_ARG, BMG_ERR_STATE, and the coarse solve's. */
bmg_status bmg_aux_estimate_gamma(bmg_aux* aux, int k, const double* y0, double tol, double* gamma,
                                  double* alpha, double* beta, int* steps);

/* Exports a matrix as CSR into host arrays (each may be NULL to query the
   sizes): which 0 = A_p, 1 = M_p (rows and columns: interior vertices in
   increasing vertex order), 2 = C (rows: interior vertices; columns: the
   coarse grid's interior nodes, as j*n + i).  nrows and nnz are always
   written; rowptr has nrows+1 entries. */
bmg_status bmg_aux_export(const bmg_aux* aux, int which, int* nrows, long long* nnz, long long* rowptr, int* col,
                          double* val);

void bmg_aux_destroy(bmg_aux* aux);

#ifdef __cplusplus
}
#endif
#endif /* BMG_H */
