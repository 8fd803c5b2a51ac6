/*
 * mgdg.h -- C ABI of the GB300 polynomial multigrid solver for the nodal
 * symmetric interior penalty DG (SIPG) Poisson equation on periodic 3D
 * Cartesian grids (Stiller, "Robust Multigrid for Cartesian Interior Penalty
 * DG Formulations of the Poisson Equation in 3D", arXiv 1612.04796).
 *
 * Problem (Section 2, Eq. poisson): -lap u = f on the periodic box
 * [0,lx] x [0,ly] x [0,lz], nx*ny*nz equal cuboid elements, tensor-product
 * Lagrange basis of order P on the Gauss-Lobatto-Legendre (GLL) points
 * (Eq. u_h), SIPG form with GLL quadrature (Eq. ip), A u = f (Eq. discrete)
 * with A = Mz(x)My(x)Lx + Mz(x)Ly(x)Mx + Lz(x)My(x)Mx (Eq. A).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Vectors are DEVICE pointers (unless a name says _host) to element-blocked
 * coefficient vectors: element e = ex + nx*(ey + ny*ez), node (i,j,k) of an
 * element of order p at index e*(p+1)^3 + i + (p+1)*(j + (p+1)*k).  Level l
 * has order P_l = 2^l (level L = log2 P is the fine level, level 0 has P_0 = 1);
 * its vectors have mg_num_dofs(ctx, l) entries.  Right-hand sides are weak
 * (assembled) vectors b = M f_nodal with 1^T b = 0 (see mg_rhs).
 *
 * Ownership: the library allocates NO device memory.  The caller allocates
 * one workspace of mg_workspace_size() bytes (256-byte aligned) and binds it
 * with mg_bind_workspace(); the caller owns all vectors it passes.  Every call
 * is ordered on the CUDA stream given in mg_opts.stream (NULL = legacy default
 * stream); calls that return host scalars synchronise that stream.
 *
 * Errors: every entry point returns an mg_status (no exceptions cross the
 * ABI, nothing aborts); mg_last_error() gives a message.  Device-side loops
 * have iteration limits that end in a status, never in a hang or trap.
 */
#ifndef MGDG_H
#define MGDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx;

typedef enum {
  MG_OK = 0,
  MG_EINVAL = 1,     /* invalid argument (sizes, pointers, level index, ...) */
  MG_ENOMEM = 2,     /* host allocation failed or workspace too small */
  MG_ECUDA = 3,      /* a CUDA runtime call failed (message in mg_last_error) */
  MG_ENOCONV = 4,    /* an iteration limit was reached (setup eigensolver, solve) */
  MG_ENOTREADY = 5   /* workspace not bound yet */
} mg_status;

/* Arithmetic of the solve (Section 3.2 method, precision is this library's choice). */
typedef enum {
  MG_FP64 = 0,  /* every kernel in FP64 */
  MG_MIXED = 1, /* FP32 multigrid (smoother, transfers, operator on the levels)
                   inside an FP64 outer iteration; FP64 outer residual, inner
                   products, updates, 1D setup and coarsest solve */
  MG_DF64 = 2   /* the same split with the multigrid in double-float arithmetic
                   (pairs of FP32, about 48 significant bits: FP64-class accuracy
                   on the FP32 pipes); the coarsest solve stays FP64 */
} mg_precision;

/* How the subdomain overlap is given (Section 3.1, Table 1). */
typedef enum {
  MG_OVERLAP_LAYERS = 0, /* N_O node layers (argument `overlap` of mg_setup) */
  MG_OVERLAP_WIDTH = 1,  /* delta_O,i = overlap_frac * dx_i on every level (Table 1 rows 3-6;
                            the "rel" overlap of Table 2) */
  MG_OVERLAP_MAX = 2     /* delta_O,i = min(overlap_frac * max_j dx_j, dx_i): the "max" overlap
                            of Table 2 for anisotropic meshes; the strip may cover the whole
                            neighbour element, and every direction has its own N_O */
} mg_overlap_mode;

/* Transition profile of the hat-shaped weight function w_H (Fig. wH). */
typedef enum {
  MG_WEIGHT_QUINTIC = 0,            /* q(t) = 10t^3 - 15t^4 + 6t^5 across the whole strip */
  MG_WEIGHT_LINEAR = 1,             /* q(t) = t */
  MG_WEIGHT_QUINTIC_HALVES = 2,     /* a quintic step on each half of the strip, 1/2 on the interface */
  MG_WEIGHT_QUINTIC_NORMALISED = 3  /* one-sided quintic hat normalised to sum to one */
} mg_weight_profile;

/* Half-width delta (reference units) of the transition of w_H (Fig. wH) when
 * the strip holds N_O >= 2 node layers; the paper defers the definition to an
 * earlier paper, so these are readings.  For N_O <= 1 all give the same weights. */
typedef enum {
  MG_DELTA_DEFAULT = 0, /* MG_DELTA_MID for MG_OVERLAP_LAYERS, MG_DELTA_STRIP otherwise */
  MG_DELTA_NODE = 1,    /* the distance of the outermost included neighbour node: its weight is 0 */
  MG_DELTA_MID = 2,     /* midway between the outermost included and the first excluded node */
  MG_DELTA_STRIP = 3    /* the strip itself, 2 delta_O / dx (MG_OVERLAP_WIDTH and MG_OVERLAP_MAX only) */
} mg_weight_delta;

typedef struct {
  int overlap_mode;      /* mg_overlap_mode, default MG_OVERLAP_LAYERS */
  double overlap_frac;   /* delta_O / dx for MG_OVERLAP_WIDTH (0 .. 0.5; paper: 0.08, 0.5),
                            delta_O / max_j dx_j for MG_OVERLAP_MAX (0 .. 1; paper: 0.08) */
  int weight_profile;    /* mg_weight_profile, default MG_WEIGHT_QUINTIC */
  int ns_pre, ns_post;   /* smoothing steps N_s1, N_s2 on the fine level (default 1, 1) */
  int ns_growth;         /* N_s,l = N_s * ns_growth^(L-l): 1 fixed V-cycle, 3 variable (Table 2) */
  int precision;         /* mg_precision, default MG_FP64 */
  int fdm_tensor_cores;  /* MG_MIXED, subdomain contractions of the FP32 smoother: 0 = FP32 CUDA
                            cores (default); 1 = tensor cores (tcgen05, TF32 inputs rounded to
                            nearest, FP32 accumulation) on every level whose tiles fit the
                            kernel; 2 = per level whichever of the two mg_bind_workspace
                            measures faster (the choice, and so the rounding, may differ
                            between contexts) */
  int outer_df64;        /* MG_MIXED with use_cg: 1 = the outer products q = A p in double-float
                            arithmetic (pairs of FP32, about 48 significant bits; FP64 vectors,
                            inner products and updates); 2 = the whole outer iteration in
                            double-float (vectors x, r, p, q stored as pairs; q = A p, inner
                            products, updates on the FP32 pipes; the initial residual and the
                            returned solution FP64); 0 = FP64 (default) */
  void* stream;          /* cudaStream_t; NULL = default stream */
  int weight_delta;      /* mg_weight_delta, default MG_DELTA_DEFAULT; MG_OVERLAP_MAX takes only
                            the default */
  int autotune;          /* 1 = mg_bind_workspace times the kernel variants of every level's
                            smoother, operator and scatter (as the hierarchy's arithmetic runs
                            them) and keeps the fastest; 0 = the fixed defaults (default) */
  int fdm_operands;      /* MG_MIXED, a precision study of the FP32 smoother of single solves:
                            every line entering a 1D product, and the 1D factors, rounded to
                            1 = BF16, or 2 = FP8 E4M3 after a power-of-two scale per line (data)
                            or per output index (factors: "scaled eigenbases"), accumulating in
                            FP32 -- the arithmetic of BF16 / FP8 tensor-core contractions, on
                            the CUDA cores (the one-kernel smoother); 0 = FP32 operands
                            (default) */
  int persistent;        /* mg_solve_batch (the first context's value): 0 = a grouped launch with
                            more blocks than the GPU holds at once runs in persistent form -- one
                            wave of blocks looping over the problems' blocks (default); 1 = every
                            grouped launch persistent; 2 = none */
} mg_opts;

/* Fill *o with the defaults above. */
void mg_default_opts(mg_opts* o);

/*
 * mg_setup -- describe a problem and its multigrid hierarchy (host only).
 * Section 2 (domain, mesh, order), Section 3.1 (overlap), Section 3.2
 * (levels P_l = 2^l), Section 4 (penalty mu = 2 mu_min).
 *   lx, ly, lz   box lengths (> 0)
 *   nx, ny, nz   elements per direction (3 .. 512)
 *   P            polynomial order, a power of two, 2 <= P <= 32
 *   penalty      mu / mu_min per direction, mu_min = P_l (P_l+1) / (2 dx) the
 *                coercivity threshold of the form; the paper's choice is 2
 *   overlap      N_O node layers (>= 0) for MG_OVERLAP_LAYERS; clamped on
 *                each level to floor(P_l/2) + 1; ignored for MG_OVERLAP_WIDTH
 *                and MG_OVERLAP_MAX
 * With MG_OVERLAP_MAX a direction whose strip covers the whole neighbour
 * element (N_O = P_l + 1) needs at least 4 elements, so that the two strips of
 * a subdomain are not coupled through the periodic boundary: MG_EINVAL
 * otherwise.
 *   opts         NULL for defaults
 *   out          receives the new context (host memory owned by the library;
 *                release with mg_destroy)
 * Returns MG_EINVAL for out-of-range arguments.  No CUDA call is made.
 */
mg_status mg_setup(double lx, double ly, double lz, int nx, int ny, int nz, int P, double penalty,
                   int overlap, const mg_opts* opts, mg_ctx** out);

/*
 * mg_setup_graded -- mg_setup for a graded mesh: element widths that vary
 * along each axis of the periodic box, the mesh staying a tensor product
 * (element (ex, ey, ez) is hx[ex] x hy[ey] x hz[ez]; its first corner lies at
 * the sums of the widths before it).  The paper's grids are uniform
 * (Section 4); the same form (Section 2, Eq. ip) applies element by element,
 * so Eq. (A) keeps its Kronecker structure with per-element 1D factors and
 * every subdomain of Section 3.1 gets the eigenbases of its own three lines.
 *   hx, hy, hz   host arrays of nx, ny, nz widths (> 0, finite); copied
 *   nx, ny, nz   3 .. 256 (the coarse eigenproblems are solved whole)
 *   penalty      as in mg_setup, per face: mu = penalty P_l (P_l+1) / (2 h_min)
 *                with h_min the smaller width of the face's two elements
 *                (the uniform threshold stays the coercivity threshold)
 *   P, overlap, opts, out   as in mg_setup
 * Supported: MG_FP64 and MG_MIXED (any outer_df64), MG_OVERLAP_LAYERS; no
 * tensor cores, no autotuning, no operand study: anything else returns
 * MG_EINVAL, as do mg_vcycle_df64, mg_smooth_df64 (the double-float
 * multigrid) and mg_solve_batch on such a context.  All other calls work as
 * on a uniform mesh (mg_node_coords gives the graded coordinates, mg_rhs the
 * graded mass; mg_get_line_table the per-line tables).  No CUDA call is made;
 * mg_bind_workspace copies the widths to the device and builds the tables.
 */
mg_status mg_setup_graded(const double* hx, const double* hy, const double* hz, int nx, int ny, int nz, int P,
                          double penalty, int overlap, const mg_opts* opts, mg_ctx** out);

/* 1 if ctx describes a graded mesh (mg_setup_graded), else 0 (host only). */
int mg_is_graded(const mg_ctx* ctx);

/* Bytes of device workspace the context needs (256-byte aligned base required). */
mg_status mg_workspace_size(const mg_ctx* ctx, size_t* bytes);

/*
 * mg_bind_workspace -- bind caller-owned device memory and run the per-level
 * 1D setup on the device (Section 3.1: GLL tables, the restricted 1D
 * generalised eigenproblems L_s S = M_s S Lambda with S^T M_s S = I, the
 * weights; Section 3.2: interpolation; coarse level eigenbases).  Synchronises
 * the stream.  Returns MG_ENOCONV if an eigensolver hit its sweep limit.
 */
mg_status mg_bind_workspace(mg_ctx* ctx, void* dptr, size_t bytes);

/* Number of levels L+1, DOFs and overlap layers of a level (host, no CUDA).
 * mg_level_layers gives N_O of the x direction; mg_level_layers_dir that of
 * direction dir (0 x, 1 y, 2 z), which differ only with MG_OVERLAP_MAX.
 * -1 for a bad level or direction. */
int mg_num_levels(const mg_ctx* ctx);
long long mg_num_dofs(const mg_ctx* ctx, int level);
int mg_level_layers(const mg_ctx* ctx, int level);
int mg_level_layers_dir(const mg_ctx* ctx, int level, int dir);

/*
 * mg_selftest_bounded_wait -- check the bounded wait of the tensor-core
 * smoother kernel on `level` (MG_MIXED context, level whose tiles fit the
 * kernel): launches it so that nothing ever arrives on its mbarrier (no MMA is
 * issued), lets its wait run out (about 10 ms), reads the status word back and
 * clears it.  *timed_out = 1 if the kernel reported the timeout.  The context
 * stays usable.  Not part of the method; a check of the failure path.
 * MG_EINVAL if the level cannot run the kernel.
 */
mg_status mg_selftest_bounded_wait(mg_ctx* ctx, int level, int* timed_out);

/* Kernel of the FP32 smoother contractions on a level after mg_bind_workspace:
 * 1 tensor cores, 0 CUDA cores, -1 bad level. */
int mg_level_fdm_tensor_cores(const mg_ctx* ctx, int level);

/* Kernel variant of single solves on a level (what mg_opts.autotune chose, or
 * the default): kind 0 smoother, 1 operator, 2 scatter; returns 0 for the
 * kernels with the 1D coefficients as kernel parameters (FP32 smoother;
 * FP32 / double-float operator on shared-memory element blocks,
 * direction-split on meshes of few elements) and the element-aligned
 * scatter; 1 for the alternative
 * (shared-memory smoother, plain operator, plain scatter); for the FP32
 * smoother 2 for the passes of the parameter-space kernel split over three
 * grid-wide kernels (planes of the tile, then its z-columns, then planes
 * again), the default on cubic levels with subdomain width m >= 11; -1 for
 * a bad level or kind. */
int mg_level_kernel_variant(const mg_ctx* ctx, int level, int kind);

/* Physical coordinates of the nodes of `level` into x, y, z (device, N_l each). */
mg_status mg_node_coords(mg_ctx* ctx, int level, double* x, double* y, double* z);

/*
 * mg_rhs -- weak right-hand side of the fine level from nodal values (Section 2:
 * GLL quadrature of int v f): b = M (f - (1^T M f)/(1^T M 1)) and then the
 * rounding-level Euclidean mean of b is removed, so 1^T b = 0.  Device pointers,
 * N_L values each; f_nodal and b may not alias.
 */
mg_status mg_rhs(mg_ctx* ctx, const double* f_nodal, double* b);

/* Au = A_l u: sum-factorised SIPG operator of level l (Eq. A). */
mg_status mg_apply_sipg(mg_ctx* ctx, int level, const double* u, double* Au);
/* r = f - A_l u (Eq. discrete, residual form). r may not alias u or f. */
mg_status mg_residual(mg_ctx* ctx, int level, const double* u, const double* f, double* r);

/*
 * mg_smooth -- nsteps weighted additive Schwarz steps on level l (Section 3.1):
 * u <- u + sum_s R_s^T W_s A_ss^{-1} R_s (f - A_l u), with A_ss^{-1} applied by
 * fast diagonalisation (Sz(x)Sy(x)Sx)(Lambda sum)^{-1}(Sz^T(x)Sy^T(x)Sx^T).
 * In place on u.  Uses the level's scratch vectors in the workspace.
 */
mg_status mg_smooth(mg_ctx* ctx, int level, double* u, const double* f, int nsteps);

/* f_c = I_l^T (f - A_l u): residual restriction to level l-1 (Algorithm 1). level >= 1. */
mg_status mg_restrict_residual(mg_ctx* ctx, int level, const double* u, const double* f, double* f_c);
/* u += I_l u_c: correction prolongation from level l-1 (Algorithm 1). level >= 1. */
mg_status mg_prolongate(mg_ctx* ctx, int level, const double* u_c, double* u);
/*
 * mg_coarse_solve -- u0 = A_0^+ f0 on level 0 (Algorithm 1, coarse grid
 * solution): f0 is projected onto the range of A_0 (zero mean) and the
 * minimum-norm solution is returned (zero mean).  Computed directly by fast
 * diagonalisation of the whole periodic coarse problem.
 */
mg_status mg_coarse_solve(mg_ctx* ctx, const double* f0, double* u0);

/* One multigrid V-cycle (Algorithm 1) on the fine level, in place on u. */
mg_status mg_vcycle(mg_ctx* ctx, double* u, const double* f);

/*
 * mg_solve -- solve A u = f to ||f - A u||_2 <= tol ||f - A u_0||_2 (Section 4).
 * u holds the initial guess on entry and the solution (zero Euclidean mean) on
 * return.  use_cg = 0: repeated V-cycles (MG); use_cg = 1: inexact
 * preconditioned CG with one V-cycle from zero as preconditioner (MG-CG,
 * Section 3.2).  With MG_MIXED the V-cycle runs in FP32.  iters, relres (host)
 * receive the iteration count and final relative residual; history (host, may be
 * NULL) receives maxit+1 residual norms.  Returns MG_ENOCONV if maxit is reached
 * or the residual becomes non-finite, MG_EINVAL if the initial residual is not
 * finite (NaN or Inf in u or f).
 */
mg_status mg_solve(mg_ctx* ctx, double* u, const double* f, double tol, int maxit, int use_cg, int* iters,
                   double* relres, double* history);

/* mg_solve with HOST buffers u_host, f_host (N_L doubles; pinned memory is
 * fastest): copies f (and the initial u) in, solves, copies u out. */
mg_status mg_solve_host(mg_ctx* ctx, double* u_host, const double* f_host, double tol, int maxit, int use_cg,
                        int* iters, double* relres, double* history);

/*
 * mg_solve_batch -- MG-CG solves (mg_solve with use_cg = 1) of `count`
 * independent problems advanced together: every sweep of their iterations
 * (operator, smoother, scatter, transfers, coarse passes, CG vector passes)
 * is issued as one launch for all of them, each problem keeping its own
 * blocks, tables and vectors, so that small problems share the GPU instead
 * of each paying for its own launches.  The problems may differ in box, mesh,
 * order and options; launches merge where their kernel sequences agree
 * (same order and level structure), the rest run one by one.
 *   ctxs     count distinct contexts, each with its workspace bound
 *   u, f     per problem: device vectors as in mg_solve (u: initial guess in,
 *            zero-mean solution out)
 *   count    1 .. 16
 *   tol, maxit  as in mg_solve, the same for every problem
 *   iters, relres, status  (host, count entries each, may be NULL) per problem:
 *            its iteration count, relative residual and mg_status (MG_OK,
 *            MG_ENOCONV at maxit or on a non-finite residual, MG_EINVAL on a
 *            non-finite initial residual, MG_ECUDA if a tensor-core wait ran out)
 * Every launch goes to the stream of ctxs[0] (the other contexts' streams are
 * not used); the call synchronises it once per iteration, to read the
 * residual norms of all problems together.  Each problem gets the block
 * decomposition and reduction order of its own mg_solve; the batched kernels
 * are separate compilations of the same code (a compiler may contract
 * multiply-adds differently), so results agree with mg_solve to rounding, and
 * bit for bit with any other batch that contains the problem (its result does
 * not depend on the other problems).  Returns MG_EINVAL / MG_ENOTREADY for bad
 * arguments, MG_ECUDA if a CUDA call failed (message on ctxs[0]), else MG_OK
 * (per-problem outcomes in status).
 */
mg_status mg_solve_batch(mg_ctx* const* ctxs, int count, double* const* u, const double* const* f, double tol,
                         int maxit, int* iters, double* relres, int* status);

/* mg_vcycle_df64 -- one V-cycle (Algorithm 1) like mg_vcycle on FP64 vectors u,
 * f of the finest level, with the multigrid arithmetic in double-float (the
 * preconditioner of MG_DF64).  Uses two of the outer-iteration work vectors. */
mg_status mg_vcycle_df64(mg_ctx* ctx, double* u, const double* f);

/* mg_smooth_df64 -- nsteps Schwarz steps on level l like mg_smooth (Section 3.1;
 * FP64 vectors u, f of that level), with the residual, the fast
 * diagonalisation and the weighted scatter in double-float arithmetic (the
 * smoother of MG_DF64).  Uses two of the outer-iteration work vectors. */
mg_status mg_smooth_df64(mg_ctx* ctx, int level, double* u, const double* f, int nsteps);

/* mg_apply_sipg_df64 -- Au = A_l u like mg_apply_sipg (FP64 vectors), with the
 * arithmetic in double-float (about 48 significant bits); the operator of the
 * outer iteration when mg_opts.outer_df64 = 1.  Uses the smoother's
 * correction buffer as scratch. */
mg_status mg_apply_sipg_df64(mg_ctx* ctx, int level, const double* u, double* Au);

/* FP32 versions of the level kernels used by the MG_MIXED preconditioner
 * (same semantics as the FP64 entry points; FP32 tables and arithmetic). */
mg_status mg_apply_sipg_f32(mg_ctx* ctx, int level, const float* u, float* Au);
mg_status mg_smooth_f32(mg_ctx* ctx, int level, float* u, const float* f, int nsteps);
mg_status mg_vcycle_f32(mg_ctx* ctx, float* u, const float* f);

/*
 * mg_get_table -- copy a 1D setup table of level l, direction dir (0 x, 1 y,
 * 2 z) to host memory, for inspection and tests.  what:
 *   0 GLL nodes (n)       1 GLL weights (n)      2 mass diag (h/2) w (n)
 *   3 element block of L (n*n, row-major)        4 eigenvalues Lambda (m)
 *   5 eigenvectors S (m*m, S[a*m + p] = entry a of eigenvector p)
 *   6 weights w (m)       7 interpolation J_l (n * n_c, row-major; level >= 1)
 *   8 coarse eigenvalues (2 n_d; level 0)  9 coarse eigenvectors (4 n_d^2; level 0)
 * (m = n + 2 N_O of direction dir.)  *count receives the number of values;
 * fails with MG_EINVAL if capacity is too small.
 */
mg_status mg_get_table(mg_ctx* ctx, int level, int dir, int what, double* host_out, int capacity, int* count);

/*
 * mg_get_line_table -- graded meshes: copy a table of element line `line`
 * (0 .. n_dir - 1) of level l, direction dir to host memory.  what:
 *   0 mass diag (h_line / 2) w (n)
 *   1 rows of the line's element in the 1D matrix L: blocks L[e][e-1],
 *     L[e][e], L[e][e+1] (3 n*n, each row-major)
 *   2 eigenvalues Lambda of the subdomain line centred on the element (m; l >= 1)
 *   3 its eigenvectors S (m*m, S[a*m + p] = entry a of eigenvector p, S^T M_s S = I)
 * The eigenpairs come in no particular order.  MG_EINVAL on a uniform mesh,
 * for a missing table, or if capacity is too small.
 */
mg_status mg_get_line_table(mg_ctx* ctx, int level, int dir, int line, int what, double* host_out, int capacity,
                            int* count);

/*
 * mg_coarse_solve_noalloc -- allocation-free variant of mg_coarse_solve.  The
 * paper has no counterpart: this entry point exists for callers that may not
 * allocate device memory (for example a plugin that a host framework hands
 * only its input and output buffers because the framework owns all device
 * memory, or a latency-critical path that cannot accept an allocation's
 * implicit device synchronisation) and therefore cannot provide the
 * workspace that mg_bind_workspace needs.
 * It computes u0 = A_0^+ f0 on the P_0 = 1 level of the mesh given by lx, ly,
 * lz, nx, ny, nz and penalty (same meaning as in mg_setup), with no context
 * and no workspace; it calls no cudaMalloc / cudaFree or any allocating
 * routine.  Its scratch is one file-scope device array of 4.5 MiB, which every
 * GPU that loads the library holds until the process exits.
 *   f0, u0   device pointers, N0 = 8 nx ny nz doubles each, element-blocked
 *            level-0 layout (2 nodes per direction); u0 receives the zero-mean
 *            solution; they may not alias.
 *   stream   cudaStream_t (NULL = legacy default stream); the call
 *            synchronises it once (it reads the coarse eigenvalues back).
 * Limits: 3 <= nx, ny, nz <= 32 (N0 <= 262,144); larger sizes (and other
 * invalid arguments) return MG_EINVAL before any CUDA call.  MG_ECUDA on a
 * failed CUDA call, MG_ENOCONV if an eigensolver hit its sweep limit.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current): make that first call
 * before any stream capture begins.  With lazy module loading (the CUDA
 * default) that first lookup may also load the library's device code on the
 * device, which is when the array is reserved, so the first call can take
 * device memory and synchronise; a caller for whom that matters makes one call
 * at start-up.  Later calls reserve nothing.  All calls share the one array, which
 * keeps the last call's contents: calls that overlap on the GPU (from other
 * streams or other host threads) race on it and must not be issued
 * concurrently.
 */
mg_status mg_coarse_solve_noalloc(double lx, double ly, double lz, int nx, int ny, int nz, double penalty,
                                  const double* f0, double* u0, void* stream);

/* Instrumentation (not part of the method).
 * mg_kernel_launches: number of kernels this context has launched since
 *   mg_setup (host-side count; mg_bind_workspace's setup kernels included).
 * mg_profile: enable = 1 starts recording a CUDA event pair on the context's
 *   stream around every kernel group (clearing earlier records); 0 stops.
 * mg_profile_result: summed device time in ms and number of recorded groups
 *   of one kind on one level (level -1: all levels).  kind: 0 smoother fast
 *   diagonalisation (gather + contractions), 1 smoother scatter, 2 level
 *   operator / residual inside the V-cycle, 3 restriction, 4 prolongation,
 *   5 coarse solve, 6 vector passes of the outer iteration (inner products,
 *   updates, mean projections, precision conversions), 7 the outer
 *   iteration's operator (fine-level residual of MG, q = A p of MG-CG).
 *   Synchronises the stream. */
long long mg_kernel_launches(const mg_ctx* ctx);
/* Kernels launched by the mg_solve_batch calls whose first context was ctx
 * (grouped launches, graph nodes, the gathers of the residual norms and the
 * per-problem first directions; recorded launches do not count for the
 * members' mg_kernel_launches). */
long long mg_batch_launches(const mg_ctx* ctx);
mg_status mg_profile(mg_ctx* ctx, int enable);
mg_status mg_profile_result(mg_ctx* ctx, int kind, int level, double* total_ms, long long* count);

/* Message of the last failed call on ctx (never NULL). */
const char* mg_last_error(const mg_ctx* ctx);

/* Release the context (host memory only; the workspace belongs to the caller). */
void mg_destroy(mg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MGDG_H */
