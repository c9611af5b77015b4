/*
 * stencil.h -- C ABI of the GB300 library for the coloured stencil codes of
 * Hazelwood & Weinzierl, "Coloured and task-based stencil codes" (arXiv:1810.04033).
 *
 * The library applies the matrix-free Q1 (d-linear) Laplacian on regular Cartesian
 * grids and runs the race-free coloured Gauss-Seidel sweep, damped Jacobi and the
 * residual on one CUDA device.  Every call below is asynchronous on the given stream
 * unless stated otherwise.
 *
 * Conventions shared by all calls
 * -------------------------------
 * Grid.  dim = 2 or 3; n[0], n[1], n[2] = cells along x, y, z (n[2] is ignored for
 *   dim 2).  Arrays hold all (n[0]+1) x (n[1]+1) [x (n[2]+1)] vertices, x fastest:
 *   element (i,j,k) lives at  k*pitch*(n[1]+1) + j*pitch + i,  pitch >= n[0]+1.
 *   Vertices with an index 0 or n[a] are the boundary: they hold Dirichlet data,
 *   are read by the stencil and never written by a smoother.
 * Operator.  A = S/h^2 where S is the assembled Q1 stencil (Section 2, Fig. 1):
 *   3D: centre 8/3, face neighbours 0, edge neighbours -1/6, corner neighbours -1/12;
 *   2D: centre 8/3, all eight neighbours -1/3 (the 9-point stencil of Fig. 1).
 *   A u = f discretises -Laplace u = f with f sampled at the vertices.
 * Colours.  Vertex (i,j,k) has colour (i&1) + 2(j&1) + 4(k&1) (2D: (i&1) + 2(j&1));
 *   a Gauss-Seidel sweep visits the colours in ascending order and updates every
 *   interior vertex of a colour from the current values of its neighbours
 *   (Section 3, "Colouring"; Section 2 for the in-situ update).
 * Memory.  All array arguments are DEVICE pointers owned by the caller unless a call
 *   says otherwise; the library never frees them.  Element type follows
 *   stencil_grid_t.dtype.  Pointers must be aligned to their element size; 16-byte
 *   aligned bases with rows on 16-byte boundaries (an even pitch for F64, a multiple
 *   of 4 for F32) give the fastest paths (plane staging by TMA, 16-byte accesses);
 *   other layouts give the same results on slower kernels.
 * Streams.  `stream` is a cudaStream_t passed as void*; NULL selects the legacy
 *   default stream.  Calls check their arguments synchronously and report launch
 *   failures synchronously; faults inside kernels surface at the next synchronising
 *   CUDA call.
 * Errors.  Every int-returning call returns STENCIL_OK (0) or a negative code below;
 *   stencil_last_error() then holds a message (per host thread).
 */
#ifndef STENCIL_GB300_H
#define STENCIL_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define STENCIL_OK 0
#define STENCIL_EINVAL (-1)    /* bad dimension, size, pitch, dtype, pointer or option */
#define STENCIL_ENOMEM (-2)    /* a device allocation the call needed failed */
#define STENCIL_EADMIT (-3)    /* server: request footprint exceeds the HBM budget */
#define STENCIL_ETIMEDOUT (-4) /* a bounded wait ran out */
#define STENCIL_ECUDA (-5)     /* the CUDA runtime reported an error */
#define STENCIL_ENOTCONV (-6)  /* solve stopped at max_outer; result still written */
#define STENCIL_ENOTFOUND (-7) /* server: unknown ticket */
#define STENCIL_EBUSY (-8)     /* server: request not finished yet (poll) */

/* ---------------------------------------------------------------- element types */
#define STENCIL_F64 0
#define STENCIL_F32 1
#define STENCIL_BF16 2

/* ---------------------------------------------------------------- apply forms */
#define STENCIL_FORM_ELEMENTWISE 0 /* cell-wise element matrix, 2^d-colour scatter */
#define STENCIL_FORM_STENCIL 1     /* assembled 3^d-point stencil, gathered */

/* Operators (stencil_grid_t.op).
 * STENCIL_OP_Q1: the Q1 (d-linear FE) Laplacian A = S / h^2, S the assembled 3^d-point
 *   stencil (2D: the 9-point stencil of Fig. 1, right), coloured with 2^d colours.
 * STENCIL_OP_FD: the 2d+1-point finite-difference Laplacian (2D: the 5-point stencil of
 *   Fig. 1, middle; 3D: 7-point), S u = 2d u - (sum of the face neighbours), coloured
 *   red-black (Section 3).  F64 only; supported by stencil_apply (stencil form),
 *   stencil_smooth_coloured (red-black: first the interior vertices with i+j+k odd,
 *   then even, the order of Algorithm 1), stencil_smooth_jacobi, stencil_jacobi_step
 *   and stencil_residual; the other entry points return STENCIL_EINVAL. */
#define STENCIL_OP_Q1 0
#define STENCIL_OP_FD 1

typedef struct stencil_grid {
  int32_t dim;   /* 2 or 3 */
  int32_t dtype; /* STENCIL_F64 | STENCIL_F32 | STENCIL_BF16 */
  int64_t n[3];  /* cells along x, y, z; each >= 1 (n[2] ignored when dim == 2) */
  int64_t pitch; /* elements between consecutive x-rows; 0 selects n[0] + 1 */
  double h;      /* mesh width (> 0) */
  int32_t op;    /* STENCIL_OP_Q1 (0, the default of a zeroed descriptor) or STENCIL_OP_FD */
  int32_t reserved; /* 0 */
} stencil_grid_t;

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int stencil_version(void);

/* Message for the last failing call on this host thread ("" if none). */
const char *stencil_last_error(void);

/* Calls whose device workspace stencil_workspace_size reports. */
#define STENCIL_CALL_SMOOTH_COLOURED 1
#define STENCIL_CALL_SMOOTH_JACOBI 2
#define STENCIL_CALL_RESIDUAL 3
#define STENCIL_CALL_APPLY_ELEMENTWISE 4 /* stencil_apply, element-wise form: no workspace */
#define STENCIL_CALL_APPLY_STENCIL 5     /* stencil_apply, stencil form: no workspace */

/*
 * *bytes = the device workspace (ws_bytes) that `call` needs on grid g for `sweeps`
 * sweeps (ignored for STENCIL_CALL_RESIDUAL); 0 when the call needs none.  The paper
 * has no counterpart: it lets callers own every device buffer (Memory, above).  The
 * size depends on the descriptor, the call, the sweep count and, for the residual, the
 * SM count of the current device (pass the buffer to calls on that device).  Host-only:
 * touches no device memory and launches nothing.  Returns STENCIL_EINVAL for a bad
 * descriptor, call or sweep count.
 */
int stencil_workspace_size(const stencil_grid_t *g, int call, int sweeps, size_t *bytes);

/*
 * y = A u.  Section 2: a stencil evaluation per vertex from its neighbours' values;
 * a separate output array makes it the matrix-vector product.
 *   form = STENCIL_FORM_ELEMENTWISE: every cell computes K_e u_e (K_e the Q1
 *     element stiffness matrix) and adds it into its 2^d vertices; cells are visited
 *     in 2^d colour passes (cell colour = parity of its lower-corner indices), so that
 *     no two cells of a pass share a vertex (Section 3, "Colouring").
 *   form = STENCIL_FORM_STENCIL: every interior vertex gathers the assembled stencil.
 * Both give the same y up to rounding.  Interior rows are divided by the lumped mass
 * h^d, so y = S u / h^2; boundary rows of y are set to 0.
 * u, y: device arrays of g->dtype (F64 only at present), must not overlap.
 * Returns STENCIL_EINVAL for a bad grid/form/pointer, STENCIL_ECUDA on launch failure.
 */
int stencil_apply(const stencil_grid_t *g, const void *u, void *y, int form, void *stream);

/*
 * `sweeps` coloured Gauss-Seidel sweeps on A u = f, in place on u (Section 2:
 * in-situ update; Section 3: 2^d colours in ascending order, independent updates
 * inside a colour).  Each interior vertex i of the current colour becomes
 *   u_i = (h^2 f_i - sum_{j != i} S_ij u_j) / S_ii.
 * Boundary values of u are read, never written; f on the boundary is ignored.
 * u: device array (in/out); f: device array, may not alias u.  dtype F64 (2D, 3D);
 * F32 or BF16 (3D): values stored in that type, arithmetic in FP32, every store of a
 * bf16 value rounded to nearest even.
 * ws, ws_bytes: the call's device workspace, owned by the caller: at least
 * stencil_workspace_size(g, STENCIL_CALL_SMOOTH_COLOURED, sweeps) bytes, 256-byte
 * aligned, overlapping neither u nor f (F64: up to three times the size of u; no
 * initial contents needed, contents on return unspecified).  Work queued on the stream
 * owns it until it completes.  ws = NULL is a convenience: the library then uses its
 * own workspace for (device, stream), allocated on first use, grown when a larger grid
 * needs more (which synchronises the stream) and kept until stencil_release_workspace.
 * Returns STENCIL_EINVAL (also for a short or misaligned ws), STENCIL_ENOMEM,
 * STENCIL_ECUDA.
 */
int stencil_smooth_coloured(const stencil_grid_t *g, void *u, const void *f, int sweeps, void *ws,
                            size_t ws_bytes, void *stream);

/*
 * `sweeps` damped Jacobi sweeps, out of place:
 *   u_i <- u_i + omega * (h^2 f_i - (S u)_i) / S_ii   on interior vertices,
 * every new value computed from the previous sweep's array (the contrast to the
 * in-situ update of Section 2).  work: caller-owned device array with the layout of u,
 * the second array of the out-of-place sweep (its contents on return are unspecified).
 * The result of the last sweep is in u; boundary values of u are never changed.
 * ws, ws_bytes: further device workspace of the multi-sweep kernels (int64 copies of
 * the iterate), at least stencil_workspace_size(g, STENCIL_CALL_SMOOTH_JACOBI, sweeps)
 * bytes (twice the size of u for two or more Q1 sweeps, else 0), 256-byte aligned,
 * overlapping no other argument; ws = NULL selects the library's own workspace as for
 * stencil_smooth_coloured.  dtype F64.
 * Returns STENCIL_EINVAL, STENCIL_ENOMEM, STENCIL_ECUDA.
 */
int stencil_smooth_jacobi(const stencil_grid_t *g, void *u, const void *f, void *work,
                          int sweeps, double omega, void *ws, size_t ws_bytes, void *stream);

/*
 * One damped Jacobi sweep, out of place: u_out = u_in + omega D^-1 (f - A u_in) on
 * interior vertices and u_out = u_in on the boundary (the primitive that
 * stencil_smooth_jacobi repeats).  u_in, f, u_out: device arrays of one layout, u_out
 * overlapping neither input.  dtype F64.  Returns STENCIL_EINVAL, STENCIL_ECUDA.
 */
int stencil_jacobi_step(const stencil_grid_t *g, const void *u_in, const void *f, void *u_out,
                        double omega, void *stream);

/*
 * Residual and norms: r = f - A u on interior vertices (0 on the boundary), and
 * d_norms2[0] = sum of r_i^2, d_norms2[1] = sum of f_i^2 over interior vertices, both
 * in FP64 by a fixed-order two-level reduction (the same bits on every call with the
 * same input and device).  r may be NULL (norms only).  d_norms2: device, 2 doubles.
 * ws, ws_bytes: the reduction's device workspace (a counter, which the call clears on
 * the stream, and one pair of partial sums per CTA), at least
 * stencil_workspace_size(g, STENCIL_CALL_RESIDUAL, 0) bytes, 256-byte aligned,
 * overlapping no other argument; ws = NULL selects the library's own workspace as for
 * stencil_smooth_coloured.  dtype F64.
 * Returns STENCIL_EINVAL, STENCIL_ENOMEM, STENCIL_ECUDA.
 */
int stencil_residual(const stencil_grid_t *g, const void *u, const void *f, void *r,
                     double *d_norms2, void *ws, size_t ws_bytes, void *stream);

/*
 * Allocation-free variant of stencil_residual, for callers that cannot let a library
 * allocate device memory: cudaMalloc/cudaFree may synchronise the whole device, which a
 * latency-bound loop driving several streams cannot afford; a caching allocator may
 * already own nearly all device memory; some deployments forbid device allocation
 * after start-up.  The paper has no counterpart; it is a service of this library.
 * Same results as stencil_residual up to the summation order of the norms (r is
 * identical in exact arithmetic; both are within the library's FP64 tolerance).
 * Scratch: a fixed 128 KiB array in the library's device image (present on every GPU
 * that loads the library, until process exit); nothing is allocated by the call.
 * Limit: at most 524288 x-rows, i.e. (n[2]+1)*(n[1]+1) in 3D or n[1]+1 in 2D; larger
 * grids return STENCIL_EINVAL.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  Every call reuses the same array (its counter is cleared on the stream at
 * the start of each call), so calls that overlap on the GPU race and must be ordered by
 * the caller.  Arguments as for stencil_residual; dtype F64.
 * Returns STENCIL_EINVAL, STENCIL_ECUDA.
 */
int stencil_residual_noalloc(const stencil_grid_t *g, const void *u, const void *f, void *r,
                             double *d_norms2, void *stream);

/* Options and report of stencil_solve. */
typedef struct stencil_solve_opts {
  double rel_tol;   /* stop when ||f - A u||_2 / ||f||_2 <= rel_tol (interior vertices) */
  int max_outer;    /* at most this many corrections */
  int inner_sweeps; /* coloured GS sweeps per correction, from a zero correction */
  int inner_dtype;  /* STENCIL_F64, STENCIL_F32 or STENCIL_BF16 (the last two: 3D only) */
} stencil_solve_opts_t;

typedef struct stencil_solve_info {
  int iterations;          /* corrections applied */
  int converged;           /* 1 if rel_tol was reached */
  double relres;           /* relative residual of the returned u */
  double *relres_history;  /* optional host array of max_outer + 1 entries (or NULL):
                              relative residual before each correction and at the end */
} stencil_solve_info_t;

/*
 * Iterative refinement for A u = f with the coloured Gauss-Seidel smoother as inner
 * solver (the multigrid-smoother use of Section 1; the precision split is this
 * library's).  Each outer iteration: r = f - A u and both norms in FP64 (fixed-order
 * reduction); stop when ||r|| / ||f|| <= rel_tol; round r to inner_dtype (bf16 via FP32,
 * nearest even); from e = 0 run inner_sweeps coloured GS sweeps on A e = r, stored and
 * computed in inner_dtype (bf16: FP32 arithmetic, every store rounded); u += e in FP64.
 * u: device F64 array (in: initial guess and Dirichlet data; out: result); f: device
 * F64.  g->dtype must be STENCIL_F64.  Host-synchronous: returns after the last
 * iteration (it synchronises `stream` once per outer iteration to read the norm).
 * Uses library workspaces of a few arrays of u's size (kept per stream).
 * Returns STENCIL_OK, STENCIL_ENOTCONV (u holds the last iterate), STENCIL_EINVAL,
 * STENCIL_ENOMEM, STENCIL_ECUDA.
 */
int stencil_solve(const stencil_grid_t *g, double *u, const double *f, const stencil_solve_opts_t *opts,
                  stencil_solve_info_t *info, void *stream);

/* ------------------------------------------------------------ dependency-driven sweeps */
/* The GPU form of the paper's Hyb-depend variant (Section 5, Algorithm 1): red-black
 * sweeps of the finite-difference operator (op = STENCIL_OP_FD) as tasks with data
 * dependencies instead of grid-wide barriers.  The grid is cut into blocks (2D: `rows`
 * x-rows; 3D: `rows` z-planes by `cols` y-rows); task (phase p = 2 sweep + colour,
 * block b) updates one colour of block b in place once b and its face-neighbour blocks
 * have finished phase p-1.  Tasks
 * are claimed by one persistent cooperative launch in phase-major order (the colouring
 * as issue order).  The result equals stencil_smooth_coloured with op FD (the same
 * updates in the same per-vertex order). */
typedef struct stencil_depend_opts {
  int32_t rows;        /* x-rows (2D) or z-planes (3D) per task; 0: 8 (2D), 1 (3D) */
  int32_t cols;        /* 3D: y-rows per task (blocks are numbered z-major); 0: 32 */
  int32_t ctas;        /* CTAs of the persistent launch; 0: every CTA that can be resident */
  int32_t test_stall;  /* testing only: if > 0, block test_stall - 1 never reports its
                          progress, so that a wait runs out; 0: off */
  int64_t max_wait_ns; /* limit of one dependency wait in ns; 0: 1e9 (1 s) */
  int32_t stalled_at;  /* out: the block a timed-out wait was waiting for */
  int32_t reserved;
} stencil_depend_opts_t;

/*
 * `sweeps` red-black Gauss-Seidel sweeps on A u = f, dependency-driven.  u, f: device F64
 * arrays of g's layout (g->op must be STENCIL_OP_FD).  Host-synchronous (reads the
 * launch's error flag).  Uses a small library workspace (per stream, kept).
 * Returns STENCIL_OK; STENCIL_ETIMEDOUT if a dependency wait exceeded max_wait_ns (u is
 * then partly updated; opts->stalled_at names the block waited for; the CUDA context
 * stays usable); STENCIL_EINVAL, STENCIL_ENOMEM, STENCIL_ECUDA (also if the device has
 * no cooperative launch).
 */
int stencil_smooth_depend(const stencil_grid_t *g, double *u, const double *f, int sweeps,
                          stencil_depend_opts_t *opts, void *stream);

/* ------------------------------------------------------------ expensive stencils S(k) */
/* Section 2 gives every stencil evaluation S(k) a cost parameter k; Section 4 realises
 * k > 0 by adding k evaluations of sin to the prescribed entry, the same k on every
 * vertex (homogeneous) or k running linearly over the mesh (heterogeneous).  Here, for
 * the red-black finite-difference sweep, the diagonal entry of interior vertex p becomes
 *   2d + 2^-20 sigma_k(p) / k,  sigma_k(p) = sum_{m=1..k} sin(m idx_p 2^-20),
 * with idx_p the lexicographic index of p among the interior vertices, and
 * k(p) = kmax (STENCIL_COST_UNIFORM) or floor(kmax idx_p / N) over the N interior
 * vertices (STENCIL_COST_LINEAR: the first 1/kmax of the vertices use the plain stencil,
 * the next one sin evaluation, ...).  The operator changes by less than 2^-20 relative;
 * each update pays for its k FP64 sin evaluations. */
#define STENCIL_COST_NONE 0
#define STENCIL_COST_UNIFORM 1
#define STENCIL_COST_LINEAR 2

/*
 * `sweeps` red-black sweeps of S(k) on A u = f (g->op must be STENCIL_OP_FD; F64), in
 * place on u.  depend == NULL: one launch per colour pass (colouring with barriers);
 * otherwise the dependency-driven sweep of stencil_smooth_depend with those options
 * (host-synchronous, may return STENCIL_ETIMEDOUT).  mode STENCIL_COST_NONE gives the
 * plain sweep with the update written as (h^2 f + neighbours) / 2d.
 * Returns STENCIL_OK, STENCIL_EINVAL, STENCIL_ENOMEM, STENCIL_ETIMEDOUT, STENCIL_ECUDA.
 */
int stencil_smooth_expensive(const stencil_grid_t *g, double *u, const double *f, int sweeps, int cost_mode,
                             int kmax, stencil_depend_opts_t *depend, void *stream);

/* ------------------------------------------------------------ geometric multigrid */
/* The paper's sweeps are the smoothers of matrix-free multigrid codes (Section 1).
 * Hierarchy: the coarse grid has n/2 cells per axis when every n[a] is even (every
 * second vertex), or ceil(n/2) on every axis when all n[a] are equal (coarse vertices
 * then not nested in the fine ones); coarse cells are cubes of side h n / n_c; grids are
 * coarsened while every n[a] >= 4 (any other grid is its own coarsest grid).
 * Prolongation P is d-linear interpolation at the fine vertex positions; restriction
 * is R = (n_c/n)^d P^T (full weighting for nested grids, where R A_h P = A_2h holds for
 * the Q1 operator).  V(pre, post) cycle: `pre` coloured GS sweeps; r = f - A u (FP64);
 * coarse right-hand side R r; coarse correction from 0 by a V-cycle (on the coarsest
 * grid: `coarse_sweeps` sweeps); u += P e; `post` sweeps. */
typedef struct stencil_mg_opts {
  double rel_tol;        /* solve: stop when ||f - A u||_2 / ||f||_2 <= rel_tol */
  int32_t max_cycles;    /* solve: at most this many V-cycles */
  int32_t pre;           /* GS sweeps before the coarse correction (>= 0) */
  int32_t post;          /* GS sweeps after it (>= 0) */
  int32_t coarse_sweeps; /* GS sweeps on the coarsest grid (>= 1) */
  int32_t max_levels;    /* at most this many grids (0: as many as the sizes allow) */
  int32_t reserved;      /* 0 */
} stencil_mg_opts_t;

typedef struct stencil_mg_info {
  int32_t cycles;          /* V-cycles applied */
  int32_t converged;       /* 1 if rel_tol was reached */
  int32_t levels;          /* grids in the hierarchy used */
  int32_t reserved;
  double relres;           /* relative residual of the returned u */
  double *relres_history;  /* optional host array of max_cycles + 1 entries (or NULL):
                              relative residual before each cycle and at the end */
} stencil_mg_info_t;

/*
 * V-cycles for A u = f until ||f - A u|| / ||f|| <= rel_tol.  u: device F64 array (in:
 * initial guess and Dirichlet data, which are never changed; out: result); f: device F64
 * of the same layout (boundary ignored).  g->dtype must be STENCIL_F64, 2D or 3D.
 * Host-synchronous (synchronises `stream` once per cycle to read the norm).  Uses
 * library workspaces (per stream, kept): the coarse-level arrays (about 3/7 (3D) or 1
 * (2D) of u's size plus one u-sized residual) and the smoother's three u-sized arrays.
 * Returns STENCIL_OK, STENCIL_ENOTCONV (u holds the last iterate), STENCIL_EINVAL,
 * STENCIL_ENOMEM, STENCIL_ECUDA.
 */
int stencil_mg_solve(const stencil_grid_t *g, double *u, const double *f, const stencil_mg_opts_t *opts,
                     stencil_mg_info_t *info, void *stream);

/* One V-cycle on u, stream-ordered (no host synchronisation; rel_tol and max_cycles
 * are ignored).  Same arrays, workspaces and errors as stencil_mg_solve. */
int stencil_mg_vcycle(const stencil_grid_t *g, double *u, const double *f, const stencil_mg_opts_t *opts,
                      void *stream);

/* Restriction rc = R rf from a fine grid to its coarse grid in the hierarchy above (the
 * coarse descriptor must have exactly those cell counts; any pitch; same dim; its h is
 * not used): coarse interior vertices get the weighted sum, the coarse boundary 0.
 * Device F64 arrays; rf and rc must not overlap.  Returns STENCIL_EINVAL, STENCIL_ECUDA. */
int stencil_mg_restrict(const stencil_grid_t *fine, const double *rf, const stencil_grid_t *coarse, double *rc,
                        void *stream);

/* uf += P ec on the fine interior (d-linear interpolation of ec, all coarse vertices
 * read, boundary included); the fine boundary is not written.  Grids as for
 * stencil_mg_restrict.  Returns STENCIL_EINVAL, STENCIL_ECUDA. */
int stencil_mg_prolong_add(const stencil_grid_t *fine, double *uf, const stencil_grid_t *coarse, const double *ec,
                           void *stream);

/* ------------------------------------------------------------ patch batches */
/* One cubic patch of a batch: a dense (n+1)^3 vertex array, x fastest, at element
 * offset `offset` of the packed FP64 buffers.  Its boundary shell is a halo. */
typedef struct stencil_patch_desc {
  int32_t n;        /* cells per edge, 2..64 */
  int32_t reserved; /* 0 */
  int64_t offset;   /* element offset of the patch in the packed arrays */
  double h;         /* mesh width; 0 selects 1/n (a unit cube per patch) */
} stencil_patch_desc_t;

typedef struct stencil_batch stencil_batch_t; /* opaque */

/*
 * Creates a batch of `npatch` cubic patches, the regular patches of a block-structured
 * mesh (Section 2).  neighbours: host array of 27 int32 per patch, entry
 * (dx+1) + 3(dy+1) + 9(dz+1) naming the patch across the face/edge/corner in direction
 * (dx,dy,dz) (the centre entry is ignored), or -1 at the outer boundary.  Halo rule,
 * applied before every sweep: a shell vertex of p with outward direction d takes, from
 * q = neighbour(d), per axis the vertex of q nearest to its position (ties to the lower
 * index) clamped into [1, n_q - 1]; with no neighbour the value is 0.  Copies the
 * tables to the current device.  Returns STENCIL_EINVAL, STENCIL_ENOMEM.
 */
int stencil_patch_batch_create(const stencil_patch_desc_t *patches, int32_t npatch, const int32_t *neighbours,
                               stencil_batch_t **out);

/*
 * `sweeps` repetitions of [halo fill of every patch, one coloured Gauss-Seidel sweep of
 * every patch (colours as in stencil_smooth_coloured, each patch on its own grid with
 * f_all)].  All patches of a sweep run in one persistent launch; CTAs take patches
 * largest first.  u_all (in/out), f_all: device FP64 packed arrays.  Asynchronous.
 */
int stencil_patch_batch_smooth(stencil_batch_t *b, double *u_all, const double *f_all, int sweeps, void *stream);

/* Times a few launch shapes (threads per CTA x CTAs per SM) on a scratch copy of u_all
 * and keeps the fastest for later smooth calls.  Host-synchronous; u_all is not
 * modified.  Returns STENCIL_ENOMEM if the scratch copy cannot be allocated. */
int stencil_patch_batch_autotune(stencil_batch_t *b, const double *u_all, const double *f_all, void *stream);

/* The launch shape the batch uses (after autotuning, or the default 256 x 4). */
int stencil_patch_batch_config(const stencil_batch_t *b, int32_t *threads, int32_t *ctas_per_sm);

/* Frees the batch's device tables (not the caller's arrays). */
int stencil_patch_batch_destroy(stencil_batch_t *b);

/* ------------------------------------------------------------ request server */
#define STENCIL_REQ_SMOOTH 0
#define STENCIL_REQ_SOLVE 1

typedef struct stencil_server stencil_server_t; /* opaque */

typedef struct stencil_server_opts {
  int32_t streams;      /* CUDA streams requests are spread over (0: 8) */
  int32_t max_inflight; /* requests resident and in progress at once (0: 64) */
  int32_t inner_sweeps; /* SOLVE: coloured GS sweeps per correction (0: 8) */
  int32_t inner_dtype;  /* SOLVE: STENCIL_F32 (default), STENCIL_BF16 or STENCIL_F64 */
  int32_t max_outer;    /* SOLVE: at most this many corrections or V-cycles (0: 100000) */
  int32_t solver;       /* SOLVE: STENCIL_SOLVER_REFINE (0: iterative refinement with the
                           GS inner solver above) or STENCIL_SOLVER_MG (FP64 multigrid
                           V(2,2) cycles, 20 sweeps on the coarsest grid; a grid with
                           an odd cell count is its own coarsest grid) */
} stencil_server_opts_t;

#define STENCIL_SOLVER_REFINE 0
#define STENCIL_SOLVER_MG 1

typedef struct stencil_request {
  int32_t kind;      /* STENCIL_REQ_SMOOTH or STENCIL_REQ_SOLVE */
  int32_t n;         /* cells per edge of the unit-cube grid (h = 1/n), 2..2048 */
  int32_t sweeps;    /* SMOOTH: coloured GS sweeps */
  int32_t reserved;
  double rel_tol;    /* SOLVE: stop when ||f - A u|| / ||f|| <= rel_tol */
  const double *f;   /* host (n+1)^3 FP64 right-hand side, copied by submit; or NULL: */
  uint64_t f_seed;   /*   f_i = U[-1,1) from SplitMix64 at counter i (interior), 0 on the boundary */
  const double *u0;  /* host (n+1)^3 initial guess incl. Dirichlet data, or NULL (zeros) */
} stencil_request_t;

typedef struct stencil_result {
  int32_t status;    /* STENCIL_OK, STENCIL_ENOTCONV (solve hit max_outer), STENCIL_ECUDA */
  int32_t iterations; /* SMOOTH: sweeps; SOLVE: corrections */
  double relres;     /* SOLVE: relative residual of the result */
  double t_submit, t_admit, t_done; /* seconds since the server was created */
} stencil_result_t;

typedef struct stencil_server_stats {
  int64_t submitted, completed, pending, inflight;
  uint64_t hbm_used, hbm_budget;
} stencil_server_stats_t;

/*
 * Creates a request server on the current device with a device-memory budget.  A host
 * engine thread admits queued requests in arrival order (looking past a blocked head
 * at the next few) whenever a request's footprint fits the remaining budget and an
 * in-flight slot is free, keeps its grids resident on the device and advances all
 * admitted requests concurrently on several streams (continuous batching): SMOOTH =
 * `sweeps` coloured GS sweeps (as stencil_smooth_coloured); SOLVE = the refinement of
 * stencil_solve, one correction per step.  A request's result does not depend on the
 * other requests.  The paper's use case is the multigrid smoother (Section 1); the
 * serving loop is this library's.  Returns STENCIL_EINVAL, STENCIL_ECUDA.
 */
int stencil_server_create(size_t hbm_budget_bytes, const stencil_server_opts_t *opts, stencil_server_t **out);
/* Queues a request (copies its host arrays).  STENCIL_EADMIT if its footprint exceeds
 * the whole budget (it could never be admitted). */
int stencil_server_submit(stencil_server_t *s, const stencil_request_t *req, uint64_t *ticket);
/* Non-blocking: STENCIL_OK with the result once done, STENCIL_EBUSY before. */
int stencil_server_poll(stencil_server_t *s, uint64_t ticket, stencil_result_t *res);
/* Blocks until done or timeout_us (negative: no limit): STENCIL_ETIMEDOUT. */
int stencil_server_wait(stencil_server_t *s, uint64_t ticket, int64_t timeout_us, stencil_result_t *res);
/* Copies a finished request's (n+1)^3 FP64 result to host memory and releases it. */
int stencil_server_fetch(stencil_server_t *s, uint64_t ticket, double *u_host);
/* Releases a finished request without copying its result. */
int stencil_server_release(stencil_server_t *s, uint64_t ticket);
int stencil_server_stats(stencil_server_t *s, stencil_server_stats_t *st);
/* Stops the engine (waits for work in flight) and frees everything. */
int stencil_server_destroy(stencil_server_t *s);

/* Frees the internal workspaces of the current device (not thread-safe against
 * concurrent calls on that device). */
int stencil_release_workspace(void);

/* Bits of stencil_device_status: a kernel's bounded wait on a TMA plane load ran out
 * and the CTA left without its outputs (the results of that call are incomplete). */
#define STENCIL_STATUS_TMA_OPS3 1u   /* 3D applies, Jacobi step, residual */
#define STENCIL_STATUS_TMA_GS3 2u    /* 3D Gauss-Seidel half sweeps */
#define STENCIL_STATUS_TMA_JAC3 4u   /* 3D multi-sweep Jacobi */
#define STENCIL_STATUS_TMA_GS_LP 8u  /* 3D FP32 / bf16 Gauss-Seidel */

/*
 * *flags = the STENCIL_STATUS_* bits set on the current device since the flags were
 * last cleared (0: every bounded device wait completed); clear != 0 clears them.  The
 * paper has no counterpart: the kernels bound every wait (a TMA completion, a
 * neighbour's progress), and this call reports the ones that ran out, which an
 * asynchronous call cannot return.  Synchronises the device first.
 * Returns STENCIL_EINVAL (flags NULL), STENCIL_ECUDA.
 */
int stencil_device_status(uint32_t *flags, int clear);

/* ---------------------------------------------------------------- launch-shape tuning
 * The plane-streaming 3D kernels process a chunk of z-planes per CTA and the 2D kernels
 * a chunk of rows per warp; the 2D multi-sweep smoothers run one or two sweeps per pass
 * over memory.  The built-in rule picks these from the grid size and the SM count;
 * stencil_autotune measures the alternatives instead.  The paper has no counterpart (its
 * Sections 5-6 discuss tile sizes and the fusion of colours as the levers of a
 * coloured sweep).  Tuned shapes apply to F64 Q1 calls of the same call kind, grid
 * shape (n, pitch) and device name, process-wide.  The smoothers give identical bits
 * under every chunk; the 2D depth (one fixed-point scale for the two sweeps of a pass)
 * and, in the single-pass applies, the per-CTA (3D) or per-warp (2D) fixed-point scale
 * make results differ between shapes by rounding only (within the FP64 tolerance).
 */
typedef struct stencil_tuning {
  int32_t chunk; /* 3D: z-planes per CTA; 2D: rows per warp (even); 0 = built-in rule */
  int32_t depth; /* 2D GS/Jacobi: sweeps per pass over memory, 1 or 2; 0 = built-in (2) */
  double ms;     /* stencil_autotune: time of one call with this shape, else as set */
} stencil_tuning_t;

/*
 * Times every candidate shape of `call` (STENCIL_CALL_APPLY_ELEMENTWISE,
 * STENCIL_CALL_APPLY_STENCIL, STENCIL_CALL_SMOOTH_COLOURED with `sweeps` sweeps,
 * STENCIL_CALL_SMOOTH_JACOBI with omega 2/3) on grid g, on scratch arrays it allocates
 * and fills itself (3D candidates: 4, 8, 16, 32 planes per CTA, 2..16 for GS; 2D: 16..256
 * rows per warp for the applies, 64..1024 rows x 1 or 2 sweeps per pass for the
 * smoothers), one untimed call and the best of three per candidate, CUDA events on
 * `stream`.  Records the fastest for (device, call, g) and returns it in *out.
 * Blocking (synchronises the stream); allocates about four arrays of g's size, plus the
 * call's workspace, and frees them before returning.  Run it when no other thread
 * launches calls on this grid shape.  F64, STENCIL_OP_Q1; smoothers 2..1000 sweeps.
 * Returns STENCIL_EINVAL, STENCIL_ENOMEM, STENCIL_ECUDA.
 */
int stencil_autotune(const stencil_grid_t *g, int call, int sweeps, stencil_tuning_t *out, void *stream);

/* Sets (t != NULL) or removes (t == NULL) the shape used for (device, call, g). */
int stencil_tuning_set(const stencil_grid_t *g, int call, const stencil_tuning_t *t);
/* The recorded shape for (device, call, g); STENCIL_ENOTFOUND if there is none. */
int stencil_tuning_get(const stencil_grid_t *g, int call, stencil_tuning_t *t);
/* Forgets every recorded shape. */
int stencil_tuning_clear(void);
/*
 * Writes every recorded shape to `path` as JSON ({"format": "stencil_gb300_tuning",
 * "version": 1, "entries": [{"device", "call", "dim", "n": [nx, ny, nz], "pitch",
 * "chunk", "depth", "ms"}, ...]}), through a temporary file renamed into place; or
 * reads such a file and adds its entries (all or none).  The first tuning lookup of the
 * process also loads the file named by the environment variable STENCIL_TUNING_CACHE,
 * if that file exists, so a saved cache steers later processes without code changes.
 * Returns STENCIL_EINVAL for an unreadable/unwritable path or a malformed file.
 */
int stencil_tuning_save(const char *path);
int stencil_tuning_load(const char *path);

#ifdef __cplusplus
}
#endif
#endif /* STENCIL_GB300_H */
