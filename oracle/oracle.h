/*
 * Oracle for the coloured stencil codes of Hazelwood & Weinzierl,
 * "Coloured and task-based stencil codes" (arXiv:1810.04033).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU statement of what the
 * GPU library computes.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA library and the library never calls it.
 *
 * Grid convention (all functions):
 *   dim  = 2 or 3.  n[0], n[1], n[2] = cells along x, y, z (n[2] is ignored for dim 2).
 *   Vertices 0..n[a] per axis; the array holds every vertex, x fastest:
 *   index(i,j,k) = (k*(n[1]+1) + j)*(n[0]+1) + i.   Boundary vertices (an index equal
 *   to 0 or n[a]) carry Dirichlet data and are never written by a smoother.
 *   h = mesh width (cells are squares / cubes of side h).
 *   Colour of vertex or cell (i,j,k) = (i&1) + 2(j&1) + 4(k&1)  (2D: (i&1) + 2(j&1)),
 *   colours are visited in ascending order (Section 3, "Colouring": 2^d colours,
 *   one pass per colour, updates inside a pass independent).
 *
 * The operator is the Q1 (d-linear) finite-element Laplacian divided by the lumped
 * mass h^d, i.e. A = S/h^2 with S the assembled 3^d-point stencil; in 2D S is the
 * 9-point stencil the paper prints in Fig. 1 (centre 8/3, neighbours -1/3).
 */
#ifndef STENCIL_ORACLE_H
#define STENCIL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element stiffness matrix K_e (2^d x 2^d, row-major, local vertex v = bx + 2by + 4bz)
 * built from the 1D stiffness [1 -1; -1 1]/h and 1D mass h/6 [2 1; 1 2] by tensor
 * products (Section 2: cell-wise weighted sums; 9-point FE stencil of Fig. 1). */
void oracle_q1_element_matrix(int dim, double h, double *Ke);

/* Assembled stencil weight S at offset (dx,dy,dz) in {-1,0,1}^d (h-free). */
double oracle_stencil_weight(int dim, int dx, int dy, int dz);

/* y = A u by cell-wise element scatter in 2^d-colour order (Section 2 blueprint,
 * Section 3 colouring); interior rows divided by h^d, boundary rows set to 0.
 * nthreads > 1 splits each colour pass over rows of cells (same-colour cells share
 * no vertex); the result does not depend on nthreads. */
void oracle_apply_elementwise(int dim, const int64_t *n, double h,
                              const double *u, double *y, int nthreads);

/* y = A u by the assembled stencil (gather, separate output array: Section 2,
 * matrix-vector product); boundary rows 0. */
void oracle_apply_stencil(int dim, const int64_t *n, double h,
                          const double *u, double *y, int nthreads);

/* `sweeps` in-situ coloured Gauss-Seidel sweeps on A u = f (Section 2 in-situ update,
 * Section 3 colouring).  nthreads > 1 splits each colour pass with OpenMP
 * `parallel for` over the outer loop, as the paper's colouring does; the result does
 * not depend on nthreads. */
void oracle_gs_coloured(int dim, const int64_t *n, double h, double *u,
                        const double *f, int sweeps, int nthreads);

/* Same sweeps in FP32 arithmetic and storage (inner solver of the refinement loop). */
void oracle_gs_coloured_f32(int dim, const int64_t *n, double h, float *u,
                            const float *f, int sweeps);

/* Same sweeps with bf16 storage (round to nearest even on every store) and FP32
 * arithmetic.  u, f hold raw bf16 bit patterns. */
void oracle_gs_coloured_bf16(int dim, const int64_t *n, double h, uint16_t *u,
                             const uint16_t *f, int sweeps);

/* Damped Jacobi, out of place: u <- u + omega * D^-1 (f - A u), boundary copied.
 * work has the size of u; the result of the last sweep is left in u. */
void oracle_jacobi(int dim, const int64_t *n, double h, double *u,
                   const double *f, double *work, double omega, int sweeps,
                   int nthreads);

/* r = f - A u on interior vertices (0 on the boundary; r may be NULL) and
 * norms2[0] = sum r_i^2, norms2[1] = sum f_i^2 over interior vertices,
 * summed in lexicographic order by one thread (r itself may be computed by
 * nthreads threads; the result does not depend on nthreads). */
void oracle_residual(int dim, const int64_t *n, double h, const double *u,
                     const double *f, double *r, double *norms2, int nthreads);

/* The two norms of oracle_residual computed in long double throughout from the same
 * FP64 inputs (rounded to double on return): a near-exact value that bounds the FP64
 * oracle's own rounding. */
void oracle_residual_ld(int dim, const int64_t *n, double h, const double *u,
                        const double *f, double *norms2_ld);

/* Mixed-precision iterative refinement (see oracle.c for the steps).
 * inner_prec: 0 = FP64, 1 = FP32, 2 = bf16 storage / FP32 arithmetic.
 * x (in/out) holds the FP64 iterate incl. its Dirichlet boundary.
 * relres[0..max_outer] receives ||r||/||f|| before each correction (may be NULL).
 * x_hist, if non-NULL, receives the interior-and-boundary iterate after each
 * correction: x_hist[k * npts + p].  Returns the number of corrections made;
 * *converged = 1 if the relative residual reached tol. */
int oracle_ir_solve(int dim, const int64_t *n, double h, double *x,
                    const double *f, double tol, int max_outer, int inner_sweeps,
                    int inner_prec, double *relres, double *x_hist,
                    int *converged);

/* Halo fill of a lattice of cubic patches (rule in oracle.c), then `sweeps`
 * repetitions of [halo fill, one coloured GS sweep per patch].
 * lat[3] = patches per axis, np[p] = cells per edge of patch p (p = Px + lat0*(Py +
 * lat1*Pz)), off[p] = element offset of patch p in u_all / f_all, each patch dense
 * (np+1)^3 with h = 1/np. */
void oracle_patch_halo_fill(const int32_t *lat, const int32_t *np,
                            const int64_t *off, double *u_all);
void oracle_patch_smooth(const int32_t *lat, const int32_t *np,
                         const int64_t *off, double *u_all, const double *f_all,
                         int sweeps, int nthreads);

/* Geometric multigrid (Section 1: the sweeps as smoothers of multigrid codes).
 * Coarse grid nc: n/2 per axis when all n are even, else ceil(n/2) when all n are equal
 * (coarse vertices not nested); coarsened while every n >= 4.  Restriction of a fine
 * residual (R = (nc/nf)^d P^T, full weighting when nested; coarse boundary 0) and
 * d-linear prolongation added to the fine interior (uf += P ec, interpolating ec at
 * every coarse vertex, boundary included: in the V-cycle the coarse correction's
 * boundary is 0).
 * oracle_mg_levels: grids in the hierarchy.
 * oracle_mg_vcycle: one V(pre, post) cycle with coloured GS smoothing and
 * `coarse_sweeps` sweeps on the coarsest of `levels` grids.
 * oracle_mg_solve: V-cycles until ||f - A u|| / ||f|| <= tol (relres[k] before cycle
 * k); returns the number of cycles. */
int oracle_mg_levels(int dim, const int64_t *n, int max_levels);
void oracle_mg_restrict(int dim, const int64_t *nf, const int64_t *nc, const double *rf,
                        double *rc);
void oracle_mg_prolong_add(int dim, const int64_t *nf, const int64_t *nc, const double *ec,
                           double *uf);
void oracle_mg_vcycle(int dim, const int64_t *n, double h, double *u, const double *f,
                      int levels, int pre, int post, int coarse_sweeps);
int oracle_mg_solve(int dim, const int64_t *n, double h, double *u, const double *f,
                    double tol, int max_cycles, int levels, int pre, int post,
                    int coarse_sweeps, double *relres, int *converged);

/* 5-point (2D) / 7-point (3D) finite differences (Fig. 1 middle, Section 2) with the
 * red-black colouring of Section 3: A u = (2d u - sum of face neighbours) / h^2.
 * Red-black GS: first all interior vertices with (i+j+k) odd, then (i+j+k) even
 * (Algorithm 1's order with its 1-based unknowns on our interior vertices).
 * Jacobi: u <- u + omega h^2/(2d) (f - A u), boundary copied.  Residual as
 * oracle_residual (sums in lexicographic order). */
double oracle_fd_weight(int dim, int dx, int dy, int dz);
void oracle_fd_apply(int dim, const int64_t *n, double h, const double *u, double *y);
void oracle_fd_gs_redblack(int dim, const int64_t *n, double h, double *u,
                           const double *f, int sweeps);
void oracle_fd_jacobi(int dim, const int64_t *n, double h, double *u, const double *f,
                      double *work, double omega, int sweeps);
void oracle_fd_residual(int dim, const int64_t *n, double h, const double *u,
                        const double *f, double *r, double *norms2);

/* Expensive stencil evaluations S(k) (Section 2; Section 4: k sin evaluations added to
 * the prescribed entry, k = kmax everywhere or running linearly over the mesh), for the
 * red-black FD sweep.  mode: 0 none, 1 uniform k = kmax, 2 linear k = floor(kmax idx/N).
 * oracle_cost_diagonal: the diagonal entry 2d + 2^-20 sigma_k / k of vertex (i,j,k)
 * (definition in oracle.c).  oracle_fd_gs_redblack_cost: the sweep with it. */
double oracle_cost_diagonal(int dim, const int64_t *n, int mode, int kmax, int64_t i,
                            int64_t j, int64_t k);
void oracle_fd_gs_redblack_cost(int dim, const int64_t *n, double h, double *u,
                                const double *f, int sweeps, int mode, int kmax);

/* Round-to-nearest-even conversion helpers exposed for tests. */
uint16_t oracle_f32_to_bf16(float x);
float oracle_bf16_to_f32(uint16_t b);

#ifdef __cplusplus
}
#endif
#endif
