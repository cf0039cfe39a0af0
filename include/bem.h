/*
 * bem.h -- C ABI of the GB300 (sm_103a) dense P0 single-layer BEM capacity library.
 *
 * The library computes the electrostatic capacity of a closed polyhedral surface
 * Gamma by the Galerkin boundary element method of Betcke, Haberl and Praetorius,
 * "Adaptive boundary element methods for the computation of the electrostatic
 * capacity on complex polyhedra" (arXiv 1901.08393), in its primal piecewise-
 * constant form (App. A, Eq. A.1):
 *
 *   V[i][j] = (1/4pi) int_Ti int_Tj 1/|x-y| dy dx          (Eq. 2.1, 2.4-2.5)
 *   solve V x = b, b[i] = |T_i|                             (Eq. 2.5 with f = 1)
 *   Cap = (1/4pi) sum_i |T_i| x_i                           (Eq. 2.8)
 *   eta(T)^2 = diam(T) ||x_T - I x||^2_{L2(T)}              (Eq. 1.6, Sec. 2.4)
 *   Doerfler marking, newest-vertex bisection               (Eq. 2.6, Alg. 1, Fig. 3)
 *
 * Conventions (all entry points):
 *   - Every call returns a bem_status: 0 on success, a negative code otherwise;
 *     bem_last_error(ctx) then holds a message.  No C++ exception crosses the ABI.
 *   - Handles (bem_ctx, bem_mesh, bem_operator) are owned by the library and freed
 *     by the matching *_destroy.  Arrays passed in are owned by the caller and only
 *     borrowed for the duration of the call; the library never keeps a pointer.
 *   - Array arguments may be host or device (CUDA) memory; the library inspects
 *     each pointer (cudaPointerGetAttributes) and copies as needed.
 *   - All GPU work is enqueued on the context's CUDA stream.  Calls that return
 *     values through host pointers synchronise that stream before returning.
 *   - Layouts: vertices M x 3 float64 row-major (x,y,z per vertex); triangles
 *     N x 3 int32 row-major, 0-based vertex indices.  V (float64 or float32 by
 *     precision) lives on the device, row-major with each row padded to a multiple
 *     of 64 entries; bem_operator_read returns compact row-major blocks.
 *   - Meshes must be closed (every edge shared by an even number >= 2 of
 *     triangles; non-manifold edges are allowed) with non-degenerate triangles;
 *     otherwise BEM_ERR_MESH.
 */
#ifndef BEM_GB300_H
#define BEM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t bem_status;
#define BEM_OK 0
#define BEM_ERR_INVALID (-1)        /* bad argument (null handle, size out of range) */
#define BEM_ERR_OOM (-2)            /* device allocation failed or HBM budget exceeded */
#define BEM_ERR_NOT_CONVERGED (-3)  /* Krylov solve hit max_it before the tolerance */
#define BEM_ERR_MESH (-4)           /* mesh not closed, degenerate or too irregular */
#define BEM_ERR_CUDA (-5)           /* CUDA runtime error */

typedef struct bem_ctx bem_ctx;
typedef struct bem_mesh bem_mesh;
typedef struct bem_operator bem_operator;

/* Storage/arithmetic precision of V. */
#define BEM_PREC_F64 0  /* V stored and applied in native FP64 */
#define BEM_PREC_F32 1  /* V stored in FP32 (near field computed in FP64, rounded) */
#define BEM_PREC_DF64 2 /* FP64-accurate "double-float": V stored as pairs hi + lo of FP32
                           (48-bit significand, entries within ~4e-15 relative of FP64);
                           far field and V x computed with error-free FP32 transformations
                           on the FP32 pipe, near field in FP64 */

typedef struct {
    int32_t precision; /* BEM_PREC_F64, BEM_PREC_F32 or BEM_PREC_DF64 */
    int32_t ss_order;  /* Gauss-Legendre points per variable for touching pairs (2..16, default 4;
                          the radial variables are integrated exactly, which equals the
                          n-point rule in them for n >= 2) */
    int32_t tile;      /* far-field pair tile (no counterpart in the paper; V is bit-identical
                          for every choice): 0 = autotuned -- the first assembly of each size
                          class (N < 1,024, < 4,096, < 16,384, larger) and precision in a
                          context times every variant on its own far-field block and the
                          context keeps the fastest; k = 1..BEM_FAR_TILE_VARIANTS: variant k,
                          rows x columns per CTA 32x256, 16x256, 64x256, 8x128, 16x128, 32x128,
                          and (DF64: point loops rolled, at least m CTAs per SM) 8x128 m8,
                          16x128 m8, 32x128 m8, 8x128 m9, 8x64 m16, 8x64 m18, and with the
                          point loops unrolled 8x128 m6, 32x128 m6 */
} bem_assembly_opts;
#define BEM_FAR_TILE_VARIANTS 14

#define BEM_PRECOND_NONE 0
#define BEM_PRECOND_JACOBI 1
/* Block Jacobi on spatial clusters: the triangles sorted by the Morton code of their
 * centroid (10 bits per axis over the centroids' bounding box, ties by index) form
 * consecutive clusters of 64; M = the block diagonal of V over the clusters, each
 * block inverted in FP64 (Cholesky).  DF64 operators, persistent solver. */
#define BEM_PRECOND_BLOCK 2
/* Operator preconditioning with the regularised hypersingular operator (Sec. 2.6),
 * for dual operators (bem_operator_dual): C = S D^reg S with D^reg = sum_m Q_m^T V^bary
 * Q_m + a a^T and S the degree-6 Chebyshev approximation of M^-1 (M the mass matrix of
 * hats against dual cells, Jacobi-scaled spectrum in [15/22, 36/22]; S agrees with M^-1
 * to 2e-4 relative), formed once with the operator (FP32, M x M) and applied as one
 * product per iteration.  C is SPD, so CG on V^dual x = f with C has the spectrum of the
 * paper's M^-T V^dual M^-1 D^reg (solved there by GMRES) and reaches the same x.
 * DF64 dual operators, persistent solver, not in a batch. */
#define BEM_PRECOND_CALDERON 3

typedef struct {
    double tol;            /* relative residual ||b - V x|| / ||b|| to reach (e.g. 1e-10) */
    int32_t max_it;        /* iteration cap (inner iterations for FP32 operators) */
    int32_t precond;       /* BEM_PRECOND_NONE, _JACOBI (diag(V), Sec. 3), _BLOCK or _CALDERON */
    int32_t max_outer;     /* FP32 operators: FP64 iterative-refinement sweeps (default 20) */
    double inner_tol;      /* FP32 operators: relative tolerance of each inner solve (default 1e-5) */
    double reliable_delta; /* DF64 operators, persistent solver: the iteration's products use the
                              FP32 hi parts of V (a packed copy of the upper triangle, 2 N^2 bytes
                              while the solve runs), and r is replaced by b - V x formed with the
                              DF64 product whenever ||r|| has dropped by this factor since the
                              last such residual and before convergence is declared, so tol
                              holds for the DF64 operator.  0: default 1e-4; < 0 or >= 1: DF64
                              products only */
    double inexact_lambda; /* > 0 (persistent solver): stop as soon as the update's energy norm
                              |||x_k - x_(k-1)||| <= inexact_lambda * eta(x_k), eta the ZZ estimator
                              of the iterate (Remark (i) after Alg. 1; the paper uses ~1e-3);
                              such a stop counts as converged.  0: off (tol only) */
    int32_t h_mode;        /* ZZ weight of that estimator, as bem_zz_estimate (bem_adaptive_run
                              takes its own h_mode) */
    int32_t products;      /* persistent solver, DF64 and FP32 operators: the source of the CG
                              iteration's products.  BEM_PRODUCTS_DEFAULT (0): _FP16 for FP32
                              operators under BEM_PRECOND_BLOCK, else _FP32.  _FP32: the packed FP32 copy with
                              double-float sums (above).  _FP16: a further copy in
                              FP16 (each 64 x 64 tile divided by a power of two above its largest
                              entry; N^2 bytes) with FP32 sums, the residual replaced by the
                              operator's own product (DF64, or the exact FP32 one) after every
                              10^2-fold drop of ||r|| (or after 400 iterations without it), and
                              the FP32 copy taken for the rest of the solve if a replaced residual
                              has fallen by less than 10x since the previous one.  tol holds for
                              the operator in every mode. */
} bem_solve_opts;
#define BEM_PRODUCTS_DEFAULT 0
#define BEM_PRODUCTS_FP32 1
#define BEM_PRODUCTS_FP16 2

typedef struct {
    int32_t iterations;    /* CG iterations (summed over refinement sweeps) */
    int32_t outer;         /* FP32 operators: refinement sweeps; DF64 operators: residuals formed
                              with the DF64 product (initial one included); FP64: 1 */
    double relres;         /* final ||b - V x|| / ||b|| in FP64 */
    int32_t converged;     /* 1 if relres <= tol */
    /* Estimates of the extreme eigenvalues of the preconditioned operator M^-1 V (the
     * condition number of Sec. 3, Figs. 6 and 12, is lambda_max / lambda_min): the
     * extreme eigenvalues of the Lanczos tridiagonal matrix formed from the CG
     * coefficients (diagonal 1/alpha_j + beta_(j-1)/alpha_(j-1), off-diagonal
     * sqrt(beta_j)/alpha_j).  Persistent solver only; 0 otherwise.  With residual
     * replacements (mixed precision) the recurrence is perturbed at those steps. */
    double lambda_min, lambda_max;
} bem_solve_info;

/* ---------------------------------------------------------------- context */
/* Create a context on the current CUDA device.  cuda_stream: a cudaStream_t (NULL:
 * the legacy default stream).  hbm_budget_bytes: device bytes the context may
 * allocate in total (<= 0: no limit).  */
bem_status bem_context_create(void *cuda_stream, int64_t hbm_budget_bytes, bem_ctx **out);
bem_status bem_context_destroy(bem_ctx *ctx);
/* Last error message of the context (never NULL; "" if none). */
const char *bem_last_error(const bem_ctx *ctx);
/* Device bytes currently held by handles of this context. */
bem_status bem_context_memory(const bem_ctx *ctx, int64_t *bytes_in_use);
/* The autotuned far-field tiles of the context: out[4 p + c] for precision p (BEM_PREC_*)
 * and size class c, the variant 1..BEM_FAR_TILE_VARIANTS, or 0 while not yet timed. */
bem_status bem_far_tiles(const bem_ctx *ctx, int32_t out[12]);

/* ---------------------------------------------------------------- mesh */
/* Upload a triangulation T_l of Gamma into N flat triangles with M vertices
 * (Sec. 2.1).  ref_edge (nullable, N bytes in 0..2) names each triangle's
 * reference edge for newest-vertex bisection (edge (v_e, v_{e+1 mod 3})); NULL
 * selects the longest edge, ties to the lowest local index.  Triangles are stored
 * rotated so that the reference edge comes first (orientation kept).
 * Also computes per-triangle area, diameter, quadrature points, the
 * vertex-to-triangle incidence and the list of touching pairs. */
bem_status bem_mesh_upload(bem_ctx *ctx, const double *verts, int64_t M, const int32_t *tris,
                           int64_t N, const uint8_t *ref_edge, bem_mesh **out);
bem_status bem_mesh_destroy(bem_mesh *mesh);
/* Sizes; n_near = number of touching ordered pairs i != j (shared vertex or edge). */
bem_status bem_mesh_info(const bem_mesh *mesh, int64_t *M, int64_t *N, int64_t *n_near);
/* Copy the stored (rotated) mesh out.  Any pointer may be NULL.  parent/kept are
 * filled for meshes made by bem_refine (parent = source triangle index in the
 * coarser mesh; kept = 1 if the triangle is that source triangle unchanged) and
 * are -1/0 for uploaded meshes. */
bem_status bem_mesh_download(const bem_mesh *mesh, double *verts, int32_t *tris,
                             int32_t *parent, uint8_t *kept);
/* Per-triangle area |T| and diam(T) (longest edge), FP64, in the fixed operation
 * order (no fused multiply-add) shared with the estimator. */
bem_status bem_mesh_geometry(const bem_mesh *mesh, double *area, double *diam);

/* ---------------------------------------------------------------- operator */
/* Assemble V on P0(T_l) (Eq. 2.4-2.5): pairs without a common vertex by the 7x7
 * product of Radon's degree-5 rule; pairs with a common vertex, a common edge, and
 * identical pairs by Sauter-Schwab regularising transformations in FP64 (the
 * paper defers these integrals to the Sauter-Schwab textbook).  V stays resident
 * on the device.  opts may be NULL (FP64, order 4). */
bem_status bem_assemble_V(bem_mesh *mesh, const bem_assembly_opts *opts, bem_operator **out);
/* Same operator for a mesh made by bem_refine from coarse's mesh: entries of pairs
 * of unrefined triangles are copied from coarse (their geometry and adjacency are
 * unchanged under conforming NVB), the others are computed.  Bit-identical to
 * bem_assemble_V on the same mesh. */
bem_status bem_assemble_V_update(bem_mesh *fine, const bem_operator *coarse,
                                 const bem_assembly_opts *opts, bem_operator **out);
/* An operator may be destroyed before or after its mesh; every other call on it
 * needs its mesh alive. */
bem_status bem_operator_destroy(bem_operator *op);
bem_status bem_operator_info(const bem_operator *op, int64_t *N, int32_t *precision);
/* Copy the block V[i0:i0+ni, j0:j0+nj] (row-major, ni x nj) into dst (host or
 * device): float64 for F64 and DF64 operators (DF64 entries as hi + lo), float32
 * for F32 operators. */
bem_status bem_operator_read(const bem_operator *op, int64_t i0, int64_t ni, int64_t j0,
                             int64_t nj, void *dst);
/* out[k] = V[I[k]][J[k]] as FP64 for K sampled entries (arrays host or device). */
bem_status bem_operator_entries(const bem_operator *op, const int64_t *I, const int64_t *J,
                                int64_t K, double *out);
/* y = V x, FP64 vectors of length N (host or device), in the operator's arithmetic. */
bem_status bem_operator_matvec(const bem_operator *op, const double *x, double *y);

/* No-allocation variant of bem_operator_matvec (the paper has no counterpart: it
 * serves callers that must not have device memory allocated during a call, such
 * as code being captured into a CUDA graph, where cudaMalloc and cudaFree are not
 * permitted, serving loops with a fixed pre-reserved footprint, and hosts whose
 * device memory belongs to another framework's allocator).  y = V x for a
 * BEM_PREC_DF64 operator with N <= 4096; x and y are FP64 device pointers of
 * length N (host pointers are rejected, staging them would allocate).  The
 * scratch is a static device array of about 2.1 MiB that every GPU loading the
 * library keeps until exit; the first call on a device looks up its address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * Enqueued on the context's stream without synchronising.  All calls share the
 * one array: calls that overlap on the GPU race.  Larger N, other precisions,
 * host pointers, device memory of another GPU or another current device:
 * BEM_ERR_INVALID with a message.  The looked-up address is kept for the life of
 * the process; it does not survive a cudaDeviceReset. */
bem_status bem_operator_matvec_noalloc(const bem_operator *op, const double *x, double *y);

/* ---------------------------------------------------------------- solve */
/* Solve V x = b, b[i] = |T_i|, by preconditioned CG (Jacobi: diag(V), the paper's
 * "diag" comparison preconditioner, Sec. 3), and return Cap = (1/4pi) b.x
 * (Eq. 2.8).  FP64 / DF64 operators: CG with FP64 recurrences.  FP32 operators:
 * FP64 iterative refinement (residual with FP64-accurate accumulation against the
 * stored FP32 V) around inner CG solves of the correction.
 * x0 (nullable) starts the iteration; phi_out (nullable) receives x.  Returns
 * BEM_ERR_NOT_CONVERGED (with cap and info filled) if tol is not reached. */
bem_status bem_solve_capacity(bem_operator *op, const bem_solve_opts *opts, const double *x0,
                              double *cap_out, double *phi_out, bem_solve_info *info);

/* ---------------------------------------------------------------- adaptivity */
/* ZZ-type indicators (Eq. 1.6), primal-P0 reading: the nodal value at vertex z is
 * the area-weighted mean of phi over the triangles at z (summed in ascending
 * triangle order), I phi the S1 interpolant of those values, and
 * eta(T)^2 = h_T |T|/12 (sum_k d_k^2 + (sum_k d_k)^2), d_k = u_{z_k} - phi_T, in
 * that operation order without fused multiply-add (bit-identical to a plain
 * IEEE-754 evaluation).  h_mode 0: h_T = diam(T) (Eq. 1.6); 1: h_T = |T|^{1/2}.
 * totals (nullable, 2 doubles): [sum_T eta^2, sum_T h_T |T| phi_T^2 / 12]. */
bem_status bem_zz_estimate(bem_mesh *mesh, const double *phi, int32_t h_mode, double *eta2_out,
                           double *totals);
/* Doerfler marking (Eq. 2.6): order the elements by decreasing eta^2 compared in
 * single precision (ties by index), accumulate eta^2 in FP64 in that order, mark
 * the shortest prefix reaching theta * total (total = the same ordered sum), and
 * extend it over elements whose single-precision indicator equals the last
 * marked one.  marked: N bytes (1 = marked).  Runs on the device. */
bem_status bem_dorfler(bem_ctx *ctx, const double *eta2, int64_t N, double theta, uint8_t *marked,
                       int64_t *n_marked);
#define BEM_REFINE_BISEC3 1 /* a marked triangle marks all three edges (default: reference edge) */
/* Newest-vertex bisection with closure (Fig. 3): marked triangles bisect their
 * reference edge (or all edges with BEM_REFINE_BISEC3); repeatedly, a triangle
 * with a marked edge marks its reference edge; each marked edge gets one new
 * vertex 0.5 (a + b), numbered after the old ones by first appearance in
 * (triangle, local edge) order; triangle (a,b,c) with midpoints m0 (ab), m1 (bc),
 * m2 (ca) becomes
 *   ab: (c,a,m0) (b,c,m0)          ab+bc: (c,a,m0) (m0,b,m1) (c,m0,m1)
 *   ab+ca: (m0,c,m2) (a,m0,m2) (b,c,m0)
 *   ab+bc+ca: (m0,c,m2) (a,m0,m2) (m0,b,m1) (c,m0,m1)
 * The new mesh lists the unrefined triangles first (in order), then the children,
 * parent by parent.  marked: N bytes.  Runs on the device. */
bem_status bem_refine(bem_mesh *mesh, const uint8_t *marked, int32_t flags, bem_mesh **refined_out);
/* bem_dorfler followed by bem_refine. */
bem_status bem_mark_refine(bem_mesh *mesh, const double *eta2, double theta, int32_t flags,
                           uint8_t *marked_out, int64_t *n_marked, bem_mesh **refined_out);

/* ---------------------------------------------------------------- adaptive loop */
typedef struct {
    int64_t N, M;          /* mesh size of this level */
    double cap;            /* Cap_l (Eq. 2.8) */
    double eta2_total;     /* sum of the ZZ indicators */
    int32_t iterations;    /* CG iterations */
    int32_t n_marked;      /* elements marked for the next level (0 on the last) */
    double relres;
    double ms_assemble, ms_solve, ms_adapt; /* device time per phase (CUDA events) */
    int32_t outer;          /* bem_solve_info.outer of the level's solve */
} bem_level_record;

typedef struct {
    double theta;           /* Doerfler parameter (Alg. 1), default 0.5 */
    int64_t max_N;          /* stop at the first level with N >= max_N */
    int32_t max_levels;     /* hard cap on levels */
    int32_t h_mode;         /* ZZ mesh-size weight, see bem_zz_estimate */
    bem_assembly_opts assembly;
    bem_solve_opts solve;
    int32_t incremental;    /* 1: reuse entries of unrefined pairs (bem_assemble_V_update) */
    int32_t basis;          /* BEM_BASIS_P0 (default) or BEM_BASIS_DUAL */
} bem_adaptive_opts;

/* Discrete space of the adaptive loop.  P0: piecewise constants on the triangles
 * (Eq. 2.5).  DUAL: piecewise constants on the dual cells (Sec. 2.1, 2.6): each level
 * builds the barycentric refinement, assembles its operator (assembly options; with
 * incremental, the children of unrefined primal triangles keep their entries from the
 * previous level's barycentric operator), forms V^dual (bem_operator_dual), solves
 * from zero, estimates with bem_zz_estimate_dual and marks and refines the primal
 * mesh; the warm start does not apply, and solve.inexact_lambda must be 0. */
#define BEM_BASIS_P0 0
#define BEM_BASIS_DUAL 1

/* Alg. 1: solve -> estimate -> mark -> refine, starting from the uploaded mesh, until
 * N >= max_N or max_levels, in the basis opts->basis (P0 on the triangles, or the
 * dual basis of Sec. 2.6, see BEM_BASIS_DUAL).  P0: the previous level's solution
 * copied to the children starts each solve.  When every indicator
 * vanishes up to rounding (sum eta^2 <= 1e-20 sum h|T|phi^2/12, a symmetric mesh
 * with a constant solution) Eq. 2.6 holds for the empty set and the level is
 * refined uniformly instead.  The checks of each refined mesh (closed, no degenerate
 * or duplicate triangle) are read with the sizes of the next refinement, or at the end
 * for the last mesh, so a failed check (BEM_ERR_MESH) ends the loop one level later.
 * records: caller array of max_levels entries; n_levels receives the count;
 * final_mesh (nullable) receives the last mesh (caller destroys it). */
bem_status bem_adaptive_run(bem_mesh *mesh, const bem_adaptive_opts *opts, bem_level_record *records,
                            int32_t *n_levels, bem_mesh **final_mesh);

/* ---------------------------------------------------------------- dual basis */
/* bem_operator_dual also forms the operator preconditioner of Sec. 2.6 from the same
 * V^bary (BEM_PRECOND_CALDERON): V^T = R^T V^bary R (the six children of each primal
 * triangle summed), D_ij = sum over T at i, T' at j of (curl phi_i|T . curl phi_j|T')
 * V^T[T][T'] with curl phi_k = (p_(k+1) - p_(k+2)) / (2 |T|) on T (the surface curl
 * n x grad of the hat of local vertex k), plus a_i a_j, a_i = |T_i^dual| = the integral
 * of the hat; then C = S D^reg S (S applied to the columns of D^reg, then to the columns
 * of the transpose); both stored in FP32 (8 M^2 bytes) with the operator. */
/* The paper's own discretisation (Sec. 2.1-2.6): piecewise constants on the dual mesh.
 * bem_mesh_barycentric: the barycentric refinement T^bary of the (stored, rotated)
 * mesh (Sec. 2.1): each triangle (v0, v1, v2) becomes (v0, m01, c), (m01, v1, c),
 * (v1, m12, c), (m12, v2, c), (v2, m20, c), (m20, v0, c) at positions 6T .. 6T+5;
 * new vertices: the edge midpoints 0.5 (a + b), numbered after the old vertices by the
 * first appearance of their edge in (triangle, local edge) order, then the centroids
 * ((v0 + v1) + v2) / 3; the children are uploaded like any mesh (reference edge =
 * longest edge).  The caller destroys it.
 * bem_operator_dual: from the operator of the barycentric refinement of mesh, the
 * Galerkin matrix of the dual basis V^dual = P^T V^bary P (Sec. 2.6; P maps the dual
 * cell of vertex z to its children: of triangle T, children 0 and 5 belong to v0, 1 and
 * 2 to v1, 3 and 4 to v2), an M x M operator (DF64; F64 from an F64 operator; FP64 sums
 * over the children, z <= w, mirrored).  bem_solve_capacity on it solves V^dual x = f,
 * f_z = |T_z^dual| = (sum of |T| at z) / 3, and returns Cap_l = (1/4 pi) sum f_z x_z
 * (Eq. 2.8); x has one value per vertex.  (The paper solves the same Galerkin system
 * with operator preconditioning and GMRES; any convergent solver gives the same x.)
 * Not with inexact_lambda.  At most 65,535 vertices and 32 triangles per vertex.
 * bem_zz_estimate_dual: eta(T)^2 = h_T ||Phi - I Phi||^2_{L2(T)} (Eq. 1.6) for the dual
 * solution x (M values), exact per barycentric child; totals (nullable): [sum eta^2,
 * sum h_T |T| xbar^2 / 12], xbar the mean of the three vertex values. */
bem_status bem_mesh_barycentric(bem_mesh *mesh, bem_mesh **out);
bem_status bem_operator_dual(bem_operator *bary_op, bem_mesh *mesh, bem_operator **out);
bem_status bem_zz_estimate_dual(bem_mesh *mesh, const double *x, int32_t h_mode, double *eta2_out, double *totals);
/* The FP32 D^reg (which = 0) or C = S D^reg S (which = 1) of a dual operator, M x M
 * row-major into dst (host or device); BEM_ERR_INVALID for an operator without them. */
bem_status bem_operator_preconditioner(const bem_operator *op, int32_t which, float *dst);

/* ---------------------------------------------------------------- batch */
/* Many independent capacity problems assembled and solved together (the paper has
 * no counterpart: it solves one polyhedron at a time).  bem_batch_create takes count
 * meshes of any sizes (same context; the meshes must outlive the batch) and the
 * operator precision (aopts->precision BEM_PREC_DF64 or BEM_PREC_F32).  It cuts the
 * problems, in their given order, into waves whose device memory fits what is
 * available at creation -- 90% of the device's free memory, and the context's HBM
 * budget if it has one -- and at most 3 x (number of SMs) problems per wave; one
 * arena sized for the largest wave holds the operators and the solver state of the
 * wave that runs (a problem that alone exceeds it: BEM_ERR_OOM).  It also times the
 * far-field tiles of the size classes present and, for BEM_PRECOND_BLOCK, computes the
 * cluster orders.  bem_batch_run runs every wave in turn: the assembly of all its
 * operators (Eq. 2.4-2.5) by one launch per phase -- the far field over a work list of
 * (problem, tile) items with one tile shape (the autotuned one of the wave's largest
 * size class), the mirror of the diagonal 64 x 64 blocks (the solves read only the
 * upper triangles), the Sauter-Schwab near field over all touching pairs -- upper
 * triangles bit-identical to bem_assemble_V's; then the diagonals, right-hand sides and
 * preconditioners; then the persistent solver of bem_solve_capacity (sopts: tol,
 * max_it, precond, reliable_delta; x = 0 start), one cooperative launch per group of
 * problems of similar size, in which problem p owns a share of the CTAs in proportion
 * to its work and has its own grid barrier; then every Cap (Eq. 2.8).  The work runs on a stream of
 * the batch; with use_graph each wave is recorded once as a CUDA graph on the first
 * run and later runs replay it.  The call blocks until the results are on the host;
 * results (nullable, count entries, in the given order) receive them;
 * BEM_ERR_NOT_CONVERGED if any problem missed tol. */
typedef struct bem_batch bem_batch;
typedef struct {
    double cap;
    int32_t iterations;
    int32_t outer;           /* as bem_solve_info.outer */
    double relres;
    int32_t converged;
    int32_t status;          /* BEM_OK, BEM_ERR_NOT_CONVERGED or BEM_ERR_CUDA (barrier time-out) */
} bem_batch_result;
bem_status bem_batch_create(bem_ctx *ctx, int32_t count, bem_mesh *const *meshes, const bem_assembly_opts *aopts,
                            const bem_solve_opts *sopts, int32_t use_graph, bem_batch **out);
bem_status bem_batch_run(bem_batch *b, bem_batch_result *results);
/* count: problems; ctas: CTAs of the solver launch; graph_used: 1 if the last run
 * replayed a captured graph. */
bem_status bem_batch_info(const bem_batch *b, int32_t *count, int32_t *ctas, int32_t *graph_used);
/* waves: number of waves; arena_bytes: device bytes of the arena; wave_of (nullable,
 * count entries): the wave of each problem.  Any pointer may be NULL. */
bem_status bem_batch_waves(const bem_batch *b, int32_t *waves, int64_t *arena_bytes, int32_t *wave_of);
bem_status bem_batch_destroy(bem_batch *b);

/* ---------------------------------------------------------------- serving */
/* Continuous-batching server for adaptive capacity requests (the paper has no
 * counterpart: it serves many polyhedra of different sizes arriving over time).
 * `slots` host threads, each with its own CUDA stream and context on the device
 * current at creation, take requests in arrival order; a request is admitted when
 * a slot is free and its device-memory estimate (one operator at N for a single
 * level, else two operators at min(1.5 max_N, N 2.2^(levels-1)); plus tables) fits
 * in hbm_budget_bytes next to the running requests -- the first
 * queued request that fits, so small requests backfill around large ones; with
 * nothing running the first request is always admitted.  Admitted requests run
 * bem_adaptive_run with `opts` (max_levels and max_N taken per request) on their
 * own stream, so their kernels overlap; each keeps its mesh, operator and Krylov
 * state on the device across levels and is held to its estimate by the context's
 * HBM budget.  A request's result does not depend on what else runs. */
typedef struct bem_server bem_server;
#define BEM_SERVER_HISTORY 16
typedef struct {
    int64_t id;
    int32_t status;          /* bem_status of the request */
    int32_t done;            /* 1 once finished */
    int32_t levels;
    int64_t N_final;
    double cap;              /* Cap of the last level */
    double t_submit, t_start, t_done;  /* seconds since the server started (steady clock) */
    int64_t estimate_bytes;  /* admission estimate */
    double cap_history[BEM_SERVER_HISTORY];
    int64_t N_history[BEM_SERVER_HISTORY];
    char message[256];       /* error message when status != 0 */
} bem_request_result;
typedef struct {
    int64_t queued, in_flight, peak_in_flight, in_flight_bytes, peak_bytes, budget;
    double clock;            /* seconds since the server started */
} bem_server_stats_t;

bem_status bem_server_create(int32_t slots, int64_t hbm_budget_bytes, const bem_adaptive_opts *opts,
                             bem_server **out);
/* Queue a request: the mesh arrays (host memory) are copied; max_levels >= 1 levels or
 * until N >= max_N.  Never blocks on the GPU. */
bem_status bem_server_submit(bem_server *s, const double *verts, int64_t M, const int32_t *tris, int64_t N,
                             int32_t max_levels, int64_t max_N, int64_t *id_out);
/* Block until request id has finished, return its result and forget it. */
bem_status bem_server_wait(bem_server *s, int64_t id, bem_request_result *out);
bem_status bem_server_stats(bem_server *s, bem_server_stats_t *out);
/* Profiling of the slots' hot kernels (bem_profile_enable / bem_profile_read on every
 * slot's context).  bem_server_profile_enable takes effect at each slot's next request
 * (enabling restarts its counts); bem_server_profile_read returns the sums over the
 * slots and needs an idle server -- no request queued or running -- else
 * BEM_ERR_INVALID.  The kernels of concurrent requests share the GPU, so a launch's
 * event time includes the time other requests' kernels ran beside it. */
bem_status bem_server_profile_enable(bem_server *s, int32_t on);
bem_status bem_server_profile_read(bem_server *s, int32_t kernel, int64_t *launches, double *ms, double *units);
/* Finish every queued request, then stop the slot threads and free the server. */
bem_status bem_server_destroy(bem_server *s);

/* ---------------------------------------------------------------- instrumentation */
/* Per-kernel device time, taken with CUDA events recorded on the context's stream
 * around every launch of the hot kernels while profiling is on, together with the
 * algorithmic work of those launches:
 *   BEM_KERNEL_FAR    units = far-field entries computed (pairs i <= j)
 *   BEM_KERNEL_NEAR   units = touching pairs integrated
 *   BEM_KERNEL_MATVEC units = bytes of V a product must read (N * N * element size, half
 *                     of it for the symmetric DF64 product); the persistent DF64 solver
 *                     is recorded as one launch carrying all its products */
#define BEM_KERNEL_FAR 0
#define BEM_KERNEL_NEAR 1
#define BEM_KERNEL_MATVEC 2
/* on = 1: clear the counters and start recording; 0: stop. */
bem_status bem_profile_enable(bem_ctx *ctx, int32_t on);
/* Totals since the last enable (synchronises the stream). */
bem_status bem_profile_read(bem_ctx *ctx, int32_t kernel, int64_t *launches, double *ms, double *units);
/* DF64 solves run as one persistent cooperative launch (on = 1, the default) or
 * as a host-driven loop of kernels (on = 0; also used when a cooperative launch is
 * not possible).  Both give the same iterates up to the order of the reductions. */
bem_status bem_context_set_persistent(bem_ctx *ctx, int32_t on);
/* Failure detection of the persistent solvers (the paper has no counterpart: it runs
 * on one workstation thread).  Their CTAs meet at grid barriers whose wait is bounded
 * in time; a CTA that waits longer than the limit raises an error flag and returns,
 * the others give up once they see the flag, and the solve reports BEM_ERR_CUDA
 * ("grid barrier timed out") with the context still usable.  wait_limit_ns (> 0)
 * sets that limit for later solves of ctx (<= 0: the default, 2 s); absent_cta >= 0
 * makes that CTA of later single-problem persistent solves leave at its first
 * barrier without arriving, as a CTA that stopped would, so that the others' waits
 * run out (a test of the time-out path that faults nothing); -1 turns it off. */
bem_status bem_debug_barrier_fault(bem_ctx *ctx, int64_t wait_limit_ns, int32_t absent_cta);
/* Number of CUDA kernels the context has launched so far. */
bem_status bem_launch_count(const bem_ctx *ctx, int64_t *n);

#ifdef __cplusplus
}
#endif
#endif /* BEM_GB300_H */
