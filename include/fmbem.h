/*
 * fmbem.h -- C ABI of the GB300 (sm_103a) fast-multipole boundary-element library for 3-D
 * electromagnetic scattering by homogeneous scatterers, after Wang, Zheng, Xiao, Lin & Chan,
 * "Fast multipole boundary element method for three dimensional electromagnetic scattering
 * problem" (arXiv 1211.7177).
 *
 * The library applies the Nystrom-discretised electric-field integral-equation operator of
 * Eqs. (2.9)-(2.13),  [Gamma Lambda][Phi; Psi] = Phi_inc,  with the fast multipole method of
 * Section 2.2 (octree of Appendix C, P2M Eqs. (2.18)-(2.19), M2M Eq. (2.20), M2L + L2L
 * Eq. (2.21), L2P + near field Eqs. (2.22)-(2.23), analytic self terms of Appendix B), and solves
 * the system with right-preconditioned GMRES, Eq. (3.1), using the block-diagonal
 * preconditioner M = A_self of Eq. (3.2).  Every numerical step runs in CUDA kernels on the
 * device; the host only validates input, sequences launches and runs the (m x m) Hessenberg
 * recurrences of GMRES.
 *
 * Conventions shared by every entry point
 *   - Time factor exp(-i omega t) (Section 2.1).  Relative permittivity eps_d and permeability
 *     mu_d per domain d: d = 0 is the background, d = 1..J the scatterers.  The wavenumber of
 *     domain d is k_d = k0 sqrt(eps_d mu_d), the root with Im k_d >= 0; T_j and gamma_j follow
 *     Eq. (2.13) with eps_0, mu_0 the background's relative values.
 *   - Nystrom nodes (one-point rule, Eq. 2.8): CENTROID mode uses triangle centroids weighted
 *     by the triangle area (the paper's "simplest case"); VERTEX mode uses mesh vertices weighted
 *     by one third of the incident triangle areas, with the area-weighted vertex normal.
 *   - A vector of unknowns or results holds, per right-hand side and per node in USER order
 *     (vertex order in VERTEX mode, triangle order in CENTROID mode), 6 complex numbers as
 *     interleaved (re, im) doubles: layout [n_rhs][N][6] complex128.  Unknowns per node are
 *     (Phi_x, Phi_y, Phi_z, Psi_x, Psi_y, Psi_z) with Phi = E_0 and Psi = n x curl E_0 for the
 *     scatterer's outward normal n (Eq. 2.12); results per node are (background equation x,y,z,
 *     scatterer equation x,y,z).
 *   - Device pointers are plain CUDA device addresses (for example torch.Tensor.data_ptr()),
 *     read or written only during the call and in the order of the given stream; the stream
 *     argument is a cudaStream_t (NULL = legacy default stream).  The caller keeps ownership
 *     of every buffer it passes.
 *   - Every entry point returns an fmbem_status and never throws; fmbem_last_error() gives a
 *     message for the last failure on a handle.  A handle must not be used by two host threads
 *     or two streams at the same time.
 */
#ifndef FMBEM_H
#define FMBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMBEM_OK = 0,
    FMBEM_ERR_INVALID_ARGUMENT = 1, /* a NULL pointer, a non-positive size, an unknown option  */
    FMBEM_ERR_INVALID_MESH = 2,     /* mesh not usable: see fmbem_create                       */
    FMBEM_ERR_OOM = 3,              /* a device allocation failed                              */
    FMBEM_ERR_CUDA = 4,             /* a CUDA runtime call or kernel launch failed             */
    FMBEM_ERR_NOT_CONVERGED = 5,    /* fmbem_solve reached max_iter above the tolerance        */
    FMBEM_ERR_BREAKDOWN = 6,        /* GMRES produced a non-finite value                       */
    FMBEM_ERR_DEVICE_TIMEOUT = 7    /* a bounded wait inside a kernel ran out (a pipeline stage
                                       or a work item never became ready); the kernel stopped,
                                       released what it held and returned, the context stays
                                       usable and the call's outputs are undefined              */
} fmbem_status;

typedef enum { FMBEM_NODES_VERTEX = 0, FMBEM_NODES_CENTROID = 1 } fmbem_node_mode;

/* Arithmetic of the near-field and far-field passes.  FP64: everything in double precision.
 * FP32: P2P, P2M, M2M, M2L, L2L and L2P in single precision (double-float node positions),
 * with the analytic self blocks, the final accumulation of every result and the GMRES vectors
 * in double precision.
 * TF32: as FP32, except that for 16 or more right-hand sides (and p = 4, 6 or 8) the M2L and
 * L2L products run on the tensor cores (tcgen05.mma, inputs rounded to TF32, FP32 accumulation
 * in tensor memory); meant for the inner iterations of the refined solve.  The rounding adds a
 * relative error of about 1e-5 to a matvec and makes it slightly nonlinear, so an inner GMRES
 * on it should stop at a loose tolerance (1e-2) and let the outer refinement finish.
 * BF16X3: as TF32, except that the tensor-core M2L and L2L products run on bf16 operands split
 * into hi and lo parts (x = x_hi + x_lo, each bf16) and accumulate A_hi B_hi + A_hi B_lo +
 * A_lo B_hi in FP32 (tcgen05.mma kind::f16): three times the MMAs of TF32 at twice its rate, the
 * same bytes, and a rounding error of ~2^-16 instead of ~2^-11 per product, so the product stays
 * within the FP32 path's accuracy (FP32 itself below 16 right-hand sides). */
typedef enum { FMBEM_FP64 = 0, FMBEM_FP32 = 1, FMBEM_TF32 = 2, FMBEM_BF16X3 = 3 } fmbem_precision;

/* How the scatterers are modelled (Section 2).
 * PENETRABLE: the interior fields are unknowns too; Eqs. (2.5)-(2.13), 6N equations.
 * IMPEDANCE: good conductors under the impedance boundary condition of Eq. (2.24),
 *   n x E = Z n x (n x H), Z_j = sqrt(mu_j / eps_j) (relative to the vacuum impedance, principal
 *   root) and n the scatterer's outward normal; the interior domains are not modelled
 *   (Section 2.3).  The vectors keep the 6-entry layout, and the 6N system becomes
 *     background rows of a node:  the background equation of Eq. (2.12), unchanged;
 *     scatterer rows of a node:   Psi - zeta_j (Phi - n (n.Phi)) = 0, zeta_j = i k0 mu_0 / Z_j,
 *   i.e. Eq. (2.24) itself written with Psi = n x curl E_0 = i k0 mu_0 (n x H_0).  Eliminating Psi
 *   node by node gives exactly Eq. (2.25) in Phi = E_0 alone; GMRES on the 6N form with right-hand
 *   sides whose scatterer rows are zero (as fmbem_plane_wave_rhs writes them) runs the same
 *   iterations as GMRES on Eq. (2.25) with the node-block preconditioner, and its solution carries
 *   the Psi that the far-field, near-field and cross-section routines take.  The fast multipole
 *   passes run for the background domain only; eps_j, mu_j enter through Z_j alone. */
typedef enum { FMBEM_BOUNDARY_PENETRABLE = 0, FMBEM_BOUNDARY_IMPEDANCE = 1 } fmbem_boundary;

typedef struct { double re, im; } fmbem_c64;

/* Closed, consistently oriented triangle mesh.  vertices [n_vertices][3] and triangles
 * [n_triangles][3] (counter-clockwise seen from outside, so (B-A) x (C-A) points out of the
 * scatterer) and tri_domain [n_triangles] (scatterer ids 1..n_scatterers) are HOST arrays. */
typedef struct {
    int64_t n_vertices;
    const double *vertices;
    int64_t n_triangles;
    const int32_t *triangles;
    const int32_t *tri_domain;
    int32_t n_scatterers;
} fmbem_mesh;

/* Options; fmbem_default_options() fills the defaults given in brackets. */
typedef struct {
    int node_mode;           /* fmbem_node_mode [VERTEX]                                         */
    int p;                   /* truncation number p of Eq. (2.17): degrees n = 0..p-1 [8]         */
    int leaf_size;           /* the octree (Appendix C) is refined to the smallest depth l_max >= 2
                                at which the non-empty leaves hold at most leaf_size nodes on
                                average [64]                                                     */
    int max_level;           /* upper bound on l_max [10]                                         */
    int gmres_restart;       /* GMRES restart length m [50]                                       */
    int solve_precision;     /* fmbem_precision used by fmbem_solve's Krylov iterations [FP64];
                                with FP32 the solve is refined: outer true residuals with the FP64
                                operator, inner GMRES with the FP32 operator                      */
    double inner_tol;        /* relative tolerance of each inner FP32 solve [1e-2]                */
    int outer_precision;     /* fmbem_precision of the passes in the refined solve's outer true-
                                residual matvec (vectors and the residual are always FP64) [FP64] */
    int m2l_rotation;        /* S|R translations for few right-hand sides: 0 dense p^2 x p^2
                                matrices, 1 rotation form (rotate to the translation axis, coaxial
                                translation, rotate back; ~3.3 p^3 instead of p^4 operations),
                                -1 automatic: rotation form for p >= 9 [-1]                      */
    int profile_phases;      /* non-zero: record CUDA events around the matvec phases so that
                                fmbem_last_matvec_times can report them [0]                       */
    int near_cache;          /* near-field kernel scalars g, c of every (target, source, domain)
                                pair, which depend on the geometry only, computed once at create
                                in FP64 and read by the FP64 matvecs with fewer than 4 right-hand
                                sides instead of evaluating exp, sincos and rsqrt per pair:
                                0 off, 1 on, -1 automatic: on when the cache (32 bytes per pair and
                                domain) takes at most a quarter of the free device memory [-1]    */
    int boundary;            /* fmbem_boundary: how the scatterers enter [PENETRABLE]             */
    double near_singular_radius; /* near-singular correction of the pair terms of Eq. (2.12) [0]:
                                0 keeps the paper's one-point rule (Eq. 2.8) for every pair;
                                rho > 0 replaces, for every source node beta within
                                |s_beta - s_alpha| < rho sqrt(w_beta) of the target, w_beta times the
                                kernel at s_beta by the integral of the kernel over beta's patch (its
                                density and normal held constant): the triangle (CENTROID nodes) or
                                the unprojected barycentric dual cell (VERTEX nodes), each flat piece
                                cut into 4^near_singular_levels triangles with the centroid rule.
                                The corrections are computed at create in FP64 and applied in FP64
                                by every product (either precision) and its transpose.  Needs the
                                penetrable boundary and rho sqrt(max w) <= the leaf box width
                                (FMBEM_ERR_INVALID_ARGUMENT otherwise); the vertex-position
                                gradients refuse handles with rho > 0                            */
    int near_singular_levels;    /* subdivision levels L of the correction, 0..6 [3]              */
    int fp32_only;           /* non-zero: keep only the single-precision bases and translation
                                matrices (about a third of the device memory of a handle, for many
                                small problems on one GPU, e.g. fmbem_batch_*); products, solves and
                                observables that need FP64, TF32 or BF16X3 passes are then refused
                                with FMBEM_ERR_INVALID_ARGUMENT, and the near-field cache is off [0] */
    double fmm_tol;          /* > 0: choose the truncation number from this tolerance instead of p
                                (Eq. 2.17 truncated after degree p - 1): for every level and domain
                                the relative RMS error of the truncated addition theorem (the
                                multipole expansion about the source box centre plus the local
                                expansion about the target box centre, Eq. 2.14) is sampled over
                                points of a box and its far-field neighbours at offsets (2,0,0) ...
                                (3,2,1) box widths; each level takes the smallest p in 2..20 that
                                meets the tolerance, and the handle uses the largest of them (the
                                expansions of all levels have one length); fmbem_truncation
                                reports both.  0: use p [0]                                     */
    int adaptive;            /* octree: 0 the paper's uniform tree (all leaves on l_max, chosen by the
                                mean occupancy as above); 1 per-branch adaptive: a box is split
                                while it holds more than leaf_size nodes, down to max_level, so that
                                leaves lie on several levels (strongly non-uniform meshes, e.g.
                                narrow gaps).  M2L still runs between well-separated boxes of one
                                level whose parents are adjacent (the FF lists of Appendix C); the
                                sources a leaf gets neither through its own nor an ancestor's FF
                                list are summed directly: the boxes of its level adjacent to it
                                (all nodes below them) and, for every ancestor, the leaves of the
                                ancestor's level adjacent to that ancestor.  FMBEM_ERR_INVALID_ARGUMENT
                                when a leaf's direct sources need more than 32 node ranges;
                                fmbem_batch_create refuses adaptive handles [0]                  */
} fmbem_options;

void fmbem_default_options(fmbem_options *opt);

/* Fault injection for tests of the out-of-memory paths: after this call, device allocations
 * of the library (all handles, all threads) may take `bytes` more bytes in total; one that would
 * exceed the budget fails as if cudaMalloc had, and the call that made it returns FMBEM_ERR_OOM
 * with the handle's resources released (fmbem_create) or left as before the call.  A negative
 * value removes the budget (the default). */
void fmbem_debug_set_device_budget(int64_t bytes);

typedef struct fmbem fmbem;  /* opaque handle */

/* Builds everything that depends on geometry and frequency, Sections 2.1-2.2 and Appendices
 * B-C: nodes, weights and normals (Eq. 2.8); the self-patch integrals of Appendix B (Eqs.
 * B.2-B.9) on a planar patch around each node -- the triangle itself for CENTROID nodes, the
 * barycentric dual cell projected on the node's tangent plane for VERTEX nodes -- and the 6x6
 * preconditioner blocks A_self (Eq. 3.2) with their LU factors; the octree with
 * Children/Parent/Neighbor/FF lists (Appendix C); the multipole bases and the S|S, S|R, R|R
 * translation matrices for every level and domain wavenumber (Eqs. 2.14-2.21).
 *   mesh        host mesh, copied; the caller keeps it.  Rejected with FMBEM_ERR_INVALID_MESH
 *               when an index is out of range, a triangle is degenerate, a domain id is outside
 *               1..n_scatterers, an edge is not shared by exactly two triangles of opposite
 *               orientation, or (VERTEX mode) a vertex is unused or touches two scatterers.
 *   eps, mu     host arrays [n_scatterers + 1] of relative permittivity / permeability,
 *               index 0 = background; mu must be non-zero, eps non-zero.
 *   k0          vacuum wavenumber (> 0).
 *   opt         options, NULL = defaults.
 *   stream      cudaStream_t for the set-up kernels (the call synchronises it before returning).
 *   out         receives the handle (NULL on failure).  The handle owns all device memory it
 *               allocates; fmbem_destroy frees it. */
fmbem_status fmbem_create(const fmbem_mesh *mesh, const fmbem_c64 *eps, const fmbem_c64 *mu, double k0,
                          const fmbem_options *opt, void *stream, fmbem **out);

void fmbem_destroy(fmbem *h);

/* Message of the last failure on this handle ("" if none); NULL handle: last fmbem_create
 * failure of the calling thread. */
const char *fmbem_last_error(const fmbem *h);

/* Number of Nystrom nodes N (a vector holds 6N complex numbers per right-hand side). */
int64_t fmbem_num_nodes(const fmbem *h);

/* Node positions [N][3], outward normals [N][3] and weights [N], host arrays in user order
 * (any of them may be NULL).  Eq. (2.8). */
fmbem_status fmbem_node_geometry(const fmbem *h, double *pos, double *normal, double *weight);

/* Number of (target, source) node pairs that take the near-singular correction (0 when
 * near_singular_radius is 0). */
int64_t fmbem_num_near_singular_pairs(const fmbem *h);

/* The truncation number p the handle uses, and (arrays of l_max + 1 entries, levels 0 and 1
 * unused) the truncation each level needs for fmm_tol and the sampled relative error estimate at p
 * (-1 without fmm_tol, when p is the option's).  Any pointer may be NULL. */
fmbem_status fmbem_truncation(const fmbem *h, int32_t *p, int32_t *p_level, double *err_level);

/* Boxes and leaves per level (Appendix C; with option adaptive the leaves lie on several levels):
 * boxes[l] = non-empty boxes of level l, leaves[l] = those that are leaves, for l = 0 .. n - 1
 * (0 past l_max).  Either pointer may be NULL; host arrays of n entries. */
fmbem_status fmbem_tree_levels(const fmbem *h, int32_t n, int64_t *boxes, int64_t *leaves);

/* Octree summary: l_max, number of leaves, total number of boxes on levels 2..l_max, and the
 * number of near-field (source, target) node pairs and of far-field box pairs (S|R
 * translations) per domain.  Any pointer may be NULL. */
fmbem_status fmbem_tree_info(const fmbem *h, int32_t *l_max, int64_t *n_leaves, int64_t *n_boxes,
                             int64_t *near_pairs, int64_t *ff_pairs);

/* Right-hand sides of Eq. (2.9) for plane waves E_inc = e exp(i k_0 d . r) (Eq. 2.12,
 * Phi_inc): e in the background rows, 0 in the scatterer rows (no incident field inside).
 *   dir   host [n_rhs][3] unit propagation directions; pol host [n_rhs][3] complex polarisations.
 *   b_dev device [n_rhs][N][6] complex128, written. */
fmbem_status fmbem_plane_wave_rhs(fmbem *h, int64_t n_rhs, const double *dir, const fmbem_c64 *pol, void *b_dev,
                                  void *stream);

/* y = A x for the operator of Eq. (2.9), evaluated as in Section 2.2: far field by the fast
 * multipole passes (Eqs. 2.18-2.21, L2P of Eq. 2.23), near field by direct one-point sums over
 * the node's own leaf and its Neighbor leaves (Eq. 2.23), self blocks analytically
 * (Appendix B).
 *   x_dev, y_dev  device [n_rhs][N][6] complex128 (user order); x is read, y written; they
 *                 must not overlap.
 *   precision     fmbem_precision of the passes (see above).
 * Scratch (expansion coefficients, source densities) is owned by the handle and grown on
 * demand, so the first call with a larger n_rhs allocates. */
fmbem_status fmbem_matvec(fmbem *h, const void *x_dev, void *y_dev, int64_t n_rhs, int precision, void *stream);

/* The same product with x and y in HOST memory, the copies included: the right-hand sides are
 * taken in chunks of chunk_rhs; chunk k is copied to the device, multiplied (exactly the kernels
 * of fmbem_matvec with n_rhs = the chunk's size) and copied back, with the copy of chunk k + 1 to
 * the device and of chunk k - 1 back on two internal copy streams, running beside the product
 * of chunk k.  The paper has no counterpart (its data never leave one machine's memory); this is
 * a library-level variant for callers whose right-hand sides arrive in and leave through host
 * memory.
 *   x_host, y_host  host [n_rhs][N][6] complex128 (user order), read / written; page-locked
 *                   (cudaHostAlloc, torch pin_memory) for the copies to overlap the kernels.
 *   chunk_rhs       right-hand sides per chunk (>= 0); 0 = the library's choice: chunks of
 *                   up to 128 right-hand sides (one chunk for a batch of 128 or fewer).
 *   stream          the products run on it, and it waits for the last copy back: y_host is
 *                   complete once the work queued on the stream so far has completed (the call
 *                   itself may return earlier).  x_host must stay unchanged until then.
 * Device memory: four chunk-sized buffers (two for x, two for y), owned by the handle and grown
 * on demand, plus the product's own scratch. */
fmbem_status fmbem_matvec_host(fmbem *h, const void *x_host, void *y_host, int64_t n_rhs, int precision,
                               int64_t chunk_rhs, void *stream);

/* y = A^T x, the transpose (complex bilinear, no conjugation) of the operator of Eq. (2.9) as
 * fmbem_matvec evaluates it; A^H x is conj(A^T conj(x)).  The paper has no adjoint; it is the
 * product an adjoint (gradient) solve needs.  Gathering the transposed blocks of Eq. (2.12) at a
 * node b turns each domain's sum into the field of unweighted monopoles: with phi_i the
 * potential of the strengths x_{a,i} of the d rows of x (g_d of Eq. 2.12),
 *   Phi rows += w_b T_d(b) [-sum_i n'_i grad phi_i + n' div phi + (n'.grad) phi](s_b),
 *   Psi rows += w_b sigma_d phi(s_b)   (n' = -n_b, sigma = -1 for the background; n' = n_b,
 *                                       sigma = gamma_j for the node's scatterer),
 * plus the transposed self block A_self^T x_b.  The far field of phi and grad phi runs through a
 * monopole P2M, the same M2M, M2L and L2L translations, and L2P with the local basis and its
 * gradient; the near field is summed directly over the Neighbor leaves.
 *   x_dev, y_dev  device [n_rhs][N][6] complex128 (user order); x is read, y written; they
 *                 must not overlap.
 *   precision     fmbem_precision of the passes, as for fmbem_matvec (FMBEM_TF32 puts M2L and
 *                 L2L on the tensor cores for at least 16 right-hand sides).
 * Uses the same handle-owned scratch as fmbem_matvec. */
fmbem_status fmbem_adjoint_matvec(fmbem *h, const void *x_dev, void *y_dev, int64_t n_rhs, int precision,
                                  void *stream);

/* Solves A x = b (Eq. 2.9) by right-preconditioned restarted GMRES (Eq. 3.1) with the
 * block-diagonal preconditioner M = A_self (Eq. 3.2) applied exactly (6x6 LU per node), each
 * right-hand side in its own Krylov space, all right-hand sides batched through one matvec per
 * iteration.  Arnoldi orthogonalisation (classical Gram-Schmidt applied twice) and the true
 * residual ||b - A x|| / ||b|| are computed in double precision; convergence is declared on
 * the true residual.  With solve_precision = FP32 the solve is iteratively refined: each outer
 * step computes the true residual with the FP64 operator and solves the correction with the
 * FP32 operator to inner_tol.
 *   b_dev    device [n_rhs][N][6] complex128, read.
 *   x_dev    device [n_rhs][N][6] complex128: initial guess on entry, solution on exit.
 *   tol      relative residual target (> 0); max_iter bounds the total number of Krylov
 *            iterations (matvecs) per solve.
 *   iters_host, relres_host  host [n_rhs]: iterations used and final true relative residual
 *            (either may be NULL).
 * Returns FMBEM_ERR_NOT_CONVERGED (x = last iterate) when a right-hand side stays above tol. */
fmbem_status fmbem_solve(fmbem *h, const void *b_dev, void *x_dev, int64_t n_rhs, double tol, int max_iter,
                         int32_t *iters_host, double *relres_host, void *stream);

/* Solves A^T x = b, the adjoint (transposed) system of Eq. (2.9), the way fmbem_solve solves
 * A x = b: right-preconditioned restarted GMRES with fmbem_adjoint_matvec as the operator and the
 * transposed preconditioner M^T = A_self^T (applied exactly from the same 6x6 LU), honouring
 * solve_precision, inner_tol and outer_precision (with TF32 the inner adjoint products run M2L
 * and L2L on the tensor cores, as the forward ones do).  The paper has no adjoint solve; an
 * adjoint (gradient) computation needs it: for an objective J = L^T x with A x = b,
 * dJ/dp = -lambda^T (dA/dp) x with A^T lambda = L.
 * Arguments, layout, return values and errors as for fmbem_solve. */
fmbem_status fmbem_adjoint_solve(fmbem *h, const void *b_dev, void *x_dev, int64_t n_rhs, double tol, int max_iter,
                                 int32_t *iters_host, double *relres_host, void *stream);

/* Far-field amplitude of the scattered field of solutions x (Section 4; the representation
 * formula of Appendix A in the far zone), with n0 = -n and Psi0 = -Psi the background's normal
 * and unknown:
 *   F(u) = 1/(4 pi) sum_b w_b exp(-i k0 u.s_b) { (-i k0)[n0 (u.Phi_b) - (n0.u) Phi_b - u (n0.Phi_b)]
 *                                                 - Psi0_b },   E_sca ~ exp(i k0 r)/r F(u).
 *   x_dev     device [n_rhs][N][6] complex128 (user order), read.
 *   rhat      host [n_dir][3] unit directions.
 *   F_host    host [n_rhs][n_dir][3] complex128, written.
 * Extinction by the optical theorem is C_ext = (4 pi / k0) Im[e* . F(d)] for the plane wave
 * (d, e); the scattering cross section is the integral of |F|^2 over the unit sphere. */
fmbem_status fmbem_far_field(fmbem *h, const void *x_dev, int64_t n_rhs, int64_t n_dir, const double *rhat,
                             fmbem_c64 *F_host, void *stream);

/* The far-field amplitude as a linear functional of the solution, for adjoint gradients of
 * far-field observables: out[r] holds the coefficients of x -> c_r . F(u_r) (F as for
 * fmbem_far_field, no conjugation), so that c_r . F(u_r) = sum_b out[r][b] . x[r][b].  With
 * c = (4 pi / k0) conj(e) and u = d, Im of the functional is the extinction cross section of the
 * plane wave (d, e); an adjoint solve with out as the right-hand side then gives its derivative
 * with respect to any parameter p of A as -Im(lambda^T (dA/dp) x).
 *   rhat   host [n_rhs][3] unit directions u_r.
 *   coef   host [n_rhs][3] complex128 vectors c_r.
 *   out_dev device [n_rhs][N][6] complex128 (user order), written.
 * Errors: FMBEM_ERR_INVALID_ARGUMENT (n_rhs outside 1..65535, NULL pointers), FMBEM_ERR_CUDA. */
fmbem_status fmbem_far_field_functional(fmbem *h, int64_t n_rhs, const double *rhat, const fmbem_c64 *coef,
                                        void *out_dev, void *stream);

/* Total electric (and magnetic) field at points outside every scatterer (Section 4; the
 * representation formula of Appendix A for the background domain), for solutions x of
 * plane-wave excitations:
 *   E(r) = e exp(i k d.r) + sum_b w_b { n0 (a.Phi_b) - (n0.a) Phi_b - a (n0.Phi_b) + g Psi_b },
 *   g = exp(i k R) / (4 pi R),  a = grad_s g = g (i k - 1/R) (s_b - r) / R,  R = |s_b - r|,
 *   n0 = -n_b (the background's normal), k the background wavenumber;
 *   H(r) = curl E / (i k0 mu_0) (omega = k0 with c = 1, mu_0 the background's permeability), where
 *   the curl of the bracket is (K n0) x Phi_b + n0 x (K Phi_b) with K the Hessian of g in s_b,
 *   and that of g Psi_b is -a x Psi_b; the incident wave contributes i k (d x e) exp(i k d.r).
 * Direct summation over the N nodes in double precision (no FMM: O(n_pts N) per right-hand side),
 * for field maps and stress-tensor surfaces off the boundary; a point on or inside the surface
 * gets no meaningful value.
 *   x_dev     device [n_rhs][N][6] complex128 (user order), read.
 *   pts       host [n_pts][3] points.
 *   dir, pol  host [n_rhs][3] each: the plane waves (direction, polarisation) that produced x, for
 *             the incident term; both NULL for the scattered field alone.
 *   E_host    host [n_rhs][n_pts][3] complex128, written.
 *   H_host    host [n_rhs][n_pts][3] complex128, written; NULL to skip the magnetic field.
 * Errors: FMBEM_ERR_INVALID_ARGUMENT (n_rhs outside 1..65535, n_pts < 1, a NULL x, pts or E, or
 * only one of dir and pol), FMBEM_ERR_CUDA, FMBEM_ERR_OOM. */
fmbem_status fmbem_near_field(fmbem *h, const void *x_dev, int64_t n_rhs, int64_t n_pts, const double *pts,
                              const double *dir, const fmbem_c64 *pol, fmbem_c64 *E_host, fmbem_c64 *H_host,
                              void *stream);

/* Gradient of a far-field functional with respect to the mesh vertex positions (vertex nodes,
 * penetrable scatterers), by the adjoint method of the discrete system of Eq. (2.9).  For each
 * right-hand side r, x_r solves A(V) x = b_r(V) with b_r the plane wave (dir[r], pol[r]) of
 * fmbem_plane_wave_rhs, f_r = L_r(V)^T x_r is the functional coef[r] . F(rhat[r]) of
 * fmbem_far_field_functional, and lambda_r solves A^T lambda = L_r (fmbem_adjoint_solve); then
 *   out[r][v][c] = d/dV_vc [ L_r^T x_r + lambda_r^T b_r - lambda_r^T A x_r ]  (x, lambda fixed)
 *               = d f_r / dV_vc.
 * The vertex positions enter through the node positions, weights and normals of each vertex's
 * 1-ring and through their self blocks (Appendix B); the pair blocks of Eq. (2.12) are summed
 * directly (O(N^2) FP64 pair evaluations), all derivatives are FP64 central differences with
 * steps of 1e-6 (the mean edge length for positions).  The extinction of the plane wave (d, e)
 * is Im f with rhat = d and coef = (4 pi / k0) conj(e).
 *   x_dev, lam_dev  device [n_rhs][N][6] complex128 (user order).
 *   dir, rhat       host [n_rhs][3]; pol, coef host [n_rhs][3] complex128.
 *   out_host        host [n_rhs][N][3] complex128 (N = number of vertices), written.
 * Errors: FMBEM_ERR_INVALID_ARGUMENT (counts, NULL pointers, centroid nodes, impedance boundary),
 * FMBEM_ERR_INVALID_MESH (a vertex with more than 31 neighbours), FMBEM_ERR_CUDA, FMBEM_ERR_OOM. */
fmbem_status fmbem_shape_gradient(fmbem *h, const void *x_dev, const void *lam_dev, int64_t n_rhs, const double *dir,
                                  const fmbem_c64 *pol, const double *rhat, const fmbem_c64 *coef,
                                  fmbem_c64 *out_host, void *stream);

/* As fmbem_shape_gradient, for the near-field functionals
 *   f_r = sum_p cE[r][p] . E_sca(r_p) + cH[r][p] . H_sca(r_p)
 * of fmbem_near_field_functional (E_sca, H_sca the scattered parts of fmbem_near_field's fields at
 * the fixed points pts) in place of the far-field ones: with A^T lambda_r = N_r (the functional's
 * coefficients), out[r][v][c] = d f_r / dV_vc.  The gradient of the Maxwell-stress force takes
 * the Wirtinger coefficients of each force component as cE, cH (F_i = 2 Re ... to first order).
 *   pts host [n_pts][3]; cE, cH host [n_rhs][n_pts][3] complex128 (cH may be NULL).
 * Errors as fmbem_shape_gradient. */
fmbem_status fmbem_shape_gradient_near(fmbem *h, const void *x_dev, const void *lam_dev, int64_t n_rhs,
                                       const double *dir, const fmbem_c64 *pol, int64_t n_pts, const double *pts,
                                       const fmbem_c64 *cE, const fmbem_c64 *cH, fmbem_c64 *out_host, void *stream);

/* Fields inside the scatterers: at each point r_p, inside scatterer domain[p] = j, the
 * representation formula of domain j (Appendix A; Eq. 2.5 holds it on the boundary),
 *   E_j(r) = sum over the nodes b of scatterer j of
 *            w_b { [n_b (grad'g_j . v_b) - (n_b . grad'g_j) v_b - grad'g_j (n_b . v_b)]
 *                  - g_j(s_b, r) gamma_j Psi_b },   v_b = T_j Phi_b (Eq. 2.6),
 * with n_b the scatterer's outward normal and gamma_j Psi = n x curl E_j (Eq. 2.7); no incident
 * field inside.  H_j = curl E_j / (i k0 mu_j), from the curl of the same sum.  Direct FP64
 * summation over the scatterer's nodes (one thread per point), for field maps of moderate size.
 *   x_dev    solutions [n_rhs][N][6] (device, user order).
 *   pts      host [n_pts][3]; domain host [n_pts] scatterer ids 1..n_scatterers (a point outside
 *            its domain gets the null-field integral, zero for exact data).
 *   E_host   host [n_rhs][n_pts][3] complex128, written; H_host likewise, or NULL.
 * Errors: FMBEM_ERR_INVALID_ARGUMENT (counts, NULL pointers, a domain id out of range, or a
 * handle created with the impedance boundary, which does not model the interiors),
 * FMBEM_ERR_CUDA, FMBEM_ERR_OOM. */
fmbem_status fmbem_interior_field(fmbem *h, const void *x_dev, int64_t n_rhs, int64_t n_pts, const double *pts,
                                  const int32_t *domain, fmbem_c64 *E_host, fmbem_c64 *H_host, void *stream);

/* The fields of fmbem_near_field through the fast multipole passes, for maps with many points:
 * one FP64 product of x (Eqs. 2.18-2.21) leaves the local expansions of the background domain
 * at every leaf; a point inside a leaf takes the far sources from that leaf's expansion (first
 * term of Eq. 2.23 at the point, and its gradient for H) and the sources of the leaf and its
 * Neighbor leaves directly; a point outside every (non-empty) leaf sums all nodes directly.
 * Arguments, layout and errors as fmbem_near_field; the result differs from it by the multipole
 * truncation error. */
fmbem_status fmbem_near_field_fmm(fmbem *h, const void *x_dev, int64_t n_rhs, int64_t n_pts, const double *pts,
                                  const double *dir, const fmbem_c64 *pol, fmbem_c64 *E_host, fmbem_c64 *H_host,
                                  void *stream);

/* The exterior fields as linear functionals of the solution, for adjoint gradients of
 * quantities built from them (the optical force of a Maxwell-stress surface): out[f] holds the
 * coefficients of x -> sum_p ( cE[f][p] . E_sca(r_p) + cH[f][p] . H_sca(r_p) ) with E_sca, H_sca
 * the scattered parts of fmbem_near_field's fields (no conjugation), so that the functional is
 * sum_b out[f][b] . x_b.
 *   pts      host [n_pts][3] points.
 *   cE, cH   host [n_fun][n_pts][3] complex128; cH may be NULL (no magnetic part).
 *   out_dev  device [n_fun][N][6] complex128 (user order), written.
 * Errors: FMBEM_ERR_INVALID_ARGUMENT (n_fun outside 1..65535, n_pts < 1, NULL pts, cE or out),
 * FMBEM_ERR_CUDA, FMBEM_ERR_OOM. */
fmbem_status fmbem_near_field_functional(fmbem *h, int64_t n_fun, int64_t n_pts, const double *pts,
                                         const fmbem_c64 *cE, const fmbem_c64 *cH, void *out_dev, void *stream);

/* Cross sections and the far-zone optical force of solutions x of the plane waves (dir[r],
 * pol[r]) (Section 4), all on the device: the far-field amplitude F of fmbem_far_field in the
 * forward directions and on a Gauss-Legendre (cos theta, n_theta nodes) x trapezoid (phi, n_phi
 * nodes) rule on the unit sphere, then per right-hand side
 *   C_ext = (4 pi / k) Im[conj(e) . F(d)]   (optical theorem),
 *   C_sca = sum_q w_q |F(u_q)|^2,
 *   C_abs = -(1/k) sum_b w_b Im(Phi_b . conj(Psi_b))   (Eq. 4.2),
 *   F_far = (C_ext d - sum_q w_q |F(u_q)|^2 u_q) / 2   (momentum balance in the far zone; the
 *           time-averaged force on all scatterers together in units with eps_0 = mu_0 = c = 1 and
 *           a unit-amplitude wave), k the background wavenumber.
 *   x_dev     device [n_rhs][N][6] complex128 (user order), read.
 *   dir, pol  host [n_rhs][3] each (pol complex128).
 *   out_host  host [n_rhs][6] = (C_ext, C_sca, C_abs, F_far x, y, z), written.
 * Errors: FMBEM_ERR_INVALID_ARGUMENT (counts, NULL pointers, n_theta or n_phi < 2, a lossy
 * background), FMBEM_ERR_CUDA, FMBEM_ERR_OOM. */
fmbem_status fmbem_cross_sections(fmbem *h, const void *x_dev, int64_t n_rhs, const double *dir, const fmbem_c64 *pol,
                                  int32_t n_theta, int32_t n_phi, double *out_host, void *stream);

/* Time-averaged optical force on the scatterers inside the sphere (center, radius) in the plane
 * waves (dir[r], pol[r]) (Appendix D): the total E and H of fmbem_near_field on the points
 * center + radius u_q of the sphere rule of fmbem_cross_sections, and
 *   F = sum_q w_q radius^2 T n_q,  T n = Re[E (E*.n) + H (H*.n) - (|E|^2 + |H|^2) n / 2] / 2
 * (Maxwell stress tensor, units with eps_0 = mu_0 = c = 1), reduced on the device.  The sphere
 * must lie in the background, enclosing the scatterers whose force is wanted and no others.
 *   out_host host [n_rhs][3], written.
 * Errors as fmbem_cross_sections (radius > 0). */
fmbem_status fmbem_force_stress(fmbem *h, const void *x_dev, int64_t n_rhs, const double *dir, const fmbem_c64 *pol,
                                const double *center, double radius, int32_t n_theta, int32_t n_phi, double *out_host,
                                void *stream);

/* The stress force of fmbem_force_stress for one plane wave (dir, pol) [n_rhs = 1], and, for its
 * adjoint gradient, the Wirtinger coefficients of its three components with respect to the
 * fields at the sphere points,
 *   cE[i][q][j] = w_q / 4 [delta_ij (conj(E_q) . n_q) + conj(E_q,i) n_q,j - n_q,i conj(E_q,j)]
 *   (cH likewise with H), so that dF_i = 2 Re sum_q (cE[i][q] . dE_q + cH[i][q] . dH_q),
 * mapped to the unknowns as in fmbem_near_field_functional: L[i] with F_i's first-order change
 * 2 Re(L[i]^T dx).  All on the device.
 *   force_host  host [3], written; pts_host host [P][3] (P = n_theta n_phi), written when not NULL;
 *   cE_host, cH_host host [3][P][3] complex128, written when not NULL (for fmbem_shape_gradient_near);
 *   L_dev       device [3][N][6] complex128 (user order), written.
 * Errors as fmbem_force_stress. */
fmbem_status fmbem_force_stress_functional(fmbem *h, const void *x_dev, const double *dir, const fmbem_c64 *pol,
                                           const double *center, double radius, int32_t n_theta, int32_t n_phi,
                                           double *force_host, double *pts_host, fmbem_c64 *cE_host,
                                           fmbem_c64 *cH_host, void *L_dev, void *stream);

/* s[r] = lambda_r^T (dA/deps_j) x_r (complex bilinear) for the operator of Eq. (2.9), which
 * depends holomorphically on eps_j (through k_j = k0 sqrt(eps_j mu_j), T_j of Eq. 2.13 and the self
 * blocks of Appendix B): the central difference (A(eps_j + step) - A(eps_j - step)) x / (2 step) of
 * two FP64 products on handles the library builds from the same mesh, media and options (kept for
 * the next call with the same j and step), then the bilinear reduction, on the device.  For an
 * objective f = L^T x with A x = b (b independent of eps_j) and A^T lambda = L:
 * df/deps_j = -s.  The paper has no adjoint; the adjoint gradients need it.
 *   j        scatterer 1..J; step > 0 (e.g. 1e-5 max(1, |eps_j|)).
 *   x_dev, lam_dev  device [n_rhs][N][6] complex128 (user order).
 *   out_host host [n_rhs] complex128, written.
 * Errors: FMBEM_ERR_INVALID_ARGUMENT (j, counts, NULL pointers, the impedance boundary or an
 * fp32_only handle), FMBEM_ERR_CUDA, FMBEM_ERR_OOM. */
fmbem_status fmbem_eps_sensitivity(fmbem *h, int32_t j, const void *x_dev, const void *lam_dev, int64_t n_rhs,
                                   double step, fmbem_c64 *out_host, void *stream);

/* sum_b w_b Im(Phi_b . conj(Psi_b)) per right-hand side (host [n_rhs], written): with
 * n x curl E = Psi the inward flux of the time-averaged Poynting vector, Eq. (4.2), gives the
 * absorption cross section C_abs = -(1/k0) times this sum. */
fmbem_status fmbem_absorption(fmbem *h, const void *x_dev, int64_t n_rhs, double *out_host, void *stream);

/* z = M^{-1} v with M = A_self (Eq. 3.2), per node 6x6 complex LU; v_dev, z_dev device
 * [n_rhs][N][6] complex128 (may be the same buffer). */
fmbem_status fmbem_precond_apply(fmbem *h, const void *v_dev, void *z_dev, int64_t n_rhs, void *stream);

/* Allocation-free y = A x, for callers that cannot allocate device memory when they need the
 * product: work recorded into a CUDA graph by stream capture (cudaMalloc is not allowed during
 * capture), code whose device memory is owned by a framework allocator, or callbacks that must
 * not trigger the implicit device synchronisation of cudaMalloc/cudaFree.  The paper has no
 * counterpart; this is a library-level variant of fmbem_matvec.
 * Same arguments, layouts, kernels and results as fmbem_matvec, except that precision must be
 * FMBEM_FP64 or FMBEM_FP32 (FMBEM_TF32 is refused with FMBEM_ERR_INVALID_ARGUMENT).  The scratch
 * (source densities, expansion coefficients, per-pair M2L results) lives in one file-scope device array
 * of 32 MiB that every GPU loading the library holds until the process exits; no cudaMalloc,
 * cudaFree or allocating library routine is called.  Problems whose scratch for the given n_rhs
 * and precision exceeds 32 MiB (roughly a few thousand nodes at p = 8 and one right-hand side)
 * are rejected with FMBEM_ERR_INVALID_ARGUMENT and a message giving the bytes needed.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array: calls that overlap on
 * the GPU (different streams without ordering) race on it.  Nothing needs clearing between
 * calls, because every scratch element a call reads is written earlier in the same call. */
fmbem_status fmbem_matvec_noalloc(fmbem *h, const void *x_dev, void *y_dev, int64_t n_rhs, int precision,
                                  void *stream);

/* One persistent kernel launch over many independent problems of uneven size (no counterpart in
 * the paper, which treats one problem at a time): the products y_i = A_i x_i of n_problems
 * handles, each with n_rhs right-hand sides, in FP32 passes.  A plan lays out, once, the work items
 * of every problem -- source densities per (node block, right-hand side), P2M per (leaf, domain,
 * right-hand side), M2M per (parent box, domain, column chunk) level by level upwards, M2L + L2L
 * per (box, domain, column chunk) level by level downwards (dense S|S, S|R, R|R), near field +
 * L2P + self per leaf -- in stage order, with the number of items of every stage of every
 * problem.  Each fmbem_batch_matvec is one launch of as many 128-thread blocks as can be
 * resident; a block takes the next item from a device queue counter, waits (bounded spin) until
 * the stages its item reads are complete for its problem, runs it and counts it complete.  Items
 * only wait for stages that come earlier in the queue, so the earliest unfinished item can always
 * proceed; a wait that runs out (2 s, see fmbem_debug_set_batch_wait) stops the launch and the
 * call returns FMBEM_ERR_DEVICE_TIMEOUT (outputs undefined, the context stays usable).
 *   handles     host [n_problems] handles (penetrable boundary, near_singular_radius 0, p <= 11);
 *               they must outlive the plan, and a handle must not run other work while a batch
 *               product that includes it is in flight.
 *   n_rhs       right-hand sides per problem, 1..64.  precision: FMBEM_FP32 only.
 *   x_dev, y_dev  host [n_problems] arrays of device pointers, problem i's [n_rhs][N_i][6]
 *               complex128 vectors (user order); x read, y written.
 * The plan's work items live in device memory allocated by fmbem_batch_create (cudaMalloc) and
 * freed by fmbem_batch_destroy; each handle's own scratch is grown for n_rhs if needed.
 * Errors: FMBEM_ERR_INVALID_ARGUMENT, FMBEM_ERR_OOM, FMBEM_ERR_CUDA, FMBEM_ERR_DEVICE_TIMEOUT. */
typedef struct fmbem_batch fmbem_batch;
fmbem_status fmbem_batch_create(fmbem *const *handles, int32_t n_problems, int64_t n_rhs, int precision,
                                fmbem_batch **out);
fmbem_status fmbem_batch_matvec(fmbem_batch *b, const void *const *x_dev, void *const *y_dev, void *stream);
int64_t fmbem_batch_num_items(const fmbem_batch *b);
void fmbem_batch_destroy(fmbem_batch *b);
/* Message of the last failure of a plan ("" if none); NULL: the last fmbem_batch_create failure
 * of the calling thread. */
const char *fmbem_batch_last_error(const fmbem_batch *b);
/* Fault injection for tests of the bounded waits, process-wide: wait_ns sets the spin limit of
 * the batch kernel's waits (0 restores 2 s); stall_problem >= 0 makes the next launches withhold
 * the completion count of that problem's P2M items, so that its later items wait until the limit
 * and the call returns FMBEM_ERR_DEVICE_TIMEOUT; -1 turns it off. */
void fmbem_debug_set_batch_wait(uint64_t wait_ns, int32_t stall_problem);

/* Wall-clock milliseconds of the phases of the last fmbem_matvec call, measured with CUDA
 * events on its stream: [0] source densities + P2M, [1] M2M, [2] M2L + L2L, [3] near field
 * + L2P + self, [4] total.  ms_host [5]. */
fmbem_status fmbem_last_matvec_times(const fmbem *h, double *ms_host);

#ifdef __cplusplus
}
#endif

#endif /* FMBEM_H */
