// fmbem_internal.cuh -- shared declarations of the GB300 FMM-BEM library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fmbem.h"

// ------------------------------------------------------------------------------------------
// complex arithmetic on plain (re, im) pairs, usable for double and float
template <typename R>
struct cx {
    R re, im;
};
using c64 = cx<double>;
using c32 = cx<float>;

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, R s) { return {s * a.re, s * a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> &operator+=(cx<R> &a, cx<R> b) { a.re += b.re; a.im += b.im; return a; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> &operator-=(cx<R> &a, cx<R> b) { a.re -= b.re; a.im -= b.im; return a; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> conjg(cx<R> a) { return {a.re, -a.im}; }
template <typename R>
__host__ __device__ __forceinline__ R abs2(cx<R> a) { return a.re * a.re + a.im * a.im; }
// a += b * c
template <typename R>
__host__ __device__ __forceinline__ void cfma(cx<R> &a, cx<R> b, cx<R> c) {
    a.re = fma(b.re, c.re, fma(-b.im, c.im, a.re));
    a.im = fma(b.re, c.im, fma(b.im, c.re, a.im));
}
__host__ __device__ __forceinline__ c64 cdiv(c64 a, c64 b) {
    double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__host__ __device__ __forceinline__ c64 cexpd(c64 z) {
    double e = exp(z.re), s, c;
    sincos(z.im, &s, &c);
    return {e * c, e * s};
}
__host__ __device__ __forceinline__ double cabsd(c64 z) { return hypot(z.re, z.im); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> to(c64 a) { return {(R)a.re, (R)a.im}; }

// ------------------------------------------------------------------------------------------
// handle
struct LevelInfo {
    int64_t off = 0;  // first global box index of the level
    int64_t n = 0;    // number of non-empty boxes
    double w = 0;     // box width
};

struct DevBuf {  // owning device buffer
    void *p = nullptr;
    size_t bytes = 0;
};

struct fmbem {
    fmbem_options opt{};
    std::string err;
    cudaStream_t setup_stream = nullptr;

    // problem
    int64_t N = 0;
    int J = 0;
    double k0 = 0;
    std::vector<c64> eps, mu, k, gam;  // [J+1]
    // impedance boundary condition (Section 2.3): the scatterer rows are Eq. (2.24) with
    // zeta[j] = i k0 mu_0 / Z_j; the media of the scatterers are then the background's (their
    // interiors are not modelled) and the multipole passes run over domains 0..Jf only
    bool ibc = false;
    int Jf = 0;
    std::vector<c64> zeta;  // [J+1], entry 0 unused
    c64 *d_zeta = nullptr;  // device copy
    int p = 0, p2 = 0;                 // truncation number and p^2 coefficients
    // a copy of the mesh and media as given, for the operators with a perturbed permittivity
    // (fmbem_eps_sensitivity), and those operators once built
    std::vector<double> mesh_V;
    std::vector<int32_t> mesh_F, mesh_D;
    std::vector<c64> eps_user, mu_user;
    fmbem *eps_plus = nullptr, *eps_minus = nullptr;
    int eps_j = -1;
    double eps_step = 0;
    std::vector<int> p_level;          // option fmm_tol: the truncation each level needs [lmax+1]
    std::vector<double> trunc_err;     // and the sampled error estimate at the p used

    // host copies of geometry (user order)
    std::vector<double> h_pos, h_nrm, h_w;
    std::vector<int32_t> h_F, h_vt_start, h_vt_tri;  // triangles and vertex -> triangle lists (vertex nodes)

    // device geometry in user order (from the node set-up)
    double *upos = nullptr, *unrm = nullptr, *uw = nullptr;  // [N][3], [N][3], [N]
    int32_t *udom = nullptr;                                 // [N] scatterer id 1..J
    // device geometry, sorted (Morton) order
    int32_t *perm = nullptr;   // sorted -> user
    int32_t *iperm = nullptr;  // user -> sorted
    double *pos = nullptr, *nrm = nullptr, *w = nullptr;  // [N][3], [N][3], [N]
    int32_t *dom = nullptr;                                // [N]
    float *pos_hi = nullptr, *pos_lo = nullptr, *nrm_f = nullptr;  // [N][3]
    float4 *src_rec = nullptr;  // [N][3]: position hi + scatterer id, position lo + n_x, n_y n_z (k_near_w)
    // self blocks (user order): M = A_self [N][6][6], LU factors and pivots
    c64 *Mself = nullptr, *Mlu = nullptr;
    int8_t *piv = nullptr;
    c32 *Minv32 = nullptr;  // single-precision explicit inverses for the inner iterations (lazy)

    // octree (Appendix C)
    int lmax = 0;
    double root_min[3] = {0, 0, 0};
    double root_w = 0;
    std::vector<LevelInfo> lev;  // [lmax+1]
    int64_t nbox = 0;            // total boxes, levels 0..lmax
    uint64_t *box_key = nullptr; // [nbox] Morton key at its level
    double *box_ctr = nullptr;   // [nbox][3]
    int32_t *box_parent = nullptr;                        // [nbox] global index (-1 at level 0)
    int32_t *box_cbeg = nullptr, *box_cend = nullptr;     // [nbox] children range (global)
    // [nbox + n_range_boxes] sorted-node range of every box, then of the merged node ranges that
    // the near lists of an adaptive tree refer to
    int32_t *box_nbeg = nullptr, *box_nend = nullptr;
    int64_t n_range_boxes = 0;
    // leaves (all at l_max in the paper's uniform tree; at any level in the adaptive tree), in
    // node order: global box of each leaf, and the leaf position of every box (-1: not a leaf)
    bool adaptive = false;
    int64_t n_leaves = 0;
    int32_t *leaf_box = nullptr, *box_leafpos = nullptr, *leaf_level = nullptr;
    std::vector<int32_t> h_leaf_box, h_leaf_level;
    int32_t *node_leaf = nullptr;                         // [N] global leaf box of each sorted node
    // per leaf (leaf position order), CSR of the boxes whose nodes are its direct sources
    // (uniform tree: Neighbor + self at l_max; adaptive tree: merged node ranges, see tree.cu)
    int32_t *nbr_start = nullptr, *nbr_idx = nullptr;
    int32_t *ff_start = nullptr, *ff_src = nullptr;       // CSR of FF lists over global boxes
    int16_t *ff_off = nullptr;                            // offset code 0..315 per FF entry
    int64_t n_ff = 0, n_nbr = 0, near_pairs = 0;
    int4 *near_items = nullptr;  // warp work items of the near field (leaf, target offset, tg, nsl)
    int n_near_items = 0;
    int *near_next = nullptr;    // unit counter of the persistent near-field kernels, reset per launch
    int4 *near_groups = nullptr;  // target groups of the lane-per-RHS near field (leaf, target offset, count, -):
                                  // n_near_groups in leaf order, then the same sorted by pair work
    int n_near_groups = 0;
    // near-field pair scalars (g, c) per leaf [side][source in the Neighbor list][target], double
    // precision; near_base[leaf] = pairs of the leaves before it
    void *near_cache64 = nullptr;
    int64_t *near_base = nullptr;
    // near-singular correction (nearsing.cu): pairs by target [ns_start[a], ns_start[a+1]) with
    // user-order target and source, 8 complex coefficients each (dS, dA for the background and
    // the scatterer side), and the pairs by source for the transposed product
    int64_t ns_pairs = 0;
    int64_t *ns_start = nullptr, *ns_tstart = nullptr, *ns_tpair = nullptr;
    int32_t *ns_tgt = nullptr, *ns_src = nullptr;
    c64 *ns_coef = nullptr;
    int32_t max_leaf = 0;                                 // largest leaf occupancy
    std::vector<int64_t> h_ff_count_level;
    // FF pairs of each level regrouped by translation offset, for the chunked M2L kernel:
    // pair_e[]: CSR positions sorted by (level, offset, target); chunk k of level l covers
    // pair_e[chunk_beg[k] .. chunk_beg[k] + chunk_cnt[k]) with one offset chunk_off[k]
    int32_t *pair_e = nullptr, *pair_tgt = nullptr;       // [n_ff], [n_ff] (target of each CSR entry)
    int32_t *chunk_beg = nullptr, *chunk_cnt = nullptr;
    int16_t *chunk_off = nullptr;
    std::vector<int64_t> h_chunk_first;                   // [lmax+2] first chunk of each level
    std::vector<int64_t> h_pair_first;                    // [lmax+2] first CSR position of each level
    void *ybuf = nullptr;                                 // per-pair M2L results
    size_t ybuf_bytes = 0;

    // multipole bases and translations, per domain d in 0..J
    std::vector<double> lam;  // [(J+1)*(lmax+1)] scale lambda = |k_d| w_l
    c64 *B_p2m64 = nullptr, *B_l2p64 = nullptr;   // [2][N][4][p2], [2][N][p2] (side 0 bg, 1 own)
    c32 *B_p2m32 = nullptr, *B_l2p32 = nullptr;
    c64 *B_l2pg64 = nullptr;                        // [2][N][3][p2] gradient of the L2P basis
    c32 *B_l2pg32 = nullptr;
    c64 *T_m2l64 = nullptr, *T_mm64 = nullptr, *T_ll64 = nullptr;  // see tables.cu for layout
    c32 *T_m2l32 = nullptr, *T_mm32 = nullptr, *T_ll32 = nullptr;
    // tensor-core (tcgen05, TF32) M2L tables: real-form 128-byte-swizzled images, see m2l_tc.cu
    float *Atc = nullptr, *Lltc = nullptr;
    float *Abf = nullptr, *Llbf = nullptr;  // the same matrices as bf16 hi/lo images (BF16x3)
    float *Mmbf = nullptr;                  // and the S|S matrices of M2M (BF16x3)
    void *Aofs = nullptr;  // S|R bf16 hi/lo images for the offset-stationary few-column M2L (BF16x3)
    void *chunk_pairs = nullptr;  // int2 [chunks][32]: (source box, CSR position) of each chunk's pairs
    int *tc_err = nullptr;
    bool m2l_rotation = false;
    int n_tlen = 0;
    int8_t *rot_tidx = nullptr;  // [316] index of the offset's length among the distinct lengths
    // rotation form of S|R = (back rotation) (coaxial) (forward rotation), packed by fmm.cu:
    // R_D [316][2][real degree blocks] (forward, back polar rotations), R_P [316][2][p2] (forward,
    // back azimuthal phases), R_Z [J+1][lmax+1][n_tlen][order blocks] (coaxial S|R)
    double *R_D64 = nullptr;
    float *R_D32 = nullptr;
    c64 *R_P64 = nullptr, *R_Z64 = nullptr;
    c32 *R_P32 = nullptr, *R_Z32 = nullptr;
    // the same form for M2M (S|S) and L2L (R|R) along the 8 child-parent diagonals, which share
    // their rotation factors with the far-field offsets (+-2, +-2, +-2): coaxial S|S and R|R per
    // (domain, level) [J+1][lmax+1][order blocks], and the child boxes of every level >= 3 in
    // entries grouped by octant, in chunks of up to 32 (fmm.cu: build_rot_mm_lists)
    c64 *R_Zmm64 = nullptr, *R_Zll64 = nullptr;
    c32 *R_Zmm32 = nullptr, *R_Zll32 = nullptr;
    int8_t *rot_zero = nullptr;                 // [316] zeros: one coaxial table per level
    int32_t *rmm_iota = nullptr;                // [n_rmm] entry e -> e
    int32_t *rmm_child = nullptr, *rmm_par = nullptr;  // [n_rmm] child box and its parent per entry
    int32_t *rmm_entry = nullptr;               // [nbox] entry of a box of level >= 3 (else -1)
    int32_t *rmm_chunk_beg = nullptr, *rmm_chunk_cnt = nullptr;
    int16_t *rmm_chunk_mm = nullptr, *rmm_chunk_ll = nullptr;  // far-field offset code of the direction
    std::vector<int64_t> h_rmm_first, h_rmm_chunk_first;      // per level: first entry, first chunk
    int64_t n_rmm = 0;

    // scratch grown on demand
    int64_t scratch_rhs = 0;
    void *dens = nullptr;   // source densities
    void *Cexp = nullptr;   // multipole coefficients [J+1][nbox][3 n_rhs][p2]
    void *Dexp = nullptr;   // local coefficients
    int scratch_prec = -1;

    // solver scratch
    int64_t solver_rhs = 0;
    c64 *sv = nullptr;      // Krylov basis and work vectors
    size_t sv_bytes = 0;
    double *sdots = nullptr;
    size_t sdots_bytes = 0;

    // per-domain constants (k_d, t_d = (eps_0 - eps_d)/eps_d, gamma_d), device [J+1][3] c64
    c64 *dcons = nullptr;

    // timing
    bool profile = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // a second stream for the few-column BF16x3 downward pass: the coarse levels' L2L + reduction
    // chain runs there beside the leaf level's tensor-core M2L (fork and join events)
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool have_times = false;
    // host-buffer products (fmbem_matvec_host): copy streams (to and from the device), their
    // events, and the chunk buffers (two x slots, two y slots)
    struct IoRows {
        c64 *y_host = nullptr;    // set for one product: its rows go back slab by slab
        cudaStream_t down = nullptr;
        cudaEvent_t ev[16] = {};  // one per slab of 32 right-hand sides
        bool copied = false;      // the product copied its rows back itself
    } io_rows;
    cudaStream_t io_stream[2] = {nullptr, nullptr};
    cudaEvent_t io_ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    void *io_buf = nullptr;
    size_t io_bytes = 0;

    std::vector<void *> allocations;
};

// ------------------------------------------------------------------------------------------
// helpers shared between translation units
#define FMBEM_PI 3.14159265358979323846

constexpr int M2L_CHUNK = 32;  // FF pairs per chunk of the offset-grouped M2L kernel

// layout of the translation tables, per domain d and level l (global matrix index):
//   M2L  [d][l][316]  for l = 2..lmax (levels below 2 unused)
//   M2M  [d][l][8]    child level l = 3..lmax, child octant o
//   L2L  [d][l][8]    child level l = 3..lmax
// each matrix p2 x p2 stored column-by-input: T[c][r] = coefficient from input c to output r.
__host__ __device__ __forceinline__ int64_t m2l_matrix(int d, int l, int o, int lmax) {
    return ((int64_t)d * (lmax + 1) + l) * 316 + o;
}
__host__ __device__ __forceinline__ int64_t oct_matrix(int d, int l, int o, int lmax) {
    return ((int64_t)d * (lmax + 1) + l) * 8 + o;
}

// the 316 M2L offsets: (dx,dy,dz) in [-3,3]^3 minus [-1,1]^3, enumerated in lexicographic order
__host__ __device__ __forceinline__ int m2l_offset_code(int dx, int dy, int dz) {
    int c = ((dx + 3) * 7 + (dy + 3)) * 7 + (dz + 3);  // 0..342
    // subtract the inner 27 codes that precede c
    int inner_before = 0;
    // inner codes have all |d|<=1; count those with code < c
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
            for (int e = -1; e <= 1; ++e) {
                int ci = ((a + 3) * 7 + (b + 3)) * 7 + (e + 3);
                inner_before += ci < c;
            }
    return c - inner_before;
}

// error handling inside the library
std::string cuda_msg(cudaError_t e, const char *what);
void *dev_alloc(fmbem *h, size_t bytes);  // records the allocation; throws std::bad_alloc on failure
void dev_free(fmbem *h, void *p);

struct fmbem_error {
    fmbem_status st;
    std::string msg;
};
#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) throw fmbem_error{FMBEM_ERR_CUDA, cuda_msg(e_, #call)}; \
    } while (0)
#define CKL(what)                                                                  \
    do {                                                                           \
        cudaError_t e_ = cudaGetLastError();                                       \
        if (e_ != cudaSuccess) throw fmbem_error{FMBEM_ERR_CUDA, cuda_msg(e_, what)}; \
    } while (0)

// set-up stages (each throws fmbem_error)
void build_geometry(fmbem *h, const fmbem_mesh *mesh, cudaStream_t s);
void build_tree(fmbem *h, cudaStream_t s);
void build_tables(fmbem *h, cudaStream_t s);
// per-call operations
void run_matvec(fmbem *h, const c64 *x, c64 *y, int64_t n_rhs, int precision, cudaStream_t s);
void run_matvec_noalloc(fmbem *h, const c64 *x, c64 *y, int64_t n_rhs, int precision, cudaStream_t s);
void run_matvec_host(fmbem *h, const c64 *x_host, c64 *y_host, int64_t n_rhs, int precision, int64_t chunk_rhs,
                     cudaStream_t s);
void run_adjoint_matvec(fmbem *h, const c64 *x, c64 *y, int64_t n_rhs, int precision, cudaStream_t s);
void run_near_field_functional(fmbem *h, int64_t nf, int64_t n_pts, const double *pts_host, const c64 *cE_host,
                               const c64 *cH_host, c64 *out, cudaStream_t s);
void run_shape_gradient(fmbem *h, const c64 *x, const c64 *lam, int64_t nr, const double *dir_host,
                        const c64 *pol_host, const double *rhat_host, const c64 *coef_host, int64_t n_pts,
                        const double *pts_host, const c64 *cE_host, const c64 *cH_host, c64 *out_host,
                        cudaStream_t s);
void run_vertex_shape_grad(fmbem *h, int64_t nr, const c64 *x, const c64 *lam, const c64 *sens, double hv, c64 *out,
                           cudaStream_t s);
void run_near_field_fmm(fmbem *h, const c64 *x, int64_t nr, int64_t n_pts, const double *pts_host,
                        const double *dir_host, const c64 *pol_host, c64 *E_host, c64 *H_host, cudaStream_t s);
void run_locate_leaves(fmbem *h, const double *pts_dev, int64_t n, int32_t *leaf_dev, cudaStream_t s);
void run_interior_field(fmbem *h, const c64 *x, int64_t nr, int64_t n_pts, const double *pts_host,
                        const int32_t *dom_host, c64 *E_host, c64 *H_host, cudaStream_t s);
void run_near_field(fmbem *h, const c64 *x, int64_t nr, int64_t n_pts, const double *pts_host, const double *dir_host,
                    const c64 *pol_host, c64 *E_host, c64 *H_host, cudaStream_t s);
void run_far_field_functional(fmbem *h, int64_t nr, const double *rhat_host, const c64 *coef_host, c64 *out,
                              cudaStream_t s);
void run_far_field(fmbem *h, const c64 *x, int64_t n_rhs, int64_t n_dir, const double *rhat_host, c64 *F_host,
                   cudaStream_t s);
void run_absorption(fmbem *h, const c64 *x, int64_t n_rhs, double *out_host, cudaStream_t s);
bool m2l_tc_supported(const fmbem *h);
void build_tc_tables(fmbem *h, cudaStream_t s);
void run_m2l_tc(fmbem *h, float *C, float *D, int64_t nr, cudaStream_t s, bool bf3, bool c_split = false);
void run_m2m_tc(fmbem *h, float *C, int64_t nr, cudaStream_t s, bool leaves_split = false);
bool p2m_tc_supported(const fmbem *h, int64_t nr);
void run_p2m_tc(fmbem *h, const float *dens, const float4 *densS, const float *Bp2m, float *C, int64_t nr,
                cudaStream_t s);
bool m2l_ofs_supported(const fmbem *h);
void build_ofs_tables(fmbem *h, cudaStream_t s);
void split_expansions_bf16(fmbem *h, float *C, int64_t nr, cudaStream_t s);
int64_t ofs_y_dom(const fmbem *h, int64_t nr);
void run_m2l_ofs(fmbem *h, const float *C, float *Y, int64_t nr, cudaStream_t s, int l0, int l1, int reserve_sms);
void pack_rot_tables(fmbem *h, cudaStream_t s);
void pack_rot_tables_mm(fmbem *h, cudaStream_t s);
void build_rot_mm_lists(fmbem *h, cudaStream_t s);
void pack_rot_factors(fmbem *h, const c64 *Tzf, const c64 *Tyf, const c64 *Tyb, const c64 *Tzb, cudaStream_t s);
void near_work_items(fmbem *h, cudaStream_t s);
void build_near_cache(fmbem *h, cudaStream_t s);
void choose_truncation(fmbem *h, cudaStream_t s);
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);
void run_cross_sections(fmbem *h, const c64 *x, int64_t nr, const double *dir_host, const c64 *pol_host, int nt, int np,
                        double *out_host, cudaStream_t s);
void run_force_stress_functional(fmbem *h, const c64 *x, const double *dir_host, const c64 *pol_host,
                                 const double *center, double radius, int nt, int np, double *force_host,
                                 double *pts_host, c64 *cE_host, c64 *cH_host, c64 *L, cudaStream_t s);
void run_eps_sensitivity(fmbem *h, int j, const c64 *x, const c64 *lam, int64_t nr, double step, c64 *out_host,
                         cudaStream_t s);
void run_force_stress(fmbem *h, const c64 *x, int64_t nr, const double *dir_host, const c64 *pol_host,
                      const double *center, double radius, int nt, int np, double *out_host, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// one persistent launch over many problems (batch.cu, kernel in fmm.cu)
constexpr int BATCH_MAX_LEVEL = 10;
constexpr int BATCH_COUNTERS = 24;  // per problem: prep, up[0..10], down[0..10], near
constexpr int BATCH_CHUNK_COLS = 6;  // columns per M2M / M2L item (the CC of the translation kernels)
enum BatchKind : int16_t { BK_PREP = 0, BK_P2M = 1, BK_M2M = 2, BK_DOWN = 3, BK_NEAR = 4 };
struct BatchProblem {  // one problem's device pointers and sizes (precision-specific tables)
    int64_t N, nbox;
    int p2, lmax;
    int64_t lev_off[BATCH_MAX_LEVEL + 1];
    const int32_t *perm, *dom, *nbeg, *nend, *cbeg, *cend, *parent, *ff_start, *ff_src, *nbr_start, *nbr_idx;
    const int16_t *ff_off;
    const uint64_t *key;
    const double *nrm64, *w;
    const void *pos_hi, *pos_lo, *nrm;  // the near field's positions and normals in the precision
    const void *dc;                     // DomainConsts [J+1]
    const void *Bp2m, *Bl2p, *Tmm, *Tm2l, *Tll;
    void *dens, *C, *D;
    const c64 *Mself;
    const c64 *x;
    c64 *y;
};
struct BatchItem {
    int32_t prob;
    int16_t kind, level;  // BatchKind; the level of M2M (child level) and DOWN items
    int32_t a;            // node block, leaf, parent or box index within its level
    int16_t b, c;         // domain; right-hand side or column chunk
};
// counter indices of a problem: completion of every stage, and the stage an item waits for
__host__ __device__ inline int batch_done_counter(int kind, int level, int lmax) {
    return kind == BK_PREP ? 0 : kind == BK_P2M ? 1 + lmax : kind == BK_M2M ? 1 + level - 1 : kind == BK_DOWN ? 12 + level : 23;
}
void run_batch_kernel(int precision, const BatchProblem *probs, const BatchItem *items, int64_t n_items,
                      unsigned long long *next, unsigned *cnt, const unsigned *tgt, int *err, uint64_t wait_ns,
                      int stall_problem, int p2max, int64_t nr, cudaStream_t s);
void batch_ensure_scratch(fmbem *h, int64_t nr, int precision);
void build_near_singular(fmbem *h, const fmbem_mesh *mesh, cudaStream_t s);
void apply_near_singular(fmbem *h, const c64 *x, c64 *y, int64_t nr, cudaStream_t s, bool transpose);
void run_precond(fmbem *h, const c64 *v, c64 *z, int64_t n_rhs, cudaStream_t s);
void run_precond32(fmbem *h, const c32 *v, c64 *z, int64_t n_rhs, cudaStream_t s, bool transpose = false);
void run_precond_t(fmbem *h, const c64 *v, c64 *z, int64_t n_rhs, cudaStream_t s);
void run_plane_wave(fmbem *h, int64_t n_rhs, const double *dir, const fmbem_c64 *pol, c64 *b, cudaStream_t s);
fmbem_status run_solve(fmbem *h, const c64 *b, c64 *x, int64_t n_rhs, double tol, int max_iter, int32_t *iters,
                       double *relres, cudaStream_t s, bool transpose = false);
