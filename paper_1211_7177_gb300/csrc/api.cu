// api.cu -- the C ABI of include/fmbem.h: argument checks, handle life cycle and error capture.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "fmbem_internal.cuh"

static thread_local std::string g_create_error;

std::string cuda_msg(cudaError_t e, const char *what) {
    return std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

// device bytes that later allocations may still take (fault injection, fmbem_debug_set_device_budget);
// negative: unlimited
static std::atomic<int64_t> g_device_budget{-1};

void *dev_alloc(fmbem *h, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    for (int64_t left = g_device_budget.load(); left >= 0;) {
        if ((int64_t)bytes > left)
            throw fmbem_error{FMBEM_ERR_OOM, "device allocation of " + std::to_string(bytes) +
                                                 " bytes refused: the injected budget has " + std::to_string(left) +
                                                 " bytes left"};
        if (g_device_budget.compare_exchange_weak(left, left - (int64_t)bytes)) break;
    }
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw fmbem_error{FMBEM_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e)};
    }
    h->allocations.push_back(p);
    return p;
}

void dev_free(fmbem *h, void *p) {
    if (!p) return;
    auto it = std::find(h->allocations.begin(), h->allocations.end(), p);
    if (it != h->allocations.end()) {
        *it = h->allocations.back();
        h->allocations.pop_back();
    }
    cudaFree(p);
}

static void free_all(fmbem *h) {
    for (void *p : h->allocations) cudaFree(p);
    h->allocations.clear();
    for (auto &e : h->ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    for (cudaEvent_t *e : {&h->ev_fork, &h->ev_join})
        if (*e) { cudaEventDestroy(*e); *e = nullptr; }
    if (h->aux_stream) { cudaStreamDestroy(h->aux_stream); h->aux_stream = nullptr; }
    for (auto &e : h->io_ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    for (auto &e : h->io_rows.ev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    for (auto &st : h->io_stream)
        if (st) { cudaStreamDestroy(st); st = nullptr; }
    h->io_buf = nullptr;  // freed with the allocations above
    h->io_bytes = 0;
}

// wraps a call: converts exceptions into a status and the handle's message
template <typename F>
static fmbem_status guarded(fmbem *h, F &&f) {
    try {
        f();
        if (h) h->err.clear();
        return FMBEM_OK;
    } catch (const fmbem_error &e) {
        if (h) h->err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        if (h) h->err = "host allocation failed";
        return FMBEM_ERR_OOM;
    } catch (...) {
        if (h) h->err = "unexpected C++ exception";
        return FMBEM_ERR_CUDA;
    }
}

static c64 root_with_nonneg_imag(c64 z) {
    // principal square root, then the sign that gives Im >= 0
    double r = cabsd(z);
    double a = std::sqrt(std::max(0.0, 0.5 * (r + z.re)));
    double b = std::sqrt(std::max(0.0, 0.5 * (r - z.re)));
    if (z.im < 0) b = -b;
    c64 s = {a, b};
    if (s.im < 0 || (s.im == 0 && s.re < 0)) s = -s;
    return s;
}

// principal square root (Re >= 0): the surface impedance Z = sqrt(mu / eps) of Eq. (2.24)
static c64 principal_root(c64 z) {
    double r = cabsd(z);
    double a = std::sqrt(std::max(0.0, 0.5 * (r + z.re)));
    double b = std::sqrt(std::max(0.0, 0.5 * (r - z.re)));
    if (z.im < 0) b = -b;
    return {a, b};
}

extern "C" {

void fmbem_debug_set_device_budget(int64_t bytes) { g_device_budget.store(bytes < 0 ? -1 : bytes); }

void fmbem_default_options(fmbem_options *o) {
    if (!o) return;
    o->node_mode = FMBEM_NODES_VERTEX;
    o->p = 8;
    o->leaf_size = 64;
    o->max_level = 10;
    o->gmres_restart = 50;
    o->solve_precision = FMBEM_FP64;
    o->inner_tol = 1e-2;
    o->outer_precision = FMBEM_FP64;
    o->m2l_rotation = -1;
    o->near_cache = -1;
    o->profile_phases = 0;
    o->boundary = FMBEM_BOUNDARY_PENETRABLE;
    o->near_singular_radius = 0.0;
    o->near_singular_levels = 3;
    o->fp32_only = 0;
    o->fmm_tol = 0.0;
    o->adaptive = 0;
}

fmbem_status fmbem_create(const fmbem_mesh *mesh, const fmbem_c64 *eps, const fmbem_c64 *mu, double k0,
                          const fmbem_options *opt, void *stream, fmbem **out) {
    if (out) *out = nullptr;
    if (!mesh || !eps || !mu || !out || !mesh->vertices || !mesh->triangles || !mesh->tri_domain) {
        g_create_error = "NULL argument";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    if (!(k0 > 0) || !std::isfinite(k0) || mesh->n_scatterers < 1 || mesh->n_scatterers > 64) {
        g_create_error = "k0 must be positive and n_scatterers in 1..64";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    fmbem *h = new (std::nothrow) fmbem();
    if (!h) { g_create_error = "host allocation failed"; return FMBEM_ERR_OOM; }
    fmbem_default_options(&h->opt);
    if (opt) h->opt = *opt;
    const fmbem_options &o = h->opt;
    if ((o.node_mode != FMBEM_NODES_VERTEX && o.node_mode != FMBEM_NODES_CENTROID) || o.p < 2 || o.p > 20 ||
        o.leaf_size < 1 || o.max_level < 2 || o.gmres_restart < 1 || o.gmres_restart > 500 ||
        (o.solve_precision != FMBEM_FP64 && o.solve_precision != FMBEM_FP32 && o.solve_precision != FMBEM_TF32 &&
         o.solve_precision != FMBEM_BF16X3) ||
        !(o.inner_tol > 0 && o.inner_tol < 1) ||
        (o.outer_precision != FMBEM_FP64 && o.outer_precision != FMBEM_FP32) || o.m2l_rotation < -1 ||
        o.m2l_rotation > 1 || o.near_cache < -1 || o.near_cache > 1 ||
        (o.boundary != FMBEM_BOUNDARY_PENETRABLE && o.boundary != FMBEM_BOUNDARY_IMPEDANCE) ||
        !(o.near_singular_radius >= 0 && std::isfinite(o.near_singular_radius)) || o.near_singular_levels < 0 ||
        o.near_singular_levels > 6 || o.fp32_only < 0 || o.fp32_only > 1 ||
        !(o.fmm_tol >= 0 && o.fmm_tol < 1) || o.adaptive < 0 || o.adaptive > 1) {
        g_create_error = "invalid option value";
        delete h;
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    if (h->opt.fp32_only) h->opt.near_cache = 0;  // the cache serves FP64 products only
    cudaStream_t s = (cudaStream_t)stream;
    fmbem_status st = guarded(h, [&] {
        h->J = mesh->n_scatterers;
        h->k0 = k0;
        h->adaptive = o.adaptive == 1;
        h->p = o.p;
        h->p2 = o.p * o.p;
        h->profile = o.profile_phases != 0;
        h->m2l_rotation = o.m2l_rotation == 1 || (o.m2l_rotation == -1 && o.p >= 9);
        h->eps.resize(h->J + 1);
        h->mu.resize(h->J + 1);
        h->k.resize(h->J + 1);
        h->gam.resize(h->J + 1);
        for (int d = 0; d <= h->J; ++d) {
            h->eps[d] = {eps[d].re, eps[d].im};
            h->mu[d] = {mu[d].re, mu[d].im};
            if (!(cabsd(h->eps[d]) > 0) || !(cabsd(h->mu[d]) > 0) || !std::isfinite(eps[d].re + eps[d].im + mu[d].re + mu[d].im))
                throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT, "eps and mu must be finite and non-zero"};
            // Eq. (2.13): k_d = k0 sqrt(eps_d mu_d), gamma_d = mu_d / mu_0
            h->k[d] = k0 * root_with_nonneg_imag(h->eps[d] * h->mu[d]);
            h->gam[d] = d == 0 ? c64{1.0, 0.0} : cdiv(h->mu[d], h->mu[0]);
        }
        h->mesh_V.assign(mesh->vertices, mesh->vertices + 3 * mesh->n_vertices);
        h->mesh_F.assign(mesh->triangles, mesh->triangles + 3 * mesh->n_triangles);
        h->mesh_D.assign(mesh->tri_domain, mesh->tri_domain + mesh->n_triangles);
        h->eps_user = h->eps;
        h->mu_user = h->mu;
        h->ibc = o.boundary == FMBEM_BOUNDARY_IMPEDANCE;
        h->Jf = h->ibc ? 0 : h->J;
        if (h->ibc) {
            // Eq. (2.24): zeta_j = i k0 mu_0 / Z_j with Z_j = sqrt(mu_j / eps_j); the scatterers'
            // interiors are not modelled, so their media become the background's (k_j = k_0,
            // T_j = I, gamma_j = 1), which keeps every per-domain table finite and unused
            h->zeta.assign(h->J + 1, c64{0, 0});
            for (int d = 1; d <= h->J; ++d) {
                h->zeta[d] = cdiv(c64{0.0, k0} * h->mu[0], principal_root(cdiv(h->mu[d], h->eps[d])));
                h->eps[d] = h->eps[0];
                h->mu[d] = h->mu[0];
                h->k[d] = h->k[0];
                h->gam[d] = {1.0, 0.0};
            }
            h->d_zeta = (c64 *)dev_alloc(h, sizeof(c64) * (h->J + 1));
            CK(cudaMemcpyAsync(h->d_zeta, h->zeta.data(), sizeof(c64) * (h->J + 1), cudaMemcpyHostToDevice, s));
        }
        build_geometry(h, mesh, s);
        build_tree(h, s);
        if (h->opt.fmm_tol > 0) {  // the truncation number from the tolerance, per level
            choose_truncation(h, s);
            h->m2l_rotation = o.m2l_rotation == 1 || (o.m2l_rotation == -1 && h->p >= 9);
        }
        build_tables(h, s);
        near_work_items(h, s);
        std::vector<c64> dc(3 * (h->J + 1));
        for (int d = 0; d <= h->J; ++d) {
            dc[3 * d] = h->k[d];
            dc[3 * d + 1] = d == 0 ? c64{0, 0} : cdiv(h->eps[0] - h->eps[d], h->eps[d]);
            dc[3 * d + 2] = h->gam[d];
        }
        h->dcons = (c64 *)dev_alloc(h, sizeof(c64) * dc.size());
        CK(cudaMemcpyAsync(h->dcons, dc.data(), sizeof(c64) * dc.size(), cudaMemcpyHostToDevice, s));
        build_near_cache(h, s);
        build_near_singular(h, mesh, s);
        if (h->profile)
            for (auto &e : h->ev) CK(cudaEventCreate(&e));
        if (h->Aofs) {  // the few-column BF16x3 downward pass forks onto a second stream
            CK(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        }
        CK(cudaStreamSynchronize(s));
    });
    if (st != FMBEM_OK) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return FMBEM_OK;
}

void fmbem_destroy(fmbem *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    if (h->eps_plus) fmbem_destroy(h->eps_plus);
    if (h->eps_minus) fmbem_destroy(h->eps_minus);
    free_all(h);
    delete h;
}

const char *fmbem_last_error(const fmbem *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int64_t fmbem_num_nodes(const fmbem *h) { return h ? h->N : 0; }

int64_t fmbem_num_near_singular_pairs(const fmbem *h) { return h ? h->ns_pairs : 0; }

fmbem_status fmbem_truncation(const fmbem *h, int32_t *p, int32_t *p_level, double *err_level) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (p) *p = h->p;
    for (int l = 0; l <= h->lmax; ++l) {
        if (p_level) p_level[l] = l < (int)h->p_level.size() ? h->p_level[l] : (l >= 2 ? h->p : 0);
        if (err_level) err_level[l] = l < (int)h->trunc_err.size() ? h->trunc_err[l] : -1.0;
    }
    return FMBEM_OK;
}

fmbem_status fmbem_node_geometry(const fmbem *h, double *pos, double *normal, double *weight) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (pos) std::memcpy(pos, h->h_pos.data(), sizeof(double) * 3 * h->N);
    if (normal) std::memcpy(normal, h->h_nrm.data(), sizeof(double) * 3 * h->N);
    if (weight) std::memcpy(weight, h->h_w.data(), sizeof(double) * h->N);
    return FMBEM_OK;
}

fmbem_status fmbem_tree_levels(const fmbem *h, int32_t n, int64_t *boxes, int64_t *leaves) {
    if (!h || n < 0) return FMBEM_ERR_INVALID_ARGUMENT;
    for (int32_t l = 0; l < n; ++l) {
        if (boxes) boxes[l] = l <= h->lmax ? h->lev[l].n : 0;
        if (leaves) leaves[l] = 0;
    }
    if (leaves)
        for (int32_t lv : h->h_leaf_level)
            if (lv < n) ++leaves[lv];
    return FMBEM_OK;
}

fmbem_status fmbem_tree_info(const fmbem *h, int32_t *l_max, int64_t *n_leaves, int64_t *n_boxes, int64_t *near_pairs,
                             int64_t *ff_pairs) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (l_max) *l_max = h->lmax;
    if (n_leaves) *n_leaves = h->n_leaves;
    if (n_boxes) {
        int64_t t = 0;
        for (int l = 2; l <= h->lmax; ++l) t += h->lev[l].n;
        *n_boxes = t;
    }
    if (near_pairs) *near_pairs = h->near_pairs;
    if (ff_pairs) *ff_pairs = h->n_ff;
    return FMBEM_OK;
}

fmbem_status fmbem_plane_wave_rhs(fmbem *h, int64_t n_rhs, const double *dir, const fmbem_c64 *pol, void *b_dev,
                                  void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || !dir || !pol || !b_dev) { h->err = "invalid argument"; return FMBEM_ERR_INVALID_ARGUMENT; }
    return guarded(h, [&] { run_plane_wave(h, n_rhs, dir, pol, (c64 *)b_dev, (cudaStream_t)stream); });
}

fmbem_status fmbem_matvec(fmbem *h, const void *x_dev, void *y_dev, int64_t n_rhs, int precision, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || !x_dev || !y_dev || x_dev == y_dev ||
        (precision != FMBEM_FP64 && precision != FMBEM_FP32 && precision != FMBEM_TF32 && precision != FMBEM_BF16X3)) {
        h->err = "invalid argument (n_rhs >= 1, distinct non-NULL x and y, precision FP64, FP32, TF32 or BF16X3)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] { run_matvec(h, (const c64 *)x_dev, (c64 *)y_dev, n_rhs, precision, (cudaStream_t)stream); });
}

fmbem_status fmbem_matvec_host(fmbem *h, const void *x_host, void *y_host, int64_t n_rhs, int precision,
                               int64_t chunk_rhs, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || chunk_rhs < 0 || !x_host || !y_host || x_host == y_host ||
        (precision != FMBEM_FP64 && precision != FMBEM_FP32 && precision != FMBEM_TF32 && precision != FMBEM_BF16X3)) {
        h->err = "invalid argument (n_rhs >= 1, chunk_rhs >= 0, distinct non-NULL x and y, precision FP64, FP32, "
                 "TF32 or BF16X3)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_matvec_host(h, (const c64 *)x_host, (c64 *)y_host, n_rhs, precision, chunk_rhs, (cudaStream_t)stream);
    });
}

fmbem_status fmbem_adjoint_matvec(fmbem *h, const void *x_dev, void *y_dev, int64_t n_rhs, int precision,
                                  void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || !x_dev || !y_dev || x_dev == y_dev ||
        (precision != FMBEM_FP64 && precision != FMBEM_FP32 && precision != FMBEM_TF32 && precision != FMBEM_BF16X3)) {
        h->err = "invalid argument (n_rhs >= 1, distinct non-NULL x and y, precision FP64, FP32, TF32 or BF16X3)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_adjoint_matvec(h, (const c64 *)x_dev, (c64 *)y_dev, n_rhs, precision, (cudaStream_t)stream);
    });
}

fmbem_status fmbem_matvec_noalloc(fmbem *h, const void *x_dev, void *y_dev, int64_t n_rhs, int precision,
                                  void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || !x_dev || !y_dev || x_dev == y_dev || (precision != FMBEM_FP64 && precision != FMBEM_FP32)) {
        h->err = "invalid argument (n_rhs >= 1, distinct non-NULL x and y, precision FP64 or FP32)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_matvec_noalloc(h, (const c64 *)x_dev, (c64 *)y_dev, n_rhs, precision, (cudaStream_t)stream);
    });
}

fmbem_status fmbem_solve(fmbem *h, const void *b_dev, void *x_dev, int64_t n_rhs, double tol, int max_iter,
                         int32_t *iters_host, double *relres_host, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || !b_dev || !x_dev || !(tol > 0) || max_iter < 1) {
        h->err = "invalid argument";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    fmbem_status res = FMBEM_OK;
    fmbem_status st = guarded(h, [&] {
        res = run_solve(h, (const c64 *)b_dev, (c64 *)x_dev, n_rhs, tol, max_iter, iters_host, relres_host,
                        (cudaStream_t)stream);
    });
    if (st != FMBEM_OK) return st;
    if (res == FMBEM_ERR_NOT_CONVERGED) h->err = "GMRES did not reach the tolerance within max_iter";
    if (res == FMBEM_ERR_BREAKDOWN) h->err = "GMRES produced a non-finite value";
    return res;
}

fmbem_status fmbem_adjoint_solve(fmbem *h, const void *b_dev, void *x_dev, int64_t n_rhs, double tol, int max_iter,
                                 int32_t *iters_host, double *relres_host, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || !b_dev || !x_dev || !(tol > 0) || max_iter < 1) {
        h->err = "invalid argument";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    fmbem_status res = FMBEM_OK;
    fmbem_status st = guarded(h, [&] {
        res = run_solve(h, (const c64 *)b_dev, (c64 *)x_dev, n_rhs, tol, max_iter, iters_host, relres_host,
                        (cudaStream_t)stream, true);
    });
    if (st != FMBEM_OK) return st;
    if (res == FMBEM_ERR_NOT_CONVERGED) h->err = "GMRES did not reach the tolerance within max_iter";
    if (res == FMBEM_ERR_BREAKDOWN) h->err = "GMRES produced a non-finite value";
    return res;
}

fmbem_status fmbem_far_field(fmbem *h, const void *x_dev, int64_t n_rhs, int64_t n_dir, const double *rhat,
                             fmbem_c64 *F_host, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || n_dir < 1 || !x_dev || !rhat || !F_host || n_dir > 65535 || n_rhs > 65535) {
        h->err = "invalid argument (n_rhs, n_dir in 1..65535, non-NULL pointers)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_far_field(h, (const c64 *)x_dev, n_rhs, n_dir, rhat, (c64 *)F_host, (cudaStream_t)stream);
    });
}

fmbem_status fmbem_near_field(fmbem *h, const void *x_dev, int64_t n_rhs, int64_t n_pts, const double *pts,
                              const double *dir, const fmbem_c64 *pol, fmbem_c64 *E_host, fmbem_c64 *H_host,
                              void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || n_pts < 1 || !x_dev || !pts || !E_host || n_rhs > 65535 || (!dir) != (!pol)) {
        h->err = "invalid argument (n_rhs in 1..65535, n_pts >= 1, non-NULL x, pts and E; dir and pol both or neither)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_near_field(h, (const c64 *)x_dev, n_rhs, n_pts, pts, dir, (const c64 *)pol, (c64 *)E_host, (c64 *)H_host,
                       (cudaStream_t)stream);
    });
}

fmbem_status fmbem_cross_sections(fmbem *h, const void *x_dev, int64_t n_rhs, const double *dir, const fmbem_c64 *pol,
                                  int32_t n_theta, int32_t n_phi, double *out_host, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || n_rhs > 65535 || !x_dev || !dir || !pol || !out_host || n_theta < 2 || n_phi < 2 ||
        (int64_t)n_theta * n_phi > (1 << 22)) {
        h->err = "invalid argument (n_rhs in 1..65535, non-NULL x, dir, pol, out; n_theta, n_phi >= 2)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_cross_sections(h, (const c64 *)x_dev, n_rhs, dir, (const c64 *)pol, n_theta, n_phi, out_host,
                           (cudaStream_t)stream);
    });
}

fmbem_status fmbem_force_stress(fmbem *h, const void *x_dev, int64_t n_rhs, const double *dir, const fmbem_c64 *pol,
                                const double *center, double radius, int32_t n_theta, int32_t n_phi, double *out_host,
                                void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || n_rhs > 65535 || !x_dev || !dir || !pol || !center || !out_host || !(radius > 0) ||
        n_theta < 2 || n_phi < 2 || (int64_t)n_theta * n_phi > (1 << 22)) {
        h->err = "invalid argument (n_rhs in 1..65535, non-NULL x, dir, pol, center, out; radius > 0; n_theta, n_phi >= 2)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_force_stress(h, (const c64 *)x_dev, n_rhs, dir, (const c64 *)pol, center, radius, n_theta, n_phi,
                         out_host, (cudaStream_t)stream);
    });
}

fmbem_status fmbem_force_stress_functional(fmbem *h, const void *x_dev, const double *dir, const fmbem_c64 *pol,
                                           const double *center, double radius, int32_t n_theta, int32_t n_phi,
                                           double *force_host, double *pts_host, fmbem_c64 *cE_host,
                                           fmbem_c64 *cH_host, void *L_dev, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (!x_dev || !dir || !pol || !center || !force_host || !L_dev || !(radius > 0) || n_theta < 2 || n_phi < 2 ||
        (int64_t)n_theta * n_phi > (1 << 22)) {
        h->err = "invalid argument (non-NULL x, dir, pol, center, force, L; radius > 0; n_theta, n_phi >= 2)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_force_stress_functional(h, (const c64 *)x_dev, dir, (const c64 *)pol, center, radius, n_theta, n_phi,
                                    force_host, pts_host, (c64 *)cE_host, (c64 *)cH_host, (c64 *)L_dev,
                                    (cudaStream_t)stream);
    });
}

fmbem_status fmbem_eps_sensitivity(fmbem *h, int32_t j, const void *x_dev, const void *lam_dev, int64_t n_rhs,
                                   double step, fmbem_c64 *out_host, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (j < 1 || j > h->J || !x_dev || !lam_dev || !out_host || n_rhs < 1 || n_rhs > 65535 || !(step > 0) || h->ibc ||
        h->opt.fp32_only) {
        h->err = "invalid argument (j in 1..J, non-NULL x, lambda, out; n_rhs in 1..65535; step > 0; penetrable "
                 "boundary; FP64 tables)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_eps_sensitivity(h, j, (const c64 *)x_dev, (const c64 *)lam_dev, n_rhs, step, (c64 *)out_host,
                            (cudaStream_t)stream);
    });
}

fmbem_status fmbem_shape_gradient(fmbem *h, const void *x_dev, const void *lam_dev, int64_t n_rhs, const double *dir,
                                  const fmbem_c64 *pol, const double *rhat, const fmbem_c64 *coef,
                                  fmbem_c64 *out_host, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || n_rhs > 65535 || !x_dev || !lam_dev || !dir || !pol || !rhat || !coef || !out_host) {
        h->err = "invalid argument (n_rhs in 1..65535, non-NULL x, lambda, dir, pol, rhat, coef and out)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    if (h->ns_pairs > 0) {
        h->err = "the vertex-position gradient does not differentiate the near-singular correction (near_singular_radius > 0)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_shape_gradient(h, (const c64 *)x_dev, (const c64 *)lam_dev, n_rhs, dir, (const c64 *)pol, rhat,
                           (const c64 *)coef, 0, nullptr, nullptr, nullptr, (c64 *)out_host, (cudaStream_t)stream);
    });
}

fmbem_status fmbem_shape_gradient_near(fmbem *h, const void *x_dev, const void *lam_dev, int64_t n_rhs,
                                       const double *dir, const fmbem_c64 *pol, int64_t n_pts, const double *pts,
                                       const fmbem_c64 *cE, const fmbem_c64 *cH, fmbem_c64 *out_host, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || n_rhs > 65535 || n_pts < 1 || !x_dev || !lam_dev || !dir || !pol || !pts || !cE || !out_host) {
        h->err = "invalid argument (n_rhs in 1..65535, n_pts >= 1, non-NULL x, lambda, dir, pol, pts, cE and out)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    if (h->ns_pairs > 0) {
        h->err = "the vertex-position gradient does not differentiate the near-singular correction (near_singular_radius > 0)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_shape_gradient(h, (const c64 *)x_dev, (const c64 *)lam_dev, n_rhs, dir, (const c64 *)pol, nullptr, nullptr,
                           n_pts, pts, (const c64 *)cE, (const c64 *)cH, (c64 *)out_host, (cudaStream_t)stream);
    });
}

fmbem_status fmbem_near_field_fmm(fmbem *h, const void *x_dev, int64_t n_rhs, int64_t n_pts, const double *pts,
                                  const double *dir, const fmbem_c64 *pol, fmbem_c64 *E_host, fmbem_c64 *H_host,
                                  void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || n_pts < 1 || !x_dev || !pts || !E_host || n_rhs > 65535 || (!dir) != (!pol)) {
        h->err = "invalid argument (n_rhs in 1..65535, n_pts >= 1, non-NULL x, pts and E; dir and pol both or neither)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_near_field_fmm(h, (const c64 *)x_dev, n_rhs, n_pts, pts, dir, (const c64 *)pol, (c64 *)E_host,
                           (c64 *)H_host, (cudaStream_t)stream);
    });
}

fmbem_status fmbem_interior_field(fmbem *h, const void *x_dev, int64_t n_rhs, int64_t n_pts, const double *pts,
                                  const int32_t *domain, fmbem_c64 *E_host, fmbem_c64 *H_host, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || n_pts < 1 || !x_dev || !pts || !domain || !E_host || n_rhs > 65535) {
        h->err = "invalid argument (n_rhs in 1..65535, n_pts >= 1, non-NULL x, pts, domain and E)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_interior_field(h, (const c64 *)x_dev, n_rhs, n_pts, pts, domain, (c64 *)E_host, (c64 *)H_host,
                           (cudaStream_t)stream);
    });
}

fmbem_status fmbem_far_field_functional(fmbem *h, int64_t n_rhs, const double *rhat, const fmbem_c64 *coef,
                                        void *out_dev, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || n_rhs > 65535 || !rhat || !coef || !out_dev) {
        h->err = "invalid argument (n_rhs in 1..65535, non-NULL pointers)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_far_field_functional(h, n_rhs, rhat, (const c64 *)coef, (c64 *)out_dev, (cudaStream_t)stream);
    });
}

fmbem_status fmbem_near_field_functional(fmbem *h, int64_t n_fun, int64_t n_pts, const double *pts,
                                         const fmbem_c64 *cE, const fmbem_c64 *cH, void *out_dev, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_fun < 1 || n_fun > 65535 || n_pts < 1 || !pts || !cE || !out_dev) {
        h->err = "invalid argument (n_fun in 1..65535, n_pts >= 1, non-NULL pts, cE and out)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] {
        run_near_field_functional(h, n_fun, n_pts, pts, (const c64 *)cE, (const c64 *)cH, (c64 *)out_dev,
                                  (cudaStream_t)stream);
    });
}

fmbem_status fmbem_absorption(fmbem *h, const void *x_dev, int64_t n_rhs, double *out_host, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || !x_dev || !out_host) {
        h->err = "invalid argument";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    return guarded(h, [&] { run_absorption(h, (const c64 *)x_dev, n_rhs, out_host, (cudaStream_t)stream); });
}

fmbem_status fmbem_precond_apply(fmbem *h, const void *v_dev, void *z_dev, int64_t n_rhs, void *stream) {
    if (!h) return FMBEM_ERR_INVALID_ARGUMENT;
    if (n_rhs < 1 || !v_dev || !z_dev) { h->err = "invalid argument"; return FMBEM_ERR_INVALID_ARGUMENT; }
    return guarded(h, [&] { run_precond(h, (const c64 *)v_dev, (c64 *)z_dev, n_rhs, (cudaStream_t)stream); });
}

fmbem_status fmbem_last_matvec_times(const fmbem *h, double *ms) {
    if (!h || !ms) return FMBEM_ERR_INVALID_ARGUMENT;
    if (!h->have_times) {
        for (int i = 0; i < 5; ++i) ms[i] = 0;
        return FMBEM_OK;
    }
    if (cudaEventSynchronize(h->ev[4]) != cudaSuccess) return FMBEM_ERR_CUDA;
    float t;
    for (int i = 0; i < 4; ++i) {
        cudaEventElapsedTime(&t, h->ev[i], h->ev[i + 1]);
        ms[i] = t;
    }
    cudaEventElapsedTime(&t, h->ev[0], h->ev[4]);
    ms[4] = t;
    return FMBEM_OK;
}

}  // extern "C"
