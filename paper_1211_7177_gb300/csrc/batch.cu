// batch.cu -- one persistent kernel launch over many independent problems of uneven size
// (fmbem_batch_*): the host lays out the work items of every problem's product in stage order
// and the completion targets of every stage; k_batch (fmm.cu) runs them.
#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "fmbem_internal.cuh"

struct fmbem_batch {
    std::vector<fmbem *> hs;
    int64_t nr = 0;
    int precision = FMBEM_FP32;
    int p2max = 0;
    int64_t n_items = 0;
    std::vector<BatchProblem> hp;
    std::string err;
    BatchProblem *d_probs = nullptr;
    BatchItem *d_items = nullptr;
    unsigned *d_cnt = nullptr, *d_tgt = nullptr;
    unsigned long long *d_next = nullptr;
    int *d_err = nullptr;
};

static thread_local std::string g_batch_create_error;
static std::atomic<uint64_t> g_batch_wait_ns{2000000000ull};  // 2 s
static std::atomic<int> g_batch_stall{-1};

static void batch_free(fmbem_batch *b) {
    cudaFree(b->d_probs);
    cudaFree(b->d_items);
    cudaFree(b->d_cnt);
    cudaFree(b->d_tgt);
    cudaFree(b->d_next);
    cudaFree(b->d_err);
}

template <typename T>
static T *batch_alloc(size_t n) {
    void *p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1)) != cudaSuccess)
        throw fmbem_error{FMBEM_ERR_OOM, "cudaMalloc of the batch's work items failed"};
    return (T *)p;
}

// the device pointers of one problem (single precision tables)
static BatchProblem batch_problem(const fmbem *h) {
    BatchProblem P{};
    P.N = h->N;
    P.nbox = h->nbox;
    P.p2 = h->p2;
    P.lmax = h->lmax;
    for (int l = 0; l <= h->lmax; ++l) P.lev_off[l] = h->lev[l].off;
    P.perm = h->perm;
    P.dom = h->dom;
    P.nbeg = h->box_nbeg;
    P.nend = h->box_nend;
    P.cbeg = h->box_cbeg;
    P.cend = h->box_cend;
    P.parent = h->box_parent;
    P.ff_start = h->ff_start;
    P.ff_src = h->ff_src;
    P.nbr_start = h->nbr_start;
    P.nbr_idx = h->nbr_idx;
    P.ff_off = h->ff_off;
    P.key = h->box_key;
    P.nrm64 = h->nrm;
    P.w = h->w;
    P.pos_hi = h->pos_hi;
    P.pos_lo = h->pos_lo;
    P.nrm = h->nrm_f;
    P.dc = h->dcons;
    P.Bp2m = h->B_p2m32;
    P.Bl2p = h->B_l2p32;
    P.Tmm = h->T_mm32;
    P.Tm2l = h->T_m2l32;
    P.Tll = h->T_ll32;
    P.dens = h->dens;
    P.C = h->Cexp;
    P.D = h->Dexp;
    P.Mself = h->Mself;
    return P;
}

extern "C" {

fmbem_status fmbem_batch_create(fmbem *const *handles, int32_t n_problems, int64_t n_rhs, int precision,
                                fmbem_batch **out) {
    if (out) *out = nullptr;
    if (!handles || !out || n_problems < 1 || n_rhs < 1 || n_rhs > 64) {
        g_batch_create_error = "invalid argument (non-NULL handles and out, n_problems >= 1, n_rhs in 1..64)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    if (precision != FMBEM_FP32) {
        g_batch_create_error = "the batch runs the FP32 passes (precision FMBEM_FP32)";
        return FMBEM_ERR_INVALID_ARGUMENT;
    }
    for (int32_t i = 0; i < n_problems; ++i) {
        const fmbem *h = handles[i];
        if (!h) {
            g_batch_create_error = "handle " + std::to_string(i) + " is NULL";
            return FMBEM_ERR_INVALID_ARGUMENT;
        }
        if (h->ibc || h->ns_pairs > 0 || h->p2 > 128 || h->lmax > BATCH_MAX_LEVEL || h->adaptive) {
            g_batch_create_error = "handle " + std::to_string(i) +
                                   ": the batch needs the penetrable boundary, the uniform octree, no near-singular "
                                   "correction, p <= 11";
            return FMBEM_ERR_INVALID_ARGUMENT;
        }
    }
    fmbem_batch *b = new (std::nothrow) fmbem_batch();
    if (!b) { g_batch_create_error = "host allocation failed"; return FMBEM_ERR_OOM; }
    try {
        b->hs.assign(handles, handles + n_problems);
        b->nr = n_rhs;
        b->precision = precision;
        const int64_t nr = n_rhs;
        const int nchunk = (int)((3 * nr + BATCH_CHUNK_COLS - 1) / BATCH_CHUNK_COLS);
        // work items in stage order: densities, P2M, M2M from the deepest child level up, M2L + L2L
        // from level 2 down, near field; within a stage, problem by problem
        std::vector<BatchItem> items;
        std::vector<unsigned> tgt((size_t)n_problems * BATCH_COUNTERS, 0);
        int max_lmax = 2;
        for (fmbem *h : b->hs) max_lmax = std::max(max_lmax, h->lmax);
        auto add = [&](int32_t i, int16_t kind, int16_t level, int32_t a, int16_t bb, int16_t c) {
            items.push_back(BatchItem{i, kind, level, a, bb, c});
            tgt[(size_t)i * BATCH_COUNTERS + batch_done_counter(kind, level, b->hs[i]->lmax)]++;
        };
        for (int32_t i = 0; i < n_problems; ++i) {
            const fmbem *h = b->hs[i];
            for (int64_t r = 0; r < nr; ++r)
                for (int64_t blk = 0; blk < (h->N + 127) / 128; ++blk) add(i, BK_PREP, 0, (int32_t)blk, 0, (int16_t)r);
        }
        for (int32_t i = 0; i < n_problems; ++i) {
            const fmbem *h = b->hs[i];
            for (int64_t r = 0; r < nr; ++r)
                for (int d = 0; d <= h->J; ++d)
                    for (int64_t lf = 0; lf < h->lev[h->lmax].n; ++lf) add(i, BK_P2M, 0, (int32_t)lf, (int16_t)d, (int16_t)r);
        }
        for (int k = 0; k <= max_lmax - 3; ++k)
            for (int32_t i = 0; i < n_problems; ++i) {
                const fmbem *h = b->hs[i];
                const int l = h->lmax - k;  // child level
                if (l < 3) continue;
                for (int c = 0; c < nchunk; ++c)
                    for (int d = 0; d <= h->J; ++d)
                        for (int64_t pb = 0; pb < h->lev[l - 1].n; ++pb)
                            add(i, BK_M2M, (int16_t)l, (int32_t)pb, (int16_t)d, (int16_t)c);
            }
        for (int l = 2; l <= max_lmax; ++l)
            for (int32_t i = 0; i < n_problems; ++i) {
                const fmbem *h = b->hs[i];
                if (l > h->lmax) continue;
                for (int c = 0; c < nchunk; ++c)
                    for (int d = 0; d <= h->J; ++d)
                        for (int64_t bx = 0; bx < h->lev[l].n; ++bx)
                            add(i, BK_DOWN, (int16_t)l, (int32_t)bx, (int16_t)d, (int16_t)c);
            }
        for (int32_t i = 0; i < n_problems; ++i) {
            const fmbem *h = b->hs[i];
            for (int64_t lf = 0; lf < h->lev[h->lmax].n; ++lf) add(i, BK_NEAR, 0, (int32_t)lf, 0, 0);
        }
        b->n_items = (int64_t)items.size();
        for (fmbem *h : b->hs) {
            batch_ensure_scratch(h, nr, precision);
            b->p2max = std::max(b->p2max, h->p2);
        }
        b->hp.resize(n_problems);
        b->d_probs = batch_alloc<BatchProblem>(n_problems);
        b->d_items = batch_alloc<BatchItem>(items.size());
        b->d_cnt = batch_alloc<unsigned>(tgt.size());
        b->d_tgt = batch_alloc<unsigned>(tgt.size());
        b->d_next = batch_alloc<unsigned long long>(1);
        b->d_err = batch_alloc<int>(1);
        CK(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b->d_tgt, tgt.data(), sizeof(unsigned) * tgt.size(), cudaMemcpyHostToDevice));
    } catch (const fmbem_error &e) {
        g_batch_create_error = e.msg;
        batch_free(b);
        delete b;
        return e.st;
    } catch (...) {
        g_batch_create_error = "host allocation failed";
        batch_free(b);
        delete b;
        return FMBEM_ERR_OOM;
    }
    *out = b;
    return FMBEM_OK;
}

fmbem_status fmbem_batch_matvec(fmbem_batch *b, const void *const *x_dev, void *const *y_dev, void *stream) {
    if (!b) return FMBEM_ERR_INVALID_ARGUMENT;
    const int32_t n = (int32_t)b->hs.size();
    if (!x_dev || !y_dev) { b->err = "NULL x or y pointer array"; return FMBEM_ERR_INVALID_ARGUMENT; }
    for (int32_t i = 0; i < n; ++i)
        if (!x_dev[i] || !y_dev[i] || x_dev[i] == y_dev[i]) {
            b->err = "problem " + std::to_string(i) + ": NULL or overlapping x and y";
            return FMBEM_ERR_INVALID_ARGUMENT;
        }
    cudaStream_t s = (cudaStream_t)stream;
    try {
        // a handle used alone in between may have regrown its scratch: take its pointers now
        for (int32_t i = 0; i < n; ++i) {
            batch_ensure_scratch(b->hs[i], b->nr, b->precision);
            b->hp[i] = batch_problem(b->hs[i]);
            b->hp[i].x = (const c64 *)x_dev[i];
            b->hp[i].y = (c64 *)y_dev[i];
        }
        CK(cudaMemcpyAsync(b->d_probs, b->hp.data(), sizeof(BatchProblem) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(b->d_cnt, 0, sizeof(unsigned) * (size_t)n * BATCH_COUNTERS, s));
        CK(cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), s));
        CK(cudaMemsetAsync(b->d_err, 0, sizeof(int), s));
        const int stall = g_batch_stall.load();
        run_batch_kernel(b->precision, b->d_probs, b->d_items, b->n_items, b->d_next, b->d_cnt, b->d_tgt, b->d_err,
                         g_batch_wait_ns.load(), stall < n ? stall : -1, b->p2max, b->nr, s);
        int e = 0;
        CK(cudaMemcpyAsync(&e, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (e) {
            b->err = "a work item's wait for its inputs ran out (bounded spin of the persistent batch kernel)";
            return FMBEM_ERR_DEVICE_TIMEOUT;
        }
    } catch (const fmbem_error &er) {
        b->err = er.msg;
        return er.st;
    } catch (...) {
        b->err = "host allocation failed";
        return FMBEM_ERR_OOM;
    }
    b->err.clear();
    return FMBEM_OK;
}

int64_t fmbem_batch_num_items(const fmbem_batch *b) { return b ? b->n_items : 0; }

void fmbem_batch_destroy(fmbem_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

const char *fmbem_batch_last_error(const fmbem_batch *b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

void fmbem_debug_set_batch_wait(uint64_t wait_ns, int32_t stall_problem) {
    g_batch_wait_ns.store(wait_ns > 0 ? wait_ns : 2000000000ull);
    g_batch_stall.store(stall_problem);
}

}  // extern "C"
