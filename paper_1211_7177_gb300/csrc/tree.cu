// tree.cu -- octree over the Nystrom nodes and its box relations (Appendix C, Section 2.2):
// root cube around the nodes, Morton keys, stable radix sort of the nodes, non-empty boxes on
// every level (empty boxes are dropped), Parent/Children, Neighbor lists of the leaves and FF
// lists (children of the parent's neighbours that are not neighbours themselves) on levels 2..l_max.
#include <algorithm>
#include <cstring>

#include "fmbem_internal.cuh"

namespace {

constexpr int KEY_LEVELS = 10;  // Morton keys resolve 2^10 boxes per axis

// ---------------------------------------------------------------- device-wide exclusive scan
constexpr int SCAN_TB = 1024;

__global__ void k_scan_block(const int32_t *in, int32_t *out, int32_t *block_sums, int64_t n) {
    __shared__ int32_t s[SCAN_TB];
    int64_t i = blockIdx.x * (int64_t)SCAN_TB + threadIdx.x;
    int32_t v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_TB; off <<= 1) {
        int32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive
    if (threadIdx.x == SCAN_TB - 1) block_sums[blockIdx.x] = s[SCAN_TB - 1];
}
__global__ void k_scan_add(int32_t *out, const int32_t *block_off, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)SCAN_TB + threadIdx.x;
    if (i < n) out[i] += block_off[blockIdx.x];
}

// exclusive scan of n int32 values; returns the total
int64_t scan_exclusive(fmbem *h, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    if (n == 0) return 0;
    int64_t nb = (n + SCAN_TB - 1) / SCAN_TB;
    int32_t *sums = (int32_t *)dev_alloc(h, sizeof(int32_t) * (nb + 1));
    int32_t *offs = (int32_t *)dev_alloc(h, sizeof(int32_t) * (nb + 1));
    k_scan_block<<<(unsigned)nb, SCAN_TB, 0, s>>>(in, out, sums, n);
    CKL("k_scan_block");
    int64_t total;
    if (nb > 1) {
        total = scan_exclusive(h, sums, offs, nb, s);
        k_scan_add<<<(unsigned)nb, SCAN_TB, 0, s>>>(out, offs, n);
        CKL("k_scan_add");
    } else {
        int32_t t;
        CK(cudaMemcpyAsync(&t, sums, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        total = t;
    }
    dev_free(h, sums);
    dev_free(h, offs);
    return total;
}

// ---------------------------------------------------------------- bounding box
__global__ void k_bbox(const double *pos, int64_t N, double *out /* [nblocks][6] */) {
    __shared__ double s[6][256];
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int q = 0; q < 3; ++q) { mn[q] = fmin(mn[q], pos[3 * i + q]); mx[q] = fmax(mx[q], pos[3 * i + q]); }
    for (int q = 0; q < 3; ++q) { s[q][threadIdx.x] = mn[q]; s[3 + q][threadIdx.x] = mx[q]; }
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int q = 0; q < 3; ++q) {
                s[q][threadIdx.x] = fmin(s[q][threadIdx.x], s[q][threadIdx.x + off]);
                s[3 + q][threadIdx.x] = fmax(s[3 + q][threadIdx.x], s[3 + q][threadIdx.x + off]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) out[6 * blockIdx.x + q] = s[q][0];
}

// ---------------------------------------------------------------- Morton keys
__host__ __device__ __forceinline__ uint64_t spread3(uint32_t v) {  // 10 bits -> every third bit
    uint64_t x = v & 0x3ff;
    x = (x | (x << 16)) & 0x30000ffULL;
    x = (x | (x << 8)) & 0x300f00fULL;
    x = (x | (x << 4)) & 0x30c30c3ULL;
    x = (x | (x << 2)) & 0x9249249ULL;
    return x;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x9249249ULL;
    x = (x | (x >> 2)) & 0x30c30c3ULL;
    x = (x | (x >> 4)) & 0x300f00fULL;
    x = (x | (x >> 8)) & 0x30000ffULL;
    x = (x | (x >> 16)) & 0x3ffULL;
    return (uint32_t)x;
}
__host__ __device__ __forceinline__ uint64_t morton(uint32_t ix, uint32_t iy, uint32_t iz) {
    return (spread3(ix) << 2) | (spread3(iy) << 1) | spread3(iz);
}
__host__ __device__ __forceinline__ void demorton(uint64_t key, int &ix, int &iy, int &iz) {
    ix = (int)compact3(key >> 2);
    iy = (int)compact3(key >> 1);
    iz = (int)compact3(key);
}

// box index along each axis = floor((x - x_min) / w) clamped to [0, 2^10 - 1]
__global__ void k_keys(const double *pos, int64_t N, double x0, double y0, double z0, double inv_w, uint64_t *key,
                       int32_t *idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int M = 1 << KEY_LEVELS;
    double o[3] = {x0, y0, z0};
    uint32_t c[3];
    for (int q = 0; q < 3; ++q) {
        double t = floor((pos[3 * i + q] - o[q]) * inv_w);
        int v = (int)t;
        c[q] = (uint32_t)min(max(v, 0), M - 1);
    }
    key[i] = morton(c[0], c[1], c[2]);
    idx[i] = (int32_t)i;
}

// ---------------------------------------------------------------- stable 1-bit split radix sort
__global__ void k_bitflag(const uint64_t *key, int64_t n, int bit, int32_t *zero_flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) zero_flag[i] = ((key[i] >> bit) & 1ULL) ? 0 : 1;
}
__global__ void k_bitscatter(const uint64_t *key, const int32_t *idx, const int32_t *zpos, int64_t n, int64_t nzero, int bit,
                             uint64_t *key2, int32_t *idx2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool one = (key[i] >> bit) & 1ULL;
    int64_t dst = one ? nzero + (i - zpos[i]) : zpos[i];
    key2[dst] = key[i];
    idx2[dst] = idx[i];
}

// ---------------------------------------------------------------- per-level boxes
__global__ void k_level_flags(const uint64_t *key, int64_t n, int shift, int32_t *flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || (key[i] >> shift) != (key[i - 1] >> shift)) ? 1 : 0;
}
// node -> box id (inclusive scan - 1) and box start positions
__global__ void k_level_boxes(const uint64_t *key, const int32_t *flag, const int32_t *excl, int64_t n, int shift,
                              int32_t *node_box, int32_t *box_start, uint64_t *box_key) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t b = excl[i] + flag[i] - 1;
    node_box[i] = b;
    if (flag[i]) {
        box_start[b] = (int32_t)i;
        box_key[b] = key[i] >> shift;
    }
}
__global__ void k_max_occupancy(const int32_t *box_start, int64_t nb, int64_t n, int32_t *out) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int32_t e = b + 1 < nb ? box_start[b + 1] : (int32_t)n;
    atomicMax(out, e - box_start[b]);
}

// fill global box arrays of one level
__global__ void k_fill_level(int64_t nb, int64_t off, int l, const int32_t *box_start, const uint64_t *lkey, int64_t n,
                             const int32_t *node_box_parent /* level l-1, or null */, int64_t off_parent,
                             double x0, double y0, double z0, double w, uint64_t *gkey, double *gctr,
                             int32_t *gparent, int32_t *nbeg, int32_t *nend) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int64_t g = off + b;
    uint64_t kk = lkey[b];
    gkey[g] = kk;
    int ix, iy, iz;
    demorton(kk, ix, iy, iz);
    gctr[3 * g + 0] = x0 + (ix + 0.5) * w;
    gctr[3 * g + 1] = y0 + (iy + 0.5) * w;
    gctr[3 * g + 2] = z0 + (iz + 0.5) * w;
    int32_t s = box_start[b];
    nbeg[g] = s;
    nend[g] = b + 1 < nb ? box_start[b + 1] : (int32_t)n;
    gparent[g] = node_box_parent ? (int32_t)(off_parent + node_box_parent[s]) : -1;
}
// children range of the boxes of level l from the node->box map of level l+1
__global__ void k_children(int64_t nb, int64_t off, const int32_t *nbeg, const int32_t *nend, const int32_t *node_box_child,
                           int64_t off_child, int32_t *cbeg, int32_t *cend) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int64_t g = off + b;
    cbeg[g] = (int32_t)(off_child + node_box_child[nbeg[g]]);
    cend[g] = (int32_t)(off_child + node_box_child[nend[g] - 1] + 1);
}

// binary search of a key among the sorted keys of one level; returns global index or -1
__device__ __forceinline__ int64_t find_box(const uint64_t *gkey, int64_t off, int64_t nb, uint64_t kk) {
    int64_t lo = 0, hi = nb;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (gkey[off + mid] < kk) lo = mid + 1;
        else hi = mid;
    }
    return (lo < nb && gkey[off + lo] == kk) ? off + lo : -1;
}

// Neighbor(l,q) plus the box itself, for the leaves (pass 0 counts, pass 1 fills)
__global__ void k_neighbors(int64_t nb, int64_t off, int l, const uint64_t *gkey, const int32_t *start, int32_t *cnt,
                            int32_t *idx, const int32_t *nbeg, const int32_t *nend, int64_t *pair_count) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int64_t g = off + b;
    int ix, iy, iz;
    demorton(gkey[g], ix, iy, iz);
    const int M = 1 << l;
    int c = 0;
    int64_t pairs = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                if (jx < 0 || jy < 0 || jz < 0 || jx >= M || jy >= M || jz >= M) continue;
                int64_t q = find_box(gkey, off, nb, morton(jx, jy, jz));
                if (q < 0) continue;
                if (idx) idx[start[b] + c] = (int32_t)q;
                pairs += nend[q] - nbeg[q];
                ++c;
            }
    if (cnt) cnt[b] = c;
    if (pair_count) atomicAdd((unsigned long long *)pair_count, (unsigned long long)(pairs * (nend[g] - nbeg[g])));
}

// FF(l,q) = Children(Neighbor(Parent(l,q))) \ Neighbor(l,q), with the offset code of each entry
__global__ void k_farfield(int64_t nb, int64_t off, int l, const uint64_t *gkey, int64_t off_par, int64_t nb_par,
                           const int32_t *cbeg, const int32_t *cend, const int32_t *start, int32_t *cnt, int32_t *src,
                           int16_t *code) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int64_t g = off + b;
    int ix, iy, iz;
    demorton(gkey[g], ix, iy, iz);
    int px = ix >> 1, py = iy >> 1, pz = iz >> 1;
    const int Mp = 1 << (l - 1);
    int c = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int qx = px + dx, qy = py + dy, qz = pz + dz;
                if (qx < 0 || qy < 0 || qz < 0 || qx >= Mp || qy >= Mp || qz >= Mp) continue;
                int64_t P = find_box(gkey, off_par, nb_par, morton(qx, qy, qz));
                if (P < 0) continue;
                for (int ch = cbeg[P]; ch < cend[P]; ++ch) {
                    int jx, jy, jz;
                    demorton(gkey[ch], jx, jy, jz);
                    int ex = jx - ix, ey = jy - iy, ez = jz - iz;
                    if (abs(ex) <= 1 && abs(ey) <= 1 && abs(ez) <= 1) continue;  // a neighbour
                    if (src) {
                        src[start[b] + c] = ch;
                        code[start[b] + c] = (int16_t)m2l_offset_code(ex, ey, ez);
                    }
                    ++c;
                }
            }
    if (cnt) cnt[b] = c;
}

// sorted copies of the node geometry, double-float positions for the single-precision passes
__global__ void k_sorted_geometry(int64_t N, const int32_t *perm, const double *upos, const double *unrm, const double *uw,
                                  const int32_t *udom, double *pos, double *nrm, double *w, int32_t *dom, int32_t *iperm,
                                  float *hi, float *lo, float *nf, float4 *rec) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int32_t u = perm[i];
    iperm[u] = (int32_t)i;
    for (int q = 0; q < 3; ++q) {
        double x = upos[3 * u + q];
        pos[3 * i + q] = x;
        nrm[3 * i + q] = unrm[3 * u + q];
        float xh = (float)x;
        hi[3 * i + q] = xh;
        lo[3 * i + q] = (float)(x - (double)xh);
        nf[3 * i + q] = (float)unrm[3 * u + q];
    }
    w[i] = uw[u];
    dom[i] = udom[u];
    // the single-precision near field's 48-byte source record: (x_hi, y_hi, z_hi, scatterer id
    // bits), (x_lo, y_lo, z_lo, n_x), (n_y, n_z, 0, 0)
    rec[3 * i] = make_float4(hi[3 * i], hi[3 * i + 1], hi[3 * i + 2], __int_as_float(udom[u]));
    rec[3 * i + 1] = make_float4(lo[3 * i], lo[3 * i + 1], lo[3 * i + 2], nf[3 * i]);
    rec[3 * i + 2] = make_float4(nf[3 * i + 1], nf[3 * i + 2], 0.f, 0.f);
}

// target box of every FF CSR entry
__global__ void k_pair_targets(int64_t nbox, const int32_t *ff_start, int32_t *pair_tgt) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    for (int e = ff_start[b]; e < ff_start[b + 1]; ++e) pair_tgt[e] = (int32_t)b;
}
__global__ void k_count_offsets(int64_t e0, int64_t e1, const int16_t *code, int32_t *cnt) {
    int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < e1) atomicAdd(&cnt[code[e]], 1);
}
// the order inside an offset bucket does not matter: every pair's result is stored at its own
// CSR position and reduced per target in CSR order
__global__ void k_fill_offsets(int64_t e0, int64_t e1, const int16_t *code, int32_t *next, int32_t *pair_e) {
    int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < e1) pair_e[atomicAdd(&next[code[e]], 1)] = (int32_t)e;
}

__global__ void k_add_offset(int32_t *a, int64_t n, int32_t off) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] += off;
}

inline unsigned nblk(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

// the leaf (position in the leaf order) containing each point, or -1 when the point lies outside
// the root cube or in an empty box: the key of the point's box at each level (as k_keys, without
// clamping), looked up by bisection among that level's sorted keys from the deepest level up; the
// first box found is the deepest one that contains the point, and the answer is its leaf position
// (-1 when it is not a leaf: the point lies in an empty part of a subdivided box)
__global__ void k_locate_leaf(int64_t n, const double *pts, double x0, double y0, double z0, double inv_w, int lmax,
                              const int64_t *lev_off, const uint64_t *box_key, const int32_t *box_leafpos,
                              int32_t *leaf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int M = 1 << KEY_LEVELS;
    const double o[3] = {x0, y0, z0};
    uint32_t c[3];
    bool inside = true;
    for (int q = 0; q < 3; ++q) {
        const double t = floor((pts[3 * i + q] - o[q]) * inv_w);
        inside = inside && t >= 0.0 && t < (double)M;
        c[q] = inside ? (uint32_t)t : 0u;
    }
    int32_t found = -1;
    if (inside) {
        const uint64_t full = morton(c[0], c[1], c[2]);
        for (int l = lmax; l >= 0; --l) {
            const uint64_t key = full >> (3 * (KEY_LEVELS - l));
            const int64_t off = lev_off[l], nb = lev_off[l + 1] - off;
            int64_t lo = 0, hi = nb;
            while (lo < hi) {
                const int64_t mid = (lo + hi) / 2;
                if (box_key[off + mid] < key) lo = mid + 1;
                else hi = mid;
            }
            if (lo < nb && box_key[off + lo] == key) {
                found = box_leafpos[off + lo];
                break;
            }
        }
    }
    leaf[i] = found;
}

}  // namespace

void run_locate_leaves(fmbem *h, const double *pts_dev, int64_t n, int32_t *leaf_dev, cudaStream_t s) {
    std::vector<int64_t> off(h->lmax + 2);
    for (int l = 0; l <= h->lmax; ++l) off[l] = h->lev[l].off;
    off[h->lmax + 1] = h->nbox;
    int64_t *doff = (int64_t *)dev_alloc(h, sizeof(int64_t) * off.size());
    CK(cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, s));
    k_locate_leaf<<<nblk(n, 128), 128, 0, s>>>(n, pts_dev, h->root_min[0], h->root_min[1], h->root_min[2],
                                               (double)(1 << KEY_LEVELS) / h->root_w, h->lmax, doff, h->box_key,
                                               h->box_leafpos, leaf_dev);
    CKL("k_locate_leaf");
    CK(cudaStreamSynchronize(s));
    dev_free(h, doff);
}

namespace {

// leaf arrays from h_leaf_box (global boxes of the leaves, node order): device copy, the leaf
// position of every box (-1 for the others) and the level of every leaf
void finish_leaves(fmbem *h, cudaStream_t s) {
    const int64_t nl = (int64_t)h->h_leaf_box.size();
    h->n_leaves = nl;
    h->h_leaf_level.resize(nl);
    std::vector<int32_t> pos(h->nbox, -1);
    for (int64_t i = 0; i < nl; ++i) {
        const int32_t g = h->h_leaf_box[i];
        pos[g] = (int32_t)i;
        int l = h->lmax;
        while (l > 0 && h->lev[l].off > g) --l;
        h->h_leaf_level[i] = l;
    }
    h->leaf_box = (int32_t *)dev_alloc(h, sizeof(int32_t) * std::max<int64_t>(nl, 1));
    h->leaf_level = (int32_t *)dev_alloc(h, sizeof(int32_t) * std::max<int64_t>(nl, 1));
    h->box_leafpos = (int32_t *)dev_alloc(h, sizeof(int32_t) * h->nbox);
    CK(cudaMemcpyAsync(h->leaf_box, h->h_leaf_box.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->leaf_level, h->h_leaf_level.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->box_leafpos, pos.data(), sizeof(int32_t) * h->nbox, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
}

}  // namespace

namespace {

// Per-branch adaptive octree: a box is split into its non-empty octants while it holds more than
// leaf_size nodes (levels 0 and 1 always; no box below max_level), so leaves lie on several
// levels.  The passes then count every (target, source) pair once: by M2L between well-separated
// boxes of one level whose parents are adjacent (the paper's FF lists, built as for the uniform
// tree: a parent's colleague that is a leaf has no children), or directly.  The direct sources of
// a leaf T on level l are
//   (a) the boxes of level l adjacent to T, and T itself, leaves or not (all nodes below them),
//   (b) for every ancestor A of T, the leaves on A's level adjacent to A
// (the per-target form of the U, W and X lists of adaptive FMMs with the W and X interactions
// summed directly).  The nodes below a box are contiguous in Morton order, so each entry is a node
// range; a leaf's ranges are sorted and merged, and a merged range that is not one box's becomes
// a range entry after the boxes in box_nbeg / box_nend.
constexpr int NEAR_RANGES_MAX = 32;  // the near-field kernels stage at most 32 ranges per leaf

void adaptive_boxes(fmbem *h, const uint64_t *key_dev, double side, cudaStream_t s) {
    const int64_t N = h->N;
    std::vector<uint64_t> hk(N);
    CK(cudaMemcpyAsync(hk.data(), key_dev, sizeof(uint64_t) * N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int cap = std::max(2, std::min(h->opt.max_level, KEY_LEVELS));
    const int64_t leaf_size = h->opt.leaf_size;
    struct Box {
        uint64_t key;
        int32_t nb, ne, parent, cb, ce;
        bool leaf;
    };
    std::vector<std::vector<Box>> L(1);
    L[0].push_back(Box{0, 0, (int32_t)N, -1, 0, 0, false});
    for (int l = 0;; ++l) {
        std::vector<Box> next;
        const int shift = 3 * (KEY_LEVELS - (l + 1));
        for (size_t b = 0; b < L[l].size(); ++b) {
            Box &B = L[l][b];
            B.leaf = l >= 2 && (B.ne - B.nb <= leaf_size || l == cap);
            if (B.leaf) continue;
            B.cb = (int32_t)next.size();
            for (int32_t i = B.nb; i < B.ne;) {
                const uint64_t ck = hk[i] >> shift;
                int32_t j = i + 1;
                while (j < B.ne && (hk[j] >> shift) == ck) ++j;
                next.push_back(Box{ck, i, j, (int32_t)b, 0, 0, false});
                i = j;
            }
            B.ce = (int32_t)next.size();
        }
        if (next.empty()) break;
        L.push_back(std::move(next));
    }
    const int lmax = (int)L.size() - 1;
    h->lmax = lmax;
    h->lev.assign(lmax + 1, LevelInfo{});
    int64_t tot = 0;
    for (int l = 0; l <= lmax; ++l) {
        h->lev[l].off = tot;
        h->lev[l].n = (int64_t)L[l].size();
        h->lev[l].w = side / (double)(1 << l);
        tot += h->lev[l].n;
    }
    h->nbox = tot;
    // global box arrays, and per level the sorted keys for lookups
    std::vector<uint64_t> gkey(tot);
    std::vector<double> gctr(3 * tot);
    std::vector<int32_t> gpar(tot), gcb(tot, 0), gce(tot, 0), gnb(tot), gne(tot);
    std::vector<char> is_leaf(tot, 0);
    std::vector<std::pair<int32_t, int32_t>> leaves;  // (first node, global box)
    for (int l = 0; l <= lmax; ++l)
        for (size_t b = 0; b < L[l].size(); ++b) {
            const Box &B = L[l][b];
            const int64_t g = h->lev[l].off + (int64_t)b;
            gkey[g] = B.key;
            int ix, iy, iz;
            demorton(B.key, ix, iy, iz);
            gctr[3 * g] = h->root_min[0] + (ix + 0.5) * h->lev[l].w;
            gctr[3 * g + 1] = h->root_min[1] + (iy + 0.5) * h->lev[l].w;
            gctr[3 * g + 2] = h->root_min[2] + (iz + 0.5) * h->lev[l].w;
            gpar[g] = l > 0 ? (int32_t)(h->lev[l - 1].off + B.parent) : -1;
            if (!B.leaf && l < lmax) {
                gcb[g] = (int32_t)(h->lev[l + 1].off + B.cb);
                gce[g] = (int32_t)(h->lev[l + 1].off + B.ce);
            }
            gnb[g] = B.nb;
            gne[g] = B.ne;
            if (B.leaf) {
                is_leaf[g] = 1;
                leaves.emplace_back(B.nb, (int32_t)g);
            }
        }
    std::sort(leaves.begin(), leaves.end());
    const int64_t nl = (int64_t)leaves.size();
    h->h_leaf_box.resize(nl);
    std::vector<int32_t> node_leaf(N);
    int32_t max_leaf = 0;
    for (int64_t i = 0; i < nl; ++i) {
        const int32_t g = leaves[i].second;
        h->h_leaf_box[i] = g;
        for (int32_t j = gnb[g]; j < gne[g]; ++j) node_leaf[j] = g;
        max_leaf = std::max(max_leaf, gne[g] - gnb[g]);
    }
    h->max_leaf = max_leaf;
    // box of level l at integer coordinates (ix, iy, iz), or -1
    auto find = [&](int l, int ix, int iy, int iz) -> int64_t {
        const int M = 1 << l;
        if (ix < 0 || iy < 0 || iz < 0 || ix >= M || iy >= M || iz >= M) return -1;
        const uint64_t kk = morton((uint32_t)ix, (uint32_t)iy, (uint32_t)iz);
        const uint64_t *k0 = gkey.data() + h->lev[l].off, *k1 = k0 + h->lev[l].n;
        const uint64_t *it = std::lower_bound(k0, k1, kk);
        return (it != k1 && *it == kk) ? h->lev[l].off + (it - k0) : -1;
    };
    std::vector<int32_t> nstart(nl + 1, 0), nidx, rnb, rne;
    int64_t pairs = 0;
    for (int64_t i = 0; i < nl; ++i) {
        const int32_t g = h->h_leaf_box[i];
        int l = lmax;
        while (h->lev[l].off > g) --l;
        int ix, iy, iz;
        demorton(gkey[g], ix, iy, iz);
        std::vector<int64_t> src;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    const int64_t q = find(l, ix + dx, iy + dy, iz + dz);
                    if (q >= 0) src.push_back(q);
                }
        for (int la = l - 1; la >= 0; --la) {
            const int sh = l - la, ax = ix >> sh, ay = iy >> sh, az = iz >> sh;
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        if (dx == 0 && dy == 0 && dz == 0) continue;
                        const int64_t q = find(la, ax + dx, ay + dy, az + dz);
                        if (q >= 0 && is_leaf[q]) src.push_back(q);
                    }
        }
        // node ranges in node order, merged where they touch
        std::sort(src.begin(), src.end(), [&](int64_t u, int64_t v) { return gnb[u] < gnb[v]; });
        int64_t nsrc = 0;
        for (size_t a = 0; a < src.size();) {
            size_t b = a + 1;
            while (b < src.size() && gnb[src[b]] == gne[src[b - 1]]) ++b;
            const int32_t beg = gnb[src[a]], end = gne[src[b - 1]];
            if (b == a + 1) {
                nidx.push_back((int32_t)src[a]);
            } else {
                nidx.push_back((int32_t)(tot + (int64_t)rnb.size()));
                rnb.push_back(beg);
                rne.push_back(end);
            }
            nsrc += end - beg;
            a = b;
        }
        nstart[i + 1] = (int32_t)nidx.size();
        if (nstart[i + 1] - nstart[i] > NEAR_RANGES_MAX)
            throw fmbem_error{FMBEM_ERR_INVALID_ARGUMENT,
                              "adaptive octree: a leaf has " + std::to_string(nstart[i + 1] - nstart[i]) +
                                  " direct-source node ranges (at most " + std::to_string(NEAR_RANGES_MAX) +
                                  "); use a larger leaf_size or a smaller max_level"};
        pairs += nsrc * (gne[g] - gnb[g]);
    }
    h->near_pairs = pairs - N;  // minus the self pairs
    h->n_nbr = (int64_t)nidx.size();
    h->n_range_boxes = (int64_t)rnb.size();
    // device copies
    const int64_t nr_all = tot + h->n_range_boxes;
    h->box_key = (uint64_t *)dev_alloc(h, sizeof(uint64_t) * tot);
    h->box_ctr = (double *)dev_alloc(h, sizeof(double) * 3 * tot);
    h->box_parent = (int32_t *)dev_alloc(h, sizeof(int32_t) * tot);
    h->box_cbeg = (int32_t *)dev_alloc(h, sizeof(int32_t) * tot);
    h->box_cend = (int32_t *)dev_alloc(h, sizeof(int32_t) * tot);
    h->box_nbeg = (int32_t *)dev_alloc(h, sizeof(int32_t) * nr_all);
    h->box_nend = (int32_t *)dev_alloc(h, sizeof(int32_t) * nr_all);
    h->nbr_start = (int32_t *)dev_alloc(h, sizeof(int32_t) * (nl + 1));
    h->nbr_idx = (int32_t *)dev_alloc(h, sizeof(int32_t) * std::max<size_t>(nidx.size(), 1));
    h->node_leaf = (int32_t *)dev_alloc(h, sizeof(int32_t) * N);
    gnb.insert(gnb.end(), rnb.begin(), rnb.end());
    gne.insert(gne.end(), rne.begin(), rne.end());
    CK(cudaMemcpyAsync(h->box_key, gkey.data(), sizeof(uint64_t) * tot, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->box_ctr, gctr.data(), sizeof(double) * 3 * tot, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->box_parent, gpar.data(), sizeof(int32_t) * tot, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->box_cbeg, gcb.data(), sizeof(int32_t) * tot, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->box_cend, gce.data(), sizeof(int32_t) * tot, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->box_nbeg, gnb.data(), sizeof(int32_t) * nr_all, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->box_nend, gne.data(), sizeof(int32_t) * nr_all, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->nbr_start, nstart.data(), sizeof(int32_t) * (nl + 1), cudaMemcpyHostToDevice, s));
    if (!nidx.empty())
        CK(cudaMemcpyAsync(h->nbr_idx, nidx.data(), sizeof(int32_t) * nidx.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->node_leaf, node_leaf.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    finish_leaves(h, s);
}

// The paper's octree (App. C): uniform depth l_max, the smallest level >= 2 at which the mean
// occupancy of the non-empty boxes is at most leaf_size; empty boxes dropped; all leaves at l_max;
// Neighbor lists of the leaves (with the leaf itself).  key: the sorted Morton keys.
void uniform_boxes(fmbem *h, const uint64_t *key, double side, int32_t *f, int32_t *fs, cudaStream_t s) {
    const int64_t N = h->N;
    const int TB = 256;
    // node -> box maps of every level up to KEY_LEVELS, and max occupancy per level
    std::vector<int32_t *> node_box(KEY_LEVELS + 1, nullptr), box_start(KEY_LEVELS + 1, nullptr);
    std::vector<uint64_t *> lkey(KEY_LEVELS + 1, nullptr);
    std::vector<int64_t> nbl(KEY_LEVELS + 1, 0);
    int32_t *occ = (int32_t *)dev_alloc(h, sizeof(int32_t));
    int lmax = -1;
    const int cap = std::max(2, std::min(h->opt.max_level, KEY_LEVELS));
    for (int l = 0; l <= cap; ++l) {
        int shift = 3 * (KEY_LEVELS - l);
        k_level_flags<<<nblk(N, TB), TB, 0, s>>>(key, N, shift, f);
        int64_t nb = scan_exclusive(h, f, fs, N, s);
        nbl[l] = nb;
        node_box[l] = (int32_t *)dev_alloc(h, sizeof(int32_t) * N);
        box_start[l] = (int32_t *)dev_alloc(h, sizeof(int32_t) * nb);
        lkey[l] = (uint64_t *)dev_alloc(h, sizeof(uint64_t) * nb);
        k_level_boxes<<<nblk(N, TB), TB, 0, s>>>(key, f, fs, N, shift, node_box[l], box_start[l], lkey[l]);
        CKL("k_level_boxes");
        CK(cudaMemsetAsync(occ, 0, sizeof(int32_t), s));
        k_max_occupancy<<<nblk(nb, TB), TB, 0, s>>>(box_start[l], nb, N, occ);
        int32_t mo;
        CK(cudaMemcpyAsync(&mo, occ, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        h->max_leaf = mo;
        // refine until the mean leaf occupancy is at most leaf_size ("several elements" per leaf)
        if (l >= 2 && ((double)N / (double)nb <= (double)h->opt.leaf_size || l == cap)) { lmax = l; break; }
    }
    dev_free(h, occ);
    h->lmax = lmax;
    h->lev.assign(lmax + 1, LevelInfo{});
    int64_t tot = 0;
    for (int l = 0; l <= lmax; ++l) {
        h->lev[l].off = tot;
        h->lev[l].n = nbl[l];
        h->lev[l].w = side / (double)(1 << l);
        tot += nbl[l];
    }
    h->nbox = tot;
    h->box_key = (uint64_t *)dev_alloc(h, sizeof(uint64_t) * tot);
    h->box_ctr = (double *)dev_alloc(h, sizeof(double) * 3 * tot);
    h->box_parent = (int32_t *)dev_alloc(h, sizeof(int32_t) * tot);
    h->box_cbeg = (int32_t *)dev_alloc(h, sizeof(int32_t) * tot);
    h->box_cend = (int32_t *)dev_alloc(h, sizeof(int32_t) * tot);
    h->box_nbeg = (int32_t *)dev_alloc(h, sizeof(int32_t) * tot);
    h->box_nend = (int32_t *)dev_alloc(h, sizeof(int32_t) * tot);
    CK(cudaMemsetAsync(h->box_cbeg, 0, sizeof(int32_t) * tot, s));
    CK(cudaMemsetAsync(h->box_cend, 0, sizeof(int32_t) * tot, s));
    for (int l = 0; l <= lmax; ++l) {
        k_fill_level<<<nblk(nbl[l], TB), TB, 0, s>>>(nbl[l], h->lev[l].off, l, box_start[l], lkey[l], N,
                                                     l > 0 ? node_box[l - 1] : nullptr, l > 0 ? h->lev[l - 1].off : 0,
                                                     h->root_min[0], h->root_min[1], h->root_min[2], h->lev[l].w,
                                                     h->box_key, h->box_ctr, h->box_parent, h->box_nbeg, h->box_nend);
        CKL("k_fill_level");
    }
    for (int l = 0; l < lmax; ++l) {
        k_children<<<nblk(nbl[l], TB), TB, 0, s>>>(nbl[l], h->lev[l].off, h->box_nbeg, h->box_nend, node_box[l + 1],
                                                   h->lev[l + 1].off, h->box_cbeg, h->box_cend);
        CKL("k_children");
    }

    // Neighbor lists of the leaves (including the leaf itself) and the near-pair count
    {
        const int l = lmax;
        const int64_t nb = nbl[l], off = h->lev[l].off;
        int32_t *cnt = (int32_t *)dev_alloc(h, sizeof(int32_t) * (nb + 1));
        h->nbr_start = (int32_t *)dev_alloc(h, sizeof(int32_t) * (nb + 1));
        int64_t *pc = (int64_t *)dev_alloc(h, sizeof(int64_t));
        CK(cudaMemsetAsync(pc, 0, sizeof(int64_t), s));
        CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nb + 1), s));
        k_neighbors<<<nblk(nb, TB), TB, 0, s>>>(nb, off, l, h->box_key, nullptr, cnt, nullptr, h->box_nbeg, h->box_nend, pc);
        CKL("k_neighbors count");
        int64_t total = scan_exclusive(h, cnt, h->nbr_start, nb + 1, s);
        h->n_nbr = total;
        h->nbr_idx = (int32_t *)dev_alloc(h, sizeof(int32_t) * std::max<int64_t>(total, 1));
        k_neighbors<<<nblk(nb, TB), TB, 0, s>>>(nb, off, l, h->box_key, h->nbr_start, nullptr, h->nbr_idx, h->box_nbeg,
                                                h->box_nend, nullptr);
        CKL("k_neighbors fill");
        int64_t pairs;
        CK(cudaMemcpyAsync(&pairs, pc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        h->near_pairs = pairs - N;  // minus the self pairs
        dev_free(h, cnt);
        dev_free(h, pc);
    }
    // leaf of every sorted node
    h->node_leaf = (int32_t *)dev_alloc(h, sizeof(int32_t) * N);
    CK(cudaMemcpyAsync(h->node_leaf, node_box[lmax], sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s));
    k_add_offset<<<nblk(N, TB), TB, 0, s>>>(h->node_leaf, N, (int32_t)h->lev[lmax].off);
    CKL("k_add_offset");

    // the leaves: the boxes of level l_max, in node order
    h->h_leaf_box.resize(h->lev[h->lmax].n);
    for (int64_t i = 0; i < h->lev[h->lmax].n; ++i) h->h_leaf_box[i] = (int32_t)(h->lev[h->lmax].off + i);
    finish_leaves(h, s);
    for (int l = 0; l <= KEY_LEVELS; ++l) {
        if (node_box[l]) dev_free(h, node_box[l]);
        if (box_start[l]) dev_free(h, box_start[l]);
        if (lkey[l]) dev_free(h, lkey[l]);
    }
}

}  // namespace

void build_tree(fmbem *h, cudaStream_t s) {
    const int64_t N = h->N;
    const int TB = 256;
    // root cube: centre of the bounding box, side 1.000001 x the largest extent
    int nbb = (int)std::min<int64_t>(nblk(N, TB), 1024);
    double *bb = (double *)dev_alloc(h, sizeof(double) * 6 * nbb);
    k_bbox<<<nbb, TB, 0, s>>>(h->upos, N, bb);
    CKL("k_bbox");
    std::vector<double> hb(6 * nbb);
    CK(cudaMemcpyAsync(hb.data(), bb, sizeof(double) * 6 * nbb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    dev_free(h, bb);
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int b = 0; b < nbb; ++b)
        for (int q = 0; q < 3; ++q) { mn[q] = std::min(mn[q], hb[6 * b + q]); mx[q] = std::max(mx[q], hb[6 * b + 3 + q]); }
    double ext = std::max(mx[0] - mn[0], std::max(mx[1] - mn[1], mx[2] - mn[2]));
    if (!(ext > 0)) throw fmbem_error{FMBEM_ERR_INVALID_MESH, "all nodes coincide"};
    double side = 1.000001 * ext;
    for (int q = 0; q < 3; ++q) h->root_min[q] = 0.5 * (mn[q] + mx[q]) - 0.5 * side;
    h->root_w = side;

    // keys and stable sort
    uint64_t *key = (uint64_t *)dev_alloc(h, sizeof(uint64_t) * N), *key2 = (uint64_t *)dev_alloc(h, sizeof(uint64_t) * N);
    int32_t *idx = (int32_t *)dev_alloc(h, sizeof(int32_t) * N), *idx2 = (int32_t *)dev_alloc(h, sizeof(int32_t) * N);
    int32_t *f = (int32_t *)dev_alloc(h, sizeof(int32_t) * N), *fs = (int32_t *)dev_alloc(h, sizeof(int32_t) * N);
    k_keys<<<nblk(N, TB), TB, 0, s>>>(h->upos, N, h->root_min[0], h->root_min[1], h->root_min[2],
                                      (double)(1 << KEY_LEVELS) / side, key, idx);
    CKL("k_keys");
    for (int bit = 0; bit < 3 * KEY_LEVELS; ++bit) {
        k_bitflag<<<nblk(N, TB), TB, 0, s>>>(key, N, bit, f);
        int64_t nzero = scan_exclusive(h, f, fs, N, s);
        k_bitscatter<<<nblk(N, TB), TB, 0, s>>>(key, idx, fs, N, nzero, bit, key2, idx2);
        CKL("k_bitscatter");
        std::swap(key, key2);
        std::swap(idx, idx2);
    }
    h->perm = idx;
    dev_free(h, idx2);

    if (h->adaptive) adaptive_boxes(h, key, side, s);
    else uniform_boxes(h, key, side, f, fs, s);
    const int lmax = h->lmax;
    const int64_t tot = h->nbox;

    // FF lists on levels 2..lmax (global CSR over all boxes; empty for levels 0..1)
    {
        int32_t *cnt = (int32_t *)dev_alloc(h, sizeof(int32_t) * (tot + 1));
        CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (tot + 1), s));
        for (int l = 2; l <= lmax; ++l)
            k_farfield<<<nblk(h->lev[l].n, TB), TB, 0, s>>>(h->lev[l].n, h->lev[l].off, l, h->box_key, h->lev[l - 1].off, h->lev[l - 1].n,
                                                       h->box_cbeg, h->box_cend, nullptr, cnt + h->lev[l].off, nullptr,
                                                       nullptr);
        CKL("k_farfield count");
        h->ff_start = (int32_t *)dev_alloc(h, sizeof(int32_t) * (tot + 1));
        int64_t total = scan_exclusive(h, cnt, h->ff_start, tot + 1, s);
        h->n_ff = total;
        h->ff_src = (int32_t *)dev_alloc(h, sizeof(int32_t) * std::max<int64_t>(total, 1));
        h->ff_off = (int16_t *)dev_alloc(h, sizeof(int16_t) * std::max<int64_t>(total, 1));
        for (int l = 2; l <= lmax; ++l)
            k_farfield<<<nblk(h->lev[l].n, TB), TB, 0, s>>>(h->lev[l].n, h->lev[l].off, l, h->box_key, h->lev[l - 1].off, h->lev[l - 1].n,
                                                       h->box_cbeg, h->box_cend, h->ff_start + h->lev[l].off, nullptr,
                                                       h->ff_src, h->ff_off);
        CKL("k_farfield fill");
        std::vector<int32_t> hs(tot + 1);
        CK(cudaMemcpyAsync(hs.data(), h->ff_start, sizeof(int32_t) * (tot + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        h->h_ff_count_level.assign(lmax + 1, 0);
        for (int l = 2; l <= lmax; ++l)
            h->h_ff_count_level[l] = hs[h->lev[l].off + h->lev[l].n] - hs[h->lev[l].off];
        dev_free(h, cnt);

        // regroup the FF pairs of each level by offset (counting sort) and cut chunks of at
        // most M2L_CHUNK pairs sharing one translation matrix
        const int64_t nff = std::max<int64_t>(total, 1);
        h->pair_tgt = (int32_t *)dev_alloc(h, sizeof(int32_t) * nff);
        h->pair_e = (int32_t *)dev_alloc(h, sizeof(int32_t) * nff);
        k_pair_targets<<<nblk(tot, TB), TB, 0, s>>>(tot, h->ff_start, h->pair_tgt);
        CKL("k_pair_targets");
        int32_t *ocnt = (int32_t *)dev_alloc(h, sizeof(int32_t) * 316);
        std::vector<int32_t> hb(316), hbeg(316);
        std::vector<int32_t> cbeg, ccnt;
        std::vector<int16_t> coff;
        h->h_chunk_first.assign(lmax + 2, 0);
        h->h_pair_first.assign(lmax + 2, 0);
        for (int l = 0; l <= lmax + 1; ++l) h->h_pair_first[l] = l <= lmax ? hs[h->lev[l].off] : hs[tot];
        for (int l = 0; l <= lmax; ++l) {
            h->h_chunk_first[l] = (int64_t)cbeg.size();
            const int64_t e0 = hs[h->lev[l].off], e1 = hs[h->lev[l].off + h->lev[l].n];
            if (e1 <= e0) continue;
            CK(cudaMemsetAsync(ocnt, 0, sizeof(int32_t) * 316, s));
            k_count_offsets<<<nblk(e1 - e0, TB), TB, 0, s>>>(e0, e1, h->ff_off, ocnt);
            CKL("k_count_offsets");
            CK(cudaMemcpyAsync(hb.data(), ocnt, sizeof(int32_t) * 316, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            int32_t acc = (int32_t)e0;
            for (int o = 0; o < 316; ++o) {
                hbeg[o] = acc;
                for (int32_t c = 0; c < hb[o]; c += M2L_CHUNK) {
                    cbeg.push_back(acc + c);
                    ccnt.push_back(std::min(M2L_CHUNK, hb[o] - c));
                    coff.push_back((int16_t)o);
                }
                acc += hb[o];
            }
            CK(cudaMemcpyAsync(ocnt, hbeg.data(), sizeof(int32_t) * 316, cudaMemcpyHostToDevice, s));
            k_fill_offsets<<<nblk(e1 - e0, TB), TB, 0, s>>>(e0, e1, h->ff_off, ocnt, h->pair_e);
            CKL("k_fill_offsets");
        }
        h->h_chunk_first[lmax + 1] = (int64_t)cbeg.size();
        const size_t nc = std::max<size_t>(cbeg.size(), 1);
        h->chunk_beg = (int32_t *)dev_alloc(h, sizeof(int32_t) * nc);
        h->chunk_cnt = (int32_t *)dev_alloc(h, sizeof(int32_t) * nc);
        h->chunk_off = (int16_t *)dev_alloc(h, sizeof(int16_t) * nc);
        if (!cbeg.empty()) {
            CK(cudaMemcpyAsync(h->chunk_beg, cbeg.data(), sizeof(int32_t) * cbeg.size(), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(h->chunk_cnt, ccnt.data(), sizeof(int32_t) * ccnt.size(), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(h->chunk_off, coff.data(), sizeof(int16_t) * coff.size(), cudaMemcpyHostToDevice, s));
        }
        CK(cudaStreamSynchronize(s));
        dev_free(h, ocnt);
    }

    // sorted geometry
    h->iperm = (int32_t *)dev_alloc(h, sizeof(int32_t) * N);
    h->pos = (double *)dev_alloc(h, sizeof(double) * 3 * N);
    h->nrm = (double *)dev_alloc(h, sizeof(double) * 3 * N);
    h->w = (double *)dev_alloc(h, sizeof(double) * N);
    h->dom = (int32_t *)dev_alloc(h, sizeof(int32_t) * N);
    h->pos_hi = (float *)dev_alloc(h, sizeof(float) * 3 * N);
    h->pos_lo = (float *)dev_alloc(h, sizeof(float) * 3 * N);
    h->nrm_f = (float *)dev_alloc(h, sizeof(float) * 3 * N);
    h->src_rec = (float4 *)dev_alloc(h, sizeof(float4) * 3 * N);
    k_sorted_geometry<<<nblk(N, TB), TB, 0, s>>>(N, h->perm, h->upos, h->unrm, h->uw, h->udom, h->pos, h->nrm, h->w, h->dom,
                                                 h->iperm, h->pos_hi, h->pos_lo, h->nrm_f, h->src_rec);
    CKL("k_sorted_geometry");
    CK(cudaStreamSynchronize(s));
    dev_free(h, key);
    dev_free(h, key2);
    dev_free(h, f);
    dev_free(h, fs);
}
