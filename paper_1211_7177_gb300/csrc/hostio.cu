// hostio.cu -- the product of Eq. (2.9) with x and y in host memory (fmbem_matvec_host).
//
// The right-hand sides are cut into chunks; chunk k is copied to the device on one copy stream,
// multiplied on the caller's stream (run_matvec, every kernel of the device product) and copied
// back on a second copy stream, so that the copy of chunk k + 1 to the device and of chunk k - 1
// back run while chunk k is multiplied.  Two x slots and two y slots of chunk size alternate;
// events order each slot's reuse after the work that still reads it.  In single precision with
// whole blocks of 32 right-hand sides the product itself copies its rows back per block, right
// after the near-field launch that finishes them (h->io_rows).  With pinned host memory
// the copies run at the link's rate beside the kernels; with pageable memory the driver stages
// them and they do not overlap.
#include <algorithm>

#include "fmbem_internal.cuh"

void run_matvec_host(fmbem *h, const c64 *x_host, c64 *y_host, int64_t nr, int precision, int64_t chunk_rhs,
                     cudaStream_t s) {
    const int64_t per_rhs = 6 * h->N;  // complex128 values per right-hand side
    // the library's choice: chunks of up to 128 right-hand sides (a product of fewer columns
    // costs more per column -- on the 65536-node torus 15.3 ms for 64 against 24.1 ms for 128 --
    // than the copies it would hide, 3.8 + 4.2 ms for 128 over the link)
    const int64_t chunk = chunk_rhs > 0 ? std::min(chunk_rhs, nr) : std::min<int64_t>(nr, 128);
    const int64_t nchunk = (nr + chunk - 1) / chunk;
    const size_t slot = sizeof(c64) * (size_t)chunk * per_rhs;
    if (h->io_bytes < 4 * slot) {
        if (h->io_buf) dev_free(h, h->io_buf);
        h->io_buf = nullptr;
        h->io_bytes = 0;
        h->io_buf = dev_alloc(h, 4 * slot);
        h->io_bytes = 4 * slot;
    }
    for (auto &st : h->io_stream)
        if (!st) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (auto &e : h->io_ev)
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto &e : h->io_rows.ev)
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaStream_t up = h->io_stream[0], down = h->io_stream[1];
    cudaEvent_t start = h->io_ev[0], *copied_in = h->io_ev + 1, *computed = h->io_ev + 3, *copied_out = h->io_ev + 5;
    c64 *xs[2], *ys[2];
    for (int q = 0; q < 2; ++q) {
        xs[q] = (c64 *)((char *)h->io_buf + q * slot);
        ys[q] = (c64 *)((char *)h->io_buf + (2 + q) * slot);
    }
    // the copy streams follow everything queued on s so far (earlier users of the slots)
    CK(cudaEventRecord(start, s));
    CK(cudaStreamWaitEvent(up, start, 0));
    CK(cudaStreamWaitEvent(down, start, 0));
    auto rhs_of = [&](int64_t k) { return std::min(chunk, nr - k * chunk); };
    auto copy_in = [&](int64_t k) {
        const int q = (int)(k & 1);
        if (k >= 2) CK(cudaStreamWaitEvent(up, computed[q], 0));  // chunk k - 2 has read slot q
        CK(cudaMemcpyAsync(xs[q], x_host + k * chunk * per_rhs, sizeof(c64) * rhs_of(k) * per_rhs,
                           cudaMemcpyHostToDevice, up));
        CK(cudaEventRecord(copied_in[q], up));
    };
    try {
        copy_in(0);
        for (int64_t k = 0; k < nchunk; ++k) {
            const int q = (int)(k & 1);
            if (k + 1 < nchunk) copy_in(k + 1);
            CK(cudaStreamWaitEvent(s, copied_in[q], 0));
            if (k >= 2) CK(cudaStreamWaitEvent(s, copied_out[q], 0));  // chunk k - 2's result is out
            // the product may copy its rows back itself, slab by slab as the near field finishes
            // them (single precision, whole blocks of 32 right-hand sides, rows final after the
            // near field): then the copy of the first slabs overlaps the near field of the last
            h->io_rows.y_host = y_host + k * chunk * per_rhs;
            h->io_rows.down = down;
            h->io_rows.copied = false;
            run_matvec(h, xs[q], ys[q], rhs_of(k), precision, s);
            h->io_rows.y_host = nullptr;
            CK(cudaEventRecord(computed[q], s));
            if (!h->io_rows.copied) {
                CK(cudaStreamWaitEvent(down, computed[q], 0));
                CK(cudaMemcpyAsync(y_host + k * chunk * per_rhs, ys[q], sizeof(c64) * rhs_of(k) * per_rhs,
                                   cudaMemcpyDeviceToHost, down));
            }
            CK(cudaEventRecord(copied_out[q], down));
        }
    } catch (...) {
        // a failed product: no copy may still touch the caller's host buffers after the return
        h->io_rows.y_host = nullptr;
        cudaStreamSynchronize(up);
        cudaStreamSynchronize(down);
        throw;
    }
    // s waits for the last copy back (the copies back run in order on their stream)
    CK(cudaStreamWaitEvent(s, copied_out[(nchunk - 1) & 1], 0));
}
