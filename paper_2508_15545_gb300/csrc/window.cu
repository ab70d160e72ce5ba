// States in host memory staged through windows in HBM: the paper's sliding
// window (Sec. III-B, Eq. 6) -- load a block into fast memory, apply every
// pending update there, write it back -- with HBM as the fast memory and the
// host memory behind NVLink-C2C as the slow one.
//
// When the whole state fits the window budget, one copy brings it into HBM,
// every fused pass runs there, and one copy writes it back: two crossings of
// the host link instead of a read and a write per pass. A larger state is cut
// into 2^(n - w) chunks of 2^w amplitudes (the top n - w qubits name the chunk,
// as Eq. 9 names a node) and follows the schedule of a split state
// (dist_plan.cpp): every local step streams the chunks through two device
// windows -- loading chunk j + 1 on one copy stream while chunk j computes and
// chunk j - 1 is written back on another -- and an exchange swaps one half of
// two chunks in host memory. The schedule ends in the natural qubit order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "planner.h"
#include "qv_internal.h"
#include "qv_plan.h"

namespace qv {

struct HostWindow {
    int bits = 0;
    int nwin = 0;
    qv_state *win[2] = {nullptr, nullptr};
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t loaded[2] = {}, computed[2] = {}, free_[2] = {};
};

namespace {

// a[i] <-> b[i] for `count` 16-byte words (two complex64 or one complex128 amplitude)
__global__ void swap_halves_kernel(uint4 *a, uint4 *b, uint64_t count)
{
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < count; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint4 t = a[i];
        a[i] = b[i];
        b[i] = t;
    }
}

void release_windows(HostWindow *W)
{
    for (int b = 0; b < 2; ++b) {
        if (W->win[b]) qv_destroy(W->win[b]);
        W->win[b] = nullptr;
        if (W->loaded[b]) cudaEventDestroy(W->loaded[b]);
        if (W->computed[b]) cudaEventDestroy(W->computed[b]);
        if (W->free_[b]) cudaEventDestroy(W->free_[b]);
        W->loaded[b] = W->computed[b] = W->free_[b] = nullptr;
    }
    if (W->h2d) cudaStreamDestroy(W->h2d);
    if (W->d2h) cudaStreamDestroy(W->d2h);
    W->h2d = W->d2h = nullptr;
    W->bits = W->nwin = 0;
}

qv_status ensure_windows(qv_state *s, int w, int nwin)
{
    if (!s->window) s->window = new HostWindow;
    HostWindow &W = *s->window;
    if (W.bits == w && W.nwin >= nwin) return QV_OK;
    QV_CUDA(cudaStreamSynchronize(s->stream));
    release_windows(&W);
    QV_CUDA(cudaSetDevice(s->device));
    for (int b = 0; b < nwin; ++b) {
        QV_TRY(qv_create(w, s->dt, s->stream, &W.win[b]));
        QV_CUDA(cudaEventCreateWithFlags(&W.loaded[b], cudaEventDisableTiming));
        QV_CUDA(cudaEventCreateWithFlags(&W.computed[b], cudaEventDisableTiming));
        QV_CUDA(cudaEventCreateWithFlags(&W.free_[b], cudaEventDisableTiming));
    }
    QV_CUDA(cudaStreamCreateWithFlags(&W.h2d, cudaStreamNonBlocking));
    QV_CUDA(cudaStreamCreateWithFlags(&W.d2h, cudaStreamNonBlocking));
    W.bits = w;
    W.nwin = nwin;
    return QV_OK;
}

}  // namespace

// The whole state as one window when it takes at most half of the free device
// memory; else 0: no default window. Streaming chunks moves more over the host
// link than in-place passes on circuits that touch every qubit in every layer
// (30-qubit random circuit: 1,460 GB in 4 chunks of 2^28 against 722 GB in
// place), so chunks are used only when the caller asks for them.
int default_window_bits(const qv_state *s)
{
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    const double ab = double(amp_bytes(s->dt));
    return std::ldexp(ab, s->n) <= 0.5 * double(free_b) ? s->n : 0;
}

namespace {

}  // namespace

void window_release(qv_state *s)
{
    if (!s->window) return;
    release_windows(s->window);
    delete s->window;
    s->window = nullptr;
}

qv_status apply_windowed(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts)
{
    const int n = s->n;
    int w = std::min(opts && opts->window_bits ? opts->window_bits : default_window_bits(s), n);
    if (w < plan::kMinK) return fail(QV_ERR_ARG, "window of 2^%d amplitudes below the smallest tile (2^%d)", w, plan::kMinK);
    const size_t ab = amp_bytes(s->dt);
    // the device windows run the fused passes with the caller's engine options
    qv_plan_opts o{};
    if (opts) o = *opts;
    o.mode = QV_MODE_FUSED;
    o.window_bits = 0;
    o.flags &= ~QV_PLAN_HOST_IN_PLACE;
    char *host = static_cast<char *>(s->amp);
    if (w == n) {
        QV_TRY(ensure_windows(s, w, 1));
        s->window->win[0]->stream = s->stream;  // the handle's stream may have changed
        qv_state *d = s->window->win[0];
        const size_t bytes = size_t(1) << n;
        QV_CUDA(cudaMemcpyAsync(d->amp, host, bytes * ab, cudaMemcpyDefault, s->stream));
        QV_TRY(apply_fused(d, g, ng, &o));
        QV_CUDA(cudaMemcpyAsync(host, d->amp, bytes * ab, cudaMemcpyDefault, s->stream));
        s->prof.h2d += bytes * ab;
        s->prof.d2h += bytes * ab;
        return QV_OK;
    }
    const int G = n - w;
    if (G > 20) return fail(QV_ERR_ARG, "window of 2^%d amplitudes is too small for %d qubits", w, n);
    const int nchunks = 1 << G;
    std::vector<std::vector<qv_dist_step>> steps(nchunks);
    std::vector<std::vector<qv_gate>> lg(nchunks);
    for (int j = 0; j < nchunks; ++j) {
        std::vector<int32_t> perm;
        QV_TRY(dist_plan(n, G, j, g, ng, steps[j], lg[j], perm, true));
    }
    QV_TRY(ensure_windows(s, w, 2));
    HostWindow &W = *s->window;
    W.win[0]->stream = W.win[1]->stream = s->stream;
    const size_t chunk_bytes = (size_t(1) << w) * ab;
    // everything enqueued so far on the handle's stream comes first
    cudaEvent_t start = W.computed[0];
    QV_CUDA(cudaEventRecord(start, s->stream));
    QV_CUDA(cudaStreamWaitEvent(W.h2d, start, 0));
    QV_CUDA(cudaStreamWaitEvent(W.d2h, start, 0));
    for (int b = 0; b < 2; ++b) QV_CUDA(cudaEventRecord(W.free_[b], W.d2h));
    for (size_t t = 0; t < steps[0].size(); ++t) {
        if (steps[0][t].kind == QV_DIST_LOCAL) {
            for (int j = 0; j < nchunks; ++j) {
                const qv_dist_step &st = steps[j][t];
                if (st.gate_end == st.gate_begin) continue;  // nothing to do on this chunk
                const int b = j & 1;
                qv_state *d = W.win[b];
                char *chunk = host + size_t(j) * chunk_bytes;
                QV_CUDA(cudaStreamWaitEvent(W.h2d, W.free_[b], 0));
                QV_CUDA(cudaMemcpyAsync(d->amp, chunk, chunk_bytes, cudaMemcpyDefault, W.h2d));
                QV_CUDA(cudaEventRecord(W.loaded[b], W.h2d));
                QV_CUDA(cudaStreamWaitEvent(s->stream, W.loaded[b], 0));
                QV_TRY(apply_fused(d, lg[j].data() + st.gate_begin, size_t(st.gate_end - st.gate_begin), &o));
                QV_CUDA(cudaEventRecord(W.computed[b], s->stream));
                QV_CUDA(cudaStreamWaitEvent(W.d2h, W.computed[b], 0));
                QV_CUDA(cudaMemcpyAsync(chunk, d->amp, chunk_bytes, cudaMemcpyDefault, W.d2h));
                QV_CUDA(cudaEventRecord(W.free_[b], W.d2h));
                s->prof.h2d += chunk_bytes;
                s->prof.d2h += chunk_bytes;
            }
        } else {
            // every chunk written back first; then chunk j (its bit 0) trades its
            // upper half for the lower half of chunk j + 2^bit
            for (int b = 0; b < 2; ++b) QV_CUDA(cudaStreamWaitEvent(s->stream, W.free_[b], 0));
            const int bit = steps[0][t].global_bit;
            const uint64_t words = chunk_bytes / 2 / 16;
            for (int j = 0; j < nchunks; ++j) {
                if ((j >> bit) & 1) continue;
                uint4 *a = reinterpret_cast<uint4 *>(host + size_t(j) * chunk_bytes + chunk_bytes / 2);
                uint4 *c = reinterpret_cast<uint4 *>(host + size_t(j | (1 << bit)) * chunk_bytes);
                const unsigned grid = unsigned(std::min<uint64_t>((words + 255) / 256, uint64_t(s->num_sms) * 8));
                swap_halves_kernel<<<grid, 256, 0, s->stream>>>(a, c, words);
                QV_CUDA(cudaGetLastError());
            }
            cudaEvent_t done = W.computed[0];
            QV_CUDA(cudaEventRecord(done, s->stream));
            QV_CUDA(cudaStreamWaitEvent(W.h2d, done, 0));
            QV_CUDA(cudaStreamWaitEvent(W.d2h, done, 0));
            for (int b = 0; b < 2; ++b) QV_CUDA(cudaEventRecord(W.free_[b], W.d2h));
        }
    }
    // later work on the handle's stream sees the written-back state
    for (int b = 0; b < 2; ++b) QV_CUDA(cudaStreamWaitEvent(s->stream, W.free_[b], 0));
    return QV_OK;
}

}  // namespace qv
