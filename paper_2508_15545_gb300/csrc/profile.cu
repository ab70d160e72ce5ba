// Launch counters, per-class CUDA-event timing and transfer accounting.
#include "qv_internal.h"

namespace qv {

void prof_begin(qv_state *s, int cls)
{
    s->prof.launches[cls]++;
    if (!s->prof.timing) return;
    Prof::Pending p{cls, nullptr, nullptr};
    for (cudaEvent_t *e : {&p.a, &p.b}) {
        if (!s->prof.pool.empty()) {
            *e = s->prof.pool.back();
            s->prof.pool.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
            *e = nullptr;
        }
    }
    if (p.a) cudaEventRecord(p.a, s->stream);
    s->prof.pending.push_back(p);
}

void prof_end(qv_state *s, int cls)
{
    if (!s->prof.timing || s->prof.pending.empty()) return;
    Prof::Pending &p = s->prof.pending.back();
    if (p.cls == cls && p.b) cudaEventRecord(p.b, s->stream);
}

qv_status prof_drain(qv_state *s)
{
    QV_CUDA(cudaStreamSynchronize(s->stream));
    for (auto &p : s->prof.pending) {
        float ms = 0;
        if (p.a && p.b && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) s->prof.ms[p.cls] += ms;
        if (p.a) s->prof.pool.push_back(p.a);
        if (p.b) s->prof.pool.push_back(p.b);
    }
    s->prof.pending.clear();
    (void)cudaGetLastError();
    return QV_OK;
}

void prof_release(qv_state *s)
{
    for (auto &p : s->prof.pending) {
        if (p.a) cudaEventDestroy(p.a);
        if (p.b) cudaEventDestroy(p.b);
    }
    for (auto e : s->prof.pool) cudaEventDestroy(e);
    s->prof.pending.clear();
    s->prof.pool.clear();
}

qv_status copy_h2d(qv_state *s, void *dst, const void *src, size_t bytes)
{
    QV_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream));
    s->prof.h2d += bytes;
    return QV_OK;
}

qv_status copy_d2h(qv_state *s, void *dst, const void *src, size_t bytes)
{
    QV_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->stream));
    s->prof.d2h += bytes;
    return QV_OK;
}

}  // namespace qv

using namespace qv;

extern "C" {

qv_status qv_profile(qv_state *s, int timing)
{
    if (!s) return fail(QV_ERR_ARG, "NULL state handle");
    QV_TRY(prof_drain(s));
    for (int k = 0; k < QV_K_COUNT; ++k) {
        s->prof.launches[k] = 0;
        s->prof.ms[k] = 0;
        s->prof.bytes[k] = 0;
    }
    s->prof.h2d = s->prof.d2h = 0;
    s->prof.timing = timing != 0;
    return QV_OK;
}

qv_status qv_profile_read(qv_state *s, qv_kernel_stat *out, int count)
{
    if (!s) return fail(QV_ERR_ARG, "NULL state handle");
    if (!out && count > 0) return fail(QV_ERR_ARG, "out is NULL");
    QV_TRY(prof_drain(s));
    for (int k = 0; k < count && k < QV_K_COUNT; ++k) {
        out[k].launches = s->prof.launches[k];
        out[k].ms = s->prof.ms[k];
        out[k].bytes = s->prof.bytes[k];
    }
    return QV_OK;
}

qv_status qv_transfer_bytes(qv_state *s, uint64_t *h2d, uint64_t *d2h)
{
    if (!s) return fail(QV_ERR_ARG, "NULL state handle");
    if (h2d) *h2d = s->prof.h2d;
    if (d2h) *d2h = s->prof.d2h;
    return QV_OK;
}

}  // extern "C"
