// Tile-size autotuner: times the fused path for each supported tile size on
// the caller's circuit and remembers the fastest per (qubits, dtype, engine).
#include <map>
#include <mutex>
#include <tuple>

#include "planner.h"
#include "qv_internal.h"
#include "qv_plan.h"

namespace qv {
namespace {
std::mutex g_mu;
std::map<std::tuple<int, int, int>, int> g_best;  // (n, dtype, interpreting) -> tile bits
}  // namespace

int tuned_tile_bits(int n, qv_dtype dt, bool interpreting)
{
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_best.find({n, int(dt), interpreting ? 1 : 0});
    if (it != g_best.end()) return it->second;
    // untuned: the compiled complex64 pass runs fastest with 2^11-amplitude tiles on the
    // 30-qubit random circuit (285 ms against 292 ms at 2^12 and 288 ms at 2^10)
    if (dt == QV_C64 && !interpreting) return std::min(n, 11);
    return std::min(n, plan::kMaxK);
}

qv_status autotune(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t *best_out)
{
    if (s->n < plan::kMinK) return fail(QV_ERR_UNSUPPORTED, "no fused tile fits %d qubits", s->n);
    const bool interp = opts && (opts->flags & QV_PLAN_INTERPRET);
    cudaEvent_t e0, e1;
    QV_CUDA(cudaEventCreate(&e0));
    QV_CUDA(cudaEventCreate(&e1));
    int best = -1;
    float best_ms = 0;
    qv_status st = QV_OK;
    for (int K = plan::kMinK; K <= std::min(s->n, plan::kMaxK) && st == QV_OK; ++K) {
        qv_plan_opts o{};
        o.mode = QV_MODE_FUSED;
        o.tile_bits = K;
        o.flags = opts ? opts->flags : 0;
        st = apply_fused(s, g, ng, &o);  // warm-up (compiles the passes when needed)
        if (st != QV_OK) break;
        float ms = 0;
        for (int rep = 0; rep < 2 && st == QV_OK; ++rep) {
            if (cudaEventRecord(e0, s->stream) != cudaSuccess) st = fail(QV_ERR_CUDA, "cudaEventRecord");
            if (st == QV_OK) st = apply_fused(s, g, ng, &o);
            if (st == QV_OK && cudaEventRecord(e1, s->stream) != cudaSuccess) st = fail(QV_ERR_CUDA, "cudaEventRecord");
            if (st == QV_OK && cudaEventSynchronize(e1) != cudaSuccess) st = fail(QV_ERR_CUDA, "cudaEventSynchronize");
            float t = 0;
            if (st == QV_OK) cudaEventElapsedTime(&t, e0, e1);
            ms = rep == 0 ? t : std::min(ms, t);
        }
        if (st == QV_OK && (best < 0 || ms < best_ms)) {
            best = K;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    QV_TRY(st);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_best[{s->n, int(s->dt), interp ? 1 : 0}] = best;
    }
    if (best_out) *best_out = best;
    return launch_set_basis(s, 0);
}

}  // namespace qv
