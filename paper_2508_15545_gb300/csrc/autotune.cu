// Autotuner: times the fused path on the caller's circuit for each supported
// tile size and each schedule variant of the compiled complex64 engine -- the
// FP32 passes with 4x4 pair operations, without them, and the tensor-core
// stages (their planner chooses other register sets, hence other transposes) --
// and remembers the fastest per (qubits, dtype, engine).
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "planner.h"
#include "qv_internal.h"
#include "qv_jit.h"
#include "qv_plan.h"

namespace qv {
namespace {
std::mutex g_mu;
// (n, dtype, interpreting) -> (tile bits, engine flags)
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_best;
}  // namespace

int tuned_tile_bits(int n, qv_dtype dt, bool interpreting)
{
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_best.find({n, int(dt), interpreting ? 1 : 0});
    if (it != g_best.end()) return it->second.first;
    // untuned: the compiled complex64 pass runs fastest with 2^11-amplitude tiles on the
    // 30-qubit random circuit (282 ms against 288 ms at 2^12 and 2^10)
    if (dt == QV_C64 && !interpreting) return std::min(n, 11);
    return std::min(n, plan::kMaxK);
}

int tuned_flags(int n, qv_dtype dt, bool interpreting)
{
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_best.find({n, int(dt), interpreting ? 1 : 0});
    return it != g_best.end() ? it->second.second : 0;
}

bool tile_bits_tuned(int n, qv_dtype dt, bool interpreting)
{
    std::lock_guard<std::mutex> lock(g_mu);
    return g_best.count({n, int(dt), interpreting ? 1 : 0}) != 0;
}

qv_status autotune(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t *best_k,
                   int32_t *best_fl, bool variants)
{
    if (s->n < plan::kMinK) return fail(QV_ERR_UNSUPPORTED, "no fused tile fits %d qubits", s->n);
    const int base = opts ? opts->flags : 0;
    const bool interp = (base & QV_PLAN_INTERPRET) || !jit_available(nullptr);
    // schedule variants of the compiled complex64 engine
    std::vector<int> vflags = {0};
    if (variants && !interp && s->dt == QV_C64 && !(base & QV_PLAN_NO_FUSION)) {
        vflags.push_back(QV_PLAN_NO_PAIRS);
        vflags.push_back(QV_PLAN_TENSOR);
    }
    cudaEvent_t e0, e1;
    QV_CUDA(cudaEventCreate(&e0));
    QV_CUDA(cudaEventCreate(&e1));
    int best = -1, best_flags = 0;
    float best_ms = 0;
    qv_status st = QV_OK;
    for (int K = plan::kMinK; K <= std::min(s->n, plan::kMaxK) && st == QV_OK; ++K)
        for (int vf : vflags) {
            if ((vf & QV_PLAN_TENSOR) && K < 11) continue;
            qv_plan_opts o{};
            o.mode = QV_MODE_FUSED;
            o.tile_bits = K;
            o.flags = base | vf;
            st = apply_fused(s, g, ng, &o);  // warm-up (compiles the passes when needed)
            if (st != QV_OK) break;
            float ms = 0;
            for (int rep = 0; rep < 2 && st == QV_OK; ++rep) {
                if (cudaEventRecord(e0, s->stream) != cudaSuccess) st = fail(QV_ERR_CUDA, "cudaEventRecord");
                if (st == QV_OK) st = apply_fused(s, g, ng, &o);
                if (st == QV_OK && cudaEventRecord(e1, s->stream) != cudaSuccess)
                    st = fail(QV_ERR_CUDA, "cudaEventRecord");
                if (st == QV_OK && cudaEventSynchronize(e1) != cudaSuccess)
                    st = fail(QV_ERR_CUDA, "cudaEventSynchronize");
                float t = 0;
                if (st == QV_OK) cudaEventElapsedTime(&t, e0, e1);
                ms = rep == 0 ? t : std::min(ms, t);
            }
            if (st == QV_OK && (best < 0 || ms < best_ms)) {
                best = K;
                best_flags = vf;
                best_ms = ms;
            }
            if (st != QV_OK) break;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    QV_TRY(st);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_best[{s->n, int(s->dt), interp ? 1 : 0}] = {best, best_flags};
    }
    if (best_k) *best_k = best;
    if (best_fl) *best_fl = best_flags;
    return launch_set_basis(s, 0);
}

}  // namespace qv
