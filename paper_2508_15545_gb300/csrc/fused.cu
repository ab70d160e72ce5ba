// Fused tiled passes (placeholder until the tiled kernel lands) and qubit
// permutations built from SWAP passes.
#include <vector>

#include "qv_plan.h"

namespace qv {

bool fused_supported(const qv_state *, const qv_plan_opts *) { return false; }

qv_status apply_fused(qv_state *, const qv_gate *, size_t, const qv_plan_opts *)
{
    return fail(QV_ERR_UNSUPPORTED, "fused mode not built");
}

qv_status apply_permutation(qv_state *s, const int32_t *perm)
{
    // cur[p] = original qubit whose bit now sits at position p; want[perm[q]] = q.
    const int n = s->n;
    std::vector<int> cur(n), want(n);
    for (int p = 0; p < n; ++p) cur[p] = p;
    for (int q = 0; q < n; ++q) want[perm[q]] = q;
    for (int p = 0; p < n; ++p) {
        if (cur[p] == want[p]) continue;
        int p2 = p + 1;
        while (cur[p2] != want[p]) ++p2;
        QV_TRY(launch_swap(s, p, p2));
        std::swap(cur[p], cur[p2]);
    }
    return QV_OK;
}

void plan_cache_release(qv_state *) {}

}  // namespace qv
