// Fused-pass planning and execution (the on-chip form of the paper's
// sliding-window cache and block storage, Sec. III-B/C/E) and qubit
// permutations.
#pragma once

#include "qv_internal.h"

namespace qv {

// True when qv_apply_circuit in QV_MODE_AUTO should take the fused path.
bool fused_supported(const qv_state *s, const qv_plan_opts *opts);
qv_status apply_fused(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts);
qv_status plan_info(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t out[4]);

// Bit q of every index moves to bit perm[q].
qv_status apply_permutation(qv_state *s, const int32_t *perm);
// Frees per-handle planning buffers.
void plan_cache_release(qv_state *s);

}  // namespace qv
