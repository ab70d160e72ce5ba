// Compiled (NVRTC) fused passes; see fused_jit.cu.
#pragma once

#include <string>
#include <vector>

#include "planner.h"
#include "qv_internal.h"

namespace qv {

// True when NVRTC could be loaded; otherwise `why` (if given) says why not.
bool jit_available(std::string *why);
// Compiles (or takes from the process-wide cache) one kernel per pass and
// launches the passes in order on the handle's stream.
qv_status jit_run_plan(qv_state *s, const std::vector<plan::Pass> &passes);

}  // namespace qv
