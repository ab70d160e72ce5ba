// Compiled (NVRTC) fused passes; see fused_jit.cu.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "planner.h"
#include "qv_internal.h"

namespace qv {

// True when NVRTC could be loaded; otherwise `why` (if given) says why not.
bool jit_available(std::string *why);

// Compiled kernels and packed coefficients of a plan, ready to launch again.
struct JitProgram;
// Forward passes: compile (or take from the cache) and pack.
qv_status jit_prepare(qv_state *s, const std::vector<plan::Pass> &passes, std::shared_ptr<JitProgram> &out);
qv_status jit_launch(qv_state *s, const JitProgram &prog);
// Adjoint passes (see jit_run_adjoint).
qv_status jit_prepare_adjoint(qv_state *s, const std::vector<plan::Pass> &passes, std::shared_ptr<JitProgram> &out);
qv_status jit_launch_adjoint(qv_state *s, const JitProgram &prog, void *lam, double *part, int G);
// Compiles (or takes from the process-wide cache) one kernel per pass and
// launches the passes in order on the handle's stream.
qv_status jit_run_plan(qv_state *s, const std::vector<plan::Pass> &passes);
// Reverse sweep of the adjoint gradient (complex64): plan of the daggered
// gates in reverse order; an op with derivatives (Op::nd > 0) writes its
// partials 2 Re <lambda | D psi> to part[slot * G + CTA]; part columns of CTAs
// not launched are left untouched.
qv_status jit_run_adjoint(qv_state *s, const std::vector<plan::Pass> &passes, void *lam, double *part, int G);

}  // namespace qv
