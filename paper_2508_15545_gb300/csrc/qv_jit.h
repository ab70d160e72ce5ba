// Compiled (NVRTC) fused passes; see fused_jit.cu.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "planner.h"
#include "qv_internal.h"

namespace qv {

// True when NVRTC and the driver could be loaded; otherwise `why` (if given) says why not.
bool jit_available(std::string *why);

// Host only (no driver needed): the CUDA source of one compiled pass, and
// NVRTC compilation of every pass of a plan (out[0] = passes, out[1] = source
// bytes, out[2] = most registers a thread of any pass uses, out[3] = passes
// whose registers spill; QV_ERR_UNSUPPORTED without NVRTC, QV_ERR_CUDA with
// the log if one fails).
std::string jit_pass_source(const plan::Pass &p, bool c64);
qv_status jit_compile_host(const std::vector<plan::Pass> &passes, bool c64, int64_t out[4]);

// Compiled kernels and packed coefficients of a plan, ready to launch again.
struct JitProgram;
// Forward passes: compile (or take from the cache) and pack.
qv_status jit_prepare(qv_state *s, const std::vector<plan::Pass> &passes, std::shared_ptr<JitProgram> &out);
// Launches on the handle's stream (counted in its profile), or on `on` when
// given (a batch graph being captured: not counted).
qv_status jit_launch(qv_state *s, const JitProgram &prog, cudaStream_t on = nullptr);
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

// Batched circuits of one plan structure (complex64) in one persistent kernel.
struct Compiled;
struct JitBatch {
    std::shared_ptr<Compiled> fn;
    std::vector<uint64_t> coefs;  // [circuit][pass][stride]
    int npasses = 0, stride = 0, threads = 0, per_sm = 0;
    size_t smem = 0;
};
// True when two plans differ at most in their coefficients.
bool jit_same_structure(const std::vector<plan::Pass> &a, const std::vector<plan::Pass> &b);
// Compiles the kernel of plans[0]'s structure and packs every plan's coefficients.
qv_status jit_prepare_batch(qv_state *s, const std::vector<std::vector<plan::Pass> *> &plans, int chunk_tiles,
                            JitBatch &out);
// Launches (or records into a capturing stream) the kernel with args:
// amps, coefs, items (uint2: circuit * passes + pass, chunk), nitems, next,
// done, status, ntiles, nchunks, spin_limit.
qv_status jit_launch_batch(const JitBatch &jb, cudaStream_t stream, unsigned grid, void **args);

}  // namespace qv
