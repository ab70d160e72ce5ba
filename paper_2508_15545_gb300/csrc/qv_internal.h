// Internal declarations shared by the translation units of libqv.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "qv.h"

namespace qv {

using cd = std::complex<double>;

// Per-handle state. The device buffer holds 2^n interleaved (re, im) pairs.
struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Launch counters and optional CUDA-event timing per kernel class.
struct Prof {
    bool timing = false;
    uint64_t launches[QV_K_COUNT] = {};
    double ms[QV_K_COUNT] = {};
    double bytes[QV_K_COUNT] = {};
    struct Pending {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    uint64_t h2d = 0, d2h = 0;
};

struct PlanCache;       // fused-pass buffers (fused.cu)
struct HostWindow;      // device windows of a state in host memory (window.cu)
struct AdjointBuffers;  // lambda buffer and gradient partials (adjoint.cu)

}  // namespace qv

struct qv_state {
    int n = 0;
    qv_dtype dt = QV_C64;
    void *amp = nullptr;          // device amplitudes
    bool owned = false;
    bool host_mem = false;        // amplitudes in mapped page-locked host memory
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    qv::Scratch scratch;          // reduction partials, gate programs
    double *host_out = nullptr;   // pinned host buffer for reduction results
    size_t host_out_len = 0;
    qv::Prof prof;
    qv::PlanCache *plan = nullptr;
    qv::AdjointBuffers *adj = nullptr;
    int *dev_status = nullptr;    // device status word written by kernels with bounded waits
    qv::HostWindow *window = nullptr;  // host-memory states: device windows the passes run in
};

namespace qv {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
qv_status fail(qv_status st, const char *fmt, ...);
qv_status cuda_fail(cudaError_t e, const char *what);

#define QV_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return ::qv::cuda_fail(e_, #call); \
    } while (0)

#define QV_TRY(expr)                           \
    do {                                       \
        qv_status st_ = (expr);                \
        if (st_ != QV_OK) return st_;          \
    } while (0)

// Counts a launch of class `cls` and, when timing is on, records CUDA events
// around it on the handle's stream.
void prof_begin(qv_state *s, int cls);
// Adds algorithmic HBM bytes to class `cls`.
inline void prof_bytes(qv_state *s, int cls, double b) { s->prof.bytes[cls] += b; }
void prof_end(qv_state *s, int cls);
qv_status prof_drain(qv_state *s);
void prof_release(qv_state *s);

#define QV_LAUNCH(s, cls, ...)                  \
    do {                                        \
        ::qv::prof_begin((s), (cls));           \
        __VA_ARGS__;                            \
        ::qv::prof_end((s), (cls));             \
        QV_CUDA(cudaGetLastError());            \
    } while (0)

// cudaMemcpyAsync on the handle's stream, counted in the transfer totals.
qv_status copy_h2d(qv_state *s, void *dst, const void *src, size_t bytes);
qv_status copy_d2h(qv_state *s, void *dst, const void *src, size_t bytes);

inline size_t amp_bytes(qv_dtype dt) { return dt == QV_C64 ? 8 : 16; }
inline uint64_t dim(const qv_state *s) { return uint64_t(1) << s->n; }

qv_status ensure_scratch(qv_state *s, size_t bytes);
// Raises the dynamic shared-memory limit of kernel `fn` to `bytes` on the
// current device, once per (kernel, device, bytes); thread-safe.
qv_status allow_smem(const void *fn, int bytes);
// Device status word of the handle (allocated and cleared on first use).
qv_status status_word(qv_state *s, int **out);
// Synchronises the handle's stream and reports a nonzero status word
// (QV_ERR_TIMEOUT from a bounded device wait), clearing it.
qv_status sync_and_check(qv_state *s);
qv_status ensure_host_out(qv_state *s, size_t count);

// ---------------------------------------------------------------- gates (host)
// Matrix of a gate in FP64 (row-major). Returns false for kinds without one.
bool gate_matrix(const qv_gate &g, cd U[4]);
bool is_diagonal(const cd U[4]);

// ---------------------------------------------------------------- kernels (pair_kernels.cu)
qv_status launch_set_basis(qv_state *s, uint64_t j);
// General 2x2 on target t, optional control (ctrl < 0: none).
qv_status launch_pair(qv_state *s, int t, int ctrl, const cd U[4]);
// Diagonal diag(d0, d1) on target t, optional control.
qv_status launch_diag(qv_state *s, int t, int ctrl, cd d0, cd d1);
qv_status launch_swap(qv_state *s, int a, int b);
// out[pi(i)] = in[i]; out and in distinct buffers of the same size.
qv_status launch_permute(qv_state *s, const void *in, void *out, const int32_t *perm);

// One gate through the per-gate kernels (qv_api.cu).
qv_status apply_gate_plain(qv_state *s, const qv_gate &g);
qv_status validate_gate(const qv_gate &g, int n, size_t idx);

// ---------------------------------------------------------------- adjoint (adjoint.cu)
// dst = H src for H = sum of Pauli terms; src, dst: 2^n amplitudes of s's dtype.
qv_status pauli_apply(qv_state *s, const void *src, void *dst, const qv_pauli_term *terms, size_t nt);
// Inverse-CDF samples of the Born distribution for uniforms u (sample.cu).
qv_status sample(qv_state *s, const double *u, size_t nshots, uint64_t *out);
// Amplitudes idx[0..k) copied to host (interleaved re, im in the state's precision).
qv_status get_amplitudes(qv_state *s, const uint64_t *idx, size_t k, void *host);
// sweep: QV_SWEEP_* (qv.h)
qv_status adjoint_grad(qv_state *s, const qv_gate *g, size_t ng, const qv_pauli_term *H, size_t nt, size_t nparams,
                       double *grad_out, double *expval_out, int sweep);
void adjoint_release(qv_state *s);

// ---------------------------------------------------------------- verification (verify.cu)
qv_status verify_qft(qv_state *s, uint64_t j, double *dist);
qv_status distance(qv_state *a, qv_state *b, double *out);

// ---------------------------------------------------------------- split states (dist_plan.cpp)
// restore: steps that bring the qubits back to their natural order follow the circuit
qv_status dist_plan(int n, int g, int rank, const qv_gate *gates, size_t ng, std::vector<qv_dist_step> &steps,
                    std::vector<qv_gate> &local_gates, std::vector<int32_t> &final_perm, bool restore);

// ---------------------------------------------------------------- reductions (reduce_kernels.cu)
// out[0] = sum |a|^2, out[1 + q] = sum over bit q set of |a|^2, q < n.
qv_status reduce_zsums(qv_state *s, double *out_host);
// <psi|P|psi> summed over terms.
qv_status reduce_pauli(qv_state *s, const qv_pauli_term *terms, size_t nt, double *out_host);

}  // namespace qv
