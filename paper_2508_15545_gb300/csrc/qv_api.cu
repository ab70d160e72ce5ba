// C ABI entry points (include/qv.h): handle lifetime, argument checks, gate
// matrices in FP64, and dispatch to the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <unistd.h>
#include <mutex>
#include <set>
#include <tuple>

#include "qv_device.cuh"
#include "qv_internal.h"
#include "qv_plan.h"

namespace qv {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

qv_status fail(qv_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

qv_status cuda_fail(cudaError_t e, const char *what)
{
    const qv_status st = (e == cudaErrorMemoryAllocation) ? QV_ERR_OOM : QV_ERR_CUDA;
    (void)cudaGetLastError();  // clear a sticky launch error so the handle stays usable
    return fail(st, "%s: %s", what, cudaGetErrorString(e));
}

qv_status ensure_scratch(qv_state *s, size_t bytes)
{
    if (s->scratch.bytes >= bytes) return QV_OK;
    if (s->scratch.ptr) {
        QV_CUDA(cudaStreamSynchronize(s->stream));
        QV_CUDA(cudaFree(s->scratch.ptr));
        s->scratch = Scratch{};
    }
    const size_t b = std::max<size_t>(bytes, 1 << 20);
    QV_CUDA(cudaMalloc(&s->scratch.ptr, b));
    s->scratch.bytes = b;
    return QV_OK;
}

qv_status allow_smem(const void *fn, int bytes)
{
    static std::mutex mu;
    static std::set<std::tuple<const void *, int, int>> done;
    int dev = 0;
    QV_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({fn, dev, bytes})) return QV_OK;
    QV_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.insert({fn, dev, bytes});
    return QV_OK;
}

qv_status status_word(qv_state *s, int **out)
{
    if (!s->dev_status) {
        QV_CUDA(cudaMalloc(&s->dev_status, 256));
        QV_CUDA(cudaMemsetAsync(s->dev_status, 0, 256, s->stream));
    }
    *out = s->dev_status;
    return QV_OK;
}

qv_status sync_and_check(qv_state *s)
{
    QV_CUDA(cudaStreamSynchronize(s->stream));
    if (!s->dev_status) return QV_OK;
    int v = 0;
    QV_CUDA(cudaMemcpy(&v, s->dev_status, sizeof v, cudaMemcpyDeviceToHost));
    if (v == 0) return QV_OK;
    QV_CUDA(cudaMemset(s->dev_status, 0, sizeof v));
    return fail(qv_status(v), "a bounded device-side wait gave up (status %d); the state is unspecified", v);
}

qv_status ensure_host_out(qv_state *s, size_t count)
{
    if (s->host_out_len >= count) return QV_OK;
    if (s->host_out) {
        QV_CUDA(cudaStreamSynchronize(s->stream));
        QV_CUDA(cudaFreeHost(s->host_out));
        s->host_out = nullptr;
        s->host_out_len = 0;
    }
    const size_t c = std::max<size_t>(count, 4096);
    QV_CUDA(cudaMallocHost(&s->host_out, c * sizeof(double)));
    s->host_out_len = c;
    return QV_OK;
}

// ---------------------------------------------------------------- gate matrices
bool gate_matrix(const qv_gate &g, cd U[4])
{
    const double th = g.theta[0], ph = g.theta[1], la = g.theta[2];
    const double h = 1.0 / std::sqrt(2.0);
    const cd I(0, 1);
    auto set = [&](cd a, cd b, cd c, cd d) {
        U[0] = a; U[1] = b; U[2] = c; U[3] = d;
        return true;
    };
    switch (g.kind) {
    case QV_G_H: return set(h, h, h, -h);
    case QV_G_X: return set(0, 1, 1, 0);
    case QV_G_Y: return set(0, -I, I, 0);
    case QV_G_Z: return set(1, 0, 0, -1);
    case QV_G_S: return set(1, 0, 0, I);
    case QV_G_SDG: return set(1, 0, 0, -I);
    case QV_G_T: return set(1, 0, 0, cd(h, h));
    case QV_G_TDG: return set(1, 0, 0, cd(h, -h));
    case QV_G_RX: return set(std::cos(th / 2), -I * std::sin(th / 2), -I * std::sin(th / 2), std::cos(th / 2));
    case QV_G_RY: return set(std::cos(th / 2), -std::sin(th / 2), std::sin(th / 2), std::cos(th / 2));
    case QV_G_RZ: return set(std::polar(1.0, -th / 2), 0, 0, std::polar(1.0, th / 2));
    case QV_G_P: return set(1, 0, 0, std::polar(1.0, th));
    case QV_G_U3:
        return set(std::cos(th / 2), -std::polar(1.0, la) * std::sin(th / 2), std::polar(1.0, ph) * std::sin(th / 2),
                   std::polar(1.0, ph + la) * std::cos(th / 2));
    case QV_G_MATRIX:
        return set(cd(g.u[0].re, g.u[0].im), cd(g.u[1].re, g.u[1].im), cd(g.u[2].re, g.u[2].im),
                   cd(g.u[3].re, g.u[3].im));
    default: return false;
    }
}

bool is_diagonal(const cd U[4]) { return U[1] == cd(0, 0) && U[2] == cd(0, 0); }

static bool finite(const cd U[4])
{
    for (int e = 0; e < 4; ++e)
        if (!std::isfinite(U[e].real()) || !std::isfinite(U[e].imag())) return false;
    return true;
}

qv_status validate_gate(const qv_gate &g, int n, size_t idx)
{
    if (g.target < 0 || g.target >= n) return fail(QV_ERR_ARG, "gate %zu: target %d out of range [0, %d)", idx, g.target, n);
    if (g.kind == QV_G_SWAP) {
        if (g.target2 < 0 || g.target2 >= n || g.target2 == g.target)
            return fail(QV_ERR_ARG, "gate %zu: bad swap partner %d", idx, g.target2);
        if (g.ctrl >= 0) return fail(QV_ERR_UNSUPPORTED, "gate %zu: controlled swap", idx);
        return QV_OK;
    }
    if (g.ctrl >= n || g.ctrl == g.target || g.ctrl < -1)
        return fail(QV_ERR_ARG, "gate %zu: bad control %d (target %d)", idx, g.ctrl, g.target);
    cd U[4];
    if (!gate_matrix(g, U)) return fail(QV_ERR_ARG, "gate %zu: unknown kind %d", idx, g.kind);
    if (!finite(U)) return fail(QV_ERR_ARG, "gate %zu: non-finite matrix", idx);
    return QV_OK;
}

// One gate through the per-gate kernels.
qv_status apply_gate_plain(qv_state *s, const qv_gate &g)
{
    if (g.kind == QV_G_SWAP) return launch_swap(s, g.target, g.target2);
    cd U[4];
    gate_matrix(g, U);
    if (is_diagonal(U)) return launch_diag(s, g.target, g.ctrl, U[0], U[3]);
    return launch_pair(s, g.target, g.ctrl, U);
}

}  // namespace qv

using namespace qv;

#define CHECK_HANDLE(s) \
    if (!(s)) return fail(QV_ERR_ARG, "NULL state handle")

extern "C" {

qv_status qv_wrap(void *dev_ptr, int n, qv_dtype dt, void *cuda_stream, qv_state **out)
{
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!dev_ptr) return fail(QV_ERR_ARG, "device pointer is NULL");
    if (n < 1 || n > 40) return fail(QV_ERR_ARG, "n = %d outside [1, 40]", n);
    if (dt != QV_C64 && dt != QV_C128) return fail(QV_ERR_ARG, "bad dtype %d", int(dt));
    if (reinterpret_cast<uintptr_t>(dev_ptr) % 16) return fail(QV_ERR_ARG, "device pointer not 16-byte aligned");
    qv_state *s = new qv_state;
    s->n = n;
    s->dt = dt;
    s->amp = dev_ptr;
    s->owned = false;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaGetDevice");
    }
    *out = s;
    return QV_OK;
}

qv_status qv_create(int n, qv_dtype dt, void *cuda_stream, qv_state **out)
{
    return qv_create_ex(n, dt, cuda_stream, 0, out);
}

qv_status qv_create_ex(int n, qv_dtype dt, void *cuda_stream, int32_t flags, qv_state **out)
{
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 40) return fail(QV_ERR_ARG, "n = %d outside [1, 40]", n);
    if (dt != QV_C64 && dt != QV_C128) return fail(QV_ERR_ARG, "bad dtype %d", int(dt));
    if (flags & ~int32_t(QV_ALLOC_HOST)) return fail(QV_ERR_ARG, "unknown flags 0x%x", unsigned(flags));
    const bool host = flags & QV_ALLOC_HOST;
    const size_t bytes = (size_t(1) << n) * amp_bytes(dt);
    void *p = nullptr;
    cudaError_t e;
    if (host) {
        const long pages = sysconf(_SC_AVPHYS_PAGES), psz = sysconf(_SC_PAGESIZE);
        const double avail = pages > 0 && psz > 0 ? double(pages) * double(psz) : 0.0;
        if (double(bytes) > 0.75 * avail)
            return fail(QV_ERR_OOM, "state needs %zu bytes of host memory, %.0f available", bytes, avail);
        e = cudaHostAlloc(&p, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc(state)");
        void *dp = nullptr;
        e = cudaHostGetDevicePointer(&dp, p, 0);
        if (e != cudaSuccess || dp != p) {  // kernels use the host address (unified addressing)
            cudaFreeHost(p);
            return e != cudaSuccess ? cuda_fail(e, "cudaHostGetDevicePointer")
                                    : fail(QV_ERR_UNSUPPORTED, "host memory is not mapped at its own address");
        }
    } else {
        size_t free_b = 0, total_b = 0;
        e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
        if (bytes > free_b) return fail(QV_ERR_OOM, "state needs %zu bytes, %zu free", bytes, free_b);
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(state)");
    }
    qv_status st = qv_wrap(p, n, dt, cuda_stream, out);
    if (st != QV_OK) {
        if (host) cudaFreeHost(p);
        else cudaFree(p);
        return st;
    }
    (*out)->owned = true;
    (*out)->host_mem = host;
    st = launch_set_basis(*out, 0);
    if (st != QV_OK) {
        qv_destroy(*out);
        *out = nullptr;
    }
    return st;
}

qv_status qv_destroy(qv_state *s)
{
    if (!s) return QV_OK;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    window_release(s);
    plan_cache_release(s);
    adjoint_release(s);
    prof_release(s);
    if (s->scratch.ptr) cudaFree(s->scratch.ptr);
    if (s->host_out) cudaFreeHost(s->host_out);
    if (s->owned && s->amp) {
        if (s->host_mem) cudaFreeHost(s->amp);
        else cudaFree(s->amp);
    }
    if (s->dev_status) cudaFree(s->dev_status);
    delete s;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return QV_OK;
}

qv_status qv_set_stream(qv_state *s, void *cuda_stream)
{
    CHECK_HANDLE(s);
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    return QV_OK;
}

qv_status qv_info(const qv_state *s, int *n, qv_dtype *dt, void **dev_ptr)
{
    CHECK_HANDLE(s);
    if (n) *n = s->n;
    if (dt) *dt = s->dt;
    if (dev_ptr) *dev_ptr = s->amp;
    return QV_OK;
}

qv_status qv_set_basis(qv_state *s, uint64_t j)
{
    CHECK_HANDLE(s);
    if (j >= dim(s)) return fail(QV_ERR_ARG, "basis index out of range");
    return launch_set_basis(s, j);
}

qv_status qv_get_state(qv_state *s, void *host, size_t bytes)
{
    CHECK_HANDLE(s);
    if (!host) return fail(QV_ERR_ARG, "host is NULL");
    if (bytes != dim(s) * amp_bytes(s->dt)) return fail(QV_ERR_ARG, "bytes != state size");
    QV_CUDA(cudaMemcpyAsync(host, s->amp, bytes, cudaMemcpyDefault, s->stream));
    return sync_and_check(s);
}

qv_status qv_set_state(qv_state *s, const void *host, size_t bytes)
{
    CHECK_HANDLE(s);
    if (!host) return fail(QV_ERR_ARG, "host is NULL");
    if (bytes != dim(s) * amp_bytes(s->dt)) return fail(QV_ERR_ARG, "bytes != state size");
    QV_CUDA(cudaMemcpyAsync(s->amp, host, bytes, cudaMemcpyDefault, s->stream));
    QV_CUDA(cudaStreamSynchronize(s->stream));
    return QV_OK;
}

qv_status qv_apply_1q(qv_state *s, int target, const qv_c128 U[4])
{
    CHECK_HANDLE(s);
    if (!U) return fail(QV_ERR_ARG, "U is NULL");
    qv_gate g{};
    g.kind = QV_G_MATRIX;
    g.target = target;
    g.target2 = -1;
    g.ctrl = -1;
    for (int e = 0; e < 4; ++e) g.u[e] = U[e];
    QV_TRY(validate_gate(g, s->n, 0));
    cd M[4];
    gate_matrix(g, M);
    return launch_pair(s, target, -1, M);
}

qv_status qv_apply_controlled(qv_state *s, int ctrl, int target, const qv_c128 U[4])
{
    CHECK_HANDLE(s);
    if (!U) return fail(QV_ERR_ARG, "U is NULL");
    if (ctrl < 0) return fail(QV_ERR_ARG, "control %d out of range", ctrl);
    qv_gate g{};
    g.kind = QV_G_MATRIX;
    g.target = target;
    g.target2 = -1;
    g.ctrl = ctrl;
    for (int e = 0; e < 4; ++e) g.u[e] = U[e];
    QV_TRY(validate_gate(g, s->n, 0));
    cd M[4];
    gate_matrix(g, M);
    return launch_pair(s, target, ctrl, M);
}

qv_status qv_apply_circuit(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts)
{
    CHECK_HANDLE(s);
    if (ng && !g) return fail(QV_ERR_ARG, "gate list is NULL");
    for (size_t k = 0; k < ng; ++k) QV_TRY(validate_gate(g[k], s->n, k));
    const int mode = opts ? opts->mode : QV_MODE_AUTO;
    if (mode != QV_MODE_AUTO && mode != QV_MODE_PLAIN && mode != QV_MODE_FUSED)
        return fail(QV_ERR_ARG, "bad mode %d", mode);
    if (mode == QV_MODE_PLAIN || (mode == QV_MODE_AUTO && !fused_supported(s, opts))) {
        for (size_t k = 0; k < ng; ++k) QV_TRY(apply_gate_plain(s, g[k]));
        return QV_OK;
    }
    return apply_fused(s, g, ng, opts);
}

namespace {
// Arguments of the host-only planning calls: size, dtype and every gate.
qv_status check_plan_args(int n, qv_dtype dt, const qv_gate *g, size_t ng)
{
    if (n < 1 || n > 40) return fail(QV_ERR_ARG, "n = %d outside [1, 40]", n);
    if (dt != QV_C64 && dt != QV_C128) return fail(QV_ERR_ARG, "bad dtype %d", int(dt));
    if (ng && !g) return fail(QV_ERR_ARG, "gate list is NULL");
    for (size_t k = 0; k < ng; ++k) QV_TRY(validate_gate(g[k], n, k));
    return QV_OK;
}
}  // namespace

qv_status qv_plan_info(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t out[4])
{
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    QV_TRY(check_plan_args(n, dt, g, ng));
    return plan_info(n, dt, g, ng, opts, out, nullptr);
}

qv_status qv_plan_cost(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, double out[2])
{
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    QV_TRY(check_plan_args(n, dt, g, ng));
    return plan_info(n, dt, g, ng, opts, nullptr, out);
}

qv_status qv_plan_source(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t pass,
                         char *buf, size_t cap, size_t *len)
{
    if (!len) return fail(QV_ERR_ARG, "len is NULL");
    if (cap && !buf) return fail(QV_ERR_ARG, "buf is NULL");
    QV_TRY(check_plan_args(n, dt, g, ng));
    std::string src;
    QV_TRY(plan_source(n, dt, g, ng, opts, pass, src));
    *len = src.size();
    if (cap) {
        const size_t m = std::min(cap - 1, src.size());
        std::memcpy(buf, src.data(), m);
        buf[m] = '\0';
    }
    return QV_OK;
}

qv_status qv_dist_plan(int n, int global_bits, int rank, const qv_gate *g, size_t ng, int32_t flags,
                       qv_dist_step *steps, size_t steps_cap, size_t *nsteps, qv_gate *local_gates, size_t gates_cap,
                       size_t *ngates, int32_t *final_perm)
{
    if (flags & ~int32_t(QV_DIST_RESTORE)) return fail(QV_ERR_ARG, "unknown flags 0x%x", unsigned(flags));
    if (!nsteps || !ngates) return fail(QV_ERR_ARG, "nsteps or ngates is NULL");
    QV_TRY(check_plan_args(n, QV_C64, g, ng));
    if (global_bits < 1 || global_bits >= n || global_bits > 30)
        return fail(QV_ERR_ARG, "global_bits = %d outside [1, n - 1]", global_bits);
    if (rank < 0 || rank >= (1 << global_bits)) return fail(QV_ERR_ARG, "rank %d outside [0, 2^%d)", rank, global_bits);
    std::vector<qv_dist_step> st;
    std::vector<qv_gate> lg;
    std::vector<int32_t> perm;
    QV_TRY(dist_plan(n, global_bits, rank, g, ng, st, lg, perm, (flags & QV_DIST_RESTORE) != 0));
    *nsteps = st.size();
    *ngates = lg.size();
    if (final_perm) std::copy(perm.begin(), perm.end(), final_perm);
    if (!steps || !local_gates) return QV_OK;
    if (steps_cap < st.size() || gates_cap < lg.size())
        return fail(QV_ERR_ARG, "buffers too small: %zu steps and %zu gates needed", st.size(), lg.size());
    std::copy(st.begin(), st.end(), steps);
    std::copy(lg.begin(), lg.end(), local_gates);
    return QV_OK;
}

qv_status qv_plan_tc_stage(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t pass,
                           int32_t stage, qv_tc_stage *out)
{
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    QV_TRY(check_plan_args(n, dt, g, ng));
    return plan_tc_stage(n, dt, g, ng, opts, pass, stage, out);
}

qv_status qv_plan_compile(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int64_t out[4])
{
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    QV_TRY(check_plan_args(n, dt, g, ng));
    return plan_compile(n, dt, g, ng, opts, out);
}

qv_status qv_permute_qubits(qv_state *s, const int32_t *perm)
{
    CHECK_HANDLE(s);
    if (!perm) return fail(QV_ERR_ARG, "perm is NULL");
    std::vector<int> seen(s->n, 0);
    for (int q = 0; q < s->n; ++q) {
        if (perm[q] < 0 || perm[q] >= s->n || seen[perm[q]]++) return fail(QV_ERR_ARG, "not a permutation");
    }
    return apply_permutation(s, perm);
}

qv_status qv_norm2(qv_state *s, double *out)
{
    CHECK_HANDLE(s);
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    std::vector<double> z(s->n + 1);
    QV_TRY(reduce_zsums(s, z.data()));
    *out = z[0];
    return QV_OK;
}

qv_status qv_expect_z(qv_state *s, const double *weights, double *per_qubit, double *total)
{
    CHECK_HANDLE(s);
    std::vector<double> z(s->n + 1);
    QV_TRY(reduce_zsums(s, z.data()));
    Neumaier acc;
    for (int q = 0; q < s->n; ++q) {
        const double ez = z[0] - 2.0 * z[1 + q];
        if (per_qubit) per_qubit[q] = ez;
        acc.add((weights ? weights[q] : 1.0) * ez);
    }
    if (total) *total = acc.value();
    return QV_OK;
}

qv_status qv_expect_pauli(qv_state *s, const qv_pauli_term *terms, size_t nt, double *out)
{
    CHECK_HANDLE(s);
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    if (nt && !terms) return fail(QV_ERR_ARG, "terms is NULL");
    const uint64_t lim = s->n >= 64 ? ~uint64_t(0) : (uint64_t(1) << s->n) - 1;
    for (size_t k = 0; k < nt; ++k)
        if ((terms[k].xmask | terms[k].zmask) & ~lim) return fail(QV_ERR_ARG, "term %zu acts on a qubit >= n", k);
    return reduce_pauli(s, terms, nt, out);
}

qv_status qv_apply_pauli(qv_state *s, const qv_pauli_term *terms, size_t nt, qv_state *out)
{
    CHECK_HANDLE(s);
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    if (out == s || out->amp == s->amp) return fail(QV_ERR_ARG, "out must be a different buffer");
    if (out->n != s->n || out->dt != s->dt) return fail(QV_ERR_ARG, "out must have the same n and dtype");
    if (out->stream != s->stream) return fail(QV_ERR_ARG, "out must use the same stream");
    if (nt && !terms) return fail(QV_ERR_ARG, "terms is NULL");
    const uint64_t lim = (uint64_t(1) << s->n) - 1;
    for (size_t k = 0; k < nt; ++k)
        if ((terms[k].xmask | terms[k].zmask) & ~lim) return fail(QV_ERR_ARG, "term %zu acts on a qubit >= n", k);
    return pauli_apply(s, s->amp, out->amp, terms, nt);
}

qv_status qv_adjoint_grad(qv_state *s, const qv_gate *g, size_t ng, const qv_pauli_term *H, size_t nt,
                          size_t nparams, double *grad_out, double *expval_out)
{
    return qv_adjoint_grad_ex(s, g, ng, H, nt, nparams, grad_out, expval_out, QV_SWEEP_AUTO);
}

qv_status qv_adjoint_grad_ex(qv_state *s, const qv_gate *g, size_t ng, const qv_pauli_term *H, size_t nt,
                             size_t nparams, double *grad_out, double *expval_out, int32_t sweep_mode)
{
    CHECK_HANDLE(s);
    if (sweep_mode < QV_SWEEP_AUTO || sweep_mode > QV_SWEEP_COMPILED)
        return fail(QV_ERR_ARG, "bad sweep mode %d", int(sweep_mode));
    if (ng && !g) return fail(QV_ERR_ARG, "gate list is NULL");
    if (nt && !H) return fail(QV_ERR_ARG, "terms is NULL");
    if (nparams && !grad_out) return fail(QV_ERR_ARG, "grad_out is NULL");
    const uint64_t lim = (uint64_t(1) << s->n) - 1;
    for (size_t k = 0; k < nt; ++k)
        if ((H[k].xmask | H[k].zmask) & ~lim) return fail(QV_ERR_ARG, "term %zu acts on a qubit >= n", k);
    for (size_t l = 0; l < ng; ++l) {
        QV_TRY(validate_gate(g[l], s->n, l));
        const qv_gate &G = g[l];
        const int nangles = G.kind == QV_G_U3 ? 3 : (G.kind == QV_G_RX || G.kind == QV_G_RY || G.kind == QV_G_RZ ||
                                                     G.kind == QV_G_P) ? 1 : 0;
        for (int a = 0; a < 3; ++a) {
            if (G.param[a] < -1) return fail(QV_ERR_ARG, "gate %zu: bad parameter index %d", l, G.param[a]);
            if (G.param[a] >= 0 && a >= nangles)
                return fail(QV_ERR_ARG, "gate %zu: angle %d of this gate kind is not trainable", l, a);
            if (G.param[a] >= 0 && size_t(G.param[a]) >= nparams)
                return fail(QV_ERR_ARG, "gate %zu: parameter index %d >= nparams", l, G.param[a]);
        }
    }
    return adjoint_grad(s, g, ng, H, nt, nparams, grad_out, expval_out, sweep_mode);
}

qv_status qv_autotune(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t *best_tile_bits)
{
    CHECK_HANDLE(s);
    if (ng && !g) return fail(QV_ERR_ARG, "gate list is NULL");
    for (size_t k = 0; k < ng; ++k) QV_TRY(validate_gate(g[k], s->n, k));
    return autotune(s, g, ng, opts, best_tile_bits, nullptr);
}

qv_status qv_autotune_ex(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t out[2])
{
    CHECK_HANDLE(s);
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    if (ng && !g) return fail(QV_ERR_ARG, "gate list is NULL");
    for (size_t k = 0; k < ng; ++k) QV_TRY(validate_gate(g[k], s->n, k));
    return autotune(s, g, ng, opts, out, out + 1);
}

int32_t qv_batch_info(const qv_batch *b, int32_t *out, size_t cap)
{
    if (!b) return -1;
    if (cap && !out) return -1;
    return int32_t(batch_info(b, out, cap));
}

qv_status qv_batch_create(const qv_batch_item *items, size_t count, const qv_pauli_term *H, size_t nt,
                          const qv_plan_opts *opts, qv_batch **out)
{
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!items || count == 0) return fail(QV_ERR_ARG, "empty batch");
    if (count > 65535) return fail(QV_ERR_ARG, "batch of %zu circuits exceeds 65535", count);
    if (nt && !H) return fail(QV_ERR_ARG, "terms is NULL");
    std::vector<const qv_state *> seen;
    for (size_t c = 0; c < count; ++c) {
        const qv_state *s = items[c].state;
        if (!s) return fail(QV_ERR_ARG, "batch item %zu: NULL state", c);
        if (s->dt != items[0].state->dt) return fail(QV_ERR_ARG, "batch item %zu: dtype differs", c);
        if (s->device != items[0].state->device) return fail(QV_ERR_ARG, "batch item %zu: other device", c);
        for (const qv_state *o : seen)
            if (o == s || o->amp == s->amp) return fail(QV_ERR_ARG, "batch item %zu: state used twice", c);
        seen.push_back(s);
        if (items[c].ngates && !items[c].gates) return fail(QV_ERR_ARG, "batch item %zu: gate list is NULL", c);
        for (size_t k = 0; k < items[c].ngates; ++k) QV_TRY(validate_gate(items[c].gates[k], s->n, k));
        const uint64_t lim = (uint64_t(1) << s->n) - 1;
        for (size_t k = 0; k < nt; ++k)
            if ((H[k].xmask | H[k].zmask) & ~lim) return fail(QV_ERR_ARG, "term %zu acts on a qubit >= n of item %zu", k, c);
    }
    return batch_create(items, count, H, nt, opts, out);
}

qv_status qv_batch_run(qv_batch *b, double *expvals)
{
    if (!b) return fail(QV_ERR_ARG, "NULL batch");
    return batch_run(b, expvals);
}

qv_status qv_batch_destroy(qv_batch *b)
{
    batch_release(b);
    return QV_OK;
}

qv_status qv_apply_batch(const qv_batch_item *items, size_t count, const qv_pauli_term *H, size_t nt,
                         const qv_plan_opts *opts, double *expvals)
{
    qv_batch *b = nullptr;
    QV_TRY(qv_batch_create(items, count, H, nt, opts, &b));
    const qv_status st = qv_batch_run(b, expvals);
    batch_release(b);
    return st;
}

qv_status qv_verify_qft(qv_state *s, uint64_t j, double *dist)
{
    CHECK_HANDLE(s);
    if (!dist) return fail(QV_ERR_ARG, "dist is NULL");
    if (j >= dim(s)) return fail(QV_ERR_ARG, "basis index out of range");
    return verify_qft(s, j, dist);
}

qv_status qv_distance(qv_state *a, qv_state *b, double *out)
{
    CHECK_HANDLE(a);
    CHECK_HANDLE(b);
    if (!out) return fail(QV_ERR_ARG, "out is NULL");
    if (a->n != b->n) return fail(QV_ERR_ARG, "states differ in n");
    return distance(a, b, out);
}

int32_t qv_default_tile_bits(int n, qv_dtype dt, int32_t flags)
{
    if (n < 1 || n > 40) return 0;
    return tuned_tile_bits(n, dt, (flags & QV_PLAN_INTERPRET) != 0);
}

qv_status qv_sample(qv_state *s, const double *u, size_t nshots, uint64_t *out)
{
    CHECK_HANDLE(s);
    if (nshots == 0) return QV_OK;
    if (!u || !out) return fail(QV_ERR_ARG, "u or out is NULL");
    if (nshots > (size_t(1) << 31)) return fail(QV_ERR_ARG, "at most 2^31 shots per call");
    for (size_t k = 0; k < nshots; ++k)
        if (!(u[k] >= 0.0 && u[k] < 1.0)) return fail(QV_ERR_ARG, "u[%zu] = %g outside [0, 1)", k, u[k]);
    return sample(s, u, nshots, out);
}

qv_status qv_get_amplitudes(qv_state *s, const uint64_t *idx, size_t k, void *host)
{
    CHECK_HANDLE(s);
    if (k == 0) return QV_OK;
    if (!idx || !host) return fail(QV_ERR_ARG, "idx or host is NULL");
    for (size_t j = 0; j < k; ++j)
        if (idx[j] >= dim(s)) return fail(QV_ERR_ARG, "idx[%zu] = %llu >= 2^n", j, (unsigned long long)idx[j]);
    return get_amplitudes(s, idx, k, host);
}

qv_status qv_wait_selftest(qv_state *s, uint32_t limit)
{
    CHECK_HANDLE(s);
    return wait_selftest(s, limit);
}

qv_status qv_sync(qv_state *s)
{
    CHECK_HANDLE(s);
    return sync_and_check(s);
}

const char *qv_last_error(void) { return g_err; }

}  // extern "C"
