// Fused tiled passes: the on-chip form of the paper's block storage and
// sliding-window cache (Sec. III-B/C, Eq. 6-8) with the single-traversal idea
// of Sec. III-E. Each pass loads every 2^K-amplitude tile once (16-byte vector
// loads of contiguous 2^5-amplitude runs), applies all gates the planner gave
// the pass in registers -- changing which tile qubits are register-local with
// swizzled shared-memory transposes -- and stores the tile once.
//
// Register file of a thread: 16 amplitudes ("slots" m = 0..15, one slot bit
// per layout register bit). Complex64 keeps tile qubit 0 on register bit 3 and
// packs the two amplitudes that differ in it into one f32x2 register pair for
// the real parts and one for the imaginary parts, so a gate on register bit
// 0..2 updates two amplitude pairs per fma.rn.f32x2 (Blackwell's paired FP32
// instructions), and a transpose moves each packed pair as one 8-byte word.
// Gates on register bit 3 pair the two lanes of one register (scalar FP32).
// Complex128 keeps scalar doubles.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "fused_device.cuh"
#include "planner.h"
#include "qv_internal.h"
#include "qv_jit.h"
#include "qv_plan.h"

namespace qv {

struct PlanCache {
    void *dev = nullptr;   // interpreter programs on the device
    size_t bytes = 0;
    // the last gate list planned on this handle, its plan and compiled program:
    // applying the same list again (same bytes, tile size and flags) skips the
    // planning and the code generation
    std::vector<qv_gate> key;
    int K = 0, flags = 0;
    std::vector<plan::Pass> passes;
    std::shared_ptr<JitProgram> jit;
};

namespace {
// One pass. Persistent CTAs walk the tiles; the pass program is copied to
// shared memory once per CTA.
template <typename R, int K>
__global__ void __launch_bounds__(1 << (K - kRegBits), QV_FUSED_MINB(R, K)) fused_pass_kernel(R *__restrict__ amp,
                                                                         const unsigned char *__restrict__ blob,
                                                                         uint64_t ntiles)
{
    constexpr int T = 1 << (K - kRegBits);
    constexpr int NQ = K - kRegBits;
    constexpr int NH = K - kChunkBits;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *tile = smem;
    uint64_t *phys_hi = reinterpret_cast<uint64_t *>(smem + tile_smem<R, K>());
    unsigned char *prog = smem + tile_smem<R, K>() + table_smem<K>();

    const DHdr *gh = reinterpret_cast<const DHdr *>(blob);
    const int nstages = gh->nstages, nops = gh->nops;
    const size_t nb = blob_bytes<R>(nstages, nops);
    for (size_t i = size_t(threadIdx.x) * 16; i < nb; i += size_t(T) * 16)
        *reinterpret_cast<uint4 *>(prog + i) = *reinterpret_cast<const uint4 *>(blob + i);
    __syncthreads();
    const DHdr &h = *reinterpret_cast<const DHdr *>(prog);
    const DStage *stg = reinterpret_cast<const DStage *>(prog + sizeof(DHdr));
    const DOp<R> *ops = reinterpret_cast<const DOp<R> *>(prog + ops_offset<R>(nstages));
    for (int i = threadIdx.x; i < (1 << NH); i += T) {
        uint64_t v = 0;
        for (int j = 0; j < NH; ++j)
            if ((i >> j) & 1) v |= uint64_t(1) << h.s_high[j];
        phys_hi[i] = v;
    }
    __syncthreads();

    const int tid = threadIdx.x;
    Regs<R> x;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint64_t base = 0;
        for (int s = 0; s < h.nseg; ++s)
            base |= ((t >> h.seg_src[s]) & ((uint64_t(1) << h.seg_w[s]) - 1)) << h.seg_dst[s];
        load_tile<NQ>(amp, base, stg[0].P, stg[0].Q, tid, phys_hi, x);
        for (int s = 0; s < nstages; ++s) {
            if (s > 0) transpose<K, NQ>(tile, stg[s - 1], stg[s], tid, x);
            run_ops<R>(ops + stg[s].op_begin, stg[s].op_end - stg[s].op_begin, tid, base, x);
        }
        // With one stage no transpose separates the loads from the stores; a SWAP
        // relabel can send a warp's data to positions another warp still has to load.
        if (nstages == 1) __syncthreads();
        store_tile<NQ>(amp, base, stg[nstages - 1].Po, stg[nstages - 1].Qo, tid, phys_hi, x);
    }
}

template <typename R, int K> size_t smem_for(size_t blob)
{
    return tile_smem<R, K>() + table_smem<K>() + blob;
}

template <typename R, int K> qv_status launch_pass(qv_state *s, const unsigned char *dblob, size_t blob)
{
    QV_TRY(allow_smem(reinterpret_cast<const void *>(fused_pass_kernel<R, K>), 227 * 1024));
    constexpr int T = 1 << (K - kRegBits);
    const size_t smem = smem_for<R, K>(blob);
    int per_sm = 0;
    QV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_pass_kernel<R, K>, T, smem));
    if (per_sm < 1) return fail(QV_ERR_UNSUPPORTED, "fused pass does not fit on an SM (%zu bytes smem)", smem);
    const uint64_t ntiles = dim(s) >> K;
    const unsigned grid = unsigned(std::min<uint64_t>(ntiles, uint64_t(per_sm) * s->num_sms));
    prof_bytes(s, QV_K_FUSED, 2.0 * double(dim(s)) * 2 * sizeof(R));
    QV_LAUNCH(s, QV_K_FUSED, fused_pass_kernel<R, K><<<grid, T, smem, s->stream>>>(static_cast<R *>(s->amp), dblob,
                                                                                  ntiles));
    return QV_OK;
}

template <typename R> qv_status run_plan(qv_state *s, const std::vector<plan::Pass> &passes, int K)
{
    std::vector<unsigned char> buf;
    std::vector<size_t> offs, sizes;
    for (const auto &p : passes) {
        for (const plan::Op &op : p.ops)
            if (op.type == plan::OP_GEN2) return fail(QV_ERR_UNSUPPORTED, "4x4 operations need the compiled kernel");
        buf.resize((buf.size() + 255) & ~size_t(255), 0);
        offs.push_back(buf.size());
        serialize<R>(p, buf);
        sizes.push_back(buf.size() - offs.back());
    }
    if (buf.empty()) return QV_OK;
    if (!s->plan) s->plan = new PlanCache;
    if (s->plan->bytes < buf.size()) {
        if (s->plan->dev) {
            QV_CUDA(cudaStreamSynchronize(s->stream));
            QV_CUDA(cudaFree(s->plan->dev));
            s->plan->dev = nullptr;
            s->plan->bytes = 0;
        }
        const size_t b = std::max<size_t>(buf.size() * 2, 1 << 16);
        QV_CUDA(cudaMalloc(&s->plan->dev, b));
        s->plan->bytes = b;
    } else {
        // earlier passes may still read the old programs
        QV_CUDA(cudaStreamSynchronize(s->stream));
    }
    QV_TRY(copy_h2d(s, s->plan->dev, buf.data(), buf.size()));
    const unsigned char *d = static_cast<const unsigned char *>(s->plan->dev);
    for (size_t i = 0; i < passes.size(); ++i) {
        switch (K) {
        case 10: QV_TRY((launch_pass<R, 10>(s, d + offs[i], sizes[i]))); break;
        case 11: QV_TRY((launch_pass<R, 11>(s, d + offs[i], sizes[i]))); break;
        case 12: QV_TRY((launch_pass<R, 12>(s, d + offs[i], sizes[i]))); break;
        default: return fail(QV_ERR_ARG, "tile bits %d unsupported", K);
        }
    }
    return QV_OK;
}

int default_tile_bits(const qv_state *s, const qv_plan_opts *opts)
{
    // a state in host memory is bound by the host link on every pass: the largest
    // tile, for the fewest passes (30 qubits: 2.25 s at 2^12 against 3.03 s at 2^11)
    if (s->host_mem) return std::min(s->n, plan::kMaxK);
    return tuned_tile_bits(s->n, s->dt, (opts && (opts->flags & QV_PLAN_INTERPRET)) || !jit_available(nullptr));
}

}  // namespace

bool fused_supported(const qv_state *s, const qv_plan_opts *) { return s->n >= plan::kMinK; }

qv_status to_pgates(const qv_gate *g, size_t ng, std::vector<plan::PGate> &out)
{
    out.resize(ng);
    for (size_t i = 0; i < ng; ++i) {
        plan::PGate &p = out[i];
        p.t = g[i].target;
        p.t2 = -1;
        p.c = g[i].ctrl;
        if (g[i].kind == QV_G_SWAP) {
            p.cls = plan::G_SWAP;
            p.t2 = g[i].target2;
            continue;
        }
        if (!gate_matrix(g[i], p.U)) return fail(QV_ERR_ARG, "gate %zu: unknown kind", i);
        p.cls = plan::classify(p.U);
    }
    return QV_OK;
}

// The fused-mode plan of g as a device-memory state would get it (host only:
// NVRTC is not consulted; the compiled complex64 engine's 4x4 pair ops unless
// interpreting or QV_PLAN_NO_PAIRS).
qv_status plan_host(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts,
                    std::vector<plan::Pass> &passes, plan::PlanStats &st)
{
    int K = (opts && opts->tile_bits) ? opts->tile_bits
                                      : tuned_tile_bits(n, dt, opts && (opts->flags & QV_PLAN_INTERPRET));
    if (K < plan::kMinK || K > plan::kMaxK || K > n) return fail(QV_ERR_ARG, "tile_bits %d unsupported for n = %d", K, n);
    std::vector<plan::PGate> pg;
    QV_TRY(to_pgates(g, ng, pg));
    std::string err;
    const int flags = opts ? opts->flags : 0;
    const bool fuse = !(flags & QV_PLAN_NO_FUSION);
    const bool pairs = dt == QV_C64 && !(flags & (QV_PLAN_INTERPRET | QV_PLAN_NO_PAIRS));
    const bool tc = (flags & QV_PLAN_TENSOR) != 0;
    if (tc && (dt != QV_C64 || (flags & QV_PLAN_INTERPRET)))
        return fail(QV_ERR_ARG, "tensor-core passes are compiled and complex64 only");
    if (!plan::make_plan(n, K, dt == QV_C64, fuse, pairs, pg, passes, st, err, tc))
        return fail(QV_ERR_UNSUPPORTED, "planner: %s", err.c_str());
    return QV_OK;
}

qv_status plan_tc_stage(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int pass,
                        int stage, qv_tc_stage *out)
{
    if (!opts || !(opts->flags & QV_PLAN_TENSOR)) return fail(QV_ERR_ARG, "not a tensor-core plan (QV_PLAN_TENSOR)");
    std::vector<plan::Pass> passes;
    plan::PlanStats st;
    QV_TRY(plan_host(n, dt, g, ng, opts, passes, st));
    if (pass < 0 || size_t(pass) >= passes.size()) return fail(QV_ERR_ARG, "pass %d outside [0, %zu)", pass, passes.size());
    const plan::Pass &P = passes[size_t(pass)];
    if (stage < 0 || size_t(stage) >= P.stages.size())
        return fail(QV_ERR_ARG, "stage %d outside [0, %zu)", stage, P.stages.size());
    const plan::Stage &S = P.stages[size_t(stage)];
    std::memset(out, 0, sizeof(*out));
    out->k = P.k;
    out->nstages = int32_t(P.stages.size());
    for (int p = 0; p < 12; ++p) out->tile_qubit[p] = -1;
    for (int p = 0; p < plan::kChunkBits; ++p) out->tile_qubit[p] = p;
    for (int j = 0; j < P.k - plan::kChunkBits; ++j) out->tile_qubit[plan::kChunkBits + j] = P.s_high[j];
    for (int j = 0; j < plan::kRegBits; ++j) {
        out->in_reg[j] = S.in.P[j];
        out->out_reg[j] = S.out.P[j];
    }
    for (int b = 0; b < 8; ++b) {
        out->in_thr[b] = b < P.k - plan::kRegBits ? S.in.Q[b] : -1;
        out->out_thr[b] = b < P.k - plan::kRegBits ? S.out.Q[b] : -1;
    }
    out->has_matrix = S.mat >= 0;
    out->ext = S.ext;
    if (S.mat >= 0)
        for (int v = 0; v < (S.ext >= 0 ? 2 : 1); ++v)
            for (int e = 0; e < plan::kTcSlot; ++e) {
                const cd z = P.tcm[size_t(S.mat + v) * plan::kTcSlot + e];
                out->m[v][e].re = z.real();
                out->m[v][e].im = z.imag();
            }
    return QV_OK;
}

qv_status plan_source(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int pass,
                      std::string &src)
{
    if (opts && (opts->flags & QV_PLAN_INTERPRET)) return fail(QV_ERR_ARG, "the interpreting engine compiles no passes");
    std::vector<plan::Pass> passes;
    plan::PlanStats st;
    QV_TRY(plan_host(n, dt, g, ng, opts, passes, st));
    if (pass < 0 || size_t(pass) >= passes.size())
        return fail(QV_ERR_ARG, "pass %d outside [0, %zu)", pass, passes.size());
    src = jit_pass_source(passes[size_t(pass)], dt == QV_C64);
    return QV_OK;
}

qv_status plan_compile(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int64_t out[4])
{
    if (opts && (opts->flags & QV_PLAN_INTERPRET)) return fail(QV_ERR_ARG, "the interpreting engine compiles no passes");
    std::vector<plan::Pass> passes;
    plan::PlanStats st;
    QV_TRY(plan_host(n, dt, g, ng, opts, passes, st));
    return jit_compile_host(passes, dt == QV_C64, out);
}

qv_status plan_info(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t out[4],
                    double cost[2])
{
    std::vector<plan::Pass> passes;
    plan::PlanStats st;
    QV_TRY(plan_host(n, dt, g, ng, opts, passes, st));
    if (out) {
        out[0] = st.passes;
        out[1] = st.stages;
        out[2] = st.transposes;
        out[3] = (opts && (opts->flags & QV_PLAN_TENSOR)) ? st.tc_mats : st.ops;
    }
    if (cost) {
        const double N = std::ldexp(1.0, n);
        cost[0] = 2.0 * st.passes * N * double(amp_bytes(dt));
        cost[1] = st.flops_per_amp * N;
    }
    return QV_OK;
}

qv_status apply_fused(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts)
{
    if (ng == 0) return QV_OK;
    if (opts && opts->window_bits && (opts->window_bits < plan::kMinK || opts->window_bits > s->n))
        return fail(QV_ERR_ARG, "window_bits %d outside [%d, n = %d]", opts->window_bits, plan::kMinK, s->n);
    if (s->host_mem && !(opts && (opts->flags & QV_PLAN_HOST_IN_PLACE)) &&
        ((opts && opts->window_bits) || default_window_bits(s) > 0))
        return apply_windowed(s, g, ng, opts);
    int K = (opts && opts->tile_bits) ? opts->tile_bits : default_tile_bits(s, opts);
    if (K < plan::kMinK || K > plan::kMaxK) return fail(QV_ERR_ARG, "tile_bits %d outside [10, 12]", K);
    if (K > s->n) return fail(QV_ERR_ARG, "tile_bits %d exceeds n = %d", K, s->n);
    int flags = opts ? opts->flags : 0;
    // the autotuner's schedule variant goes with its tile size
    if (!(opts && opts->tile_bits) && !s->host_mem &&
        !(flags & (QV_PLAN_NO_FUSION | QV_PLAN_INTERPRET | QV_PLAN_NO_PAIRS | QV_PLAN_TENSOR)))
        flags |= tuned_flags(s->n, s->dt, !jit_available(nullptr));
    const bool fuse = !(flags & QV_PLAN_NO_FUSION);
    const bool jit = !(flags & QV_PLAN_INTERPRET) && jit_available(nullptr);
    const bool tc = (flags & QV_PLAN_TENSOR) != 0;
    if (tc) {
        if (s->dt != QV_C64 || (flags & QV_PLAN_INTERPRET))
            return fail(QV_ERR_ARG, "tensor-core passes are compiled and complex64 only");
        if (K < 11) return fail(QV_ERR_ARG, "tensor-core passes need tiles of 2^11 or 2^12 amplitudes");
        std::string why;
        if (!jit_available(&why)) return fail(QV_ERR_UNSUPPORTED, "tensor-core passes need NVRTC: %s", why.c_str());
    }
    if (!s->plan) s->plan = new PlanCache;
    PlanCache &C = *s->plan;
    const bool hit = C.K == K && C.flags == flags && C.key.size() == ng &&
                     std::memcmp(C.key.data(), g, ng * sizeof(qv_gate)) == 0;
    if (!hit) {
        std::vector<plan::PGate> pg;
        QV_TRY(to_pgates(g, ng, pg));
        std::vector<plan::Pass> passes;
        plan::PlanStats st;
        std::string err;
        // 4x4 operations exist only in the compiled complex64 kernel
        const bool pairs = jit && s->dt == QV_C64 && !(flags & QV_PLAN_NO_PAIRS);
        if (!plan::make_plan(s->n, K, s->dt == QV_C64, fuse, pairs, pg, passes, st, err, tc))
            return fail(QV_ERR_UNSUPPORTED, "planner: %s", err.c_str());
        C.key.clear();  // invalid until the new plan is complete
        C.passes = std::move(passes);
        C.jit.reset();
        if (jit) QV_TRY(jit_prepare(s, C.passes, C.jit));
        C.key.assign(g, g + ng);
        C.K = K;
        C.flags = flags;
    }
    if (jit) return jit_launch(s, *C.jit);
    return s->dt == QV_C64 ? run_plan<float>(s, C.passes, K) : run_plan<double>(s, C.passes, K);
}

qv_status apply_permutation(qv_state *s, const int32_t *perm)
{
    // Transpositions turning the identity into perm; the fused planner turns
    // SWAPs into relabelings inside tiles, the per-gate path into swap passes.
    const int n = s->n;
    std::vector<int> cur(n), want(n);
    for (int p = 0; p < n; ++p) cur[p] = p;
    for (int q = 0; q < n; ++q) want[perm[q]] = q;
    std::vector<qv_gate> swaps;
    for (int p = 0; p < n; ++p) {
        if (cur[p] == want[p]) continue;
        int p2 = p + 1;
        while (cur[p2] != want[p]) ++p2;
        qv_gate g{};
        g.kind = QV_G_SWAP;
        g.target = p;
        g.target2 = p2;
        g.ctrl = -1;
        swaps.push_back(g);
        std::swap(cur[p], cur[p2]);
    }
    if (swaps.empty()) return QV_OK;
    if (fused_supported(s, nullptr)) return apply_fused(s, swaps.data(), swaps.size(), nullptr);
    for (const auto &g : swaps) QV_TRY(launch_swap(s, g.target, g.target2));
    return QV_OK;
}

void plan_cache_release(qv_state *s)
{
    if (s->plan) {
        if (s->plan->dev) cudaFree(s->plan->dev);
        delete s->plan;
        s->plan = nullptr;
    }
}

}  // namespace qv
