// Batched circuits: many states, each with its own circuit (same or uneven
// qubit counts), captured together with the per-state initialisation and the
// batched <H> reduction in one CUDA graph that is replayed by qv_batch_run.
// Members with enough tiles per pass run their own compiled fused passes, on
// side streams of the graph so that their kernels share the GPU; the others
// run as one persistent launch per tile size.
//
// Persistent launches: work items are (circuit, pass, chunk of tiles) in round order: every
// circuit's pass 0, then every circuit's pass 1, ... (larger circuits first
// within a round). A CTA claims items with an atomic counter; before a pass-p
// item of circuit c it waits until all chunks of pass p-1 of c are done
// (per-pass completion counters, release/acquire). An item only waits on
// items claimed before it, so the queue cannot deadlock. Every wait is bounded:
// on timeout the kernel writes QV_ERR_TIMEOUT to a status word and returns.
#include <algorithm>
#include <map>
#include <memory>
#include <vector>

#include "fused_device.cuh"
#include "qv_internal.h"
#include "qv_jit.h"
#include "qv_plan.h"

namespace qv {
namespace {

constexpr uint32_t kChunkTiles = 32;    // tiles per work item
// A circuit whose passes have at least 2^kSoloTileBits tiles (and that shares
// its gate structure with another member, else 2^12 tiles) runs on its own
// compiled passes (coefficients as kernel parameters, the next tile held in
// registers); such circuits are spread over kSideStreams capture streams so
// that their kernels share the GPU.
constexpr int kSoloTileBits = 8;
constexpr int kSideStreams = 16;
constexpr uint32_t kSpinLimit = 1u << 24;  // ~ seconds of __nanosleep(128) before giving up

struct BPass {
    uint64_t blob_off;     // program offset in the blob buffer
    uint64_t ntiles;
    uint32_t nchunks;
    int32_t dep;           // global index of the pass this one waits for (-1: none)
    int32_t circuit;
    uint32_t pad;
};
struct BItem {
    uint32_t gpass;
    uint32_t chunk;
};

template <typename R, int K>
__global__ void __launch_bounds__(1 << (K - kRegBits), 1)
    batch_kernel(R *const *amps, const unsigned char *__restrict__ blobs, const BPass *__restrict__ passes,
                 const BItem *__restrict__ items, uint32_t nitems, unsigned *next, unsigned *done, int *status,
                 uint32_t spin_limit)
{
    constexpr int T = 1 << (K - kRegBits);
    constexpr int NQ = K - kRegBits;
    constexpr int NH = K - kChunkBits;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *tile = smem;
    uint64_t *phys_hi = reinterpret_cast<uint64_t *>(smem + tile_smem<R, K>());
    unsigned char *prog = smem + tile_smem<R, K>() + table_smem<K>();
    __shared__ uint32_t s_item;
    __shared__ int s_abort;
    __shared__ int32_t s_cached;
    const int tid = threadIdx.x;
    if (tid == 0) s_cached = -1;
    Regs<R> x;
    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(next, 1u);
            s_abort = 0;
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= nitems) break;
        const BItem it = items[item];
        const BPass P = passes[it.gpass];
        if (tid == 0 && P.dep >= 0 &&
            !wait_counter(&done[P.dep], passes[P.dep].nchunks, spin_limit, status, int(QV_ERR_TIMEOUT)))
            s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        if (s_cached != int32_t(it.gpass)) {
            const unsigned char *blob = blobs + P.blob_off;
            const DHdr *gh = reinterpret_cast<const DHdr *>(blob);
            const size_t nb = blob_bytes<R>(gh->nstages, gh->nops);
            for (size_t i = size_t(tid) * 16; i < nb; i += size_t(T) * 16)
                *reinterpret_cast<uint4 *>(prog + i) = *reinterpret_cast<const uint4 *>(blob + i);
            __syncthreads();
            const DHdr &h = *reinterpret_cast<const DHdr *>(prog);
            for (int i = tid; i < (1 << NH); i += T) {
                uint64_t v = 0;
                for (int j = 0; j < NH; ++j)
                    if ((i >> j) & 1) v |= uint64_t(1) << h.s_high[j];
                phys_hi[i] = v;
            }
            if (tid == 0) s_cached = int32_t(it.gpass);
            __syncthreads();
        }
        const DHdr &h = *reinterpret_cast<const DHdr *>(prog);
        const DStage *stg = reinterpret_cast<const DStage *>(prog + sizeof(DHdr));
        const DOp<R> *ops = reinterpret_cast<const DOp<R> *>(prog + ops_offset<R>(h.nstages));
        R *amp = amps[P.circuit];
        const uint64_t t0 = uint64_t(it.chunk) * kChunkTiles;
        const uint64_t t1 = min(P.ntiles, t0 + kChunkTiles);
        for (uint64_t t = t0; t < t1; ++t) {
            uint64_t base = 0;
            for (int s = 0; s < h.nseg; ++s)
                base |= ((t >> h.seg_src[s]) & ((uint64_t(1) << h.seg_w[s]) - 1)) << h.seg_dst[s];
            load_tile<NQ, true>(amp, base, stg[0].P, stg[0].Q, tid, phys_hi, x);
            for (int s = 0; s < h.nstages; ++s) {
                if (s > 0) transpose<K, NQ>(tile, stg[s - 1], stg[s], tid, x);
                run_ops<R>(ops + stg[s].op_begin, stg[s].op_end - stg[s].op_begin, tid, base, x);
            }
            if (h.nstages == 1) __syncthreads();  // loads of other warps before a relabelled store
            store_tile<NQ>(amp, base, stg[h.nstages - 1].Po, stg[h.nstages - 1].Qo, tid, phys_hi, x);
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(&done[it.gpass], 1u);
        }
    }
}

// Every state <- |0...0>.
template <typename R> __global__ void batch_init_kernel(R *const *amps, const int *nq, int count)
{
    const int c = blockIdx.y;
    if (c >= count) return;
    R *a = amps[c];
    const uint64_t N = uint64_t(1) << nq[c];
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += uint64_t(gridDim.x) * blockDim.x) {
        a[2 * i] = R(i == 0 ? 1 : 0);
        a[2 * i + 1] = R(0);
    }
}

// ---------------------------------------------------------------- batched <H>
constexpr int kBThreads = 256;
constexpr int kBlocksPerState = 64;
constexpr int kMaxGroupTerms = 64;
struct BGroup {
    uint64_t x;
    int nt;
    int zero_z;   // every z mask is 0: c(i) is the constant (c0re, c0im)
    int has_im;   // some coefficient has an imaginary part
    int tab;      // chunks of Z-term tables (pure-Z group), 0: none
    double c0re, c0im;
    float f0re, f0im;
    uint64_t z[kMaxGroupTerms];
    double cre[kMaxGroupTerms], cim[kMaxGroupTerms];
    float fre[kMaxGroupTerms], fim[kMaxGroupTerms];  // the same in FP32, for complex64 states
};

// part[state * kBlocksPerState + block] = sum over this block's share of the
// state of Re( conj(a_{i^x}) c(i) a_i ), summed over all X-mask groups.
template <typename R>
__global__ void __launch_bounds__(kBThreads) batch_pauli_kernel(R *const *amps, const int *nq, const BGroup *groups,
                                                                int ng, const R *ztab, int tab_words, double *part)
{
    extern __shared__ unsigned char sraw[];
    BGroup *g = reinterpret_cast<BGroup *>(sraw);
    R *tab = reinterpret_cast<R *>(sraw + size_t(ng) * sizeof(BGroup));
    for (int k = threadIdx.x; k < ng * int(sizeof(BGroup) / 8); k += kBThreads)
        reinterpret_cast<uint64_t *>(g)[k] = reinterpret_cast<const uint64_t *>(groups)[k];
    for (int k = threadIdx.x; k < tab_words; k += kBThreads) tab[k] = ztab[k];
    __syncthreads();
    const int c = blockIdx.y;
    const R *a = amps[c];
    const uint64_t N = uint64_t(1) << nq[c];
    const uint64_t per = (N + kBlocksPerState - 1) / kBlocksPerState;
    const uint64_t i0 = uint64_t(blockIdx.x) * per, i1 = min(N, i0 + per);
    CompSum<R> acc;
    // per amplitude a plain sum over the groups, across amplitudes with compensation;
    // four amplitudes a thread at a time (the group fields read once for the four)
    uint64_t i = i0 + threadIdx.x;
    for (; i + 3 * kBThreads < i1; i += 4 * kBThreads) {
        R s4[4];
        pauli_amp_sums<R, 4, 4>(a, i, kBThreads, g, ng, tab, s4);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.add(s4[k]);
    }
    for (; i < i1; i += kBThreads) acc.add(pauli_amp_sum<R>(a, i, g, ng, tab));
    double v = acc.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double ws[kBThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < kBThreads / 32; ++w) s += ws[w];
        part[size_t(c) * kBlocksPerState + blockIdx.x] = s;
    }
}

__global__ void batch_combine_kernel(const double *part, int count, double *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count) return;
    Neumaier a;
    for (int b = 0; b < kBlocksPerState; ++b) a.add(part[size_t(c) * kBlocksPerState + b]);
    out[c] = a.value();
}

// Waits on a counter that nothing increments: runs the timeout path of the
// bounded wait the batch kernel uses, with no fault and no hang.
__global__ void wait_selftest_kernel(const unsigned *ctr, uint32_t limit, int *status)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) wait_counter(ctr, 1u, limit, status, int(QV_ERR_TIMEOUT));
}

}  // namespace

qv_status wait_selftest(qv_state *s, uint32_t limit)
{
    if (limit > kSpinLimit) return fail(QV_ERR_ARG, "limit %u above %u", limit, kSpinLimit);
    int *status = nullptr;
    QV_TRY(status_word(s, &status));
    QV_TRY(ensure_scratch(s, 256));
    unsigned *ctr = static_cast<unsigned *>(s->scratch.ptr);
    QV_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned), s->stream));
    QV_LAUNCH(s, QV_K_BATCH, wait_selftest_kernel<<<1, 32, 0, s->stream>>>(ctr, limit, status));
    return sync_and_check(s);
}

// ---------------------------------------------------------------- host side
struct BatchGroup {
    int K = 0;
    std::vector<int> circuits;
    void *blobs = nullptr, *passes = nullptr, *items = nullptr, *done = nullptr;
    uint32_t nitems = 0, npasses = 0;
    size_t smem = 0;
    unsigned grid = 0;
    // compiled path: every circuit of the group has the same plan structure
    bool jit = false;
    JitBatch jb;
    void *jamps = nullptr, *jcoefs = nullptr;
    uint64_t ntiles = 0;
    uint32_t nchunks = 0;

};

}  // namespace qv

struct qv_batch {
    std::vector<qv_state *> states;
    qv_dtype dt = QV_C64;
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    std::vector<qv::BatchGroup> groups;
    void *amps = nullptr, *nq = nullptr;     // device arrays of state pointers and qubit counts
    unsigned *next = nullptr;                 // one work counter per group
    int *status = nullptr;                    // device status word
    void *hgroups = nullptr;                  // Pauli groups (device)
    int nhgroups = 0;
    void *ztab = nullptr;                     // Z-term tables of the pure-Z group (device), or none
    int ztab_words = 0;
    double *part = nullptr, *energies = nullptr;
    double *host = nullptr;                   // pinned: energies then status
    size_t nt = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> owned;
    // circuits that fill the GPU alone: their own compiled fused passes, in the same graph
    struct Solo {
        int circuit = 0, K = 0;
        std::shared_ptr<qv::JitProgram> prog;
    };
    std::vector<Solo> solo;
    std::vector<cudaStream_t> side;  // capture streams of the solo circuits
    std::vector<cudaEvent_t> side_ev;  // fork event, then one join event per side stream
};

namespace qv {
namespace {

template <typename R, int K> qv_status set_attr_once()
{
    return allow_smem(reinterpret_cast<const void *>(batch_kernel<R, K>), 220 * 1024);
}

template <typename R, int K> qv_status occupancy(size_t smem, int *per_sm)
{
    QV_TRY((set_attr_once<R, K>()));
    QV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<R, K>, 1 << (K - kRegBits), smem));
    return QV_OK;
}

template <typename R> qv_status group_occupancy(int K, size_t smem, int *per_sm)
{
    switch (K) {
    case 10: return occupancy<R, 10>(smem, per_sm);
    case 11: return occupancy<R, 11>(smem, per_sm);
    case 12: return occupancy<R, 12>(smem, per_sm);
    default: return fail(QV_ERR_ARG, "tile bits %d unsupported", K);
    }
}

// Enqueues the group's persistent launch; false when the driver refused the
// compiled launch (the runtime's error state does not see driver API calls).
template <typename R>
bool launch_group(qv_batch *b, const BatchGroup &g, unsigned *next)
{
    if (g.jit) {
        uint32_t nitems = g.nitems, nchunks = g.nchunks, spin = kSpinLimit;
        uint64_t ntiles = g.ntiles;
        void *amps = g.jamps, *coefs = g.jcoefs, *items = g.items, *done = g.done, *st = b->status;
        void *nx = next;
        void *args[] = {&amps, &coefs, &items, &nitems, &nx, &done, &st, &ntiles, &nchunks, &spin};
        return jit_launch_batch(g.jb, b->stream, g.grid, args) == QV_OK;
    }
    R *const *amps = static_cast<R *const *>(b->amps);
    auto args = [&](auto kern) {
        kern<<<g.grid, 1 << (g.K - kRegBits), g.smem, b->stream>>>(
            amps, static_cast<const unsigned char *>(g.blobs), static_cast<const BPass *>(g.passes),
            static_cast<const BItem *>(g.items), g.nitems, next, static_cast<unsigned *>(g.done), b->status,
            kSpinLimit);
    };
    if (g.K == 10) args(batch_kernel<R, 10>);
    else if (g.K == 11) args(batch_kernel<R, 11>);
    else args(batch_kernel<R, 12>);
    return true;
}

qv_status dmalloc(qv_batch *b, void **p, size_t bytes)
{
    QV_CUDA(cudaMalloc(p, std::max<size_t>(bytes, 16)));
    b->owned.push_back(*p);
    return QV_OK;
}

template <typename R>
qv_status build(qv_batch *b, const qv_batch_item *items, size_t count, const qv_pauli_term *H, size_t nt,
                const qv_plan_opts *opts)
{
    const bool fuse = !(opts && (opts->flags & QV_PLAN_NO_FUSION));
    const bool jit_ok = sizeof(R) == 4 && jit_available(nullptr) && !(opts && (opts->flags & QV_PLAN_INTERPRET));
    const bool fixed_k = opts && opts->tile_bits;
    // ---- circuits whose every pass fills the GPU (at least 2^12 tiles) run on
    // their own compiled passes, as qv_apply_circuit would run them; the
    // persistent queue takes the rest
    std::vector<char> solo(count, 0);
    auto solo_k = [&](int n) { return fixed_k ? opts->tile_bits : tuned_tile_bits(n, b->dt, false); };
    if (jit_ok) {
        // members with the same gate structure share their compiled passes (the
        // kernel cache is keyed by source), so they go to their own passes from
        // 2^kSoloTileBits tiles on; a structure of its own only from 2^12 tiles,
        // where compiling its passes pays off
        std::map<std::vector<int32_t>, int> shape_count;
        std::vector<std::vector<int32_t>> shape(count);
        for (size_t c = 0; c < count; ++c) {
            shape[c].push_back(items[c].state->n);
            for (size_t k = 0; k < items[c].ngates; ++k) {
                const qv_gate &x = items[c].gates[k];
                shape[c].insert(shape[c].end(), {int32_t(x.kind), x.target, x.target2, x.ctrl});
            }
            ++shape_count[shape[c]];
        }
        for (size_t c = 0; c < count; ++c) {
            const int tiles = items[c].state->n - solo_k(items[c].state->n);
            solo[c] = tiles >= 12 || (tiles >= kSoloTileBits && shape_count[shape[c]] > 1);
        }
    }
    // qubit counts whose queued circuits all share one gate structure run in the
    // compiled persistent kernel, the others in the interpreting one
    std::map<int, bool> uniform;
    {
        std::map<int, size_t> first;
        for (size_t c = 0; c < count; ++c) {
            if (solo[c]) continue;
            const int n = items[c].state->n;
            auto it = first.find(n);
            if (it == first.end()) {
                first[n] = c;
                uniform[n] = jit_ok;
                continue;
            }
            const qv_batch_item &a = items[it->second], &x = items[c];
            bool same = a.ngates == x.ngates;
            for (size_t k = 0; same && k < x.ngates; ++k)
                same = a.gates[k].kind == x.gates[k].kind && a.gates[k].target == x.gates[k].target &&
                       a.gates[k].target2 == x.gates[k].target2 && a.gates[k].ctrl == x.gates[k].ctrl;
            uniform[n] = uniform[n] && same;
        }
    }
    auto engine_interp = [&](size_t c) { return !solo[c] && !uniform[items[c].state->n]; };
    // ---- with QV_PLAN_AUTOTUNE, time the tile sizes once per qubit count not tuned yet,
    // with the engine that will run it (on the first state of that size, with its
    // circuit; the run resets the states)
    if (opts && (opts->flags & QV_PLAN_AUTOTUNE) && !fixed_k) {
        std::map<int, size_t> first;
        for (size_t c = 0; c < count; ++c) first.emplace(items[c].state->n, c);
        for (auto &kv : first) {
            const bool interp = engine_interp(kv.second) || !jit_ok;
            if (kv.first < plan::kMinK || tile_bits_tuned(kv.first, b->dt, interp)) continue;
            qv_plan_opts o{};
            o.flags = interp ? QV_PLAN_INTERPRET : 0;
            QV_TRY(autotune(items[kv.second].state, items[kv.second].gates, items[kv.second].ngates, &o, nullptr,
                            nullptr, false));
            QV_CUDA(cudaStreamSynchronize(items[kv.second].state->stream));
        }
    }
    // ---- plan every circuit, group by tile size
    std::map<int, std::vector<int>> by_k;
    std::vector<std::vector<plan::Pass>> plans(count);
    for (size_t c = 0; c < count; ++c) {
        const int n = items[c].state->n;
        if (solo[c]) {
            const int K = std::min(n, solo_k(n));
            std::vector<plan::PGate> pg;
            QV_TRY(to_pgates(items[c].gates, items[c].ngates, pg));
            plan::PlanStats st;
            std::string err;
            if (!plan::make_plan(n, K, true, fuse, fuse, pg, plans[c], st, err))
                return fail(QV_ERR_UNSUPPORTED, "batch item %zu: planner: %s", c, err.c_str());
            qv_batch::Solo so;
            so.circuit = int(c);
            so.K = K;
            QV_TRY(jit_prepare(items[c].state, plans[c], so.prog));
            b->solo.push_back(std::move(so));
            continue;
        }
        // the tile size the autotuner chose for the engine that will run it;
        // untuned, 2^12 (the batch kernels hold no next tile in registers: 256 x
        // 20 qubits took 47 ms at 2^12, 51 ms at 2^11)
        const bool interp = engine_interp(c) || !jit_ok;
        int K = fixed_k ? opts->tile_bits
                : tile_bits_tuned(n, b->dt, interp) ? tuned_tile_bits(n, b->dt, interp) : std::min(n, plan::kMaxK);
        if (K > n) K = n;
        if (K < plan::kMinK || K > plan::kMaxK)
            return fail(QV_ERR_UNSUPPORTED, "batch item %zu: %d qubits is below the smallest tile (%d)", c, n,
                        plan::kMinK);
        std::vector<plan::PGate> pg;
        QV_TRY(to_pgates(items[c].gates, items[c].ngates, pg));
        plan::PlanStats st;
        std::string err;
        if (!plan::make_plan(n, K, b->dt == QV_C64, fuse, false, pg, plans[c], st, err))
            return fail(QV_ERR_UNSUPPORTED, "batch item %zu: planner: %s", c, err.c_str());
        by_k[K].push_back(int(c));
    }
    // ---- device arrays of amplitude pointers and qubit counts
    std::vector<void *> amps(count);
    std::vector<int> nq(count);
    for (size_t c = 0; c < count; ++c) {
        amps[c] = items[c].state->amp;
        nq[c] = items[c].state->n;
    }
    QV_TRY(dmalloc(b, &b->amps, count * sizeof(void *)));
    QV_TRY(dmalloc(b, &b->nq, count * sizeof(int)));
    QV_CUDA(cudaMemcpy(b->amps, amps.data(), count * sizeof(void *), cudaMemcpyHostToDevice));
    QV_CUDA(cudaMemcpy(b->nq, nq.data(), count * sizeof(int), cudaMemcpyHostToDevice));
    void *nextv = nullptr;
    QV_TRY(dmalloc(b, &nextv, by_k.size() * sizeof(unsigned)));
    b->next = static_cast<unsigned *>(nextv);
    void *st = nullptr;
    QV_TRY(dmalloc(b, &st, sizeof(int)));
    b->status = static_cast<int *>(st);
    // ---- one persistent launch per tile size
    for (auto &kv : by_k) {
        BatchGroup g;
        g.K = kv.first;
        g.circuits = kv.second;
        bool same = jit_ok;
        for (int c : g.circuits)
            same = same && nq[c] == nq[g.circuits[0]] && jit_same_structure(plans[c], plans[g.circuits[0]]);
        if (same) {  // compiled persistent kernel over (circuit, pass, chunk) items
            g.jit = true;
            std::vector<std::vector<plan::Pass> *> pl;
            std::vector<void *> ga;
            for (int c : g.circuits) {
                pl.push_back(&plans[c]);
                ga.push_back(amps[c]);
            }
            QV_TRY(jit_prepare_batch(items[g.circuits[0]].state, pl, int(kChunkTiles), g.jb));
            const uint32_t np = uint32_t(g.jb.npasses);
            g.ntiles = uint64_t(1) << (nq[g.circuits[0]] - g.K);
            g.nchunks = uint32_t((g.ntiles + kChunkTiles - 1) / kChunkTiles);
            std::vector<uint2> it;
            for (uint32_t r = 0; r < np; ++r)
                for (uint32_t cl = 0; cl < uint32_t(g.circuits.size()); ++cl)
                    for (uint32_t k = 0; k < g.nchunks; ++k) it.push_back(make_uint2(cl * np + r, k));
            g.nitems = uint32_t(it.size());
            g.npasses = uint32_t(g.circuits.size()) * np;
            QV_TRY(dmalloc(b, &g.jamps, ga.size() * sizeof(void *)));
            QV_TRY(dmalloc(b, &g.jcoefs, g.jb.coefs.size() * sizeof(uint64_t)));
            QV_TRY(dmalloc(b, &g.items, it.size() * sizeof(uint2)));
            QV_TRY(dmalloc(b, &g.done, g.npasses * sizeof(unsigned)));
            QV_CUDA(cudaMemcpy(g.jamps, ga.data(), ga.size() * sizeof(void *), cudaMemcpyHostToDevice));
            QV_CUDA(cudaMemcpy(g.jcoefs, g.jb.coefs.data(), g.jb.coefs.size() * sizeof(uint64_t),
                               cudaMemcpyHostToDevice));
            QV_CUDA(cudaMemcpy(g.items, it.data(), it.size() * sizeof(uint2), cudaMemcpyHostToDevice));
            g.jb.coefs.clear();
            g.jb.coefs.shrink_to_fit();
            g.grid = unsigned(g.jb.per_sm) * b->num_sms;
            b->groups.push_back(g);
            continue;
        }
        // larger circuits first within a round
        std::stable_sort(g.circuits.begin(), g.circuits.end(),
                         [&](int a, int c) { return nq[a] > nq[c]; });
        std::vector<unsigned char> blob;
        std::vector<BPass> bp;
        std::vector<std::vector<int>> gidx(count);
        size_t max_blob = 0;
        for (int c : g.circuits) {
            int prev = -1;
            for (const plan::Pass &p : plans[c]) {
                blob.resize((blob.size() + 255) & ~size_t(255), 0);
                BPass q{};
                q.blob_off = blob.size();
                serialize<R>(p, blob);
                max_blob = std::max(max_blob, blob.size() - q.blob_off);
                q.ntiles = uint64_t(1) << (nq[c] - p.k);
                q.nchunks = uint32_t((q.ntiles + kChunkTiles - 1) / kChunkTiles);
                q.dep = prev;
                q.circuit = c;
                prev = int(bp.size());
                gidx[c].push_back(prev);
                bp.push_back(q);
            }
        }
        std::vector<BItem> it;
        for (size_t r = 0;; ++r) {
            bool any = false;
            for (int c : g.circuits) {
                if (r >= gidx[c].size()) continue;
                any = true;
                const uint32_t gp = uint32_t(gidx[c][r]);
                for (uint32_t k = 0; k < bp[gp].nchunks; ++k) it.push_back({gp, k});
            }
            if (!any) break;
        }
        g.nitems = uint32_t(it.size());
        g.npasses = uint32_t(bp.size());
        QV_TRY(dmalloc(b, &g.blobs, blob.size()));
        QV_TRY(dmalloc(b, &g.passes, bp.size() * sizeof(BPass)));
        QV_TRY(dmalloc(b, &g.items, it.size() * sizeof(BItem)));
        QV_TRY(dmalloc(b, &g.done, bp.size() * sizeof(unsigned)));
        if (!blob.empty()) QV_CUDA(cudaMemcpy(g.blobs, blob.data(), blob.size(), cudaMemcpyHostToDevice));
        if (!bp.empty()) QV_CUDA(cudaMemcpy(g.passes, bp.data(), bp.size() * sizeof(BPass), cudaMemcpyHostToDevice));
        if (!it.empty()) QV_CUDA(cudaMemcpy(g.items, it.data(), it.size() * sizeof(BItem), cudaMemcpyHostToDevice));
        g.smem = tile_smem<R, 12>() / (size_t(1) << (12 - g.K)) + (sizeof(uint64_t) << (g.K - kChunkBits)) + max_blob;
        int per_sm = 0;
        QV_TRY(group_occupancy<R>(g.K, g.smem, &per_sm));
        if (per_sm < 1) return fail(QV_ERR_UNSUPPORTED, "batch pass programs too large for shared memory");
        g.grid = unsigned(per_sm) * b->num_sms;
        b->groups.push_back(g);
    }
    // ---- Hamiltonian groups for the batched <H>
    b->nt = nt;
    if (nt) {
        std::vector<BGroup> hg;
        for (size_t k = 0; k < nt; ++k) {
            const uint64_t x = H[k].xmask, z = H[k].zmask;
            const int ny = __builtin_popcountll(x & z);
            static const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, 1, 0, -1};
            BGroup *g = nullptr;
            for (auto &gg : hg)
                if (gg.x == x && gg.nt < kMaxGroupTerms) { g = &gg; break; }
            if (!g) {
                hg.emplace_back();
                g = &hg.back();
                std::memset(g, 0, sizeof *g);
                g->x = x;
            }
            g->z[g->nt] = z;
            g->cre[g->nt] = H[k].coeff * pr[ny & 3];
            g->cim[g->nt] = H[k].coeff * pi[ny & 3];
            g->fre[g->nt] = float(g->cre[g->nt]);
            g->fim[g->nt] = float(g->cim[g->nt]);
            g->nt++;
            g->c0re += g->cre[g->nt - 1];
            g->c0im += g->cim[g->nt - 1];
            g->f0re = float(g->c0re);
            g->f0im = float(g->c0im);
        }
        for (BGroup &gg : hg) {
            gg.zero_z = 1;
            gg.has_im = 0;
            for (int k = 0; k < gg.nt; ++k) {
                gg.zero_z &= gg.z[k] == 0;
                gg.has_im |= gg.cim[k] != 0.0;
            }
        }
        // the pure-Z group's terms that lie inside one 8-bit chunk of the index go into tables
        int maxn = 0;
        for (int v : nq) maxn = std::max(maxn, v);
        // (only when the tables fit in shared memory beside the groups)
        const std::vector<R> htab = hg.size() * sizeof(BGroup) + kZTabWords * sizeof(R) <= 200 * 1024
                                        ? ztab_for_group<R>(maxn, hg)
                                        : std::vector<R>();
        for (BGroup &gg : hg)
            for (int k = 0; k < gg.nt; ++k) {
                gg.fre[k] = float(gg.cre[k]);
                gg.fim[k] = float(gg.cim[k]);
            }
        if (hg.size() * sizeof(BGroup) + htab.size() * sizeof(R) > 200 * 1024)
            return fail(QV_ERR_UNSUPPORTED, "Hamiltonian too large");
        if (!htab.empty()) {
            QV_TRY(dmalloc(b, &b->ztab, htab.size() * sizeof(R)));
            QV_CUDA(cudaMemcpy(b->ztab, htab.data(), htab.size() * sizeof(R), cudaMemcpyHostToDevice));
            b->ztab_words = int(htab.size());
        }
        b->nhgroups = int(hg.size());
        QV_TRY(dmalloc(b, &b->hgroups, hg.size() * sizeof(BGroup)));
        QV_CUDA(cudaMemcpy(b->hgroups, hg.data(), hg.size() * sizeof(BGroup), cudaMemcpyHostToDevice));
        void *pp = nullptr, *ee = nullptr;
        QV_TRY(dmalloc(b, &pp, count * kBlocksPerState * sizeof(double)));
        QV_TRY(dmalloc(b, &ee, count * sizeof(double)));
        b->part = static_cast<double *>(pp);
        b->energies = static_cast<double *>(ee);
        QV_TRY(allow_smem(reinterpret_cast<const void *>(batch_pauli_kernel<R>), 200 * 1024));
    }
    QV_CUDA(cudaMallocHost(reinterpret_cast<void **>(&b->host), (count + 2) * sizeof(double)));
    // solo circuits, largest first, round-robin over the side streams
    std::stable_sort(b->solo.begin(), b->solo.end(), [&](const qv_batch::Solo &x, const qv_batch::Solo &y) {
        return nq[size_t(x.circuit)] > nq[size_t(y.circuit)];
    });
    const size_t nside = std::min<size_t>(b->solo.size(), kSideStreams);
    for (size_t j = 0; j < nside; ++j) {
        cudaStream_t st = nullptr;
        QV_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b->side.push_back(st);
    }
    for (size_t j = 0; j < (nside ? nside + 1 : 0); ++j) {
        cudaEvent_t ev = nullptr;
        QV_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->side_ev.push_back(ev);
    }
    // ---- capture the whole run in one graph
    QV_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    {
        ce = cudaMemsetAsync(b->next, 0, b->groups.size() * sizeof(unsigned), b->stream);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(b->status, 0, sizeof(int), b->stream);
        for (auto &g : b->groups)
            if (ce == cudaSuccess) ce = cudaMemsetAsync(g.done, 0, g.npasses * sizeof(unsigned), b->stream);
        if (ce == cudaSuccess) {
            int maxn = 0;
            for (int v : nq) maxn = std::max(maxn, v);
            const unsigned gx = unsigned(std::min<uint64_t>(uint64_t(b->num_sms) * 4, ((uint64_t(1) << maxn) + 255) / 256));
            batch_init_kernel<R><<<dim3(gx, unsigned(count)), 256, 0, b->stream>>>(static_cast<R *const *>(b->amps),
                                                                                   static_cast<const int *>(b->nq),
                                                                                   int(count));
            ce = cudaGetLastError();
        }
        // fork: the side streams start after the initialisation
        if (ce == cudaSuccess && !b->side.empty()) {
            ce = cudaEventRecord(b->side_ev[0], b->stream);
            for (size_t j = 0; j < b->side.size() && ce == cudaSuccess; ++j)
                ce = cudaStreamWaitEvent(b->side[j], b->side_ev[0], 0);
        }
        for (size_t gi = 0; gi < b->groups.size() && ce == cudaSuccess; ++gi) {
            const bool ok = launch_group<R>(b, b->groups[gi], b->next + gi);
            ce = ok ? cudaGetLastError() : cudaErrorLaunchFailure;
        }
        for (size_t k = 0; k < b->solo.size(); ++k) {
            if (ce != cudaSuccess) break;
            const auto &so = b->solo[k];
            const qv_status r = jit_launch(items[so.circuit].state, *so.prog, b->side[k % b->side.size()]);
            ce = r == QV_OK ? cudaGetLastError() : cudaErrorLaunchFailure;
        }
        // join: the reduction and the copies wait for every side stream
        for (size_t j = 0; j < b->side.size() && ce == cudaSuccess; ++j) {
            ce = cudaEventRecord(b->side_ev[j + 1], b->side[j]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->stream, b->side_ev[j + 1], 0);
        }
        if (nt && ce == cudaSuccess) {
            batch_pauli_kernel<R><<<dim3(kBlocksPerState, unsigned(count)), kBThreads,
                                    b->nhgroups * sizeof(BGroup) + b->ztab_words * sizeof(R), b->stream>>>(
                static_cast<R *const *>(b->amps), static_cast<const int *>(b->nq),
                static_cast<const BGroup *>(b->hgroups), b->nhgroups, static_cast<const R *>(b->ztab), b->ztab_words,
                b->part);
            ce = cudaGetLastError();
            if (ce == cudaSuccess) {
                batch_combine_kernel<<<unsigned((count + 127) / 128), 128, 0, b->stream>>>(b->part, int(count),
                                                                                            b->energies);
                ce = cudaGetLastError();
            }
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(b->host, b->energies, count * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        }
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(b->host + count, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    }
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &b->graph);
    QV_CUDA(ce);
    QV_CUDA(ee);
    QV_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return QV_OK;
}

}  // namespace

void batch_release(qv_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void *p : b->owned) cudaFree(p);
    for (cudaEvent_t ev : b->side_ev) cudaEventDestroy(ev);
    for (cudaStream_t st : b->side) cudaStreamDestroy(st);
    if (b->host) cudaFreeHost(b->host);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

qv_status batch_create(const qv_batch_item *items, size_t count, const qv_pauli_term *H, size_t nt,
                       const qv_plan_opts *opts, qv_batch **out)
{
    qv_batch *b = new qv_batch;
    b->dt = items[0].state->dt;
    b->device = items[0].state->device;
    b->num_sms = items[0].state->num_sms;
    for (size_t c = 0; c < count; ++c) b->states.push_back(items[c].state);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "cudaStreamCreate");
    }
    for (size_t c = 0; c < count; ++c) {
        e = cudaStreamSynchronize(items[c].state->stream);
        if (e != cudaSuccess) {
            batch_release(b);
            return cuda_fail(e, "cudaStreamSynchronize");
        }
    }
    const qv_status st = b->dt == QV_C64 ? build<float>(b, items, count, H, nt, opts)
                                         : build<double>(b, items, count, H, nt, opts);
    if (st != QV_OK) {
        (void)cudaGetLastError();
        batch_release(b);
        return st;
    }
    *out = b;
    return QV_OK;
}

size_t batch_info(const qv_batch *b, int32_t *out, size_t cap)
{
    for (size_t g = 0; g < b->groups.size() && g < cap; ++g) {
        const BatchGroup &G = b->groups[g];
        int32_t *o = out + 6 * g;
        o[0] = G.K;
        o[1] = int32_t(G.circuits.size());
        o[2] = b->states[size_t(G.circuits.front())]->n;
        o[3] = G.jit ? 1 : 0;
        o[4] = int32_t(G.jit ? G.circuits.size() : 0);  // one round of every circuit at a time
        o[5] = int32_t(kChunkTiles);
    }
    size_t g = b->groups.size();
    for (const auto &so : b->solo) {
        if (g < cap) {
            int32_t *o = out + 6 * g;
            o[0] = so.K;
            o[1] = 1;
            o[2] = b->states[size_t(so.circuit)]->n;
            o[3] = 2;  // its own compiled passes
            o[4] = 0;
            o[5] = 0;
        }
        ++g;
    }
    return g;
}

qv_status batch_run(qv_batch *b, double *expvals)
{
    for (qv_state *s : b->states) QV_CUDA(cudaStreamSynchronize(s->stream));
    QV_CUDA(cudaGraphLaunch(b->exec, b->stream));
    QV_CUDA(cudaStreamSynchronize(b->stream));
    int status = 0;
    std::memcpy(&status, b->host + b->states.size(), sizeof(int));
    if (status != 0) return fail(qv_status(status), "batched launch: a dependency wait timed out");
    if (expvals && b->nt)
        for (size_t c = 0; c < b->states.size(); ++c) expvals[c] = b->host[c];
    return QV_OK;
}

}  // namespace qv
