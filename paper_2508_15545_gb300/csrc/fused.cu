// Fused tiled passes: the on-chip form of the paper's block storage and
// sliding-window cache (Sec. III-B/C, Eq. 6-8) with the single-traversal idea
// of Sec. III-E. Each pass loads every 2^K-amplitude tile once (16-byte vector
// loads of contiguous 2^5-amplitude runs), applies all gates the planner gave
// the pass in registers -- changing which tile qubits are register-local with
// swizzled shared-memory transposes -- and stores the tile once.
#include <algorithm>
#include <mutex>
#include <vector>

#include "planner.h"
#include "qv_device.cuh"
#include "qv_internal.h"
#include "qv_plan.h"

namespace qv {

struct PlanCache {
    void *dev = nullptr;
    size_t bytes = 0;
};

namespace {

using plan::kChunkBits;
using plan::kRegBits;
constexpr int kNR = 1 << kRegBits;  // amplitudes per thread

// Device form of a pass program: header, stages, ops (one blob per pass).
struct DHdr {
    int32_t k, nstages, nops, nseg;
    int32_t s_high[8];
    int32_t seg_src[8], seg_w[8], seg_dst[8];
};
struct DStage {
    int8_t P[4], Q[8], Po[4], Qo[8];
    int32_t op_begin, op_end;
};
template <typename R> struct DOp {
    int8_t type, treg, creg, d0one;
    uint32_t cthr, tthr, pad;
    uint64_t cext, text;
    R m[8];
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
template <typename R> __host__ __device__ inline size_t ops_offset(int nstages)
{
    return align16(sizeof(DHdr) + sizeof(DStage) * size_t(nstages));
}
template <typename R> __host__ __device__ inline size_t blob_bytes(int nstages, int nops)
{
    return align16(ops_offset<R>(nstages) + sizeof(DOp<R>) * size_t(nops));
}

template <typename R> struct V2T;
template <> struct V2T<float> { using T = float2; };
template <> struct V2T<double> { using T = double2; };

// Bank-conflict-free slot of tile index l: fold higher index bits onto the
// bits that select a bank slot (8-byte: 16 slots per 128 bytes, 16-byte: 8).
template <typename R> __device__ __forceinline__ uint32_t swz(uint32_t l);
template <> __device__ __forceinline__ uint32_t swz<float>(uint32_t l) { return l ^ (((l >> 4) ^ (l >> 8)) & 15u); }
template <> __device__ __forceinline__ uint32_t swz<double>(uint32_t l)
{
    return l ^ (((l >> 3) ^ (l >> 6) ^ (l >> 9)) & 7u);
}

template <int NQ> __device__ __forceinline__ uint32_t thr_part(const int8_t *Q, int tid)
{
    uint32_t l = 0;
#pragma unroll
    for (int b = 0; b < NQ; ++b)
        if ((tid >> b) & 1) l |= 1u << Q[b];
    return l;
}

struct RegMasks {
    uint32_t pm[kRegBits];
    __device__ __forceinline__ void set(const int8_t *P)
    {
#pragma unroll
        for (int j = 0; j < kRegBits; ++j) pm[j] = 1u << P[j];
    }
    __device__ __forceinline__ uint32_t part(int m) const
    {
        uint32_t l = 0;
#pragma unroll
        for (int j = 0; j < kRegBits; ++j)
            if ((m >> j) & 1) l |= pm[j];
        return l;
    }
};

__device__ __forceinline__ uint64_t phys(uint32_t l, const uint64_t *phys_hi)
{
    return (l & ((1u << kChunkBits) - 1)) | phys_hi[l >> kChunkBits];
}

// ---- tile load / store in the canonical layouts
template <int NQ>
__device__ __forceinline__ void load_tile(const float *amp, uint64_t base, const DStage &st, int tid,
                                          const uint64_t *phys_hi, float (&re)[kNR], float (&im)[kNR])
{
    RegMasks rm;
    rm.set(st.P);
    const uint32_t tp = thr_part<NQ>(st.Q, tid);
    float4 v[kNR / 2];
#pragma unroll
    for (int h = 0; h < kNR / 2; ++h) {
        const uint64_t g = base | phys(tp | rm.part(2 * h), phys_hi);
        v[h] = *reinterpret_cast<const float4 *>(amp + 2 * g);
    }
#pragma unroll
    for (int h = 0; h < kNR / 2; ++h) {
        re[2 * h] = v[h].x; im[2 * h] = v[h].y; re[2 * h + 1] = v[h].z; im[2 * h + 1] = v[h].w;
    }
}

template <int NQ>
__device__ __forceinline__ void store_tile(float *amp, uint64_t base, const DStage &st, int tid,
                                           const uint64_t *phys_hi, const float (&re)[kNR], const float (&im)[kNR])
{
    RegMasks rm;
    rm.set(st.Po);
    const uint32_t tp = thr_part<NQ>(st.Qo, tid);
#pragma unroll
    for (int h = 0; h < kNR / 2; ++h) {
        const uint64_t g = base | phys(tp | rm.part(2 * h), phys_hi);
        *reinterpret_cast<float4 *>(amp + 2 * g) = make_float4(re[2 * h], im[2 * h], re[2 * h + 1], im[2 * h + 1]);
    }
}

template <int NQ>
__device__ __forceinline__ void load_tile(const double *amp, uint64_t base, const DStage &st, int tid,
                                          const uint64_t *phys_hi, double (&re)[kNR], double (&im)[kNR])
{
    RegMasks rm;
    rm.set(st.P);
    const uint32_t tp = thr_part<NQ>(st.Q, tid);
    double2 v[kNR];
#pragma unroll
    for (int m = 0; m < kNR; ++m) {
        const uint64_t g = base | phys(tp | rm.part(m), phys_hi);
        v[m] = reinterpret_cast<const double2 *>(amp)[g];
    }
#pragma unroll
    for (int m = 0; m < kNR; ++m) {
        re[m] = v[m].x;
        im[m] = v[m].y;
    }
}

template <int NQ>
__device__ __forceinline__ void store_tile(double *amp, uint64_t base, const DStage &st, int tid,
                                           const uint64_t *phys_hi, const double (&re)[kNR], const double (&im)[kNR])
{
    RegMasks rm;
    rm.set(st.Po);
    const uint32_t tp = thr_part<NQ>(st.Qo, tid);
#pragma unroll
    for (int m = 0; m < kNR; ++m) {
        const uint64_t g = base | phys(tp | rm.part(m), phys_hi);
        reinterpret_cast<double2 *>(amp)[g] = make_double2(re[m], im[m]);
    }
}

// ---- layout change through shared memory
template <typename R, int NQ>
__device__ __forceinline__ void transpose(typename V2T<R>::T *tile, const DStage &from, const DStage &to, int tid,
                                          R (&re)[kNR], R (&im)[kNR])
{
    using V2 = typename V2T<R>::T;
    RegMasks ro, ri;
    ro.set(from.Po);
    ri.set(to.P);
    const uint32_t to_ = thr_part<NQ>(from.Qo, tid), ti = thr_part<NQ>(to.Q, tid);
#pragma unroll
    for (int m = 0; m < kNR; ++m) {
        V2 v;
        v.x = re[m];
        v.y = im[m];
        tile[swz<R>(to_ | ro.part(m))] = v;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kNR; ++m) {
        const V2 v = tile[swz<R>(ti | ri.part(m))];
        re[m] = v.x;
        im[m] = v.y;
    }
    __syncthreads();
}

// ---- on-chip gate application
template <typename R, int J>
__device__ __forceinline__ void op_gen(const DOp<R> &op, int creg, R (&re)[kNR], R (&im)[kNR])
{
    Mat2<R> U;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        U.r[e] = op.m[2 * e];
        U.i[e] = op.m[2 * e + 1];
    }
#pragma unroll
    for (int m = 0; m < kNR; ++m) {
        if (m & (1 << J)) continue;
        if (creg >= 0 && !((m >> creg) & 1)) continue;
        apply2(U, re[m], im[m], re[m | (1 << J)], im[m | (1 << J)]);
    }
}

template <typename R, int J> __device__ __forceinline__ void op_x(int creg, R (&re)[kNR], R (&im)[kNR])
{
#pragma unroll
    for (int m = 0; m < kNR; ++m) {
        if (m & (1 << J)) continue;
        const bool go = creg < 0 || ((m >> creg) & 1);
        const int m1 = m | (1 << J);
        const R a = re[m], b = re[m1], c = im[m], d = im[m1];
        re[m] = go ? b : a;
        re[m1] = go ? a : b;
        im[m] = go ? d : c;
        im[m1] = go ? c : d;
    }
}

template <typename R, int J>
__device__ __forceinline__ void op_diag(const DOp<R> &op, int creg, R (&re)[kNR], R (&im)[kNR])
{
    const R d0r = op.m[0], d0i = op.m[1], d1r = op.m[2], d1i = op.m[3];
    const bool skip0 = op.d0one;
#pragma unroll
    for (int m = 0; m < kNR; ++m) {
        if (creg >= 0 && !((m >> creg) & 1)) continue;
        if ((m >> J) & 1) cmul(d1r, d1i, re[m], im[m]);
        else if (!skip0) cmul(d0r, d0i, re[m], im[m]);
    }
}

template <typename R>
__device__ __forceinline__ void run_ops(const DOp<R> *ops, int nops, int tid, uint64_t base, R (&re)[kNR],
                                        R (&im)[kNR])
{
    for (int o = 0; o < nops; ++o) {
        const DOp<R> &op = ops[o];
        if ((uint32_t(tid) & op.cthr) != op.cthr || (base & op.cext) != op.cext) continue;
        const int creg = op.creg;
        if (op.type == plan::OP_DIAG && op.treg < 0) {
            const bool sel = (uint32_t(tid) & op.tthr) != 0 || (base & op.text) != 0;
            if (!sel && op.d0one) continue;
            const R dr = sel ? op.m[2] : op.m[0], di = sel ? op.m[3] : op.m[1];
#pragma unroll
            for (int m = 0; m < kNR; ++m)
                if (creg < 0 || ((m >> creg) & 1)) cmul(dr, di, re[m], im[m]);
            continue;
        }
        switch (op.type * 4 + op.treg) {
        case 0: op_gen<R, 0>(op, creg, re, im); break;
        case 1: op_gen<R, 1>(op, creg, re, im); break;
        case 2: op_gen<R, 2>(op, creg, re, im); break;
        case 3: op_gen<R, 3>(op, creg, re, im); break;
        case 4: op_x<R, 0>(creg, re, im); break;
        case 5: op_x<R, 1>(creg, re, im); break;
        case 6: op_x<R, 2>(creg, re, im); break;
        case 7: op_x<R, 3>(creg, re, im); break;
        case 8: op_diag<R, 0>(op, creg, re, im); break;
        case 9: op_diag<R, 1>(op, creg, re, im); break;
        case 10: op_diag<R, 2>(op, creg, re, im); break;
        case 11: op_diag<R, 3>(op, creg, re, im); break;
        default: break;
        }
    }
}

template <typename R, int K> __host__ __device__ constexpr size_t tile_smem() { return sizeof(typename V2T<R>::T) << K; }
template <int K> __host__ __device__ constexpr size_t table_smem() { return sizeof(uint64_t) << (K - kChunkBits); }

// One pass. Persistent CTAs walk the tiles; the pass program is copied to
// shared memory once per CTA.
template <typename R, int K>
__global__ void __launch_bounds__(1 << (K - kRegBits)) fused_pass_kernel(R *__restrict__ amp,
                                                                         const unsigned char *__restrict__ blob,
                                                                         uint64_t ntiles)
{
    constexpr int T = 1 << (K - kRegBits);
    constexpr int NQ = K - kRegBits;
    constexpr int NH = K - kChunkBits;
    using V2 = typename V2T<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    V2 *tile = reinterpret_cast<V2 *>(smem);
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
    R re[kNR], im[kNR];
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint64_t base = 0;
        for (int s = 0; s < h.nseg; ++s)
            base |= ((t >> h.seg_src[s]) & ((uint64_t(1) << h.seg_w[s]) - 1)) << h.seg_dst[s];
        load_tile<NQ>(amp, base, stg[0], tid, phys_hi, re, im);
        for (int s = 0; s < nstages; ++s) {
            if (s > 0) transpose<R, NQ>(tile, stg[s - 1], stg[s], tid, re, im);
            run_ops<R>(ops + stg[s].op_begin, stg[s].op_end - stg[s].op_begin, tid, base, re, im);
        }
        store_tile<NQ>(amp, base, stg[nstages - 1], tid, phys_hi, re, im);
    }
}

// ---------------------------------------------------------------- host side
template <typename R> void serialize(const plan::Pass &p, std::vector<unsigned char> &buf)
{
    const size_t off = buf.size();
    const int ns = int(p.stages.size()), no = int(p.ops.size());
    buf.resize(off + blob_bytes<R>(ns, no), 0);
    unsigned char *b = buf.data() + off;
    DHdr hd{};
    hd.k = p.k;
    hd.nstages = ns;
    hd.nops = no;
    hd.nseg = p.nseg;
    for (int j = 0; j < p.k - kChunkBits; ++j) hd.s_high[j] = p.s_high[j];
    for (int s = 0; s < p.nseg; ++s) {
        hd.seg_src[s] = p.seg_src[s];
        hd.seg_w[s] = p.seg_w[s];
        hd.seg_dst[s] = p.seg_dst[s];
    }
    memcpy(b, &hd, sizeof hd);
    for (int s = 0; s < ns; ++s) {
        DStage d{};
        const plan::Stage &st = p.stages[s];
        for (int j = 0; j < 4; ++j) {
            d.P[j] = st.in.P[j];
            d.Po[j] = st.out.P[j];
        }
        for (int q = 0; q < 8; ++q) {
            d.Q[q] = st.in.Q[q];
            d.Qo[q] = st.out.Q[q];
        }
        d.op_begin = st.op_begin;
        d.op_end = st.op_end;
        memcpy(b + sizeof(DHdr) + s * sizeof(DStage), &d, sizeof d);
    }
    DOp<R> *dop = reinterpret_cast<DOp<R> *>(b + ops_offset<R>(ns));
    for (int o = 0; o < no; ++o) {
        const plan::Op &op = p.ops[o];
        DOp<R> d{};
        d.type = op.type;
        d.treg = op.treg;
        d.creg = op.creg;
        d.d0one = (op.type == plan::OP_DIAG && op.m[0] == 1.0 && op.m[1] == 0.0) ? 1 : 0;
        d.cthr = op.cthr;
        d.tthr = op.tthr;
        d.cext = op.cext;
        d.text = op.text;
        for (int e = 0; e < 8; ++e) d.m[e] = R(op.m[e]);
        memcpy(&dop[o], &d, sizeof d);
    }
}

template <typename R, int K> size_t smem_for(size_t blob)
{
    return tile_smem<R, K>() + table_smem<K>() + blob;
}

template <typename R, int K> qv_status launch_pass(qv_state *s, const unsigned char *dblob, size_t blob)
{
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(fused_pass_kernel<R, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        227 * 1024);
    });
    QV_CUDA(attr_err);
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

int default_tile_bits(const qv_state *s) { return std::min(s->n, plan::kMaxK); }

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

qv_status plan_info(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t out[4])
{
    int K = (opts && opts->tile_bits) ? opts->tile_bits : std::min(n, plan::kMaxK);
    if (K < plan::kMinK || K > plan::kMaxK || K > n) return fail(QV_ERR_ARG, "tile_bits %d unsupported for n = %d", K, n);
    std::vector<plan::PGate> pg;
    QV_TRY(to_pgates(g, ng, pg));
    std::vector<plan::Pass> passes;
    plan::PlanStats st;
    std::string err;
    if (!plan::make_plan(n, K, dt == QV_C64, pg, passes, st, err))
        return fail(QV_ERR_UNSUPPORTED, "planner: %s", err.c_str());
    out[0] = st.passes;
    out[1] = st.stages;
    out[2] = st.transposes;
    out[3] = st.ops;
    return QV_OK;
}

qv_status apply_fused(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts)
{
    if (ng == 0) return QV_OK;
    int K = (opts && opts->tile_bits) ? opts->tile_bits : default_tile_bits(s);
    if (K < plan::kMinK || K > plan::kMaxK) return fail(QV_ERR_ARG, "tile_bits %d outside [10, 12]", K);
    if (K > s->n) return fail(QV_ERR_ARG, "tile_bits %d exceeds n = %d", K, s->n);
    std::vector<plan::PGate> pg;
    QV_TRY(to_pgates(g, ng, pg));
    std::vector<plan::Pass> passes;
    plan::PlanStats st;
    std::string err;
    if (!plan::make_plan(s->n, K, s->dt == QV_C64, pg, passes, st, err))
        return fail(QV_ERR_UNSUPPORTED, "planner: %s", err.c_str());
    return s->dt == QV_C64 ? run_plan<float>(s, passes, K) : run_plan<double>(s, passes, K);
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
