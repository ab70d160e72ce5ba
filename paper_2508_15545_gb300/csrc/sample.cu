// Measurement sampling and partial amplitudes (not in the paper; the paper
// notes that its strategies carry over to partial-amplitude simulation).
//
// Sampling is inverse-CDF sampling of the Born distribution p_i = |a_i|^2 /
// sum |a|^2: for a uniform u in [0, 1), the outcome is the smallest i whose
// cumulative probability exceeds u. The uniforms are inputs. Single
// probabilities are FP64 (a squared FP32 component is exact in FP64); sums of
// complex64 probabilities over runs of amplitudes are two-float sums of exact
// squares (see Slot), and everything from segment totals on is FP64. Every step
// runs on the device:
//  1. per segment of kSeg amplitudes: its probability sum (one read of the state);
//  2. one block: compensated exclusive prefix P over the segments (P[nseg] = total)
//     and the last segment of nonzero probability;
//  3. per shot: its segment by binary search over P (upper bound of u * total),
//     counted per segment;
//  4. one block: exclusive prefix of the counts; then each shot's place in the
//     shot list ordered by segment (counting sort);
//  5. per segment holding shots: its amplitudes in shared memory, sums of runs of
//     16 probabilities (FP64 per run), a prefix over the runs, and per shot a
//     binary search over the runs and a short sequential search inside one.
#include <algorithm>

#include "qv_device.cuh"
#include "qv_internal.h"

namespace qv {
namespace {

constexpr int kSegBitsS = 12;  // amplitudes per segment: 4096
constexpr int kSeg = 1 << kSegBitsS;
constexpr int kThreadsS = 256;
constexpr int kScanThreads = 1024;  // one block for the prefix over segments

// Per-amplitude slot of a segment in shared memory and the sums over runs of
// them. complex64: the raw FP32 components; a square of an FP32 value is
// exact as an FP32 product plus its FMA error term, and run sums are kept as
// two FP32 values (Dekker's two-sum), about 2^-44 relative, then one FP64
// conversion per run, which spares GB300's slow FP64 pipe. Single
// probabilities are FP64 (exact squares), as in the oracle. complex128: FP64
// probabilities and plain FP64 sums.
template <typename R> struct Slot;
template <> struct Slot<float> {
    using T = float2;
    static __device__ __forceinline__ T load(const float *a, uint64_t i) { return make_float2(a[2 * i], a[2 * i + 1]); }
    static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ double p(T v)
    {
        const double re = v.x, im = v.y;
        return re * re + im * im;
    }
    static __device__ __forceinline__ bool nonzero(T v) { return v.x != 0.f || v.y != 0.f; }
    struct Acc {
        float h = 0.f, l = 0.f;
        __device__ __forceinline__ void two_sum(float x)
        {
            const float s = __fadd_rn(h, x), bb = __fsub_rn(s, h);
            l = __fadd_rn(l, __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
            h = s;
        }
        __device__ __forceinline__ void square(float x)
        {
            const float q = __fmul_rn(x, x);
            two_sum(q);
            l = __fadd_rn(l, fmaf(x, x, -q));
        }
        __device__ __forceinline__ void add(T v)
        {
            square(v.x);
            square(v.y);
        }
        __device__ __forceinline__ void merge(const Acc &o)
        {
            two_sum(o.h);
            l = __fadd_rn(l, o.l);
        }
        __device__ __forceinline__ Acc shfl_xor(int m) const
        {
            Acc o;
            o.h = __shfl_xor_sync(0xffffffffu, h, m);
            o.l = __shfl_xor_sync(0xffffffffu, l, m);
            return o;
        }
        __device__ __forceinline__ double value() const { return double(h) + double(l); }
    };
};
template <> struct Slot<double> {
    using T = double;
    static __device__ __forceinline__ T load(const double *a, uint64_t i)
    {
        const double re = a[2 * i], im = a[2 * i + 1];
        return re * re + im * im;
    }
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ double p(T v) { return v; }
    static __device__ __forceinline__ bool nonzero(T v) { return v > 0.0; }
    struct Acc {
        double s = 0.0;
        __device__ __forceinline__ void add(T v) { s += v; }
        __device__ __forceinline__ void merge(const Acc &o) { s += o.s; }
        __device__ __forceinline__ Acc shfl_xor(int m) const
        {
            Acc o;
            o.s = __shfl_xor_sync(0xffffffffu, s, m);
            return o;
        }
        __device__ __forceinline__ double value() const { return s; }
    };
};

// seg[s] = sum of the probabilities of segment s
template <typename R>
__global__ void __launch_bounds__(kThreadsS) seg_prob_kernel(const R *__restrict__ a, uint64_t N, double *seg)
{
    const uint64_t s0 = uint64_t(blockIdx.x) * kSeg;
    const uint64_t s1 = min(N, s0 + kSeg);
    using Acc = typename Slot<R>::Acc;
    Acc acc;
    for (uint64_t i = s0 + threadIdx.x; i < s1; i += kThreadsS) acc.add(Slot<R>::load(a, i));
    // combine across the block with shuffles in the same arithmetic: a serial
    // FP64 loop in one thread would hold the FP64 pipe for whole warps
    for (int m = 16; m > 0; m >>= 1) acc.merge(acc.shfl_xor(m));
    __shared__ Acc ws[kThreadsS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        Acc t = ws[0];
        for (int w = 1; w < kThreadsS / 32; ++w) t.merge(ws[w]);
        seg[blockIdx.x] = t.value();
    }
}

// Exclusive compensated prefix over x[0..m): P[i] = x[0] + ... + x[i-1],
// P[m] = the total; *last = the largest i with x[i] > 0 (left as set when none).
// One block: each thread sums a contiguous run, thread 0 chains the runs.
__global__ void __launch_bounds__(kScanThreads) seg_prefix_kernel(const double *x, uint64_t m, double *P,
                                                                  unsigned long long *last)
{
    __shared__ double hs[kScanThreads], hc[kScanThreads];
    const uint64_t per = (m + kScanThreads - 1) / kScanThreads;
    const uint64_t b0 = min(m, per * threadIdx.x), b1 = min(m, b0 + per);
    Neumaier acc;
    unsigned long long lst = 0;
    bool any = false;
    for (uint64_t i = b0; i < b1; ++i) {
        acc.add(x[i]);
        if (x[i] > 0.0) {
            lst = i;
            any = true;
        }
    }
    if (any) atomicMax(last, lst);
    hs[threadIdx.x] = acc.s;
    hc[threadIdx.x] = acc.c;
    __syncthreads();
    if (threadIdx.x == 0) {
        Neumaier run;
        for (int t = 0; t < kScanThreads; ++t) {
            const double sv = hs[t], cv = hc[t];
            hs[t] = run.s;
            hc[t] = run.c;
            run.add(sv);
            run.add(cv);
        }
        P[m] = run.value();
    }
    __syncthreads();
    Neumaier r;
    r.s = hs[threadIdx.x];
    r.c = hc[threadIdx.x];
    for (uint64_t i = b0; i < b1; ++i) {
        P[i] = r.value();
        r.add(x[i]);
    }
}

// Exclusive prefix of the counts cnt[0..m) into off[0..m], one block.
__global__ void __launch_bounds__(kScanThreads) count_prefix_kernel(const uint32_t *cnt, uint64_t m, uint32_t *off)
{
    __shared__ uint32_t hs[kScanThreads];
    const uint64_t per = (m + kScanThreads - 1) / kScanThreads;
    const uint64_t b0 = min(m, per * threadIdx.x), b1 = min(m, b0 + per);
    uint32_t acc = 0;
    for (uint64_t i = b0; i < b1; ++i) acc += cnt[i];
    hs[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < kScanThreads; ++t) {
            const uint32_t v = hs[t];
            hs[t] = run;
            run += v;
        }
        off[m] = run;
    }
    __syncthreads();
    uint32_t r = hs[threadIdx.x];
    for (uint64_t i = b0; i < b1; ++i) {
        off[i] = r;
        r += cnt[i];
    }
}

// Segment of each shot: the last i with P[i] <= u * total (zero-mass segments
// are skipped); a target at or past the total, or past the last segment of
// nonzero probability, takes that segment. Counted per segment.
__global__ void shot_segment_kernel(const double *u, uint32_t nshots, const double *P, uint64_t nseg,
                                    const unsigned long long *last, uint32_t *sseg, uint32_t *cnt)
{
    const double total = P[nseg];
    const uint64_t lst = *last;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nshots; k += gridDim.x * blockDim.x) {
        const double t = __dmul_rn(u[k], total);
        uint64_t lo = 0, hi = nseg;  // first index with P[i] > t
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (P[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        uint64_t i = lo ? lo - 1 : 0;
        if (!(t < total) || i > lst) i = lst;
        sseg[k] = uint32_t(i);
        atomicAdd(&cnt[i], 1u);
    }
}

// Place of each shot in the list ordered by segment (order inside a segment
// is arbitrary: each shot's result depends on its own uniform only).
__global__ void shot_scatter_kernel(const uint32_t *sseg, uint32_t nshots, const uint32_t *off, uint32_t *cursor,
                                    uint32_t *sorted)
{
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nshots; k += gridDim.x * blockDim.x) {
        const uint32_t sg = sseg[k];
        sorted[off[sg] + atomicAdd(&cursor[sg], 1u)] = k;
    }
}

// One block per segment; segments without shots return at once. Shots of
// segment s are sorted[off[s] .. off[s+1]); the target inside the segment is
// t = u * total - P[s]. Thread j sums the run of kRun probabilities
// [j kRun, (j + 1) kRun); cs[] is the inclusive prefix over the runs. A shot
// takes the first run whose prefix exceeds t, then the first outcome inside it
// whose running sum exceeds t; a target at or past the segment's total (rounding
// at u -> 1) takes the last outcome with nonzero probability.
template <typename R>
__global__ void __launch_bounds__(kThreadsS) seg_search_kernel(const R *__restrict__ a, uint64_t N, const double *P,
                                                               uint64_t nseg, const uint32_t *off,
                                                               const uint32_t *sorted, const double *u, uint64_t *out)
{
    constexpr int kRun = kSeg / kThreadsS;
    const uint64_t sg = blockIdx.x;
    const uint32_t j0 = off[sg], j1 = off[sg + 1];
    if (j0 == j1) return;
    using S = Slot<R>;
    __shared__ typename S::T el[kSeg];
    __shared__ double cs[kThreadsS + 1];
    __shared__ int lastnz;
    const uint64_t s0 = sg * kSeg;
    const int len = int(N - s0 < uint64_t(kSeg) ? N - s0 : uint64_t(kSeg));
    if (threadIdx.x == 0) lastnz = 0;
    for (int l = threadIdx.x; l < kSeg; l += kThreadsS) el[l] = l < len ? S::load(a, s0 + l) : S::zero();
    __syncthreads();
    typename S::Acc acc;
    int lz = -1;
    for (int i = 0; i < kRun; ++i) {  // rotated start: the threads of a warp hit distinct banks
        const int x = int(threadIdx.x) * kRun + ((i + int(threadIdx.x)) & (kRun - 1));
        const typename S::T v = el[x];
        acc.add(v);
        if (S::nonzero(v)) lz = max(lz, x);
    }
    if (lz >= 0) atomicMax(&lastnz, lz);
    // inclusive prefix over the runs: within each warp by shuffles, then the warp offsets
    __shared__ double wtot[kThreadsS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v = acc.value();
    for (int d = 1; d < 32; d <<= 1) {
        const double o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    if (lane == 31) wtot[warp] = v;
    __syncthreads();
    double woff = 0.0;
    for (int w = 0; w < warp; ++w) woff += wtot[w];
    cs[threadIdx.x + 1] = woff + v;
    if (threadIdx.x == 0) cs[0] = 0.0;
    __syncthreads();
    const double segtot = cs[kThreadsS], total = P[nseg], base = P[sg];
    for (uint32_t j = j0 + threadIdx.x; j < j1; j += kThreadsS) {
        const uint32_t k = sorted[j];
        const double t = __dsub_rn(__dmul_rn(u[k], total), base);
        int l = lastnz;
        if (t < segtot) {
            int lo = 0, hi = kThreadsS - 1;  // first run r with cs[r + 1] > t
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cs[mid + 1] > t) hi = mid;
                else lo = mid + 1;
            }
            double run = cs[lo];
            int last_in_run = -1;
            l = -1;
            for (int i = 0; i < kRun; ++i) {
                const int x = lo * kRun + i;
                if (S::nonzero(el[x])) last_in_run = x;
                run += S::p(el[x]);
                if (run > t) {
                    l = x;
                    break;
                }
            }
            // the running sum can round to at most t inside the run: its last outcome
            if (l < 0) l = last_in_run >= 0 ? last_in_run : lastnz;
        }
        out[k] = s0 + uint64_t(l);
    }
}

template <typename R> __global__ void gather_kernel(const R *__restrict__ a, const uint64_t *idx, size_t k, R *out)
{
    for (size_t j = size_t(blockIdx.x) * blockDim.x + threadIdx.x; j < k; j += size_t(gridDim.x) * blockDim.x) {
        out[2 * j] = a[2 * idx[j]];
        out[2 * j + 1] = a[2 * idx[j] + 1];
    }
}

template <typename R> qv_status sample_impl(qv_state *s, const double *u, size_t nshots, uint64_t *out)
{
    const uint64_t N = dim(s);
    const uint64_t nseg = (N + kSeg - 1) / kSeg;
    const uint32_t ns = uint32_t(nshots);
    auto up16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    // scratch: seg, P, last, cnt (then the scatter cursor), off, u, sseg, sorted, out
    const size_t b_seg = up16(nseg * sizeof(double)), b_P = up16((nseg + 1) * sizeof(double)), b_last = 16;
    const size_t b_cnt = up16((nseg + 1) * sizeof(uint32_t)), b_u = up16(nshots * sizeof(double));
    const size_t b_idx = up16(nshots * sizeof(uint32_t)), b_out = up16(nshots * sizeof(uint64_t));
    QV_TRY(ensure_scratch(s, b_seg + b_P + b_last + 2 * b_cnt + b_u + 2 * b_idx + b_out));
    char *p = static_cast<char *>(s->scratch.ptr);
    double *seg = reinterpret_cast<double *>(p);
    double *P = reinterpret_cast<double *>(p += b_seg);
    unsigned long long *last = reinterpret_cast<unsigned long long *>(p += b_P);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(p += b_last);
    uint32_t *off = reinterpret_cast<uint32_t *>(p += b_cnt);
    double *du = reinterpret_cast<double *>(p += b_cnt);
    uint32_t *sseg = reinterpret_cast<uint32_t *>(p += b_u);
    uint32_t *sorted = reinterpret_cast<uint32_t *>(p += b_idx);
    uint64_t *dout = reinterpret_cast<uint64_t *>(p += b_idx);
    const R *a = static_cast<const R *>(s->amp);

    prof_bytes(s, QV_K_REDUCE, double(N) * 2 * sizeof(R));
    QV_LAUNCH(s, QV_K_REDUCE, seg_prob_kernel<R><<<unsigned(nseg), kThreadsS, 0, s->stream>>>(a, N, seg));
    QV_CUDA(cudaMemsetAsync(last, 0, sizeof(unsigned long long), s->stream));
    QV_LAUNCH(s, QV_K_REDUCE, seg_prefix_kernel<<<1, kScanThreads, 0, s->stream>>>(seg, nseg, P, last));
    double total = 0;
    QV_TRY(copy_d2h(s, &total, P + nseg, sizeof(double)));
    QV_TRY(sync_and_check(s));
    if (!(total > 0)) return fail(QV_ERR_ARG, "the state has zero norm");
    QV_TRY(copy_h2d(s, du, u, nshots * sizeof(double)));
    QV_CUDA(cudaMemsetAsync(cnt, 0, (nseg + 1) * sizeof(uint32_t), s->stream));
    const unsigned grid = unsigned(std::min<size_t>((nshots + 255) / 256, size_t(s->num_sms) * 8));
    QV_LAUNCH(s, QV_K_REDUCE,
              shot_segment_kernel<<<grid, 256, 0, s->stream>>>(du, ns, P, nseg, last, sseg, cnt));
    QV_LAUNCH(s, QV_K_REDUCE, count_prefix_kernel<<<1, kScanThreads, 0, s->stream>>>(cnt, nseg, off));
    QV_CUDA(cudaMemsetAsync(cnt, 0, (nseg + 1) * sizeof(uint32_t), s->stream));
    QV_LAUNCH(s, QV_K_REDUCE, shot_scatter_kernel<<<grid, 256, 0, s->stream>>>(sseg, ns, off, cnt, sorted));
    prof_bytes(s, QV_K_REDUCE, double(N) * 2 * sizeof(R));
    QV_LAUNCH(s, QV_K_REDUCE,
              seg_search_kernel<R><<<unsigned(nseg), kThreadsS, 0, s->stream>>>(a, N, P, nseg, off, sorted, du, dout));
    QV_TRY(copy_d2h(s, out, dout, nshots * sizeof(uint64_t)));
    return sync_and_check(s);
}

template <typename R> qv_status gather_impl(qv_state *s, const uint64_t *idx, size_t k, void *host)
{
    const size_t bi = (k * sizeof(uint64_t) + 15) & ~size_t(15);
    QV_TRY(ensure_scratch(s, bi + k * 2 * sizeof(R)));
    char *base = static_cast<char *>(s->scratch.ptr);
    uint64_t *d_idx = reinterpret_cast<uint64_t *>(base);
    R *d_out = reinterpret_cast<R *>(base + bi);
    QV_TRY(copy_h2d(s, d_idx, idx, k * sizeof(uint64_t)));
    const unsigned grid = unsigned(std::min<size_t>((k + 255) / 256, size_t(s->num_sms) * 4));
    QV_LAUNCH(s, QV_K_REDUCE, gather_kernel<R><<<grid, 256, 0, s->stream>>>(static_cast<const R *>(s->amp), d_idx, k,
                                                                            d_out));
    QV_TRY(copy_d2h(s, host, d_out, k * 2 * sizeof(R)));
    return sync_and_check(s);
}

}  // namespace

qv_status sample(qv_state *s, const double *u, size_t nshots, uint64_t *out)
{
    return s->dt == QV_C64 ? sample_impl<float>(s, u, nshots, out) : sample_impl<double>(s, u, nshots, out);
}

qv_status get_amplitudes(qv_state *s, const uint64_t *idx, size_t k, void *host)
{
    return s->dt == QV_C64 ? gather_impl<float>(s, idx, k, host) : gather_impl<double>(s, idx, k, host);
}

}  // namespace qv
