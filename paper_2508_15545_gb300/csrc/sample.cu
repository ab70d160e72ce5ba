// Measurement sampling and partial amplitudes (not in the paper; the paper
// notes that its strategies carry over to partial-amplitude simulation).
//
// Sampling is inverse-CDF sampling of the Born distribution p_i = |a_i|^2 /
// sum |a|^2: for a uniform u in [0, 1), the outcome is the smallest i whose
// cumulative probability exceeds u. The uniforms are inputs. Probabilities and
// all sums are FP64 (a squared FP32 component is exact in FP64).
//  1. per segment of kSeg amplitudes: its probability sum (one read of the state);
//  2. host: compensated prefix over the segments, then each shot's segment by
//     binary search and its offset inside the segment;
//  3. per segment holding shots: an inclusive FP64 scan of its probabilities in
//     shared memory and a binary search per shot.
#include <algorithm>
#include <cmath>
#include <vector>

#include "qv_device.cuh"
#include "qv_internal.h"

namespace qv {
namespace {

constexpr int kSegBitsS = 12;  // amplitudes per segment: 4096
constexpr int kSeg = 1 << kSegBitsS;
constexpr int kThreadsS = 256;

template <typename R> __device__ __forceinline__ double prob(const R *a, uint64_t i)
{
    const double re = a[2 * i], im = a[2 * i + 1];
    return re * re + im * im;
}

// seg[s] = sum of the probabilities of segment s (FP64, compensated)
template <typename R>
__global__ void __launch_bounds__(kThreadsS) seg_prob_kernel(const R *__restrict__ a, uint64_t N, double *seg)
{
    const uint64_t s0 = uint64_t(blockIdx.x) * kSeg;
    const uint64_t s1 = min(N, s0 + kSeg);
    Neumaier acc;
    for (uint64_t i = s0 + threadIdx.x; i < s1; i += kThreadsS) acc.add(prob(a, i));
    __shared__ double hs[kThreadsS], cs[kThreadsS];
    hs[threadIdx.x] = acc.s;
    cs[threadIdx.x] = acc.c;
    __syncthreads();
    if (threadIdx.x == 0) {
        Neumaier t;
        double c = 0;
        for (int k = 0; k < kThreadsS; ++k) {
            t.add(hs[k]);
            c += cs[k];
        }
        seg[blockIdx.x] = t.value() + c;
    }
}

// One block per segment that holds shots: segments[b], shots [first[b], first[b+1]).
// local[k] = the shot's target measured from the segment's start.
template <typename R>
__global__ void __launch_bounds__(kThreadsS) seg_search_kernel(const R *__restrict__ a, uint64_t N,
                                                               const uint64_t *segments, const uint32_t *first,
                                                               const double *local, uint64_t *out)
{
    __shared__ double cdf[kSeg];
    const uint64_t s0 = segments[blockIdx.x] * kSeg;
    const int len = int(N - s0 < uint64_t(kSeg) ? N - s0 : uint64_t(kSeg));
    for (int l = threadIdx.x; l < kSeg; l += kThreadsS) cdf[l] = l < len ? prob(a, s0 + l) : 0.0;
    __syncthreads();
    // inclusive scan (Hillis-Steele) in FP64
    for (int off = 1; off < kSeg; off <<= 1) {
        double v[kSeg / kThreadsS];
#pragma unroll
        for (int k = 0; k < kSeg / kThreadsS; ++k) {
            const int l = threadIdx.x + k * kThreadsS;
            v[k] = l >= off ? cdf[l - off] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSeg / kThreadsS; ++k) cdf[threadIdx.x + k * kThreadsS] += v[k];
        __syncthreads();
    }
    const double segtot = cdf[len - 1];
    for (uint32_t k = first[blockIdx.x] + threadIdx.x; k < first[blockIdx.x + 1]; k += kThreadsS) {
        const double t = local[k];
        // smallest l with cdf[l] > t; a target at or past the segment's total (rounding
        // at u -> 1) takes the last outcome with nonzero probability
        const bool past = !(t < segtot);
        int lo = 0, hi = len - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (past ? cdf[mid] >= segtot : cdf[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        out[k] = s0 + uint64_t(lo);
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
    QV_TRY(ensure_scratch(s, nseg * sizeof(double)));
    double *seg = static_cast<double *>(s->scratch.ptr);
    prof_bytes(s, QV_K_REDUCE, double(N) * 2 * sizeof(R));
    QV_LAUNCH(s, QV_K_REDUCE, seg_prob_kernel<R><<<unsigned(nseg), kThreadsS, 0, s->stream>>>(
                                  static_cast<const R *>(s->amp), N, seg));
    std::vector<double> hseg(nseg);
    QV_TRY(copy_d2h(s, hseg.data(), seg, nseg * sizeof(double)));
    QV_TRY(sync_and_check(s));
    // exclusive prefix P[i] and total (compensated running sum)
    std::vector<double> P(nseg + 1);
    Neumaier run;
    for (uint64_t i = 0; i < nseg; ++i) {
        P[i] = run.value();
        run.add(hseg[i]);
    }
    P[nseg] = run.value();
    const double total = P[nseg];
    if (!(total > 0)) return fail(QV_ERR_ARG, "the state has zero norm");
    // shots per segment, in segment order
    std::vector<uint64_t> sseg(nshots);
    uint64_t last = nseg - 1;  // last segment with nonzero probability
    while (last > 0 && !(hseg[last] > 0.0)) --last;
    for (size_t k = 0; k < nshots; ++k) {
        const double t = u[k] * total;
        // P[i] <= t < P[i + 1]; upper_bound skips segments of zero mass
        uint64_t i = uint64_t(std::upper_bound(P.begin(), P.begin() + nseg, t) - P.begin());
        i = i ? i - 1 : 0;
        if (!(t < total) || i > last) i = last;
        sseg[k] = i;
    }
    // shots in segment order (counting sort over the segments)
    std::vector<uint32_t> count(nseg + 1, 0), order(nshots);
    for (size_t k = 0; k < nshots; ++k) ++count[sseg[k] + 1];
    for (uint64_t i = 0; i < nseg; ++i) count[i + 1] += count[i];
    for (size_t k = 0; k < nshots; ++k) order[count[sseg[k]]++] = uint32_t(k);
    std::vector<uint64_t> segs;
    std::vector<uint32_t> first;
    std::vector<double> local(nshots);
    for (size_t j = 0; j < nshots; ++j) {
        const uint32_t k = order[j];
        if (segs.empty() || segs.back() != sseg[k]) {
            segs.push_back(sseg[k]);
            first.push_back(uint32_t(j));
        }
        local[j] = u[k] * total - P[sseg[k]];
    }
    first.push_back(uint32_t(nshots));
    // device buffers: segments, first, local, result
    const size_t b_seg = segs.size() * sizeof(uint64_t), b_first = first.size() * sizeof(uint32_t);
    const size_t b_loc = nshots * sizeof(double), b_out = nshots * sizeof(uint64_t);
    const size_t a8 = [](size_t x) { return (x + 15) & ~size_t(15); }(b_seg);
    const size_t a_first = (b_first + 15) & ~size_t(15), a_loc = (b_loc + 15) & ~size_t(15);
    QV_TRY(ensure_scratch(s, a8 + a_first + a_loc + b_out));
    char *base = static_cast<char *>(s->scratch.ptr);
    uint64_t *d_seg = reinterpret_cast<uint64_t *>(base);
    uint32_t *d_first = reinterpret_cast<uint32_t *>(base + a8);
    double *d_loc = reinterpret_cast<double *>(base + a8 + a_first);
    uint64_t *d_out = reinterpret_cast<uint64_t *>(base + a8 + a_first + a_loc);
    QV_TRY(copy_h2d(s, d_seg, segs.data(), b_seg));
    QV_TRY(copy_h2d(s, d_first, first.data(), b_first));
    QV_TRY(copy_h2d(s, d_loc, local.data(), b_loc));
    prof_bytes(s, QV_K_REDUCE, double(segs.size()) * kSeg * 2 * sizeof(R));
    QV_LAUNCH(s, QV_K_REDUCE, seg_search_kernel<R><<<unsigned(segs.size()), kThreadsS, 0, s->stream>>>(
                                  static_cast<const R *>(s->amp), N, d_seg, d_first, d_loc, d_out));
    std::vector<uint64_t> res(nshots);
    QV_TRY(copy_d2h(s, res.data(), d_out, b_out));
    QV_TRY(sync_and_check(s));
    for (size_t j = 0; j < nshots; ++j) out[order[j]] = res[j];
    return QV_OK;
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
