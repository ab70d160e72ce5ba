// Reductions over the state: norm and per-qubit Z sums, and Pauli-string
// expectation values. Not part of the paper (which reports no observables);
// they read the state once and never write it.
//
// Precision: |a|^2 is formed exactly as hi + lo (each square as its rounded
// product plus the FMA error term) in the norm and Z sums, and short runs
// inside a thread are summed in the state's precision with error-free two-sum
// compensation, so a thread's partial carries about twice the working
// precision. complex64 partials are merged across a block in the same
// two-float arithmetic and converted to FP64 once per block; complex128 ones
// by FP64 shuffle trees. Blocks are combined with Neumaier-compensated FP64 sums.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "qv_device.cuh"
#include "qv_internal.h"

namespace qv {
namespace {

template <typename R> struct Traits;
template <> struct Traits<float> { static constexpr int W = 4, LOGW = 2; };
template <> struct Traits<double> { static constexpr int W = 2, LOGW = 1; };

constexpr int kThreads = 256;         // 8 warps, 8 thread-index bits
constexpr int kSegBits = 14;          // a block reduces 2^14 consecutive amplitudes
constexpr int kSmallMaxN = 13;        // below this one block reduces the whole state
constexpr int kParts = kSegBits + 1;  // per block: total, then S_q for q < kSegBits

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sums V values per thread over the block; result valid in thread 0.
template <int V> __device__ void block_sum(double (&x)[V], double (*smem)[V])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = warp_sum(x[v]);
    if (lane == 0)
#pragma unroll
        for (int v = 0; v < V; ++v) smem[warp][v] = x[v];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int v = 0; v < V; ++v) {
            double s = 0;
            for (int w = 0; w < kThreads / 32; ++w) s += smem[w][v];
            x[v] = s;
        }
    }
}

// Combines V running sums over the block and writes their values to out[0..V).
// complex64: in FP32 two-sum arithmetic with shuffles, converted to FP64 once
// per value (GB300's FP64 pipe is about 1/64 of FP32: FP64 shuffle trees over
// every block cost more than reading the state). complex128: FP64 trees.
template <typename R, int V> __device__ void block_merge(CompSum<R> (&x)[V], double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (sizeof(R) == 4) {
        __shared__ R sh_hi[kThreads / 32][V], sh_lo[kThreads / 32][V];
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                x[v].merge(__shfl_xor_sync(0xffffffffu, x[v].hi, o), __shfl_xor_sync(0xffffffffu, x[v].lo, o));
        if (lane == 0)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                sh_hi[warp][v] = x[v].hi;
                sh_lo[warp][v] = x[v].lo;
            }
        __syncthreads();
        if (threadIdx.x < V) {
            CompSum<R> s;
            s.hi = sh_hi[0][threadIdx.x];
            s.lo = sh_lo[0][threadIdx.x];
            for (int w = 1; w < kThreads / 32; ++w) s.merge(sh_hi[w][threadIdx.x], sh_lo[w][threadIdx.x]);
            out[threadIdx.x] = s.value();
        }
    } else {
        __shared__ double smem[kThreads / 32][V];
        double y[V];
#pragma unroll
        for (int v = 0; v < V; ++v) y[v] = x[v].value();
        block_sum<V>(y, smem);
        if (threadIdx.x == 0)
            for (int v = 0; v < V; ++v) out[v] = y[v];
    }
}

// ---------------------------------------------------------------- small states
// One block: out[0] = sum |a|^2, out[1+q] = sum_{bit q set} |a|^2.
template <typename R> __global__ void __launch_bounds__(kThreads) zsum_small_kernel(const R *amp, int n, double *out)
{
    __shared__ double smem[kThreads / 32][kSmallMaxN + 1];
    double x[kSmallMaxN + 1];
#pragma unroll
    for (int v = 0; v <= kSmallMaxN; ++v) x[v] = 0;
    const uint64_t N = uint64_t(1) << n;
    for (uint64_t i = threadIdx.x; i < N; i += kThreads) {
        const double re = amp[2 * i], im = amp[2 * i + 1];
        const double p = re * re + im * im;
        x[0] += p;
#pragma unroll
        for (int q = 0; q < kSmallMaxN; ++q)
            if (q < n && ((i >> q) & 1)) x[1 + q] += p;
    }
    block_sum<kSmallMaxN + 1>(x, smem);
    if (threadIdx.x == 0)
        for (int v = 0; v <= n; ++v) out[v] = x[v];
}

// ---------------------------------------------------------------- segmented
// Block b reduces amplitudes [b 2^14, (b+1) 2^14). Thread t reads W-groups
// g = t + 256 v, so index bits split into: element bits [0, LOGW), thread
// bits [LOGW, LOGW+8), loop bits [LOGW+8, 14). Writes kParts doubles per block.
template <typename R> __global__ void __launch_bounds__(kThreads) zsum_seg_kernel(const R *__restrict__ amp, double *part)
{
    constexpr int W = Traits<R>::W, LOGW = Traits<R>::LOGW;
    constexpr int TB = 8;                         // thread bits
    constexpr int VB = kSegBits - LOGW - TB;      // loop bits
    CompSum<R> tot, eb[LOGW], vb[VB];
    const uint64_t seg = uint64_t(blockIdx.x) << kSegBits;
    const int t = threadIdx.x;
#pragma unroll 4
    for (int v = 0; v < (1 << VB); ++v) {
        AmpGroup<R, W> a;
        load_group(amp, seg + (uint64_t(t) << LOGW) + (uint64_t(v) << (LOGW + TB)), a);
        R ph[W], pl[W];  // |a|^2 exactly as ph + pl (up to the rounding of pl)
#pragma unroll
        for (int e = 0; e < W; ++e) exact_norm2(a.re[e], a.im[e], ph[e], pl[e]);
        CompSum<R> w;
#pragma unroll
        for (int e = 0; e < W; ++e) w.merge(ph[e], pl[e]);
        tot.merge(w.hi, w.lo);
#pragma unroll
        for (int k = 0; k < LOGW; ++k) {
            CompSum<R> sk;
#pragma unroll
            for (int e = 0; e < W; ++e)
                if ((e >> k) & 1) sk.merge(ph[e], pl[e]);
            eb[k].merge(sk.hi, sk.lo);
        }
#pragma unroll
        for (int k = 0; k < VB; ++k)
            if ((v >> k) & 1) vb[k].merge(w.hi, w.lo);
    }
    CompSum<R> x[kParts];
    x[0] = tot;
#pragma unroll
    for (int k = 0; k < LOGW; ++k) x[1 + k] = eb[k];
#pragma unroll
    for (int k = 0; k < TB; ++k) x[1 + LOGW + k] = ((t >> k) & 1) ? tot : CompSum<R>();
#pragma unroll
    for (int k = 0; k < VB; ++k) x[1 + LOGW + TB + k] = vb[k];
    block_merge<R, kParts>(x, part + uint64_t(blockIdx.x) * kParts);
}

// Output o = 0: total; o = 1 + q: S_q. For q < 14 sum column 1+q of the
// partials; for q >= 14 sum the totals of blocks whose bit (q - 14) is set.
__global__ void __launch_bounds__(kThreads) zsum_combine_kernel(const double *part, uint64_t nblk, double *out)
{
    __shared__ double sh_s[kThreads], sh_c[kThreads];
    const int o = blockIdx.x;
    Neumaier acc;
    for (uint64_t b = threadIdx.x; b < nblk; b += kThreads) {
        if (o <= kSegBits) acc.add(part[b * kParts + o]);
        else if ((b >> (o - 1 - kSegBits)) & 1) acc.add(part[b * kParts]);
    }
    sh_s[threadIdx.x] = acc.s;
    sh_c[threadIdx.x] = acc.c;
    __syncthreads();
    if (threadIdx.x == 0) {
        Neumaier f;
        for (int k = 0; k < kThreads; ++k) f.add(sh_s[k]);
        double c = 0;
        for (int k = 0; k < kThreads; ++k) c += sh_c[k];
        out[o] = f.value() + c;
    }
}

// ---------------------------------------------------------------- Pauli strings
// Terms sharing one X mask x: sum_i Re( conj(a_{i^x}) c(i) a_i ) with
// c(i) = sum_t coeff_t i^{ny_t} (-1)^{popcount(i & z_t)} (complex coefficient
// kept as re/im). One partial per block.
constexpr int kMaxTermsPerGroup = 64;
struct PauliGroup {
    uint64_t x;
    int nt;
    uint64_t z[kMaxTermsPerGroup];
    double cre[kMaxTermsPerGroup], cim[kMaxTermsPerGroup];
};

template <typename R>
__global__ void __launch_bounds__(kThreads) pauli_kernel(const R *__restrict__ amp, uint64_t N, const PauliGroup *g,
                                                         double *part)
{
    __shared__ double smem[kThreads / 32][1];
    __shared__ PauliGroup sg;
    __shared__ R cre[kMaxTermsPerGroup], cim[kMaxTermsPerGroup];  // in the state's precision, converted once
    if (threadIdx.x == 0) sg = *g;
    __syncthreads();
    for (int k = threadIdx.x; k < sg.nt; k += kThreads) {
        cre[k] = R(sg.cre[k]);
        cim[k] = R(sg.cim[k]);
    }
    __syncthreads();
    CompSum<R> acc;
    for (uint64_t i = uint64_t(blockIdx.x) * kThreads + threadIdx.x; i < N; i += uint64_t(gridDim.x) * kThreads) {
        const uint64_t j = i ^ sg.x;
        const R ar = amp[2 * i], ai = amp[2 * i + 1];
        const R br = amp[2 * j], bi = amp[2 * j + 1];
        // conj(b) a
        const R pr = br * ar + bi * ai, pi = br * ai - bi * ar;
        R cr, ci;
        zsign_sum<R>(i, sg.z, cre, cim, sg.nt, true, cr, ci);
        acc.add(pr * cr - pi * ci);
    }
    double x[1] = {acc.value()};
    block_sum<1>(x, smem);
    if (threadIdx.x == 0) part[blockIdx.x] = x[0];
}

// All X-mask groups in one pass over the state: part[block] = this block's
// share of sum_i sum_groups Re( conj(a_{i^x}) c(i) a_i ).
struct PauliGroupAll {
    uint64_t x;
    int nt;
    int zero_z;   // every z mask is 0: c(i) is the constant (c0re, c0im)
    int has_im;   // some coefficient has an imaginary part
    int tab;      // chunks of Z-term tables (pure-Z group), 0: none
    double c0re, c0im;
    float f0re, f0im;
    uint64_t z[kMaxTermsPerGroup];
    double cre[kMaxTermsPerGroup], cim[kMaxTermsPerGroup];
    float fre[kMaxTermsPerGroup], fim[kMaxTermsPerGroup];
};
constexpr size_t kPauliAllSmem = 200 * 1024;

template <typename R>
__global__ void __launch_bounds__(kThreads) pauli_all_kernel(const R *__restrict__ amp, uint64_t N,
                                                             const PauliGroupAll *groups, int ng, const R *ztab,
                                                             int tab_words, double *part)
{
    __shared__ double smem[kThreads / 32][1];
    extern __shared__ unsigned char sraw[];
    PauliGroupAll *g = reinterpret_cast<PauliGroupAll *>(sraw);
    R *tab = reinterpret_cast<R *>(sraw + size_t(ng) * sizeof(PauliGroupAll));
    static_assert(sizeof(PauliGroupAll) % 8 == 0, "copied as 8-byte words");
    for (int k = threadIdx.x; k < ng * int(sizeof(PauliGroupAll) / 8); k += kThreads)
        reinterpret_cast<uint64_t *>(g)[k] = reinterpret_cast<const uint64_t *>(groups)[k];
    for (int k = threadIdx.x; k < tab_words; k += kThreads) tab[k] = ztab[k];
    __syncthreads();
    CompSum<R> acc;
    // the terms of one amplitude are summed plainly (a few dozen of similar size);
    // the amplitudes' sums are added with compensation. Four amplitudes a thread
    // at a time: the group fields are read once for the four, and more partner
    // loads are in flight.
    const uint64_t S = uint64_t(gridDim.x) * kThreads;
    uint64_t i = uint64_t(blockIdx.x) * kThreads + threadIdx.x;
    for (; i + 3 * S < N; i += 4 * S) {
        R s4[4];
        pauli_amp_sums<R, 4, 4>(amp, i, S, g, ng, tab, s4);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.add(s4[k]);
    }
    for (; i < N; i += S) acc.add(pauli_amp_sum<R>(amp, i, g, ng, tab));
    double x[1] = {acc.value()};
    block_sum<1>(x, smem);
    if (threadIdx.x == 0) part[blockIdx.x] = x[0];
}

__global__ void sum_parts_kernel(const double *part, int np, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        Neumaier a;
        for (int k = 0; k < np; ++k) a.add(part[k]);
        *out = a.value();
    }
}

template <typename R> qv_status zsums_impl(qv_state *s, double *out_host)
{
    const int n = s->n;
    const R *amp = static_cast<const R *>(s->amp);
    QV_TRY(ensure_host_out(s, n + 1));
    if (n <= kSmallMaxN) {
        QV_TRY(ensure_scratch(s, sizeof(double) * (n + 1)));
        double *out = static_cast<double *>(s->scratch.ptr);
        prof_bytes(s, QV_K_REDUCE, double(dim(s)) * 2 * sizeof(R));
        QV_LAUNCH(s, QV_K_REDUCE, zsum_small_kernel<R><<<1, kThreads, 0, s->stream>>>(amp, n, out));
        QV_TRY(copy_d2h(s, s->host_out, out, sizeof(double) * (n + 1)));
    } else {
        const uint64_t nblk = dim(s) >> kSegBits;
        const size_t part_bytes = sizeof(double) * nblk * kParts;
        QV_TRY(ensure_scratch(s, part_bytes + sizeof(double) * (n + 1)));
        double *part = static_cast<double *>(s->scratch.ptr);
        double *out = part + nblk * kParts;
        prof_bytes(s, QV_K_REDUCE, double(dim(s)) * 2 * sizeof(R));
        QV_LAUNCH(s, QV_K_REDUCE, zsum_seg_kernel<R><<<unsigned(nblk), kThreads, 0, s->stream>>>(amp, part));
        QV_LAUNCH(s, QV_K_REDUCE, zsum_combine_kernel<<<n + 1, kThreads, 0, s->stream>>>(part, nblk, out));
        QV_TRY(copy_d2h(s, s->host_out, out, sizeof(double) * (n + 1)));
    }
    QV_TRY(sync_and_check(s));
    std::copy(s->host_out, s->host_out + n + 1, out_host);
    return QV_OK;
}

template <typename R> qv_status pauli_impl(qv_state *s, const qv_pauli_term *terms, size_t nt, double *out_host)
{
    // Group terms by X mask.
    std::vector<PauliGroup> groups;
    for (size_t k = 0; k < nt; ++k) {
        const uint64_t x = terms[k].xmask, z = terms[k].zmask;
        const int ny = __builtin_popcountll(x & z);
        // coeff * i^ny
        static const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, 1, 0, -1};
        const double cre = terms[k].coeff * pr[ny & 3], cim = terms[k].coeff * pi[ny & 3];
        PauliGroup *g = nullptr;
        for (auto &gg : groups)
            if (gg.x == x && gg.nt < kMaxTermsPerGroup) { g = &gg; break; }
        if (!g) {
            groups.emplace_back();
            g = &groups.back();
            g->x = x;
            g->nt = 0;
        }
        g->z[g->nt] = z;
        g->cre[g->nt] = cre;
        g->cim[g->nt] = cim;
        g->nt++;
    }
    const unsigned grid = unsigned(std::min<uint64_t>((dim(s) + kThreads - 1) / kThreads, uint64_t(s->num_sms) * 4));
    const size_t ng = groups.size();
    if (ng == 0) {
        *out_host = 0;
        return QV_OK;
    }
    if (ng * sizeof(PauliGroupAll) + kZTabWords * sizeof(R) <= kPauliAllSmem) {
        // one pass over the state for all groups
        std::vector<PauliGroupAll> ga(ng);
        for (size_t q = 0; q < ng; ++q) {
            PauliGroupAll &a = ga[q];
            std::memset(&a, 0, sizeof a);
            a.x = groups[q].x;
            a.nt = groups[q].nt;
            a.zero_z = 1;
            for (int k = 0; k < a.nt; ++k) {
                a.z[k] = groups[q].z[k];
                a.cre[k] = groups[q].cre[k];
                a.cim[k] = groups[q].cim[k];
                a.fre[k] = float(a.cre[k]);
                a.fim[k] = float(a.cim[k]);
                a.c0re += a.cre[k];
                a.c0im += a.cim[k];
                a.zero_z &= a.z[k] == 0;
                a.has_im |= a.cim[k] != 0.0;
            }
            a.f0re = float(a.c0re);
            a.f0im = float(a.c0im);
        }
        // the pure-Z group's terms that lie inside one 8-bit chunk of the index go into tables
        std::vector<R> htab = ztab_for_group<R>(s->n, ga);
        for (PauliGroupAll &a : ga)
            for (int k = 0; k < a.nt; ++k) {
                a.fre[k] = float(a.cre[k]);
                a.fim[k] = float(a.cim[k]);
            }
        const size_t gb = ng * sizeof(PauliGroupAll), tb = htab.size() * sizeof(R);
        QV_TRY(ensure_scratch(s, gb + tb + sizeof(double) * (grid + 1)));
        char *base = static_cast<char *>(s->scratch.ptr);
        PauliGroupAll *dg = reinterpret_cast<PauliGroupAll *>(base);
        R *dtab = reinterpret_cast<R *>(base + gb);
        double *part = reinterpret_cast<double *>(base + gb + tb), *res = part + grid;
        QV_TRY(copy_h2d(s, dg, ga.data(), gb));
        if (tb) QV_TRY(copy_h2d(s, dtab, htab.data(), tb));
        QV_TRY(allow_smem(reinterpret_cast<const void *>(pauli_all_kernel<R>), int(kPauliAllSmem)));
        prof_bytes(s, QV_K_PAULI, double(dim(s)) * 2 * sizeof(R) * double(ng + 1));
        QV_LAUNCH(s, QV_K_PAULI, pauli_all_kernel<R><<<grid, kThreads, gb + tb, s->stream>>>(
                                      static_cast<const R *>(s->amp), dim(s), dg, int(ng), dtab, int(htab.size()), part));
        QV_LAUNCH(s, QV_K_PAULI, sum_parts_kernel<<<1, 32, 0, s->stream>>>(part, int(grid), res));
        QV_TRY(ensure_host_out(s, 1));
        QV_TRY(copy_d2h(s, s->host_out, res, sizeof(double)));
        QV_TRY(sync_and_check(s));
        *out_host = s->host_out[0];
        return QV_OK;
    }
    // more groups than shared memory holds: one pass per group
    const size_t bytes = ng * sizeof(PauliGroup) + sizeof(double) * (ng * grid + ng + 1);
    QV_TRY(ensure_scratch(s, bytes));
    QV_TRY(ensure_host_out(s, ng + 1));
    char *base = static_cast<char *>(s->scratch.ptr);
    PauliGroup *dg = reinterpret_cast<PauliGroup *>(base);
    double *part = reinterpret_cast<double *>(base + ng * sizeof(PauliGroup));
    double *res = part + ng * grid;
    QV_TRY(copy_h2d(s, dg, groups.data(), ng * sizeof(PauliGroup)));
    const R *amp = static_cast<const R *>(s->amp);
    for (size_t k = 0; k < ng; ++k) {
        prof_bytes(s, QV_K_PAULI, double(dim(s)) * 2 * sizeof(R));
        QV_LAUNCH(s, QV_K_PAULI,
                  pauli_kernel<R><<<grid, kThreads, 0, s->stream>>>(amp, dim(s), dg + k, part + k * grid));
        QV_LAUNCH(s, QV_K_PAULI, sum_parts_kernel<<<1, 32, 0, s->stream>>>(part + k * grid, int(grid), res + k));
    }
    QV_TRY(copy_d2h(s, s->host_out, res, sizeof(double) * ng));
    QV_TRY(sync_and_check(s));
    Neumaier tot;
    for (size_t k = 0; k < ng; ++k) tot.add(s->host_out[k]);
    *out_host = tot.value();
    return QV_OK;
}

}  // namespace

qv_status reduce_zsums(qv_state *s, double *out_host)
{
    return s->dt == QV_C64 ? zsums_impl<float>(s, out_host) : zsums_impl<double>(s, out_host);
}

qv_status reduce_pauli(qv_state *s, const qv_pauli_term *terms, size_t nt, double *out_host)
{
    return s->dt == QV_C64 ? pauli_impl<float>(s, terms, nt, out_host) : pauli_impl<double>(s, terms, nt, out_host);
}

// ---------------------------------------------------------------- allocation-free Z sums
// Same kernels as reduce_zsums, but the per-block partials live in a fixed
// device array owned by this library instead of per-handle cudaMalloc'd
// scratch. Sized for states up to kStaticMaxN qubits: 2^(30-14) blocks x 15
// doubles = 7,864,320 bytes, held on every device that loads the library.
constexpr int kStaticMaxN = 30;
constexpr uint64_t kStaticBlocks = uint64_t(1) << (kStaticMaxN - kSegBits);
__device__ __align__(256) double g_zsum_static[kStaticBlocks * kParts];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double *g_static_ptr[kMaxDevices] = {};

// Device address of g_zsum_static on the current device, looked up once per
// device (host code cannot use the symbol itself as a device pointer).
qv_status static_scratch(double **out)
{
    int dev = 0;
    QV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(QV_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        QV_CUDA(cudaGetSymbolAddress(&p, g_zsum_static));
        g_static_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_static_ptr[dev];
    return QV_OK;
}

template <typename R>
qv_status zsums_noalloc_impl(const void *dev_amp, int n, cudaStream_t stream, double *dev_out)
{
    const R *amp = static_cast<const R *>(dev_amp);
    if (n <= kSmallMaxN) {
        zsum_small_kernel<R><<<1, kThreads, 0, stream>>>(amp, n, dev_out);
        QV_CUDA(cudaGetLastError());
        return QV_OK;
    }
    double *part = nullptr;
    QV_TRY(static_scratch(&part));
    const uint64_t nblk = (uint64_t(1) << n) >> kSegBits;
    // Every block writes all kParts of its partials, so nothing needs clearing.
    zsum_seg_kernel<R><<<unsigned(nblk), kThreads, 0, stream>>>(amp, part);
    QV_CUDA(cudaGetLastError());
    zsum_combine_kernel<<<n + 1, kThreads, 0, stream>>>(part, nblk, dev_out);
    QV_CUDA(cudaGetLastError());
    return QV_OK;
}
}  // namespace

}  // namespace qv

extern "C" qv_status qv_zsums_noalloc(const void *dev_amp, int n, qv_dtype dt, void *cuda_stream, double *dev_out)
{
    using namespace qv;
    if (!dev_amp || !dev_out) return fail(QV_ERR_ARG, "NULL device pointer");
    if (reinterpret_cast<uintptr_t>(dev_amp) % 16) return fail(QV_ERR_ARG, "amplitudes not 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(dev_out) % 8) return fail(QV_ERR_ARG, "output not 8-byte aligned");
    if (dt != QV_C64 && dt != QV_C128) return fail(QV_ERR_ARG, "bad dtype %d", int(dt));
    if (n < 1 || n > kStaticMaxN)
        return fail(QV_ERR_ARG, "qv_zsums_noalloc: n = %d outside [1, %d] (its fixed scratch holds the partials of "
                                "at most 2^%d amplitudes)", n, kStaticMaxN, kStaticMaxN);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the fixed array belongs to the current device: the buffers and the stream must too
    int dev = 0;
    QV_CUDA(cudaGetDevice(&dev));
    for (const void *p : {dev_amp, static_cast<const void *>(dev_out)}) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(QV_ERR_ARG, "qv_zsums_noalloc: %p is not memory CUDA knows", p);
        }
        if (a.type == cudaMemoryTypeDevice && a.device != dev)
            return fail(QV_ERR_ARG, "qv_zsums_noalloc: buffer %p is on device %d, the current device is %d", p,
                        a.device, dev);
    }
    if (st) {
        int sdev = dev;
        if (cudaStreamGetDevice(st, &sdev) == cudaSuccess && sdev != dev)
            return fail(QV_ERR_ARG, "qv_zsums_noalloc: the stream belongs to device %d, the current device is %d",
                        sdev, dev);
        (void)cudaGetLastError();
    }
    return dt == QV_C64 ? zsums_noalloc_impl<float>(dev_amp, n, st, dev_out)
                        : zsums_noalloc_impl<double>(dev_amp, n, st, dev_out);
}
