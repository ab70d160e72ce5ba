// Device-side helpers: index arithmetic and vectorised amplitude access.
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

namespace qv {

// Load with acquire semantics at GPU scope (pairs with a release increment).
__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait: polls *ctr until it reaches `need`. Gives up after `limit`
// polls (128 ns apart) or as soon as another wait has set *status; a wait
// that gives up sets *status to `code` (if still 0) and returns false.
__device__ __forceinline__ bool wait_counter(const unsigned *ctr, unsigned need, uint32_t limit, int *status,
                                             int code)
{
    uint32_t spins = 0;
    while (ld_acquire_u32(ctr) < need) {
        if (++spins > limit || *reinterpret_cast<volatile int *>(status) != 0) {
            atomicCAS(status, 0, code);
            return false;
        }
        __nanosleep(128);
    }
    return true;
}

// c(i) = sum_k c_k (-1)^{popcount(i & z_k)} over the nt terms of one X-mask
// group (Pauli strings: coefficients c_k already carry the i^{#Y} factor).
// Parities from 32-bit popcounts of the two halves of the index; the
// imaginary part is skipped for groups whose coefficients are all real.
template <typename R>
__device__ __forceinline__ void zsign_sum(uint64_t i, const uint64_t *z, const R *cre, const R *cim, int nt,
                                          bool has_im, R &cr, R &ci)
{
    const uint32_t lo = uint32_t(i), hi = uint32_t(i >> 32);
    cr = R(0);
    ci = R(0);
#pragma unroll 4
    for (int k = 0; k < nt; ++k) {
        const uint64_t zk = z[k];
        const uint32_t par = (__popc(lo & uint32_t(zk)) ^ __popc(hi & uint32_t(zk >> 32))) & 1u;
        const R sg = par ? R(-1) : R(1);
        cr += sg * cre[k];
        if (has_im) ci += sg * cim[k];
    }
}

// Insert a 0 at bit position b of x (bits >= b move up by one).
__host__ __device__ __forceinline__ uint64_t insert_zero(uint64_t x, int b)
{
    const uint64_t lo = x & ((uint64_t(1) << b) - 1);
    return ((x >> b) << (b + 1)) | lo;
}

// A group of W consecutive amplitudes held as separate re / im registers.
// Loads and stores use 16-byte vector accesses: C64 packs 2 amplitudes per
// float4, C128 one per double2. The group start must be W-aligned.
template <typename R, int W> struct AmpGroup {
    R re[W], im[W];
};

template <int W>
__device__ __forceinline__ void load_group(const float *base, uint64_t idx, AmpGroup<float, W> &g)
{
    static_assert(W % 2 == 0, "C64 groups hold pairs of amplitudes");
    const float4 *p = reinterpret_cast<const float4 *>(base + 2 * idx);
#pragma unroll
    for (int v = 0; v < W / 2; ++v) {
        const float4 x = p[v];
        g.re[2 * v] = x.x; g.im[2 * v] = x.y; g.re[2 * v + 1] = x.z; g.im[2 * v + 1] = x.w;
    }
}

template <int W>
__device__ __forceinline__ void store_group(float *base, uint64_t idx, const AmpGroup<float, W> &g)
{
    float4 *p = reinterpret_cast<float4 *>(base + 2 * idx);
#pragma unroll
    for (int v = 0; v < W / 2; ++v)
        p[v] = make_float4(g.re[2 * v], g.im[2 * v], g.re[2 * v + 1], g.im[2 * v + 1]);
}

template <int W>
__device__ __forceinline__ void load_group(const double *base, uint64_t idx, AmpGroup<double, W> &g)
{
    const double2 *p = reinterpret_cast<const double2 *>(base + 2 * idx);
#pragma unroll
    for (int v = 0; v < W; ++v) {
        const double2 x = p[v];
        g.re[v] = x.x; g.im[v] = x.y;
    }
}

template <int W>
__device__ __forceinline__ void store_group(double *base, uint64_t idx, const AmpGroup<double, W> &g)
{
    double2 *p = reinterpret_cast<double2 *>(base + 2 * idx);
#pragma unroll
    for (int v = 0; v < W; ++v) p[v] = make_double2(g.re[v], g.im[v]);
}

// 2x2 complex matrix in working precision, row-major.
template <typename R> struct Mat2 {
    R r[4], i[4];
};

// (a, b) <- U (a, b)
template <typename R>
__device__ __forceinline__ void apply2(const Mat2<R> &U, R &ar, R &ai, R &br, R &bi)
{
    const R xr = ar, xi = ai, yr = br, yi = bi;
    ar = U.r[0] * xr - U.i[0] * xi + U.r[1] * yr - U.i[1] * yi;
    ai = U.r[0] * xi + U.i[0] * xr + U.r[1] * yi + U.i[1] * yr;
    br = U.r[2] * xr - U.i[2] * xi + U.r[3] * yr - U.i[3] * yi;
    bi = U.r[2] * xi + U.i[2] * xr + U.r[3] * yi + U.i[3] * yr;
}

// a <- d a
template <typename R>
__device__ __forceinline__ void cmul(R dr, R di, R &ar, R &ai)
{
    const R xr = ar;
    ar = dr * xr - di * ai;
    ai = dr * ai + di * xr;
}

// Knuth's two-sum: s + e == a + b exactly (round-to-nearest).
template <typename R>
__device__ __forceinline__ void two_sum(R a, R b, R &s, R &e)
{
    s = a + b;
    const R bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// re^2 + im^2 = h + l exactly up to the rounding of l: each square as its
// rounded product plus the FMA error term, the two high parts by two-sum.
// The products use explicit round-to-nearest so they are not contracted.
__device__ __forceinline__ void exact_norm2(float re, float im, float &h, float &l)
{
    const float hr = __fmul_rn(re, re), hi = __fmul_rn(im, im);
    float e;
    two_sum(hr, hi, h, e);
    l = e + (fmaf(re, re, -hr) + fmaf(im, im, -hi));
}
__device__ __forceinline__ void exact_norm2(double re, double im, double &h, double &l)
{
    const double hr = __dmul_rn(re, re), hi = __dmul_rn(im, im);
    double e;
    two_sum(hr, hi, h, e);
    l = e + (fma(re, re, -hr) + fma(im, im, -hi));
}

// Running compensated sum in precision R: hi + lo carries the exact sum of
// everything added so far up to the rounding of lo.
// One complex amplitude (re, im) as one 8-byte (complex64) or 16-byte
// (complex128) load.
template <typename R> struct Cplx;
template <> struct Cplx<float> { using V = float2; };
template <> struct Cplx<double> { using V = double2; };
template <typename R> __device__ __forceinline__ typename Cplx<R>::V load_amp(const R *amp, uint64_t i)
{
    return reinterpret_cast<const typename Cplx<R>::V *>(amp)[i];
}

// Tables of the Z terms of a pure-Z group (X mask 0). A term whose Z mask lies
// inside one 8-bit chunk of the index (bits 8c .. 8c + 7) adds coef (-1)^popcount(v & m)
// to entry v of chunk c's table (m: the mask shifted down by 8c); the group's
// coefficient at index i is then the sum over chunks of entry (i >> 8c) & 255, plus
// the terms that span two chunks, which the group keeps in its term list. Layout:
// real parts at [c * 256 + v], imaginary parts at [(kZChunks + c) * 256 + v].
constexpr int kZChunks = 5;  // indices up to 40 bits
constexpr int kZTabWords = 2 * kZChunks * 256;

// Host side: fills the tables (2 kZTabWords values, double) from the terms that fit a
// chunk, moves the others to the front of z / cre / cim, and returns their count.
// *nch gets the number of chunks that cover n qubits.
inline int ztab_build(int n, uint64_t *z, double *cre, double *cim, int nt, double *tab, int *nch)
{
    const int nc = (n + 7) / 8;
    for (int e = 0; e < kZTabWords; ++e) tab[e] = 0.0;
    int keep = 0;
    for (int k = 0; k < nt; ++k) {
        int chunk = -1;
        for (int c = 0; c < nc && chunk < 0; ++c)
            if ((z[k] & ((uint64_t(1) << (8 * c)) - 1)) == 0 && (z[k] >> (8 * c)) < 256) chunk = c;
        if (chunk < 0) {
            z[keep] = z[k];
            cre[keep] = cre[k];
            cim[keep] = cim[k];
            ++keep;
            continue;
        }
        const unsigned m = unsigned(z[k] >> (8 * chunk));
        for (unsigned v = 0; v < 256; ++v) {
            const double sg = (__builtin_popcount(v & m) & 1) ? -1.0 : 1.0;
            tab[chunk * 256 + v] += sg * cre[k];
            tab[(kZChunks + chunk) * 256 + v] += sg * cim[k];
        }
    }
    *nch = nc;
    return keep;
}

// Host side, for a list of X-mask groups (fields x, zero_z, nt, z, cre, cim, tab): the
// first pure-Z group with at least four terms that fit a chunk gets its tables
// (returned in the state's precision, kZTabWords values) and keeps only its other
// terms; returns an empty vector when no group qualifies. Callers refresh any
// per-precision copies of the kept coefficients.
template <typename R, typename G> std::vector<R> ztab_for_group(int n, std::vector<G> &groups)
{
    for (G &g : groups) {
        if (g.x != 0 || g.zero_z || g.nt < 4) continue;
        uint64_t z[64];
        double cr[64], ci[64];
        for (int k = 0; k < g.nt; ++k) {
            z[k] = g.z[k];
            cr[k] = double(g.cre[k]);
            ci[k] = double(g.cim[k]);
        }
        std::vector<double> tab(kZTabWords);
        int nch = 0;
        const int keep = ztab_build(n, z, cr, ci, g.nt, tab.data(), &nch);
        if (g.nt - keep < 4) return {};
        for (int k = 0; k < keep; ++k) {
            g.z[k] = z[k];
            g.cre[k] = decltype(+g.cre[0])(cr[k]);
            g.cim[k] = decltype(+g.cim[0])(ci[k]);
        }
        g.nt = keep;
        g.tab = nch;
        return std::vector<R>(tab.begin(), tab.end());
    }
    return {};
}

// Device side: adds the tables' entries for index i (nch chunks).
template <typename R>
__device__ __forceinline__ void ztab_add(const R *tab, int nch, uint64_t i, bool him, R &cr, R &ci)
{
    for (int c = 0; c < nch; ++c) {
        const uint32_t v = uint32_t(i >> (8 * c)) & 255u;
        cr += tab[c * 256 + v];
        if (him) ci += tab[(kZChunks + c) * 256 + v];
    }
}

// Sum over the X-mask groups of Re( conj(a_{i^x}) c(i) a_i ) for amplitude i
// (a group has x, zero_z, has_im, nt, z, the coefficients c0re/c0im, cre/cim in
// double and f0re/f0im, fre/fim in float), in the state's precision.
template <typename R, typename G>
__device__ __forceinline__ R pauli_amp_sum(const R *__restrict__ amp, uint64_t i, const G *g, int ng, const R *tab)
{
    using V = typename Cplx<R>::V;
    const V a = load_amp(amp, i);
    R s = 0;
    // the partner loads of eight groups are issued before any is used: the far
    // partners come from DRAM, and the sum is bound by their latency
    for (int q0 = 0; q0 < ng; q0 += 8) {
        V b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u;
            b[u] = (q < ng && g[q].x) ? load_amp(amp, i ^ g[q].x) : a;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u;
            if (q >= ng) break;
            const R pr = b[u].x * a.x + b[u].y * a.y, pi = b[u].x * a.y - b[u].y * a.x;  // conj(b) a
            R cr, ci;
            if (g[q].zero_z) {
                if constexpr (sizeof(R) == 4) {
                    cr = g[q].f0re;
                    ci = g[q].f0im;
                } else {
                    cr = g[q].c0re;
                    ci = g[q].c0im;
                }
            } else {
                if constexpr (sizeof(R) == 4) zsign_sum<R>(i, g[q].z, g[q].fre, g[q].fim, g[q].nt, g[q].has_im != 0, cr, ci);
                else zsign_sum<R>(i, g[q].z, g[q].cre, g[q].cim, g[q].nt, g[q].has_im != 0, cr, ci);
                if (g[q].tab) ztab_add(tab, g[q].tab, i, g[q].has_im != 0, cr, ci);
            }
            s += pr * cr - pi * ci;
        }
    }
    return s;
}

// The same for NA amplitudes i0 + a * stride at once: each group's fields and
// each Z term are read once for all of them, and the partner loads of QB
// groups are issued before any is used. s[a] gets amplitude a's sum (a plain
// sum in the state's precision).
template <typename R, int NA, int QB, typename G>
__device__ __forceinline__ void pauli_amp_sums(const R *__restrict__ amp, uint64_t i0, uint64_t stride, const G *g,
                                               int ng, const R *tab, R (&s)[NA])
{
    using V = typename Cplx<R>::V;
    V a[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) {
        a[k] = load_amp(amp, i0 + k * stride);
        s[k] = 0;
    }
    for (int q0 = 0; q0 < ng; q0 += QB) {
        V b[QB][NA];
#pragma unroll
        for (int u = 0; u < QB; ++u) {
            const int q = q0 + u;
            const uint64_t x = q < ng ? g[q].x : 0;
#pragma unroll
            for (int k = 0; k < NA; ++k) b[u][k] = x ? load_amp(amp, (i0 + k * stride) ^ x) : a[k];
        }
#pragma unroll
        for (int u = 0; u < QB; ++u) {
            const int q = q0 + u;
            if (q >= ng) break;
            R cr[NA], ci[NA];
            if (g[q].zero_z) {
                R c0r, c0i;
                if constexpr (sizeof(R) == 4) {
                    c0r = g[q].f0re;
                    c0i = g[q].f0im;
                } else {
                    c0r = g[q].c0re;
                    c0i = g[q].c0im;
                }
#pragma unroll
                for (int k = 0; k < NA; ++k) {
                    cr[k] = c0r;
                    ci[k] = c0i;
                }
            } else {
#pragma unroll
                for (int k = 0; k < NA; ++k) cr[k] = ci[k] = R(0);
                const bool him = g[q].has_im != 0;
                for (int t = 0; t < g[q].nt; ++t) {
                    const uint64_t zk = g[q].z[t];
                    R fr, fi;
                    if constexpr (sizeof(R) == 4) {
                        fr = g[q].fre[t];
                        fi = g[q].fim[t];
                    } else {
                        fr = g[q].cre[t];
                        fi = g[q].cim[t];
                    }
#pragma unroll
                    for (int k = 0; k < NA; ++k) {
                        const uint64_t i = i0 + k * stride;
                        const uint32_t par = (__popc(uint32_t(i) & uint32_t(zk)) ^ __popc(uint32_t(i >> 32) & uint32_t(zk >> 32))) & 1u;
                        const R sg = par ? R(-1) : R(1);
                        cr[k] += sg * fr;
                        if (him) ci[k] += sg * fi;
                    }
                }
                if (g[q].tab) {
#pragma unroll
                    for (int k = 0; k < NA; ++k) ztab_add(tab, g[q].tab, i0 + k * stride, him, cr[k], ci[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                const R pr = b[u][k].x * a[k].x + b[u][k].y * a[k].y, pi = b[u][k].x * a[k].y - b[u][k].y * a[k].x;
                s[k] += pr * cr[k] - pi * ci[k];
            }
        }
    }
}

template <typename R> struct CompSum {
    R hi = 0, lo = 0;
    __device__ __forceinline__ void add(R x)
    {
        R s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo += e;
    }
    // adds another running sum (two-sum of the high parts, low parts added)
    __device__ __forceinline__ void merge(R ohi, R olo)
    {
        R s, e;
        two_sum(hi, ohi, s, e);
        hi = s;
        lo += e + olo;
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

// Neumaier-compensated FP64 accumulator.
struct Neumaier {
    double s = 0, c = 0;
    __host__ __device__ __forceinline__ void add(double x)
    {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __host__ __device__ __forceinline__ double value() const { return s + c; }
};

}  // namespace qv
