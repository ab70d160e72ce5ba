// Device side of the interpreting fused kernel: the pass-program format,
// register files, addressing, tile load/store, transposes and on-chip ops.
// Shared by the per-pass kernel (fused.cu) and the persistent batched kernel
// (batch.cu); the comment at the top of fused.cu describes the design.
#pragma once

#include <cstring>
#include <vector>

#include "coef.h"
#include "planner.h"
#include "qv_device.cuh"

namespace qv {
namespace {


using plan::kChunkBits;
using plan::kRegBits;
constexpr int kNR = 1 << kRegBits;  // amplitudes per thread

// Minimum resident CTAs per SM the register allocation must allow.
#ifndef QV_FUSED_MINB
#define QV_FUSED_MINB(R, K) ((K) == 12 ? (sizeof(R) == 4 ? 3 : 1) : (sizeof(R) == 4 ? 4 : 2))
#endif

// ---------------------------------------------------------------- device program
// One blob per pass: header, stages, ops.
struct DHdr {
    int32_t k, nstages, nops, nseg;
    int32_t s_high[8];
    int32_t seg_src[8], seg_w[8], seg_dst[8];
};
struct DStage {
    int8_t P[4], Q[8], Po[4], Qo[8];
    int32_t op_begin, op_end;
};
// code = type * 20 + treg * 5 + (sreg + 1) for a register-bit target (type
// GEN 0, X 1, DIAG 2); treg = 4 (code 60 + sreg + 1) for a diagonal op whose
// target is a thread bit or a qubit outside the tile.
struct DOpHdr {
    int32_t code;
    uint32_t sthr;    // select on this thread-index bit
    uint32_t tthr;    // uniform diagonal: target on this thread-index bit
    uint32_t m0id;    // the select = 0 matrix is the identity
    uint64_t sext;    // select on this physical qubit outside the tile
    uint64_t text;    // uniform diagonal: target physical qubit outside the tile
};
// Coefficients for select = 0 / 1. complex64: 12 broadcast f32x2 pairs per set
// -- (re, re), (im, im), (-im, -im) of U00, U01, U10, U11 (GEN), or of d0, d1
// (DIAG) -- with the two lanes resolved on the host where they differ (select
// or diagonal target on register bit 3). complex128: re, im of the 4 entries.
template <typename R> struct DOp;
template <> struct DOp<float> {
    DOpHdr h;
    uint64_t c[2][12];
};
template <> struct DOp<double> {
    DOpHdr h;
    double m[2][8];
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

// ---------------------------------------------------------------- packed f32x2
__device__ __forceinline__ uint64_t pk(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(uint64_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---------------------------------------------------------------- register files
// complex64: r[v] = (Re slot v, Re slot v + 8), i[v] likewise (slot bit 3 =
// tile position 0). complex128: plain arrays.
template <typename R> struct Regs;
template <> struct Regs<float> {
    uint64_t r[8], i[8];
};
template <> struct Regs<double> {
    double r[kNR], i[kNR];
};

// ---------------------------------------------------------------- addressing
template <int NQ> __device__ __forceinline__ uint32_t thr_part(const int8_t *Q, int tid)
{
    uint32_t l = 0;
#pragma unroll
    for (int b = 0; b < NQ; ++b)
        if ((tid >> b) & 1) l |= 1u << Q[b];
    return l;
}

// Physical index bits of tile index l (a linear scatter of its bits).
__device__ __forceinline__ uint64_t phys(uint32_t l, const uint64_t *phys_hi)
{
    return (l & ((1u << kChunkBits) - 1)) | phys_hi[l >> kChunkBits];
}

// XOR of u[j] over the set bits j of the compile-time M, onto b0.
template <int M, typename T, int NU> __device__ __forceinline__ T xor_sel(T b0, const T (&u)[NU])
{
    T a = b0;
#pragma unroll
    for (int j = 0; j < NU; ++j)
        if ((M >> j) & 1) a ^= u[j];
    return a;
}

// Shared-memory word swizzles (linear over GF(2)): complex64 words are 8-byte
// packed pairs (16 per 128-byte row), complex128 words 16-byte amplitudes (8).
__device__ __forceinline__ uint32_t swz8(uint32_t w) { return w ^ (((w >> 4) ^ (w >> 8)) & 15u); }
__device__ __forceinline__ uint32_t swz16(uint32_t w) { return w ^ (((w >> 3) ^ (w >> 6) ^ (w >> 9)) & 7u); }

// ---------------------------------------------------------------- tile load / store
// complex64 load/store layout: position 0 on register bit 3, lanes on
// positions 1..5; one float4 = (re, im) of the amplitudes l and l + 1.
// CG: load through L2 only (ld.global.cg), for data another CTA may have just
// written (the persistent batched kernel).
template <int NQ, bool CG = false>
__device__ __forceinline__ void load_tile(const float *amp, uint64_t base, const int8_t *P, const int8_t *Q, int tid,
                                          const uint64_t *phys_hi, Regs<float> &x)
{
    uint64_t u[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) u[j] = phys(1u << P[j], phys_hi);
    const uint64_t gb = base + phys(thr_part<NQ>(Q, tid), phys_hi);
    float4 f[8];
#define QV_LD(V)                                                                            \
    {                                                                                       \
        const float4 *p_ = reinterpret_cast<const float4 *>(amp + 2 * xor_sel<V>(gb, u));   \
        f[V] = CG ? __ldcg(p_) : *p_;                                                       \
    }
    QV_LD(0) QV_LD(1) QV_LD(2) QV_LD(3) QV_LD(4) QV_LD(5) QV_LD(6) QV_LD(7)
#undef QV_LD
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        x.r[v] = pk(f[v].x, f[v].z);
        x.i[v] = pk(f[v].y, f[v].w);
    }
}

template <int NQ>
__device__ __forceinline__ void store_tile(float *amp, uint64_t base, const int8_t *P, const int8_t *Q, int tid,
                                           const uint64_t *phys_hi, const Regs<float> &x)
{
    uint64_t u[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) u[j] = phys(1u << P[j], phys_hi);
    const uint64_t gb = base + phys(thr_part<NQ>(Q, tid), phys_hi);
    float a, b, c, d;
#define QV_ST(V)                                                                                 \
    upk(x.r[V], a, b);                                                                           \
    upk(x.i[V], c, d);                                                                           \
    *reinterpret_cast<float4 *>(amp + 2 * xor_sel<V>(gb, u)) = make_float4(a, c, b, d);
    QV_ST(0) QV_ST(1) QV_ST(2) QV_ST(3) QV_ST(4) QV_ST(5) QV_ST(6) QV_ST(7)
#undef QV_ST
}

// complex128 load/store layout: lanes on positions 0..4; one double2 per amplitude.
template <int NQ, bool CG = false>
__device__ __forceinline__ void load_tile(const double *amp, uint64_t base, const int8_t *P, const int8_t *Q,
                                          int tid, const uint64_t *phys_hi, Regs<double> &x)
{
    uint64_t u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = phys(1u << P[j], phys_hi);
    const uint64_t gb = base + phys(thr_part<NQ>(Q, tid), phys_hi);
    double2 v[kNR];
#define QV_LD(M)                                                                         \
    {                                                                                    \
        const double2 *p_ = reinterpret_cast<const double2 *>(amp) + xor_sel<M>(gb, u);  \
        v[M] = CG ? __ldcg(p_) : *p_;                                                    \
    }
    QV_LD(0) QV_LD(1) QV_LD(2) QV_LD(3) QV_LD(4) QV_LD(5) QV_LD(6) QV_LD(7)
    QV_LD(8) QV_LD(9) QV_LD(10) QV_LD(11) QV_LD(12) QV_LD(13) QV_LD(14) QV_LD(15)
#undef QV_LD
#pragma unroll
    for (int m = 0; m < kNR; ++m) {
        x.r[m] = v[m].x;
        x.i[m] = v[m].y;
    }
}

template <int NQ>
__device__ __forceinline__ void store_tile(double *amp, uint64_t base, const int8_t *P, const int8_t *Q, int tid,
                                           const uint64_t *phys_hi, const Regs<double> &x)
{
    uint64_t u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = phys(1u << P[j], phys_hi);
    const uint64_t gb = base + phys(thr_part<NQ>(Q, tid), phys_hi);
#define QV_ST(M) reinterpret_cast<double2 *>(amp)[xor_sel<M>(gb, u)] = make_double2(x.r[M], x.i[M]);
    QV_ST(0) QV_ST(1) QV_ST(2) QV_ST(3) QV_ST(4) QV_ST(5) QV_ST(6) QV_ST(7)
    QV_ST(8) QV_ST(9) QV_ST(10) QV_ST(11) QV_ST(12) QV_ST(13) QV_ST(14) QV_ST(15)
#undef QV_ST
}

// ---------------------------------------------------------------- layout change
// complex64: two planes of 2^(K-1) 8-byte words (real, imaginary); word index =
// tile index >> 1 (tile position 0 is the lane inside the word).
template <int K, int NQ>
__device__ __forceinline__ void transpose(unsigned char *tile, const DStage &from, const DStage &to, int tid,
                                          Regs<float> &x)
{
    uint64_t *re = reinterpret_cast<uint64_t *>(tile);
    uint64_t *im = re + (1 << (K - 1));
    {
        uint32_t u[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) u[j] = swz8((1u << from.Po[j]) >> 1);
        const uint32_t b = swz8(thr_part<NQ>(from.Qo, tid) >> 1);
#define QV_W(V)                                \
    {                                          \
        const uint32_t w = xor_sel<V>(b, u);   \
        re[w] = x.r[V];                        \
        im[w] = x.i[V];                        \
    }
        QV_W(0) QV_W(1) QV_W(2) QV_W(3) QV_W(4) QV_W(5) QV_W(6) QV_W(7)
#undef QV_W
    }
    __syncthreads();
    {
        uint32_t u[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) u[j] = swz8((1u << to.P[j]) >> 1);
        const uint32_t b = swz8(thr_part<NQ>(to.Q, tid) >> 1);
#define QV_R(V)                                \
    {                                          \
        const uint32_t w = xor_sel<V>(b, u);   \
        x.r[V] = re[w];                        \
        x.i[V] = im[w];                        \
    }
        QV_R(0) QV_R(1) QV_R(2) QV_R(3) QV_R(4) QV_R(5) QV_R(6) QV_R(7)
#undef QV_R
    }
    __syncthreads();
}

// complex128: one plane of 2^K 16-byte words.
template <int K, int NQ>
__device__ __forceinline__ void transpose(unsigned char *tile, const DStage &from, const DStage &to, int tid,
                                          Regs<double> &x)
{
    double2 *t = reinterpret_cast<double2 *>(tile);
    {
        uint32_t u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = swz16(1u << from.Po[j]);
        const uint32_t b = swz16(thr_part<NQ>(from.Qo, tid));
#define QV_W(M) t[xor_sel<M>(b, u)] = make_double2(x.r[M], x.i[M]);
        QV_W(0) QV_W(1) QV_W(2) QV_W(3) QV_W(4) QV_W(5) QV_W(6) QV_W(7)
        QV_W(8) QV_W(9) QV_W(10) QV_W(11) QV_W(12) QV_W(13) QV_W(14) QV_W(15)
#undef QV_W
    }
    __syncthreads();
    {
        uint32_t u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = swz16(1u << to.P[j]);
        const uint32_t b = swz16(thr_part<NQ>(to.Q, tid));
#define QV_R(M)                                      \
    {                                                \
        const double2 v = t[xor_sel<M>(b, u)];       \
        x.r[M] = v.x;                                \
        x.i[M] = v.y;                                \
    }
        QV_R(0) QV_R(1) QV_R(2) QV_R(3) QV_R(4) QV_R(5) QV_R(6) QV_R(7)
        QV_R(8) QV_R(9) QV_R(10) QV_R(11) QV_R(12) QV_R(13) QV_R(14) QV_R(15)
#undef QV_R
    }
    __syncthreads();
}

// ---------------------------------------------------------------- gate math, complex64
// (a, b) <- U (a, b) on two packed amplitude pairs; c = 12 coefficient pairs.
__device__ __forceinline__ void apply2_f2(const uint64_t (&c)[12], uint64_t &ar, uint64_t &ai, uint64_t &br,
                                          uint64_t &bi)
{
    const uint64_t xr = ar, xi = ai, yr = br, yi = bi;
    ar = f2fma(c[0], xr, f2fma(c[2], xi, f2fma(c[3], yr, f2mul(c[5], yi))));
    ai = f2fma(c[0], xi, f2fma(c[1], xr, f2fma(c[3], yi, f2mul(c[4], yr))));
    br = f2fma(c[6], xr, f2fma(c[8], xi, f2fma(c[9], yr, f2mul(c[11], yi))));
    bi = f2fma(c[6], xi, f2fma(c[7], xr, f2fma(c[9], yi, f2mul(c[10], yr))));
}

// a <- d a on a packed pair; d given as (re, im, -im) pairs
__device__ __forceinline__ void cmul_f2(uint64_t dr, uint64_t di, uint64_t dn, uint64_t &ar, uint64_t &ai)
{
    const uint64_t xr = ar, xi = ai;
    ar = f2fma(dr, xr, f2mul(dn, xi));
    ai = f2fma(dr, xi, f2mul(di, xr));
}

template <int N> __device__ __forceinline__ void load_c(const uint64_t *src, uint64_t (&c)[12])
{
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(src);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
        const ulonglong2 v = p[k];
        c[2 * k] = v.x;
        c[2 * k + 1] = v.y;
    }
}

// Lane-0 (scalar) matrix of a coefficient set.
__device__ __forceinline__ void scalar_mat(const uint64_t (&c)[12], Mat2<float> &U)
{
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float a, b;
        upk(c[3 * e], U.r[e], a);
        upk(c[3 * e + 1], U.i[e], b);
    }
}

// uniform select value of an op for this thread and tile
__device__ __forceinline__ int usel(const DOpHdr &h, int tid, uint64_t base)
{
    return ((uint32_t(tid) & h.sthr) != 0) || ((base & h.sext) != 0);
}

template <int T, int J, int C>
__device__ __forceinline__ void op_impl(const DOp<float> &op, Regs<float> &x, int tid, uint64_t base)
{
    if constexpr (C == J) {
        return;
    } else if constexpr (T == plan::OP_GEN) {
        uint64_t c[12];
        if constexpr (C < 0 || C == 3) {
            int s = 0;
            if constexpr (C < 0) {
                s = usel(op.h, tid, base);
                if (!s && op.h.m0id) return;
            }
            load_c<12>(op.c[s], c);
            if constexpr (J < 3) {
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    if (!((v >> J) & 1)) apply2_f2(c, x.r[v], x.i[v], x.r[v | (1 << J)], x.i[v | (1 << J)]);
            } else {
                Mat2<float> U;
                scalar_mat(c, U);
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    float a0, a1, b0, b1;
                    upk(x.r[v], a0, a1);
                    upk(x.i[v], b0, b1);
                    apply2(U, a0, b0, a1, b1);
                    x.r[v] = pk(a0, a1);
                    x.i[v] = pk(b0, b1);
                }
            }
        } else {  // select on register bit C in 0..2: set 0 for bit C = 0, set 1 for bit C = 1
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (s == 0 && op.h.m0id) continue;
                load_c<12>(op.c[s], c);
                if constexpr (J < 3) {
#pragma unroll
                    for (int v = 0; v < 8; ++v)
                        if (!((v >> J) & 1) && ((v >> C) & 1) == s)
                            apply2_f2(c, x.r[v], x.i[v], x.r[v | (1 << J)], x.i[v | (1 << J)]);
                } else {
                    Mat2<float> U;
                    scalar_mat(c, U);
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        if (((v >> C) & 1) != s) continue;
                        float a0, a1, b0, b1;
                        upk(x.r[v], a0, a1);
                        upk(x.i[v], b0, b1);
                        apply2(U, a0, b0, a1, b1);
                        x.r[v] = pk(a0, a1);
                        x.i[v] = pk(b0, b1);
                    }
                }
            }
        }
    } else if constexpr (T == plan::OP_X) {
        // unfused bit flip: M0 = I (controlled) or X (uncontrolled), M1 = X
        if constexpr (C < 0) {
            if (!usel(op.h, tid, base) && op.h.m0id) return;
        }
        if constexpr (J < 3 && C != 3) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                if ((v >> J) & 1) continue;
                if (C >= 0 && !((v >> C) & 1)) continue;
                const int w = v | (1 << J);
                const uint64_t tr = x.r[v], ti = x.i[v];
                x.r[v] = x.r[w];
                x.i[v] = x.i[w];
                x.r[w] = tr;
                x.i[w] = ti;
            }
        } else if constexpr (J < 3) {  // select on the lane bit: swap lane 1 only
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                if ((v >> J) & 1) continue;
                const int w = v | (1 << J);
                float a0, a1, b0, b1, c0, c1, d0, d1;
                upk(x.r[v], a0, a1);
                upk(x.i[v], b0, b1);
                upk(x.r[w], c0, c1);
                upk(x.i[w], d0, d1);
                x.r[v] = pk(a0, c1);
                x.i[v] = pk(b0, d1);
                x.r[w] = pk(c0, a1);
                x.i[w] = pk(d0, b1);
            }
        } else {  // J == 3: swap the two lanes
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                if (C >= 0 && !((v >> C) & 1)) continue;
                float a0, a1, b0, b1;
                upk(x.r[v], a0, a1);
                upk(x.i[v], b0, b1);
                x.r[v] = pk(a1, a0);
                x.i[v] = pk(b1, b0);
            }
        }
    } else {  // OP_DIAG: J = 0..3 register target, 4 = uniform target (thread bit / outside)
        uint64_t c[12];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int ss = s;
            if constexpr (C < 0 || C == 3) {
                if (s == 1) break;
                if constexpr (C < 0) {
                    ss = usel(op.h, tid, base);
                    if (!ss && op.h.m0id) return;
                }
            } else {
                if (s == 0 && op.h.m0id) continue;
            }
            load_c<6>(op.c[ss], c);  // c[0..2] = d0, c[3..5] = d1 (lane-resolved for J == 3 or C == 3)
            if constexpr (J == 4) {
                const bool t1 = (uint32_t(tid) & op.h.tthr) != 0 || (base & op.h.text) != 0;
                const uint64_t dr = t1 ? c[3] : c[0], di = t1 ? c[4] : c[1], dn = t1 ? c[5] : c[2];
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    if (C < 0 || C == 3 || ((v >> C) & 1) == s) cmul_f2(dr, di, dn, x.r[v], x.i[v]);
            } else if constexpr (J < 3) {
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    if (!(C < 0 || C == 3 || ((v >> C) & 1) == s)) continue;
                    if ((v >> J) & 1) cmul_f2(c[3], c[4], c[5], x.r[v], x.i[v]);
                    else cmul_f2(c[0], c[1], c[2], x.r[v], x.i[v]);
                }
            } else {  // J == 3: c[0..2] carry d0 in lane 0 and d1 in lane 1
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    if (C < 0 || ((v >> C) & 1) == s) cmul_f2(c[0], c[1], c[2], x.r[v], x.i[v]);
            }
        }
    }
}

// ---------------------------------------------------------------- gate math, complex128
template <int T, int J, int C>
__device__ __forceinline__ void op_impl(const DOp<double> &op, Regs<double> &x, int tid, uint64_t base)
{
    if constexpr (C == J) {
        return;
    } else {
        const int su = (C < 0) ? usel(op.h, tid, base) : 0;
        if (C < 0 && !su && op.h.m0id) return;
        if constexpr (T == plan::OP_GEN) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (C < 0 && s != su) continue;
                if (C >= 0 && s == 0 && op.h.m0id) continue;
                Mat2<double> U;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    U.r[e] = op.m[s][2 * e];
                    U.i[e] = op.m[s][2 * e + 1];
                }
#pragma unroll
                for (int m = 0; m < kNR; ++m) {
                    if ((m >> J) & 1) continue;
                    if (C >= 0 && ((m >> C) & 1) != s) continue;
                    apply2(U, x.r[m], x.i[m], x.r[m | (1 << J)], x.i[m | (1 << J)]);
                }
            }
        } else if constexpr (T == plan::OP_X) {
#pragma unroll
            for (int m = 0; m < kNR; ++m) {
                if ((m >> J) & 1) continue;
                if (C >= 0 && !((m >> C) & 1)) continue;
                const int w = m | (1 << J);
                const double tr = x.r[m], ti = x.i[m];
                x.r[m] = x.r[w];
                x.i[m] = x.i[w];
                x.r[w] = tr;
                x.i[w] = ti;
            }
        } else {
            const bool t1 = J == 4 && ((uint32_t(tid) & op.h.tthr) != 0 || (base & op.h.text) != 0);
#pragma unroll
            for (int m = 0; m < kNR; ++m) {
                const int s = C < 0 ? su : ((m >> C) & 1);
                if (s == 0 && op.h.m0id) continue;
                const bool one = J == 4 ? t1 : (((m >> (J & 3)) & 1) != 0);
                cmul(op.m[s][one ? 6 : 0], op.m[s][one ? 7 : 1], x.r[m], x.i[m]);
            }
        }
    }
}

#define QV_C5(T, J)                                                            \
    case (T)*20 + (J)*5 + 0: op_impl<T, J, -1>(op, x, tid, base); break;       \
    case (T)*20 + (J)*5 + 1: op_impl<T, J, 0>(op, x, tid, base); break;        \
    case (T)*20 + (J)*5 + 2: op_impl<T, J, 1>(op, x, tid, base); break;        \
    case (T)*20 + (J)*5 + 3: op_impl<T, J, 2>(op, x, tid, base); break;        \
    case (T)*20 + (J)*5 + 4: op_impl<T, J, 3>(op, x, tid, base); break;
#define QV_C20(T) QV_C5(T, 0) QV_C5(T, 1) QV_C5(T, 2) QV_C5(T, 3)

template <typename R>
__device__ __forceinline__ void run_ops(const DOp<R> *ops, int nops, int tid, uint64_t base, Regs<R> &x)
{
    for (int o = 0; o < nops; ++o) {
        const DOp<R> &op = ops[o];
        switch (op.h.code) {
            QV_C20(0)
            QV_C20(1)
            QV_C20(2)
            QV_C5(2, 4)
        default: break;
        }
    }
}
#undef QV_C20
#undef QV_C5

template <typename R, int K> __host__ __device__ constexpr size_t tile_smem() { return (2 * sizeof(R)) << K; }
template <int K> __host__ __device__ constexpr size_t table_smem() { return sizeof(uint64_t) << (K - kChunkBits); }


// ---------------------------------------------------------------- host side
void fill_coeffs(DOp<float> &d, const plan::Op &op) { op_coeffs_c64(op, &d.c[0][0]); }
void fill_coeffs(DOp<double> &d, const plan::Op &op) { op_coeffs_c128(op, &d.m[0][0]); }

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
    unsigned char *dop = b + ops_offset<R>(ns);
    for (int o = 0; o < no; ++o) {
        const plan::Op &op = p.ops[o];
        DOp<R> d{};
        const int treg = (op.type == plan::OP_DIAG && op.treg < 0) ? 4 : op.treg;
        d.h.code = op.type * 20 + treg * 5 + op.sreg + 1;
        d.h.sthr = op.sthr;
        d.h.tthr = op.tthr;
        d.h.m0id = op.m0id ? 1u : 0u;
        d.h.sext = op.sext;
        d.h.text = op.text;
        fill_coeffs(d, op);
        memcpy(dop + o * sizeof(DOp<R>), &d, sizeof d);
    }
}

}  // namespace
}  // namespace qv
