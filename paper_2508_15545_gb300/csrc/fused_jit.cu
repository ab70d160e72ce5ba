// Compiled fused passes. The planner's program for one pass (tile qubits,
// register layouts, the op sequence) is turned into CUDA C++ with every
// layout, address offset, target and select bit baked in as constants, then
// compiled with NVRTC for sm_103a and launched through the driver API. The
// gate coefficients stay runtime data (a by-value kernel parameter, read
// from the constant bank), so circuits that differ only in their angles --
// the same circuit run again, or a variational ansatz with new parameters --
// reuse the compiled kernel. Compared with the interpreted kernel in
// fused.cu this removes the per-op dispatch, the register moves at the
// dispatch merge points, and the runtime index arithmetic.
#include <cuda.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "coef.h"
#include "planner.h"
#include "ptxas_report.h"
#include "qv_internal.h"
#include "qv_jit.h"

namespace qv {
namespace {

using plan::kChunkBits;
using plan::kRegBits;

// ---------------------------------------------------------------- NVRTC + driver, loaded on demand
// Both are opened with dlopen so that libqv.so itself loads on machines
// without a GPU driver (the host-only entry points still work there).
struct JitApi {
    bool ok = false;        // NVRTC and the driver: compile and launch
    bool nvrtc_ok = false;  // NVRTC alone: compile on a host without a GPU driver
    std::string why;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *, const char *const *);
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *);
    nvrtcResult (*log_size)(nvrtcProgram, size_t *);
    nvrtcResult (*log)(nvrtcProgram, char *);
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *);
    nvrtcResult (*cubin)(nvrtcProgram, char *);
    nvrtcResult (*destroy)(nvrtcProgram *);
    CUresult (*module_load)(CUmodule *, const void *);
    CUresult (*get_function)(CUfunction *, CUmodule, const char *);
    CUresult (*set_attr)(CUfunction, CUfunction_attribute, int);
    CUresult (*get_attr)(int *, CUfunction_attribute, CUfunction);
    CUresult (*occupancy)(int *, CUfunction, int, size_t);
    CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                       void **, void **);
    CUresult (*err_string)(CUresult, const char **);
};

const JitApi &api()
{
    static JitApi n;
    static std::once_flag once;
    std::call_once(once, [] {
        void *h = dlopen("libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL);
        if (!h) h = dlopen("libnvrtc.so", RTLD_NOW | RTLD_LOCAL);
        void *d = dlopen("libcuda.so.1", RTLD_NOW | RTLD_LOCAL);
        if (!h) {
            n.why = "libnvrtc.so not found";
            return;
        }
        bool all = true;
        auto sym = [&](void *lib, auto &f, const char *name) {
            f = reinterpret_cast<std::remove_reference_t<decltype(f)>>(dlsym(lib, name));
            all &= f != nullptr;
        };
        sym(h, n.create, "nvrtcCreateProgram");
        sym(h, n.compile, "nvrtcCompileProgram");
        sym(h, n.log_size, "nvrtcGetProgramLogSize");
        sym(h, n.log, "nvrtcGetProgramLog");
        sym(h, n.cubin_size, "nvrtcGetCUBINSize");
        sym(h, n.cubin, "nvrtcGetCUBIN");
        sym(h, n.destroy, "nvrtcDestroyProgram");
        n.nvrtc_ok = all;
        if (!all) {
            n.why = "libnvrtc.so lacks a needed symbol";
            return;
        }
        if (!d) {
            n.why = "libcuda.so.1 not found";
            return;
        }
        sym(d, n.module_load, "cuModuleLoadData");
        sym(d, n.get_function, "cuModuleGetFunction");
        sym(d, n.set_attr, "cuFuncSetAttribute");
        sym(d, n.get_attr, "cuFuncGetAttribute");
        sym(d, n.occupancy, "cuOccupancyMaxActiveBlocksPerMultiprocessor");
        sym(d, n.launch, "cuLaunchKernel");
        sym(d, n.err_string, "cuGetErrorString");
        n.ok = all;
        if (!all) n.why = "libnvrtc.so or libcuda.so.1 lacks a needed symbol";
    });
    return n;
}

// ---------------------------------------------------------------- device prelude
const char *kPrelude = R"PRELUDE(
typedef unsigned long long u64;
typedef unsigned int u32;
#define QI __device__ __forceinline__
QI u64 pk(float lo, float hi) { u64 r; asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi)); return r; }
QI void upk(u64 v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
QI u64 f2fma(u64 a, u64 b, u64 c) { u64 d; asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c)); return d; }
QI u64 f2mul(u64 a, u64 b) { u64 d; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
// asynchronous 16-byte copy global -> shared (through L2 only), and waiting for this thread's copies
QI u32 sh_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }
QI void cp16(u32 dst, const void *src) { asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory"); }
QI void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
QI void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// complex64: (a, b) <- U (a, b) on two packed pairs; c = (re, im, -im) pairs of U00 U01 U10 U11
QI void ap2(const u64 (&c)[12], u64 &ar, u64 &ai, u64 &br, u64 &bi) {
    const u64 xr = ar, xi = ai, yr = br, yi = bi;
    ar = f2fma(c[0], xr, f2fma(c[2], xi, f2fma(c[3], yr, f2mul(c[5], yi))));
    ai = f2fma(c[0], xi, f2fma(c[1], xr, f2fma(c[3], yi, f2mul(c[4], yr))));
    br = f2fma(c[6], xr, f2fma(c[8], xi, f2fma(c[9], yr, f2mul(c[11], yi))));
    bi = f2fma(c[6], xi, f2fma(c[7], xr, f2fma(c[9], yi, f2mul(c[10], yr))));
}
QI void cm2(u64 dr, u64 di, u64 dn, u64 &ar, u64 &ai) {
    const u64 xr = ar, xi = ai;
    ar = f2fma(dr, xr, f2mul(dn, xi));
    ai = f2fma(dr, xi, f2mul(di, xr));
}
// sign flips: amplitude v (both packed lanes, real and imaginary parts) XOR m[v]
QI void xs8(u64 (&r)[8], u64 (&i)[8], u64 m0, u64 m1, u64 m2, u64 m3, u64 m4, u64 m5, u64 m6, u64 m7) {
    const u64 m[8] = {m0, m1, m2, m3, m4, m5, m6, m7};
#pragma unroll
    for (int v = 0; v < 8; ++v) { r[v] ^= m[v]; i[v] ^= m[v]; }
}
// scalar pair with the lane-0 values of c
QI void ap1(const u64 (&c)[12], float &ar, float &ai, float &br, float &bi) {
    float u[8], t;
    for (int e = 0; e < 4; ++e) { upk(c[3 * e], u[2 * e], t); upk(c[3 * e + 1], u[2 * e + 1], t); }
    const float xr = ar, xi = ai, yr = br, yi = bi;
    ar = u[0] * xr - u[1] * xi + u[2] * yr - u[3] * yi;
    ai = u[0] * xi + u[1] * xr + u[2] * yi + u[3] * yr;
    br = u[4] * xr - u[5] * xi + u[6] * yr - u[7] * yi;
    bi = u[4] * xi + u[5] * xr + u[6] * yi + u[7] * yr;
}
template <int J> QI void g_all(u64 (&r)[8], u64 (&i)[8], const u64 (&c)[12]) {
#pragma unroll
    for (int v = 0; v < 8; ++v) if (!((v >> J) & 1)) ap2(c, r[v], i[v], r[v | (1 << J)], i[v | (1 << J)]);
}
template <int J, int C, int S> QI void g_sel(u64 (&r)[8], u64 (&i)[8], const u64 (&c)[12]) {
#pragma unroll
    for (int v = 0; v < 8; ++v)
        if (!((v >> J) & 1) && ((v >> C) & 1) == S) ap2(c, r[v], i[v], r[v | (1 << J)], i[v | (1 << J)]);
}
template <int C, int S> QI void g_lane(u64 (&r)[8], u64 (&i)[8], const u64 (&c)[12]) {
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if (C >= 0 && ((v >> C) & 1) != S) continue;
        float a0, a1, b0, b1;
        upk(r[v], a0, a1); upk(i[v], b0, b1);
        ap1(c, a0, b0, a1, b1);
        r[v] = pk(a0, a1); i[v] = pk(b0, b1);
    }
}
template <int J, int C> QI void x_op(u64 (&r)[8], u64 (&i)[8]) {
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if (J < 3) {
            if ((v >> J) & 1) continue;
            const int w = v | (1 << (J & 3));
            if (C == 3) {
                float a0, a1, b0, b1, c0, c1, d0, d1;
                upk(r[v], a0, a1); upk(i[v], b0, b1); upk(r[w], c0, c1); upk(i[w], d0, d1);
                r[v] = pk(a0, c1); i[v] = pk(b0, d1); r[w] = pk(c0, a1); i[w] = pk(d0, b1);
            } else {
                if (C >= 0 && !((v >> (C & 3)) & 1)) continue;
                const u64 tr = r[v], ti = i[v];
                r[v] = r[w]; i[v] = i[w]; r[w] = tr; i[w] = ti;
            }
        } else {
            if (C >= 0 && !((v >> (C & 3)) & 1)) continue;
            float a0, a1, b0, b1;
            upk(r[v], a0, a1); upk(i[v], b0, b1);
            r[v] = pk(a1, a0); i[v] = pk(b1, b0);
        }
    }
}
// diagonal: c[0..2] = d0, c[3..5] = d1 (lane-resolved by the host where lanes differ);
// J = 0..2 register target, 3 = lane target, 4 = uniform target given by t1
template <int J, int C, int S> QI void d_op(u64 (&r)[8], u64 (&i)[8], const u64 (&c)[12], bool t1) {
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if (!(C < 0 || C == 3 || ((v >> (C & 3)) & 1) == S)) continue;
        bool one;
        if (J == 4) one = t1; else if (J == 3) one = false; else one = ((v >> (J & 3)) & 1) != 0;
        if (one) cm2(c[3], c[4], c[5], r[v], i[v]); else cm2(c[0], c[1], c[2], r[v], i[v]);
    }
}

// adjoint: sum over the pairs along register bit J (with select bit C == S when
// C >= 0) of Re( conj(l) . (D x) ), x the psi pair, l the lambda pair (packed)
template <int J, int C, int S> QI float gd_reg(const u64 (&r)[8], const u64 (&i)[8], const u64 (&lr)[8],
                                               const u64 (&li)[8], const u64 (&d)[12]) {
    u64 acc = 0ull;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if ((v >> J) & 1) continue;
        if (C >= 0 && ((v >> C) & 1) != S) continue;
        const int w = v | (1 << J);
        u64 xr = r[v], xi = i[v], yr = r[w], yi = i[w];
        ap2(d, xr, xi, yr, yi);
        acc = f2fma(lr[v], xr, acc); acc = f2fma(li[v], xi, acc);
        acc = f2fma(lr[w], yr, acc); acc = f2fma(li[w], yi, acc);
    }
    float a0, a1; upk(acc, a0, a1); return a0 + a1;
}
// adjoint, generator form: the derivative term Re <lambda | dU psi'> of a gate
// U = exp(-i theta G / 2), psi' = U^dagger psi, equals Im <lambda | G psi> / 2 with psi
// before the gate is undone (GEN = 1, 2, 3: G = X, Y, Z); for P(theta) (GEN = 4,
// dP = i |1><1| P) it is -Im <lambda_1 | psi_1>. Sums over the pairs along
// register bit J (with select bit C == S when C >= 0); (a, b) = (bit 0, bit 1).
template <int J, int C, int S, int GEN> QI float gg_reg(const u64 (&r)[8], const u64 (&i)[8], const u64 (&lr)[8],
                                                        const u64 (&li)[8]) {
    u64 p = 0ull, m = 0ull;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if ((v >> J) & 1) continue;
        if (C >= 0 && ((v >> C) & 1) != S) continue;
        const int w = v | (1 << J);
        if (GEN == 1) {        // Im(conj(la) pb + conj(lb) pa)
            p = f2fma(lr[v], i[w], f2fma(lr[w], i[v], p));
            m = f2fma(li[v], r[w], f2fma(li[w], r[v], m));
        } else if (GEN == 2) { // Re(conj(lb) pa - conj(la) pb)
            p = f2fma(lr[w], r[v], f2fma(li[w], i[v], p));
            m = f2fma(lr[v], r[w], f2fma(li[v], i[w], m));
        } else if (GEN == 3) { // Im(conj(la) pa - conj(lb) pb)
            p = f2fma(lr[v], i[v], f2fma(li[w], r[w], p));
            m = f2fma(li[v], r[v], f2fma(lr[w], i[w], m));
        } else {               // -Im(conj(lb) pb)
            p = f2fma(li[w], r[w], p);
            m = f2fma(lr[w], i[w], m);
        }
    }
    float p0, p1, m0, m1;
    upk(p, p0, p1); upk(m, m0, m1);
    const float d = (p0 + p1) - (m0 + m1);
    return GEN == 4 ? d : 0.5f * d;
}
// real 2x2 (imaginary parts zero): (re, re) pairs of U00 U01 U10 U11 at c[0], c[3], c[6], c[9]
QI void ap2r(const u64 (&c)[12], u64 &ar, u64 &ai, u64 &br, u64 &bi) {
    const u64 xr = ar, xi = ai, yr = br, yi = bi;
    ar = f2fma(c[0], xr, f2mul(c[3], yr)); ai = f2fma(c[0], xi, f2mul(c[3], yi));
    br = f2fma(c[6], xr, f2mul(c[9], yr)); bi = f2fma(c[6], xi, f2mul(c[9], yi));
}
template <int J, int C, int S> QI void g_real(u64 (&r)[8], u64 (&i)[8], const u64 (&c)[12]) {
#pragma unroll
    for (int v = 0; v < 8; ++v)
        if (!((v >> J) & 1) && (C < 0 || ((v >> C) & 1) == S)) ap2r(c, r[v], i[v], r[v | (1 << J)], i[v | (1 << J)]);
}
template <int J, int C, int S> QI float gd_real(const u64 (&r)[8], const u64 (&i)[8], const u64 (&lr)[8],
                                                const u64 (&li)[8], const u64 (&d)[12]) {
    u64 acc = 0ull;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if ((v >> J) & 1) continue;
        if (C >= 0 && ((v >> C) & 1) != S) continue;
        const int w = v | (1 << J);
        u64 xr = r[v], xi = i[v], yr = r[w], yi = i[w];
        ap2r(d, xr, xi, yr, yi);
        acc = f2fma(lr[v], xr, acc); acc = f2fma(li[v], xi, acc);
        acc = f2fma(lr[w], yr, acc); acc = f2fma(li[w], yi, acc);
    }
    float a0, a1; upk(acc, a0, a1); return a0 + a1;
}
// diagonal 2x2 in the general layout: d0 = c[0..2] (U00), d1 = c[9..11] (U11)
template <int J, int C, int S> QI void g_diag(u64 (&r)[8], u64 (&i)[8], const u64 (&c)[12]) {
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if (C >= 0 && ((v >> C) & 1) != S) continue;
        if ((v >> J) & 1) cm2(c[9], c[10], c[11], r[v], i[v]); else cm2(c[0], c[1], c[2], r[v], i[v]);
    }
}
template <int J, int C, int S> QI float gd_diag(const u64 (&r)[8], const u64 (&i)[8], const u64 (&lr)[8],
                                                const u64 (&li)[8], const u64 (&d)[12]) {
    u64 acc = 0ull;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if (C >= 0 && ((v >> C) & 1) != S) continue;
        u64 xr = r[v], xi = i[v];
        if ((v >> J) & 1) cm2(d[9], d[10], d[11], xr, xi); else cm2(d[0], d[1], d[2], xr, xi);
        acc = f2fma(lr[v], xr, acc); acc = f2fma(li[v], xi, acc);
    }
    float a0, a1; upk(acc, a0, a1); return a0 + a1;
}
// the same for a target on the packed lane (tile qubit 0): scalar pairs
template <int C, int S> QI float gd_lane(const u64 (&r)[8], const u64 (&i)[8], const u64 (&lr)[8],
                                         const u64 (&li)[8], const u64 (&d)[12]) {
    float acc = 0.f;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if (C >= 0 && ((v >> C) & 1) != S) continue;
        float a0, a1, b0, b1, p0, p1, q0, q1;
        upk(r[v], a0, a1); upk(i[v], b0, b1);
        ap1(d, a0, b0, a1, b1);
        upk(lr[v], p0, p1); upk(li[v], q0, q1);
        acc += p0 * a0 + q0 * b0 + p1 * a1 + q1 * b1;
    }
    return acc;
}

// complex128, scalar slots m = 0..15; m8 = re, im of U00 U01 U10 U11
QI void ap1d(const double (&m)[8], double &ar, double &ai, double &br, double &bi) {
    const double xr = ar, xi = ai, yr = br, yi = bi;
    ar = m[0] * xr - m[1] * xi + m[2] * yr - m[3] * yi;
    ai = m[0] * xi + m[1] * xr + m[2] * yi + m[3] * yr;
    br = m[4] * xr - m[5] * xi + m[6] * yr - m[7] * yi;
    bi = m[4] * xi + m[5] * xr + m[6] * yi + m[7] * yr;
}
template <int J, int C, int S> QI void g_d(double (&r)[16], double (&i)[16], const double (&m)[8]) {
#pragma unroll
    for (int s = 0; s < 16; ++s)
        if (!((s >> J) & 1) && (C < 0 || ((s >> (C & 3)) & 1) == S)) ap1d(m, r[s], i[s], r[s | (1 << J)], i[s | (1 << J)]);
}
template <int J, int C> QI void x_d(double (&r)[16], double (&i)[16]) {
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        if (((s >> J) & 1) || (C >= 0 && !((s >> (C & 3)) & 1))) continue;
        const int w = s | (1 << J);
        const double tr = r[s], ti = i[s];
        r[s] = r[w]; i[s] = i[w]; r[w] = tr; i[w] = ti;
    }
}
template <int J, int C, int S> QI void d_d(double (&r)[16], double (&i)[16], const double (&m)[8], bool t1) {
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        if (!(C < 0 || ((s >> (C & 3)) & 1) == S)) continue;
        const bool one = J == 4 ? t1 : (((s >> (J & 3)) & 1) != 0);
        const double dr = one ? m[6] : m[0], di = one ? m[7] : m[1];
        const double xr = r[s];
        r[s] = dr * xr - di * i[s];
        i[s] = dr * i[s] + di * xr;
    }
}
)PRELUDE";

// ---------------------------------------------------------------- source generation
uint32_t swz8(uint32_t w) { return w ^ (((w >> 4) ^ (w >> 8)) & 15u); }
uint32_t swz16(uint32_t w) { return w ^ (((w >> 3) ^ (w >> 6) ^ (w >> 9)) & 7u); }

struct PassGeom {
    int k, nq, nh;
    const plan::Pass *p;
    uint64_t phys(uint32_t l) const
    {
        uint64_t g = l & ((1u << kChunkBits) - 1);
        for (int j = 0; j < nh; ++j)
            if ((l >> (kChunkBits + j)) & 1) g |= uint64_t(1) << p->s_high[j];
        return g;
    }
};

std::string hex64(uint64_t v)
{
    char b[32];
    snprintf(b, sizeof b, "0x%llxull", (unsigned long long)v);
    return b;
}
std::string hex32(uint32_t v)
{
    char b[32];
    snprintf(b, sizeof b, "0x%xu", v);
    return b;
}

// XOR over thread bits b of (bit b of tid ? mask[b] : 0)
std::string thread_expr(const std::vector<uint64_t> &mask, bool wide)
{
    std::string e = wide ? "0ull" : "0u";
    for (size_t b = 0; b < mask.size(); ++b) {
        if (!mask[b]) continue;
        if (wide)
            e += " ^ ((0ull - (u64)((tid >> " + std::to_string(b) + ") & 1u)) & " + hex64(mask[b]) + ")";
        else
            e += " ^ ((0u - ((tid >> " + std::to_string(b) + ") & 1u)) & " + hex32(uint32_t(mask[b])) + ")";
    }
    return "(" + e + ")";
}

std::string coef_load(int base, const std::string &sel, int n, bool dbl)
{
    std::ostringstream o;
    o << (dbl ? "double m[8];" : "u64 c[12];");
    for (int e = 0; e < n; ++e)
        o << (dbl ? " m[" : " c[") << e << "] = cf.c[" << base << " + " << (dbl ? 8 : 12) << " * (" << sel << ") + " << e
          << "];";
    return o.str();
}

// GEN2: (v_0..v_3) <- M4 (v_0..v_3) for the four packed vectors that differ
// in register bits A = treg, B = treg2, in both groups of the third bit E.
// Coefficients are read straight from the parameter bank.
void emit_gen2_c64(std::ostream &o, const plan::Op &op, int O)
{
    const int A = op.treg, B = op.treg2, E = 3 - A - B;
    auto C = [&](int j) { return "cf.c[" + std::to_string(O + j) + "]"; };
    for (int g = 0; g < 2; ++g) {
        int v[4];
        v[0] = g << E;
        v[1] = v[0] | (1 << A);
        v[2] = v[0] | (1 << B);
        v[3] = v[1] | (1 << B);
        o << "    {";
        for (int n = 0; n < 4; ++n) o << " const u64 xr" << n << " = r[" << v[n] << "], xi" << n << " = i[" << v[n] << "];";
        o << "\n";
        for (int m = 0; m < 4; ++m) {
            std::string er = "f2mul(" + C(3 * (4 * m)) + ", xr0)", ei = "f2mul(" + C(3 * (4 * m)) + ", xi0)";
            er = "f2fma(" + C(3 * (4 * m) + 2) + ", xi0, " + er + ")";
            ei = "f2fma(" + C(3 * (4 * m) + 1) + ", xr0, " + ei + ")";
            for (int n = 1; n < 4; ++n) {
                const int e = 4 * m + n;
                er = "f2fma(" + C(3 * e + 2) + ", xi" + std::to_string(n) + ", f2fma(" + C(3 * e) + ", xr" +
                     std::to_string(n) + ", " + er + "))";
                ei = "f2fma(" + C(3 * e + 1) + ", xr" + std::to_string(n) + ", f2fma(" + C(3 * e) + ", xi" +
                     std::to_string(n) + ", " + ei + "))";
            }
            o << "      r[" << v[m] << "] = " << er << ";\n      i[" << v[m] << "] = " << ei << ";\n";
        }
        o << "    }\n";
    }
}

// A diagonal op of +1 / -1 entries as sign-bit XORs (integer pipe, exact): the
// mask of register v has bit 31 set where lane 0 is negated and bit 63 where
// lane 1 is. Target bit b and select value s of each amplitude come from its
// register index (bits 0-2), its lane (bit 3: packed qubit), or a runtime
// expression (a thread bit or a qubit outside the tile).
void emit_sign_c64(std::ostream &o, const plan::Op &op, const std::string &sel)
{
    const int J = op.treg, C = op.sreg;
    const bool rs = C < 0 && (op.sthr || op.sext);  // runtime select
    const bool rt = J < 0;                           // runtime target bit
    const std::string t1 = rt ? "(((tid & " + hex32(op.tthr) + ") != 0u) | ((base & " + hex64(op.text) + ") != 0ull))"
                              : "false";
    auto mask = [&](int v, int s_rt, int b_rt) {
        uint64_t m = 0;
        for (int l = 0; l < 2; ++l) {
            const int b = rt ? b_rt : J == 3 ? l : (v >> J) & 1;
            const int s = C < 0 ? (rs ? s_rt : 0) : C == 3 ? l : (v >> C) & 1;
            if (op.M[s][b ? 3 : 0].real() < 0) m |= uint64_t(1) << (l ? 63 : 31);
        }
        return m;
    };
    o << "    { const int s = " << (rs ? sel : std::string("0")) << "; const bool tb = " << t1 << "; (void)s; (void)tb;\n";
    o << "      xs8(r, i";
    for (int v = 0; v < 8; ++v) {
        const uint64_t m00 = mask(v, 0, 0), m01 = mask(v, 0, 1), m10 = mask(v, 1, 0), m11 = mask(v, 1, 1);
        o << ", ";
        if (m00 == m01 && m00 == m10 && m00 == m11) o << hex64(m00);
        else
            o << "(s ? (tb ? " << hex64(m11) << " : " << hex64(m10) << ") : (tb ? " << hex64(m01) << " : "
              << hex64(m00) << "))";
    }
    o << ");\n    }\n";
}

void emit_op_c64(std::ostream &o, const plan::Op &op, int O)
{
    if (op.type == plan::OP_GEN2) {
        emit_gen2_c64(o, op, O);
        return;
    }
    const bool us = op.sthr || op.sext;
    const std::string sel =
        us ? "(((tid & " + hex32(op.sthr) + ") != 0u) | ((base & " + hex64(op.sext) + ") != 0ull))" : "0";
    const int J = op.treg, C = op.sreg;
    if (op.type == plan::OP_GEN) {
        if (C < 0) {
            o << "    { const int s = " << sel << "; if (s || " << (op.m0id ? 0 : 1) << ") { " << coef_load(O, "s", 12, false);
            o << (J < 3 ? " g_all<" + std::to_string(J) + ">(r, i, c);" : " g_lane<-1, 0>(r, i, c);") << " } }\n";
        } else if (C == 3) {
            o << "    { " << coef_load(O, "0", 12, false) << " g_all<" << J << ">(r, i, c); }\n";
        } else {
            for (int s = 0; s < 2; ++s) {
                if (s == 0 && op.m0id) continue;
                o << "    { " << coef_load(O, std::to_string(s), 12, false);
                if (J < 3) o << " g_sel<" << J << ", " << C << ", " << s << ">(r, i, c); }\n";
                else o << " g_lane<" << C << ", " << s << ">(r, i, c); }\n";
            }
        }
    } else if (op.type == plan::OP_X) {
        if (C < 0 && us && op.m0id) o << "    if (" << sel << ") x_op<" << J << ", -1>(r, i);\n";
        else o << "    x_op<" << J << ", " << C << ">(r, i);\n";
    } else if (plan::sign_only(op)) {
        emit_sign_c64(o, op, sel);
    } else {
        const int Jd = J >= 0 ? J : 4;
        const std::string t1 = Jd == 4 ? "(((tid & " + hex32(op.tthr) + ") != 0u) | ((base & " + hex64(op.text) +
                                             ") != 0ull))"
                                       : "false";
        if (C < 0) {
            o << "    { const int s = " << sel << "; if (s || " << (op.m0id ? 0 : 1) << ") { " << coef_load(O, "s", 6, false)
              << " d_op<" << Jd << ", -1, 0>(r, i, c, " << t1 << "); } }\n";
        } else if (C == 3) {
            o << "    { " << coef_load(O, "0", 6, false) << " d_op<" << Jd << ", 3, 0>(r, i, c, " << t1 << "); }\n";
        } else {
            for (int s = 0; s < 2; ++s) {
                if (s == 0 && op.m0id) continue;
                o << "    { " << coef_load(O, std::to_string(s), 6, false) << " d_op<" << Jd << ", " << C << ", " << s
                  << ">(r, i, c, " << t1 << "); }\n";
            }
        }
    }
}

void emit_op_c128(std::ostream &o, const plan::Op &op, int k)
{
    const int O = 16 * k;
    const bool us = op.sthr || op.sext;
    const std::string sel =
        us ? "(((tid & " + hex32(op.sthr) + ") != 0u) | ((base & " + hex64(op.sext) + ") != 0ull))" : "0";
    const int J = op.treg, C = op.sreg;
    if (op.type == plan::OP_X) {
        if (C < 0 && us && op.m0id) o << "    if (" << sel << ") x_d<" << J << ", -1>(r, i);\n";
        else o << "    x_d<" << J << ", " << C << ">(r, i);\n";
        return;
    }
    const bool diag = op.type == plan::OP_DIAG;
    const int Jd = diag && J < 0 ? 4 : J;
    const std::string t1 = Jd == 4 ? "(((tid & " + hex32(op.tthr) + ") != 0u) | ((base & " + hex64(op.text) +
                                         ") != 0ull))"
                                   : "false";
    auto call = [&](int c, int s) {
        std::ostringstream x;
        if (diag) x << " d_d<" << Jd << ", " << c << ", " << s << ">(r, i, m, " << t1 << ");";
        else x << " g_d<" << J << ", " << c << ", " << s << ">(r, i, m);";
        return x.str();
    };
    if (C < 0) {
        o << "    { const int s = " << sel << "; if (s || " << (op.m0id ? 0 : 1) << ") { " << coef_load(O, "s", 8, true)
          << call(-1, 0) << " } }\n";
    } else {
        for (int s = 0; s < 2; ++s) {
            if (s == 0 && op.m0id) continue;
            o << "    { " << coef_load(O, std::to_string(s), 8, true) << call(C, s) << " }\n";
        }
    }
}

// CTAs per SM the compiled pass is built for (its register budget). The
// complex64 pass holds the next tile's loads in registers while it computes
// the current one, which needs 128 registers: measured on the 30-qubit random
// circuit, K = 12 at 2 CTAs per SM runs 292 ms (3: 326 ms, spilling), K = 11
// at 4 runs 285 ms (5: 305, 6: 322), K = 10 at 8 runs 288 ms (12: 317).
int min_blocks(bool c64, int k) { return k == 12 ? (c64 ? 2 : 1) : k == 11 ? (c64 ? 4 : 2) : (c64 ? 8 : 2); }
// The same for complex64 tile code without the register-held next tile (the
// batch kernel): 80 registers, 3 / 6 / 12 CTAs per SM.
int min_blocks_unpipelined(int k) { return k == 12 ? 3 : k == 11 ? 6 : 12; }

// Thread-invariant offsets of a pass: global offsets of the load and store
// layouts and the shared-memory word offsets of every transpose.
void emit_pass_consts(std::ostream &o, const plan::Pass &p, bool c64)
{
    PassGeom G{p.k, p.k - kRegBits, p.k - kChunkBits, &p};
    auto phys_mask = [&](const int8_t *Q) {
        std::vector<uint64_t> m(G.nq);
        for (int b = 0; b < G.nq; ++b) m[b] = G.phys(1u << Q[b]);
        return m;
    };
    auto word_mask = [&](const int8_t *Q) {
        std::vector<uint64_t> m(G.nq);
        for (int b = 0; b < G.nq; ++b) m[b] = c64 ? swz8((1u << Q[b]) >> 1) : swz16(1u << Q[b]);
        return m;
    };
    const plan::Stage &s0 = p.stages.front(), &sl = p.stages.back();
    o << "    const u64 gL = " << thread_expr(phys_mask(s0.in.Q), true) << ";\n";
    o << "    const u64 gS = " << thread_expr(phys_mask(sl.out.Q), true) << ";\n";
    for (size_t s = 1; s < p.stages.size(); ++s) {
        o << "    const u32 wW" << s << " = " << thread_expr(word_mask(p.stages[s - 1].out.Q), false) << ";\n";
        o << "    const u32 wR" << s << " = " << thread_expr(word_mask(p.stages[s].in.Q), false) << ";\n";
    }
}

// One tile of a pass (tile index t): base index, load, stages with their
// transposes and ops, store. Coefficients are read as cf.c[...]; with
// l2_loads the tile is read through L2 only (other CTAs may have written it
// since this SM last cached it).
// Tile base index of tile expression `t` (the bits outside the tile).
std::string tile_base_expr(const plan::Pass &p, const std::string &t)
{
    std::string e = "0ull";
    for (int s = 0; s < p.nseg; ++s)
        e += " | (((" + t + " >> " + std::to_string(p.seg_src[s]) + ") & " +
             hex64((uint64_t(1) << p.seg_w[s]) - 1) + ") << " + std::to_string(p.seg_dst[s]) + ")";
    return e;
}

void emit_tile_body(std::ostream &o, const plan::Pass &p, bool c64, bool l2_loads, bool pipelined = false)
{
    PassGeom G{p.k, p.k - kRegBits, p.k - kChunkBits, &p};
    const int nops = int(p.ops.size());
    std::vector<int> coff(nops + 1, 0);  // coefficient offset of each op
    for (int k = 0; k < nops; ++k) coff[k + 1] = coff[k] + (c64 ? coef_slots_c64(p.ops[k]) : 16);
    const int nreg = c64 ? 3 : 4;  // register bits addressed per vector/slot (c64: bit 3 is the lane)
    const int nvec = 1 << nreg;
    const plan::Stage &s0 = p.stages.front(), &sl = p.stages.back();
    const std::string ld0 = l2_loads ? "__ldcg(" : "*", ld1 = l2_loads ? ")" : "";
    o << "    const u64 base = 0ull";
    for (int s = 0; s < p.nseg; ++s)
        o << " | (((t >> " << p.seg_src[s] << ") & " << hex64((uint64_t(1) << p.seg_w[s]) - 1) << ") << "
          << p.seg_dst[s] << ")";
    o << ";\n";
    auto reg_offset = [&](const int8_t *P, int v) {
        uint32_t l = 0;
        for (int j = 0; j < nreg; ++j)
            if ((v >> j) & 1) l |= 1u << P[j];
        return l;
    };
    if (c64 && pipelined) {
        // this tile was loaded during the previous one; start loading the next
        o << "    u64 r[8], i[8];\n";
        for (int v = 0; v < 8; ++v)
            o << "    r[" << v << "] = pk(nf" << v << ".x, nf" << v << ".z); i[" << v << "] = pk(nf" << v << ".y, nf" << v
              << ".w);\n";
        o << "    { const u64 tn = t + gridDim.x;\n";
        o << "      if (tn < ntiles) { const float *a = amp + 2 * ((" << tile_base_expr(p, "tn") << ") + gL);\n";
        for (int v = 0; v < 8; ++v)
            o << "        nf" << v << " = *reinterpret_cast<const float4 *>(a + 2 * " << hex64(G.phys(reg_offset(s0.in.P, v)))
              << ");\n";
        o << "      }\n    }\n";
    } else if (c64) {
        o << "    u64 r[8], i[8];\n";
        o << "    { const float *a = amp + 2 * (base + gL);\n";
        for (int v = 0; v < 8; ++v)
            o << "      const float4 f" << v << " = " << ld0 << "reinterpret_cast<const float4 *>(a + 2 * "
              << hex64(G.phys(reg_offset(s0.in.P, v))) << ")" << ld1 << ";\n";
        for (int v = 0; v < 8; ++v)
            o << "      r[" << v << "] = pk(f" << v << ".x, f" << v << ".z); i[" << v << "] = pk(f" << v << ".y, f" << v
              << ".w);\n";
        o << "    }\n";
    } else {
        o << "    double r[16], i[16];\n";
        o << "    { const double2 *a = reinterpret_cast<const double2 *>(amp) + (base + gL);\n";
        for (int m = 0; m < 16; ++m)
            o << "      const double2 f" << m << " = " << ld0 << "(a + " << hex64(G.phys(reg_offset(s0.in.P, m))) << ")"
              << ld1 << ";\n";
        for (int m = 0; m < 16; ++m) o << "      r[" << m << "] = f" << m << ".x; i[" << m << "] = f" << m << ".y;\n";
        o << "    }\n";
    }
    for (size_t s = 0; s < p.stages.size(); ++s) {
        const plan::Stage &st = p.stages[s];
        if (s > 0) {
            const plan::Stage &pr = p.stages[s - 1];
            if (c64) {
                o << "    { u64 *pre = sm, *pim = sm + " << (1 << (p.k - 1)) << ";\n";
                for (int v = 0; v < nvec; ++v) {
                    const uint32_t w = swz8(reg_offset(pr.out.P, v) >> 1);
                    o << "      pre[wW" << s << " ^ " << hex32(w) << "] = r[" << v << "]; pim[wW" << s << " ^ " << hex32(w)
                      << "] = i[" << v << "];\n";
                }
                o << "      __syncthreads();\n";
                for (int v = 0; v < nvec; ++v) {
                    const uint32_t w = swz8(reg_offset(st.in.P, v) >> 1);
                    o << "      r[" << v << "] = pre[wR" << s << " ^ " << hex32(w) << "]; i[" << v << "] = pim[wR" << s
                      << " ^ " << hex32(w) << "];\n";
                }
                o << "      __syncthreads(); }\n";
            } else {
                o << "    { double2 *tl = reinterpret_cast<double2 *>(sm);\n";
                for (int v = 0; v < nvec; ++v) {
                    const uint32_t w = swz16(reg_offset(pr.out.P, v));
                    o << "      tl[wW" << s << " ^ " << hex32(w) << "] = make_double2(r[" << v << "], i[" << v << "]);\n";
                }
                o << "      __syncthreads();\n";
                for (int v = 0; v < nvec; ++v) {
                    const uint32_t w = swz16(reg_offset(st.in.P, v));
                    o << "      { const double2 q = tl[wR" << s << " ^ " << hex32(w) << "]; r[" << v << "] = q.x; i[" << v
                      << "] = q.y; }\n";
                }
                o << "      __syncthreads(); }\n";
            }
        }
        for (int k = st.op_begin; k < st.op_end; ++k) {
            if (c64) emit_op_c64(o, p.ops[k], coff[k]);
            else emit_op_c128(o, p.ops[k], k);
        }
    }
    // With one stage no transpose (and its barrier) separates the loads from the
    // stores; when SWAP relabels changed the layout, a warp may store into
    // positions another warp has not loaded yet.
    if (p.stages.size() == 1 && std::memcmp(&s0.in, &sl.out, sizeof(plan::Layout)) != 0) o << "    __syncthreads();\n";
    if (c64) {
        o << "    { float *a = amp + 2 * (base + gS); float x0, x1, y0, y1;\n";
        for (int v = 0; v < 8; ++v)
            o << "      upk(r[" << v << "], x0, x1); upk(i[" << v << "], y0, y1); *reinterpret_cast<float4 *>(a + 2 * "
              << hex64(G.phys(reg_offset(sl.out.P, v))) << ") = make_float4(x0, y0, x1, y1);\n";
        o << "    }\n";
    } else {
        o << "    { double2 *a = reinterpret_cast<double2 *>(amp) + (base + gS);\n";
        for (int m = 0; m < 16; ++m)
            o << "      a[" << hex64(G.phys(reg_offset(sl.out.P, m))) << "] = make_double2(r[" << m << "], i[" << m
              << "]);\n";
        o << "    }\n";
    }
}

// ---------------------------------------------------------------- tensor-core passes (complex64)
// A pass of a tensor-core plan: every stage multiplies the 16 amplitudes a
// thread holds (its four register positions) by the stage's 16x16 complex
// matrix on the tensor cores. Thread t of the tile is row t of an M = 128
// product (two products for 2^12 tiles): the row's 32 real components (16 re,
// 16 im) are the A operand, written to tensor memory with tcgen05.st; the
// matrix in real form [[Re, -Im], [Im, Re]] (32 x 32, K-major) is the B operand
// in shared memory; the 32 outputs land in tensor memory and return to the
// thread with tcgen05.ld. TF32 keeps 11 significant bits, so each operand is
// split into a TF32 head and a TF32 tail (x = hi + lo) and the product is
// hi*hi + lo*hi + hi*lo, accumulated in FP32 (the lo*lo term is below FP32
// rounding). Between stages the tile moves through shared memory (one 8-byte
// word per amplitude, swizzled) into the next stage's layout.

const char *kPreludeTc = R"PRELUDE(
typedef unsigned long long u64;
typedef unsigned int u32;
#define QI __device__ __forceinline__
QI u32 smem_u32(const void *p) { return (u32)__cvta_generic_to_shared(p); }
QI float tf32r(float x) { u32 r; asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x)); return __uint_as_float(r); }
// K-major operand without swizzle: 8-row x 16-byte core matrices, 1024 bytes
// between core matrices along K (64 rows of N), 128 bytes between them along N
QI u64 bdesc(u32 addr) { return (u64)((addr >> 4) & 0x3FFFu) | ((u64)(1024u >> 4) << 16) | ((u64)(128u >> 4) << 32) | ((u64)1 << 46); }
#define R16(v) "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), \
    "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), \
    "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])), \
    "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
QI void tst16(u32 ta, const float (&v)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(ta), R16(v) : "memory");
}
QI void tld32(u32 ta, float (&a)[16], float (&b)[16]) {
    u32 r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(ta) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) { a[j] = __uint_as_float(r[j]); b[j] = __uint_as_float(r[16 + j]); }
}
QI void tld16(u32 ta, u32 (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(ta) : "memory");
}
// x[j] = D[:, c + j] + D[:, c + 32 + j] (head products + products with the matrix tails)
QI void tld_pair(u32 ta, float (&x)[16]) {
    u32 p[16], q[16];
    tld16(ta, p);
    tld16(ta + 32u, q);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = __uint_as_float(p[j]) + __uint_as_float(q[j]);
}
QI void tld_sum(u32 ta, float (&a)[16], float (&b)[16]) {
    tld_pair(ta, a);
    tld_pair(ta + 16u, b);
}
QI void tst8(u32 ta, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                    "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                    "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])) : "memory");
}
// the 16 values as TF32 heads at column ta and tails at column ta + lo (this warp's lanes), 8 at a time
QI void put_split(u32 ta, u32 lo, const float (&x)[16]) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float h[8], l[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) { h[j] = tf32r(x[8 * c + j]); l[j] = tf32r(x[8 * c + j] - h[j]); }
        tst8(ta + 8u * c, h);
        tst8(ta + lo + 8u * c, l);
    }
}
// thread index read afresh (keeps per-stage offsets from being hoisted into registers)
QI u32 tid_now() { u32 t; asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t)); return t; }
QI void mma_tf32(u32 d, u32 a, u64 b, u32 idesc, u32 acc) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, q;\n\t}"
                 :: "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
// sum of v over the CTA (nw warps), every thread gets it; red: nw floats of shared memory
QI float cta_sum(float v, float *red, u32 tid, u32 nw) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((tid & 31u) == 0) red[tid >> 5] = v;
    __syncthreads();
    float s = 0.f;
    for (u32 w = 0; w < nw; ++w) s += red[w];
    return s;
}
// bounded wait for the completion of mbarrier phase `parity`
QI bool mbar_wait(u32 bar, u32 parity, u32 limit) {
    for (u32 it = 0; it < limit; ++it) {
        u32 ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}
)PRELUDE";

uint32_t swz_tc(uint32_t l) { return l ^ (((l >> 4) ^ (l >> 8)) & 15u); }

// Dynamic shared memory of a tensor-core pass: the transpose words, then 8 KB
// per matrix slot; at least enough that no more CTAs fit on an SM than tensor
// memory serves (512 columns: four CTAs of 2^11 tiles, two of 2^12).
size_t tc_smem(const plan::Pass &p)
{
    const size_t need = (size_t(8) << p.k) + (p.tcm.size() / plan::kTcSlot) * 8192;
    const size_t floor_bytes = p.k == 12 ? 78848 : 47104;
    return std::max(need, floor_bytes);
}
int tc_cols(int k) { return k == 12 ? 256 : 128; }

// Host packing of a pass's matrix slots: per slot one 64 x 32 K-major operand,
// rows n < 32 the TF32 heads and rows 32 + n the tails of row n of the real form
// [[Re, -Im], [Im, Re]] (element (n, kk) at byte (kk/4)*1024 + (n/8)*128 +
// (n%8)*16 + (kk%4)*4). One product with N = 64 gives heads and tails of the
// matrix at once; a product with N = 32 reads the heads alone.
float tf32_round_host(float f)
{
    uint32_t b;
    std::memcpy(&b, &f, 4);
    if ((b & 0x7F800000u) != 0x7F800000u) b = (b + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

void pack_tc_mats(const plan::Pass &p, std::vector<float> &out)
{
    const size_t nslot = p.tcm.size() / plan::kTcSlot;
    out.assign(nslot * 2048, 0.f);
    auto at = [](int n, int kk) { return size_t((kk / 4) * 256 + (n / 8) * 32 + (n % 8) * 4 + (kk % 4)); };
    for (size_t sl = 0; sl < nslot; ++sl) {
        const cd *G = p.tcm.data() + sl * plan::kTcSlot;
        float *B = out.data() + sl * 2048;
        for (int n = 0; n < 32; ++n)
            for (int kk = 0; kk < 32; ++kk) {
                const cd z = G[16 * (n & 15) + (kk & 15)];
                const double x = (n < 16) == (kk < 16) ? z.real() : (n < 16 ? -z.imag() : z.imag());
                const float h = tf32_round_host(float(x));
                const float l = tf32_round_host(float(x - double(h)));
                B[at(n, kk)] = h;
                B[at(32 + n, kk)] = l;
            }
    }
}

std::string gen_source_tc(const plan::Pass &p)
{
    const int K = p.k, T = 1 << (K - kRegBits), NG = T / 128, NQ = K - kRegBits;
    PassGeom G{K, NQ, K - kChunkBits, &p};
    const int cols = tc_cols(K);
    auto col_hi = [&](int g) { return 32 * g; };
    auto col_d = [&](int g) { return 64 * NG + 64 * g; };
    auto reg_off = [&](const int8_t *P, int j) {
        uint32_t l = 0;
        for (int b = 0; b < kRegBits; ++b)
            if ((j >> b) & 1) l |= 1u << P[b];
        return l;
    };
    auto phys_mask = [&](const int8_t *Q) {
        std::vector<uint64_t> m(NQ);
        for (int b = 0; b < NQ; ++b) m[b] = G.phys(1u << Q[b]);
        return m;
    };
    auto word_mask = [&](const int8_t *Q) {
        std::vector<uint64_t> m(NQ);
        for (int b = 0; b < NQ; ++b) m[b] = swz_tc(1u << Q[b]);
        return m;
    };
    const plan::Stage &s0 = p.stages.front(), &sl = p.stages.back();
    const int nslot = int(p.tcm.size() / plan::kTcSlot);
    // instruction descriptors: D FP32, A and B TF32, both K-major, M = 128, N = 64 / 32
    const uint32_t idesc64 = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t idesc32 = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    std::ostringstream o;
    o << kPreludeTc;
    o << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << (K == 12 ? 2 : 4)
      << ") qv_tc(float2 *__restrict__ amp, u64 ntiles, const float4 *__restrict__ mats, int *status, u32 spin)\n{\n";
    o << "    extern __shared__ __align__(1024) unsigned char smx[];\n";
    o << "    __shared__ __align__(8) u64 mbar;\n    __shared__ u32 tslot;\n    __shared__ int s_abort;\n";
    if (p.tc_unitary) o << "    __shared__ float red[2][" << T / 32 << "];\n";
    o << "    float2 *tw = reinterpret_cast<float2 *>(smx);\n";
    o << "    const u32 mb = smem_u32(smx + " << (8 << K) << ");\n";
    o << "    const u32 tid = threadIdx.x, warp = tid >> 5;\n";
    o << "    if (warp == 0) {\n"
         "        asm volatile(\"tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\" :: \"r\"(smem_u32(&tslot)), \"r\"("
      << cols << ") : \"memory\");\n"
         "        asm volatile(\"tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\" ::: \"memory\");\n    }\n";
    o << "    if (tid == 0) {\n"
         "        asm volatile(\"mbarrier.init.shared::cta.b64 [%0], 1;\" :: \"r\"(smem_u32(&mbar)) : \"memory\");\n"
         "        asm volatile(\"fence.mbarrier_init.release.cluster;\" ::: \"memory\");\n"
         "        s_abort = 0;\n    }\n";
    o << "    for (u32 i = tid; i < " << nslot * 512 << "u; i += " << T
      << "u) reinterpret_cast<float4 *>(smx + " << (8 << K) << ")[i] = __ldg(mats + i);\n";
    o << "    asm volatile(\"fence.proxy.async.shared::cta;\" ::: \"memory\");\n";
    o << "    asm volatile(\"tcgen05.fence::before_thread_sync;\" ::: \"memory\");\n    __syncthreads();\n";
    o << "    asm volatile(\"tcgen05.fence::after_thread_sync;\" ::: \"memory\");\n";
    o << "    const u32 tm = tslot, bar = smem_u32(&mbar);\n";
    o << "    const u32 lb = ((warp & 3u) * 32u) << 16, grp = warp >> 2;\n";
    o << "    const u32 ahi = tm + lb + 32u * grp, dcol = tm + lb + " << col_d(0) << "u + 64u * grp;\n";
    o << "    u32 phase = 0;\n";
    o << "    const u64 gL = " << thread_expr(phys_mask(s0.in.Q), true) << ";\n";
    o << "    const u64 gS = " << thread_expr(phys_mask(sl.out.Q), true) << ";\n";
    o << "    float2 nx[16];\n";
    o << "    if (blockIdx.x < ntiles) { const float2 *a = amp + ((" << tile_base_expr(p, "(u64)blockIdx.x") << ") + gL);\n";
    for (int j = 0; j < 16; ++j) o << "      nx[" << j << "] = a[" << hex64(G.phys(reg_off(s0.in.P, j))) << "];\n";
    o << "    }\n";
    o << "    for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {\n";
    o << "    const u64 base = " << tile_base_expr(p, "t") << ";\n";
    o << "    float re[16], im[16];\n";
    o << "#pragma unroll\n    for (int j = 0; j < 16; ++j) { re[j] = nx[j].x; im[j] = nx[j].y; }\n";
    if (p.tc_unitary) {
        o << "    float nin = 0.f;\n";
        o << "#pragma unroll\n    for (int j = 0; j < 16; ++j) nin = fmaf(re[j], re[j], fmaf(im[j], im[j], nin));\n";
    }
    o << "    { const u64 tn = t + gridDim.x;\n";
    o << "      if (tn < ntiles) { const float2 *a = amp + ((" << tile_base_expr(p, "tn") << ") + gL);\n";
    for (int j = 0; j < 16; ++j) o << "        nx[" << j << "] = a[" << hex64(G.phys(reg_off(s0.in.P, j))) << "];\n";
    o << "      }\n    }\n";
    for (size_t s = 0; s < p.stages.size(); ++s) {
        const plan::Stage &st = p.stages[s];
        if (s > 0) {
            const plan::Stage &pr = p.stages[s - 1];
            o << "    {\n";
            {
                std::string wW = thread_expr(word_mask(pr.out.Q), false), wR = thread_expr(word_mask(st.in.Q), false);
                for (std::string *e : {&wW, &wR})
                    for (size_t q = e->find("tid"); q != std::string::npos; q = e->find("tid", q + 2)) e->replace(q, 3, "tn");
                o << "      u32 tn = tid_now(); const u32 wW" << s << " = " << wW << ";\n";
                o << "      tn = tid_now(); const u32 wR" << s << " = " << wR << ";\n";
            }
            for (int j = 0; j < 16; ++j)
                o << "      tw[wW" << s << " ^ " << hex32(swz_tc(reg_off(pr.out.P, j))) << "] = make_float2(re[" << j
                  << "], im[" << j << "]);\n";
            o << "      __syncthreads();\n";
            for (int j = 0; j < 16; ++j)
                o << "      { const float2 w = tw[wR" << s << " ^ " << hex32(swz_tc(reg_off(st.in.P, j))) << "]; re[" << j
                  << "] = w.x; im[" << j << "] = w.y; }\n";
            if (st.mat < 0) o << "      __syncthreads();\n";
            o << "    }\n";
        }
        if (st.mat < 0) continue;
        o << "    {\n";
        o << "      put_split(ahi, " << 32 * NG << "u, re);\n      put_split(ahi + 16u, " << 32 * NG << "u, im);\n";
        o << "      asm volatile(\"tcgen05.wait::st.sync.aligned;\" ::: \"memory\");\n";
        o << "      asm volatile(\"tcgen05.fence::before_thread_sync;\" ::: \"memory\");\n";
        o << "      __syncthreads();\n";
        o << "      if (s_abort) goto done;\n";
        o << "      if (tid == 0) {\n";
        o << "        asm volatile(\"tcgen05.fence::after_thread_sync;\" ::: \"memory\");\n";
        if (st.ext >= 0)
            o << "        const u32 slot = " << st.mat << "u + (u32)((base >> " << st.ext << ") & 1ull);\n";
        else
            o << "        const u32 slot = " << st.mat << "u;\n";
        o << "        const u32 bm = mb + slot * 8192u;\n";
        // D[:, 0:64] = A_hi [B_hi | B_lo], then D[:, 0:32] += A_lo B_hi
        for (int g = 0; g < NG; ++g)
            for (int pr = 0; pr < 2; ++pr)
                for (int ks = 0; ks < 4; ++ks) {
                    const int acol = col_hi(g) + (pr == 1 ? 32 * NG : 0) + 8 * ks;
                    o << "        mma_tf32(tm + " << col_d(g) << "u, tm + " << acol << "u, bdesc(bm + " << 2048 * ks << "u), "
                      << hex32(pr == 0 ? idesc64 : idesc32) << ", " << ((pr | ks) ? 1 : 0) << "u);\n";
                }
        o << "        asm volatile(\"tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\" :: \"r\"(bar) : \"memory\");\n";
        o << "      }\n";
        o << "      if (!mbar_wait(bar, phase, spin)) { s_abort = 1; atomicCAS(status, 0, 4); }\n";
        o << "      phase ^= 1u;\n";
        o << "      asm volatile(\"tcgen05.fence::after_thread_sync;\" ::: \"memory\");\n";
        o << "      tld_sum(dcol, re, im);\n";
        o << "    }\n";
    }
    if (p.tc_unitary) {
        // The pass is a unitary acting inside each tile, so the tile keeps its
        // norm; the tensor cores truncate their FP32 sums, which shrinks every
        // stage's output by a few units in the last place. Rescaling the tile to
        // its input norm removes that systematic part of the rounding error.
        o << "    {\n";
        o << "      float nout = 0.f;\n";
        o << "#pragma unroll\n      for (int j = 0; j < 16; ++j) nout = fmaf(re[j], re[j], fmaf(im[j], im[j], nout));\n";
        o << "      const float si = cta_sum(nin, red[0], tid, " << T / 32 << "u), so = cta_sum(nout, red[1], tid, " << T / 32
          << "u);\n";
        o << "      const float f = so > 0.f ? sqrtf(si / so) : 1.f;\n";
        o << "#pragma unroll\n      for (int j = 0; j < 16; ++j) { re[j] *= f; im[j] *= f; }\n";
        o << "    }\n";
    }
    o << "    { float2 *a = amp + (base + gS);\n";
    for (int j = 0; j < 16; ++j)
        o << "      a[" << hex64(G.phys(reg_off(sl.out.P, j))) << "] = make_float2(re[" << j << "], im[" << j << "]);\n";
    o << "    }\n";
    o << "    }\n";
    o << "done:\n";
    o << "    asm volatile(\"tcgen05.fence::before_thread_sync;\" ::: \"memory\");\n    __syncthreads();\n";
    o << "    if (warp == 0) asm volatile(\"tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\" :: \"r\"(tm), \"r\"(" << cols
      << ") : \"memory\");\n";
    o << "}\n";
    return o.str();
}

std::string gen_source(const plan::Pass &p, bool c64)
{
    PassGeom G{p.k, p.k - kRegBits, p.k - kChunkBits, &p};
    const int T = 1 << G.nq;
    const int nops = int(p.ops.size());
    int ncoef = 0;
    for (int k = 0; k < nops; ++k) ncoef += c64 ? coef_slots_c64(p.ops[k]) : 16;
    ncoef = std::max(1, ncoef);
    std::ostringstream o;
    o << kPrelude;
    o << "struct QvCoef { " << (c64 ? "u64" : "double") << " c[" << ncoef << "]; };\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << min_blocks(c64, p.k) << ") qv_pass("
      << (c64 ? "float" : "double") << " *__restrict__ amp, u64 ntiles, const QvCoef cf)\n{\n";
    o << "    extern __shared__ __align__(16) u64 sm[];\n";
    o << "    const u32 tid = threadIdx.x;\n";
    emit_pass_consts(o, p, c64);
    const bool pipe = c64;
    if (pipe) {  // prologue: the first tile's loads
        const plan::Stage &s0 = p.stages.front();
        PassGeom G{p.k, p.k - kRegBits, p.k - kChunkBits, &p};
        o << "    float4 nf0, nf1, nf2, nf3, nf4, nf5, nf6, nf7;\n";
        o << "    if (blockIdx.x < ntiles) { const float *a = amp + 2 * ((" << tile_base_expr(p, "(u64)blockIdx.x")
          << ") + gL);\n";
        for (int v = 0; v < 8; ++v) {
            uint32_t l = 0;
            for (int j = 0; j < 3; ++j)
                if ((v >> j) & 1) l |= 1u << s0.in.P[j];
            o << "      nf" << v << " = *reinterpret_cast<const float4 *>(a + 2 * " << hex64(G.phys(l)) << ");\n";
        }
        o << "    }\n";
    }
    o << "    for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {\n";
    emit_tile_body(o, p, c64, false, pipe);
    o << "    }\n}\n";
    return o.str();
}

// ---------------------------------------------------------------- batched passes (complex64)
// Many circuits that share one plan structure (same passes, layouts and op
// kinds; only the coefficients differ), as one persistent kernel: CTAs claim
// work items (circuit, pass, chunk of tiles) from a counter, wait (bounded)
// until the previous pass of that circuit is complete, and run the pass's
// compiled tile code with that circuit's coefficients from global memory.

bool same_structure(const plan::Pass &a, const plan::Pass &b)
{
    if (a.k != b.k || a.nseg != b.nseg || a.stages.size() != b.stages.size() || a.ops.size() != b.ops.size())
        return false;
    for (int j = 0; j < a.k - kChunkBits; ++j)
        if (a.s_high[j] != b.s_high[j]) return false;
    for (int q = 0; q < a.nseg; ++q)
        if (a.seg_src[q] != b.seg_src[q] || a.seg_w[q] != b.seg_w[q] || a.seg_dst[q] != b.seg_dst[q]) return false;
    for (size_t s = 0; s < a.stages.size(); ++s)
        if (std::memcmp(&a.stages[s], &b.stages[s], sizeof(plan::Stage)) != 0) return false;
    for (size_t k = 0; k < a.ops.size(); ++k) {
        const plan::Op &x = a.ops[k], &y = b.ops[k];
        if (x.type != y.type || x.treg != y.treg || x.treg2 != y.treg2 || x.sreg != y.sreg || x.m0id != y.m0id ||
            x.sthr != y.sthr || x.tthr != y.tthr || x.sext != y.sext || x.text != y.text || x.nd != y.nd)
            return false;
    }
    return true;
}

std::string gen_source_batch(const std::vector<plan::Pass> &passes, int stride, int chunk_tiles)
{
    const int k = passes.front().k;
    const int T = 1 << (k - kRegBits);
    const int np = int(passes.size());
    std::ostringstream o;
    o << kPrelude;
    o << "QI u32 ld_acq(const unsigned *p) { u32 v; asm volatile(\"ld.acquire.gpu.global.u32 %0, [%1];\" : \"=r\"(v) : \"l\"(p) : \"memory\"); return v; }\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << min_blocks_unpipelined(k)
      << ") qv_batch(float *const *amps, const u64 *__restrict__ coefs, const uint2 *__restrict__ items, u32 nitems, "
         "unsigned *next, unsigned *done, int *status, u64 ntiles, u32 nchunks, u32 spin_limit)\n{\n";
    o << "    extern __shared__ __align__(16) u64 sm[];\n";
    o << "    __shared__ u32 s_item; __shared__ int s_abort;\n";
    o << "    const u32 tid = threadIdx.x;\n";
    o << "    for (;;) {\n";
    o << "    if (tid == 0) { s_item = atomicAdd(next, 1u); s_abort = 0; }\n";
    o << "    __syncthreads();\n";
    o << "    const u32 item = s_item;\n";
    o << "    if (item >= nitems) break;\n";
    o << "    const uint2 it = items[item];  // x = circuit * passes + pass, y = chunk\n";
    o << "    const u32 pass = it.x % " << np << "u, circ = it.x / " << np << "u;\n";
    o << "    if (tid == 0 && pass > 0) {  // bounded wait for the previous pass of this circuit\n";
    o << "        u32 spins = 0;\n";
    o << "        while (ld_acq(&done[it.x - 1]) < nchunks) {\n";
    o << "            if (++spins > spin_limit || *reinterpret_cast<volatile int *>(status) != 0) {\n";
    o << "                atomicCAS(status, 0, 4); s_abort = 1; break; }\n";
    o << "            __nanosleep(128);\n";
    o << "        }\n";
    o << "    }\n";
    o << "    __syncthreads();\n";
    o << "    if (s_abort) break;\n";
    o << "    float *amp = amps[circ];\n";
    o << "    const u64 *cf = coefs + (size_t)it.x * " << stride << "u;\n";
    o << "    const u64 t0 = (u64)it.y * " << chunk_tiles << "u, t1 = min(ntiles, t0 + " << chunk_tiles << "u);\n";
    o << "    switch (pass) {\n";
    for (int p = 0; p < np; ++p) {
        o << "    case " << p << ": {\n";
        emit_pass_consts(o, passes[p], true);
        o << "    for (u64 t = t0; t < t1; ++t) {\n";
        std::ostringstream body;
        emit_tile_body(body, passes[p], true, true);
        std::string bs = body.str();
        for (size_t q = bs.find("cf.c["); q != std::string::npos; q = bs.find("cf.c[", q)) bs.replace(q, 5, "cf[");
        o << bs;
        o << "    }\n    } break;\n";
    }
    o << "    default: break;\n    }\n";
    o << "    __syncthreads();\n";
    o << "    if (tid == 0) { __threadfence(); atomicAdd(&done[it.x], 1u); }\n";
    o << "    }\n}\n";
    return o.str();
}

// ---------------------------------------------------------------- adjoint passes (complex64)
// The reverse sweep of the adjoint gradient as compiled passes: psi and lambda
// tiles both live in registers (same layouts, same transposes), every op of
// the pass is applied to both, and an op that carries derivatives also sums
// 2 Re <lambda | D psi> over the thread's pairs between its psi and lambda
// updates (the planner gives such an op to its gate alone). Per tile, each
// derivative is summed over a warp (shuffles) and added to a compensated
// per-CTA accumulator in shared memory; the CTA writes one partial per slot.

std::string for_lambda(const std::string &code)
{
    std::string out;
    size_t pos = 0;
    for (;;) {
        const size_t q = code.find("(r, i", pos);
        if (q == std::string::npos) break;
        out += code.substr(pos, q - pos) + "(rl, il";
        pos = q + 5;
    }
    return out + code.substr(pos);
}

int coef_slots_adj(const plan::Op &op) { return 24 + 12 * op.nd; }

void emit_adj_op_c64(std::ostream &o, const plan::Op &op, int O, int lslot)
{
    if (op.nd == 0) {
        std::ostringstream a;
        emit_op_c64(a, op, O);
        o << a.str() << for_lambda(a.str());
        return;
    }
    // a gate with derivatives: GEN op, M[0] = I when it is controlled (m0id)
    const bool us = op.sthr || op.sext;
    const std::string sel =
        us ? "(((tid & " + hex32(op.sthr) + ") != 0u) | ((base & " + hex64(op.sext) + ") != 0ull))" : "0";
    const int J = op.treg, C = op.sreg;
    std::string apply, grad;
    int s = 0;
    // cheaper forms for a register target: diagonal (RZ, P) or real (RY) matrix and derivatives
    const int b = op.m0id ? 1 : 0;  // the branch that is not the identity
    bool diag = J < 3, real = J < 3;
    for (int d = -1; d < op.nd; ++d) {
        const std::complex<double> *m = d < 0 ? op.M[b] : op.D[d];
        diag &= m[1] == 0.0 && m[2] == 0.0;
        for (int e = 0; e < 4; ++e) real &= m[e].imag() == 0.0;
    }
    if (C == 3) diag = real = false;  // lane-resolved coefficients differ per lane
    if (diag || real) {
        const std::string f = diag ? "diag" : "real";
        const std::string cc = C < 0 ? "-1, 0" : std::to_string(C) + ", 1";
        if (C >= 0) s = 1;
        apply = "g_" + f + "<" + std::to_string(J) + ", " + cc + ">(r, i, c);";
        grad = "gd_" + f + "<" + std::to_string(J) + ", " + cc + ">";
    } else if (C < 0) {
        apply = J < 3 ? "g_all<" + std::to_string(J) + ">(r, i, c);" : "g_lane<-1, 0>(r, i, c);";
        grad = J < 3 ? "gd_reg<" + std::to_string(J) + ", -1, 0>" : "gd_lane<-1, 0>";
    } else if (C == 3) {  // select on the packed lane: coefficients resolved per lane
        apply = "g_all<" + std::to_string(J) + ">(r, i, c);";
        grad = "gd_reg<" + std::to_string(J) + ", -1, 0>";
    } else {
        s = 1;  // controlled by a register bit: only the s = 1 half changes
        apply = J < 3 ? "g_sel<" + std::to_string(J) + ", " + std::to_string(C) + ", 1>(r, i, c);"
                      : "g_lane<" + std::to_string(C) + ", 1>(r, i, c);";
        grad = J < 3 ? "gd_reg<" + std::to_string(J) + ", " + std::to_string(C) + ", 1>"
                     : "gd_lane<" + std::to_string(C) + ", 1>";
    }
    o << "    { float gsum[" << op.nd << "] = {";
    for (int d = 0; d < op.nd; ++d) o << (d ? ", " : "") << "0.f";
    o << "};\n";
    o << "      const int s = " << sel << ";\n";
    // a runtime select (control on a thread bit or outside the tile) skips the op where it is 0;
    // register selects are resolved inside the op
    const std::string cond = C < 0 ? std::string("s || ") + (op.m0id ? "0" : "1") : std::string("1");
    // generator form (a register target, no lane select): the derivative from psi before the
    // gate is undone, no derivative matrix
    const bool gen = op.nd == 1 && op.gen > 0 && J < 3 && C != 3;
    o << "      if (" << cond << ") { ";
    if (gen)
        o << "gsum[0] = gg_reg<" << J << ", " << (C >= 0 ? C : -1) << ", " << (C >= 0 ? 1 : 0) << ", " << op.gen
          << ">(r, i, rl, il);\n        ";
    o << coef_load(O, C < 0 ? "s" : std::to_string(s), 12, false) << "\n        " << apply << "\n";
    for (int d = 0; d < op.nd && !gen; ++d) {
        o << "        { u64 dc[12];";
        for (int e = 0; e < 12; ++e) o << " dc[" << e << "] = cf.c[" << O + 24 + 12 * d + e << "];";
        o << " gsum[" << d << "] = " << grad << "(r, i, rl, il, dc); }\n";
    }
    o << "        " << for_lambda(apply) << "\n      }\n";
    for (int d = 0; d < op.nd; ++d)
        o << "      acc_add(sacc, " << lslot + d << ", warp, lane, gsum[" << d << "]);\n";
    o << "    }\n";
}

std::string gen_source_adj(const plan::Pass &p, int nslots)
{
    PassGeom G{p.k, p.k - kRegBits, p.k - kChunkBits, &p};
    const int T = 1 << G.nq;
    const int nops = int(p.ops.size());
    std::vector<int> coff(nops + 1, 0), lsl(nops, 0);
    int ls = 0;
    for (int k = 0; k < nops; ++k) {
        coff[k + 1] = coff[k] + coef_slots_adj(p.ops[k]);
        lsl[k] = ls;
        ls += p.ops[k].nd;
    }
    const int ncoef = std::max(1, coff[nops]);
    std::ostringstream o;
    o << kPrelude;
    o << "struct QvAdjArgs { u64 c[" << ncoef << "]; int gslot[" << std::max(1, nslots) << "]; };\n";
    o << "#define NW " << T / 32 << "\n";
    o << "QI void acc_add(float *sacc, int q, int warp, int lane, float v) {\n"
         "#pragma unroll\n"
         "    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);\n"
         "    if (lane == 0) { float *h = sacc + 2 * (q * NW + warp); const float t = h[0] + v;\n"
         "        const float bb = t - h[0]; h[1] += (h[0] - (t - bb)) + (v - bb); h[0] = t; }\n"
         "}\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << (p.k == 12 ? 2 : p.k == 11 ? 4 : 8)
      << ") qv_adj(float *__restrict__ amp, float *__restrict__ lam, u64 ntiles, double *part, int Gc, "
         "const QvAdjArgs cf)\n{\n";
    o << "    extern __shared__ __align__(16) u64 sm[];\n";
    // shared memory: 2^k transpose words, then the next tile of psi and of lambda
    // (thread tid's eight 16-byte words at word v * T + tid of each, copied
    // asynchronously while the current tile computes), then the accumulators
    o << "    float *sacc = reinterpret_cast<float *>(sm + " << (size_t(3) << p.k) << ");\n";
    o << "    const u32 tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;\n";
    o << "    for (int q = tid; q < " << 2 * nslots * (T / 32) << "; q += " << T << ") sacc[q] = 0.f;\n";
    o << "    __syncthreads();\n";
    auto phys_mask = [&](const int8_t *Q) {
        std::vector<uint64_t> m(G.nq);
        for (int b = 0; b < G.nq; ++b) m[b] = G.phys(1u << Q[b]);
        return m;
    };
    auto word_mask = [&](const int8_t *Q) {
        std::vector<uint64_t> m(G.nq);
        for (int b = 0; b < G.nq; ++b) m[b] = swz8((1u << Q[b]) >> 1);
        return m;
    };
    const plan::Stage &s0 = p.stages.front(), &sl = p.stages.back();
    o << "    const u64 gL = " << thread_expr(phys_mask(s0.in.Q), true) << ";\n";
    o << "    const u64 gS = " << thread_expr(phys_mask(sl.out.Q), true) << ";\n";
    for (size_t s = 1; s < p.stages.size(); ++s) {
        o << "    const u32 wW" << s << " = " << thread_expr(word_mask(p.stages[s - 1].out.Q), false) << ";\n";
        o << "    const u32 wR" << s << " = " << thread_expr(word_mask(p.stages[s].in.Q), false) << ";\n";
    }
    auto reg_offset = [&](const int8_t *P, int v) {
        uint32_t l = 0;
        for (int j = 0; j < 3; ++j)
            if ((v >> j) & 1) l |= 1u << P[j];
        return l;
    };
    // copies of tile `tile` of psi and lambda into the prefetch buffers (if it exists)
    auto issue = [&](const std::string &tile, const std::string &ind) {
        o << ind << "if (" << tile << " < ntiles) { const u64 bn = " << tile_base_expr(p, tile) << ";\n";
        for (int b = 0; b < 2; ++b) {
            o << ind << "  { const float *a = " << (b ? "lam" : "amp") << " + 2 * (bn + gL); const u32 d = sh_addr(sm + "
              << ((b + 1) << p.k) << ") + 16u * tid;\n";
            for (int v = 0; v < 8; ++v)
                o << ind << "    cp16(d + " << 16 * v * T << "u, a + 2 * " << hex64(G.phys(reg_offset(s0.in.P, v))) << ");\n";
            o << ind << "  }\n";
        }
        o << ind << "}\n" << ind << "cp_commit();\n";
    };
    issue("(u64)blockIdx.x", "    ");
    o << "    for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {\n";
    o << "    const u64 base = 0ull";
    for (int s = 0; s < p.nseg; ++s)
        o << " | (((t >> " << p.seg_src[s] << ") & " << hex64((uint64_t(1) << p.seg_w[s]) - 1) << ") << "
          << p.seg_dst[s] << ")";
    o << ";\n";
    o << "    u64 r[8], i[8], rl[8], il[8];\n";
    o << "    cp_wait_all();\n";
    for (int b = 0; b < 2; ++b) {
        const char *R = b ? "rl" : "r", *I = b ? "il" : "i";
        o << "    { const float4 *pf = reinterpret_cast<const float4 *>(sm + " << ((b + 1) << p.k) << ") + tid;\n";
        for (int v = 0; v < 8; ++v)
            o << "      { const float4 f = pf[" << v * T << "]; " << R << "[" << v << "] = pk(f.x, f.z); " << I << "["
              << v << "] = pk(f.y, f.w); }\n";
        o << "    }\n";
    }
    // the next tile's copies go out once every thread has read its words of this
    // one: after the first block barrier of the tile (added when the pass has no
    // transpose)
    if (p.stages.size() == 1) {
        o << "    __syncthreads();\n";
        issue("(t + gridDim.x)", "    ");
    }
    for (size_t s = 0; s < p.stages.size(); ++s) {
        const plan::Stage &st = p.stages[s];
        if (s > 0) {
            const plan::Stage &pr = p.stages[s - 1];
            // psi through words [0, 2^k / 2) x 2 halves, lambda through the next 2^k words
            o << "    { u64 *pre = sm, *pim = sm + " << (1 << (p.k - 1)) << ";\n";
            for (int v = 0; v < 8; ++v) {
                const uint32_t w = swz8(reg_offset(pr.out.P, v) >> 1);
                o << "      pre[wW" << s << " ^ " << hex32(w) << "] = r[" << v << "]; pim[wW" << s << " ^ " << hex32(w)
                  << "] = i[" << v << "];\n";
            }
            o << "      __syncthreads();\n";
            if (s == 1) issue("(t + gridDim.x)", "      ");
            for (int v = 0; v < 8; ++v) {
                const uint32_t w = swz8(reg_offset(st.in.P, v) >> 1);
                o << "      r[" << v << "] = pre[wR" << s << " ^ " << hex32(w) << "]; i[" << v << "] = pim[wR" << s
                  << " ^ " << hex32(w) << "];\n";
            }
            o << "      __syncthreads();\n";
            for (int v = 0; v < 8; ++v) {
                const uint32_t w = swz8(reg_offset(pr.out.P, v) >> 1);
                o << "      pre[wW" << s << " ^ " << hex32(w) << "] = rl[" << v << "]; pim[wW" << s << " ^ " << hex32(w)
                  << "] = il[" << v << "];\n";
            }
            o << "      __syncthreads();\n";
            for (int v = 0; v < 8; ++v) {
                const uint32_t w = swz8(reg_offset(st.in.P, v) >> 1);
                o << "      rl[" << v << "] = pre[wR" << s << " ^ " << hex32(w) << "]; il[" << v << "] = pim[wR" << s
                  << " ^ " << hex32(w) << "];\n";
            }
            o << "      __syncthreads(); }\n";
        }
        for (int k = st.op_begin; k < st.op_end; ++k) emit_adj_op_c64(o, p.ops[k], coff[k], lsl[k]);
    }
    if (p.stages.size() == 1 && std::memcmp(&s0.in, &sl.out, sizeof(plan::Layout)) != 0) o << "    __syncthreads();\n";
    for (int b = 0; b < 2; ++b) {
        const char *dst = b ? "lam" : "amp";
        const char *R = b ? "rl" : "r", *I = b ? "il" : "i";
        o << "    { float *a = " << dst << " + 2 * (base + gS); float x0, x1, y0, y1;\n";
        for (int v = 0; v < 8; ++v)
            o << "      upk(" << R << "[" << v << "], x0, x1); upk(" << I << "[" << v
              << "], y0, y1); *reinterpret_cast<float4 *>(a + 2 * " << hex64(G.phys(reg_offset(sl.out.P, v)))
              << ") = make_float4(x0, y0, x1, y1);\n";
        o << "    }\n";
    }
    o << "    }\n";
    o << "    __syncthreads();\n";
    o << "    for (int q = tid; q < " << nslots << "; q += " << T << ") {\n";
    o << "        double v = 0;\n";
    o << "        for (int w = 0; w < NW; ++w) v += double(sacc[2 * (q * NW + w)]) + double(sacc[2 * (q * NW + w) + 1]);\n";
    o << "        part[(size_t)cf.gslot[q] * Gc + blockIdx.x] = 2.0 * v;  // 2 Re <lambda | D psi>\n";
    o << "    }\n}\n";
    return o.str();
}

}  // namespace

// ---------------------------------------------------------------- compile + cache
struct Compiled {
    CUmodule mod = nullptr;
    CUfunction fn = nullptr;
    int per_sm = 0;
    size_t smem = 0;
};

namespace {

std::mutex g_cache_mu;
std::map<std::pair<int, std::string>, std::shared_ptr<Compiled>> g_cache;

// With `log`, ptxas also reports registers and spills (-v) into *log.
bool compile_one(const std::string &src, std::vector<char> &cubin, std::string &err, std::string *log = nullptr)
{
    const JitApi &N = api();
    nvrtcProgram prog;
    if (N.create(&prog, src.c_str(), "qv_pass.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        err = "nvrtcCreateProgram failed";
        return false;
    }
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=true", "--ptxas-options=-v"};
    const nvrtcResult rc = N.compile(prog, log ? 4 : 3, opts);
    if (log && rc == NVRTC_SUCCESS) {
        size_t ls = 0;
        N.log_size(prog, &ls);
        log->assign(ls, '\0');
        if (ls) N.log(prog, &(*log)[0]);
    }
    if (rc != NVRTC_SUCCESS) {
        size_t ls = 0;
        N.log_size(prog, &ls);
        std::string log(ls, '\0');
        if (ls) N.log(prog, &log[0]);
        err = "nvrtc: " + log.substr(0, 400);
        N.destroy(&prog);
        return false;
    }
    size_t cs = 0;
    N.cubin_size(prog, &cs);
    cubin.resize(cs);
    N.cubin(prog, cubin.data());
    N.destroy(&prog);
    return true;
}

// Threads that compile passes in parallel: at most 16.
unsigned compile_threads() { return std::max(1u, std::min(16u, std::thread::hardware_concurrency())); }

qv_status cu_fail(CUresult r, const char *what)
{
    const char *s = nullptr;
    if (api().err_string) api().err_string(r, &s);
    return fail(QV_ERR_CUDA, "%s: %s", what, s ? s : "?");
}

}  // namespace

bool jit_available(std::string *why)
{
    const JitApi &N = api();
    if (!N.ok && why) *why = N.why;
    return N.ok;
}

std::string jit_pass_source(const plan::Pass &p, bool c64) { return p.tc ? gen_source_tc(p) : gen_source(p, c64); }

qv_status jit_compile_host(const std::vector<plan::Pass> &passes, bool c64, int64_t out[4])
{
    const JitApi &N = api();
    if (!N.nvrtc_ok) return fail(QV_ERR_UNSUPPORTED, "NVRTC unavailable: %s", N.why.c_str());
    const size_t np = passes.size();
    std::vector<std::string> srcs(np), errs(np), logs(np);
    std::vector<char> ok(np, 0);
    int64_t bytes = 0;
    for (size_t i = 0; i < np; ++i) {
        srcs[i] = jit_pass_source(passes[i], c64);
        bytes += int64_t(srcs[i].size());
    }
    // as many compiler threads as the kernel loader uses: NVRTC and ptxas take
    // hundreds of MB of host memory each
    const size_t nt = std::max<size_t>(1, std::min<size_t>(np, compile_threads()));
    std::atomic<size_t> next{0};
    std::vector<std::thread> th;
    for (size_t t = 0; t < nt; ++t)
        th.emplace_back([&] {
            for (size_t i; (i = next.fetch_add(1)) < np;) {
                std::vector<char> cubin;
                ok[i] = compile_one(srcs[i], cubin, errs[i], &logs[i]) ? 1 : 0;
            }
        });
    for (auto &x : th) x.join();
    int64_t regs = 0, spilling = 0;
    for (size_t i = 0; i < np; ++i) {
        if (!ok[i]) return fail(QV_ERR_CUDA, "pass %zu: %s", i, errs[i].c_str());
        regs = std::max<int64_t>(regs, ptxas_registers(logs[i]));
        spilling += ptxas_spills(logs[i]) ? 1 : 0;
    }
    out[0] = int64_t(np);
    out[1] = bytes;
    out[2] = regs;
    out[3] = spilling;
    return QV_OK;
}

namespace {

// Kernels `entry` of srcs[i] (dynamic shared memory smem[i], threads[i] per
// CTA), compiled in parallel host threads or taken from the process-wide cache.
qv_status get_kernels(qv_state *s, const std::vector<std::string> &srcs, const char *entry,
                      const std::vector<size_t> &smem, const std::vector<int> &threads,
                      std::vector<std::shared_ptr<Compiled>> &fns)
{
    std::string why;
    if (!jit_available(&why)) return fail(QV_ERR_UNSUPPORTED, "compiled passes unavailable: %s", why.c_str());
    // make sure this thread has the device's primary context current for the driver API
    QV_CUDA(cudaSetDevice(s->device));
    QV_CUDA(cudaFree(nullptr));
    fns.assign(srcs.size(), nullptr);
    std::vector<size_t> todo;
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        for (size_t i = 0; i < srcs.size(); ++i) {
            auto it = g_cache.find({s->device, srcs[i]});
            if (it != g_cache.end()) fns[i] = it->second;
            else if (std::find_if(todo.begin(), todo.end(), [&](size_t j) { return srcs[j] == srcs[i]; }) == todo.end())
                todo.push_back(i);
        }
    }
    if (!todo.empty()) {
        std::vector<std::vector<char>> cubins(todo.size());
        std::vector<std::string> errs(todo.size());
        std::vector<char> okv(todo.size(), 0);
        const unsigned hw = compile_threads();
        size_t next = 0;
        std::mutex mu;
        auto worker = [&] {
            for (;;) {
                size_t j;
                {
                    std::lock_guard<std::mutex> l(mu);
                    if (next >= todo.size()) return;
                    j = next++;
                }
                okv[j] = compile_one(srcs[todo[j]], cubins[j], errs[j]);
            }
        };
        std::vector<std::thread> th;
        for (unsigned w = 0; w < std::min<size_t>(hw, todo.size()); ++w) th.emplace_back(worker);
        for (auto &t : th) t.join();
        std::lock_guard<std::mutex> lock(g_cache_mu);
        for (size_t j = 0; j < todo.size(); ++j) {
            if (!okv[j]) return fail(QV_ERR_CUDA, "compiling a pass failed: %s", errs[j].c_str());
            auto c = std::make_shared<Compiled>();
            const JitApi &A = api();
            CUresult r = A.module_load(&c->mod, cubins[j].data());
            if (r != CUDA_SUCCESS) return cu_fail(r, "cuModuleLoadData");
            r = A.get_function(&c->fn, c->mod, entry);
            if (r != CUDA_SUCCESS) return cu_fail(r, "cuModuleGetFunction");
            c->smem = smem[todo[j]];
            // the default limit (48 KB minus the static shared memory) can be below
            // what a pass needs even at 48 KB: always raise it to the pass's size
            r = A.set_attr(c->fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, int(c->smem));
            if (r != CUDA_SUCCESS) return cu_fail(r, "cuFuncSetAttribute");
            r = A.occupancy(&c->per_sm, c->fn, threads[todo[j]], c->smem);
            if (r != CUDA_SUCCESS) return cu_fail(r, "cuOccupancyMaxActiveBlocksPerMultiprocessor");
            if (c->per_sm < 1) {
                int regs = -1, st = -1, maxdyn = -1, maxthr = -1;
                A.get_attr(&regs, CU_FUNC_ATTRIBUTE_NUM_REGS, c->fn);
                A.get_attr(&st, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, c->fn);
                A.get_attr(&maxdyn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, c->fn);
                A.get_attr(&maxthr, CU_FUNC_ATTRIBUTE_MAX_THREADS_PER_BLOCK, c->fn);
                return fail(QV_ERR_UNSUPPORTED,
                            "compiled pass does not fit on an SM (%d threads, %d registers, %d + %zu bytes of shared "
                            "memory, at most %d dynamic, %d threads per CTA)",
                            threads[todo[j]], regs, st, c->smem, maxdyn, maxthr);
            }
            g_cache[{s->device, srcs[todo[j]]}] = c;
        }
        for (size_t i = 0; i < srcs.size(); ++i)
            if (!fns[i]) fns[i] = g_cache[{s->device, srcs[i]}];
    }
    return QV_OK;
}

}  // namespace

struct JitProgram {
    std::vector<std::shared_ptr<Compiled>> fns;
    std::vector<std::vector<uint64_t>> args;  // by-value kernel parameter of each pass
    std::vector<int> threads;
    std::vector<uint64_t> ntiles;
    // tensor-core passes: matrix slots of every pass in one device buffer
    bool tc = false;
    int device = 0;
    void *mats = nullptr;
    std::vector<size_t> mat_off;  // byte offset of each pass's slots
    ~JitProgram()
    {
        if (mats) {
            int cur = 0;
            cudaGetDevice(&cur);
            cudaSetDevice(device);
            cudaFree(mats);
            cudaSetDevice(cur);
        }
    }
};

namespace {
qv_status jit_prepare_tc(qv_state *s, const std::vector<plan::Pass> &passes, std::shared_ptr<JitProgram> &out)
{
    if (s->dt != QV_C64) return fail(QV_ERR_UNSUPPORTED, "tensor-core passes are complex64 only");
    auto P = std::make_shared<JitProgram>();
    P->tc = true;
    P->device = s->device;
    std::vector<std::string> srcs(passes.size());
    std::vector<size_t> smem(passes.size());
    std::vector<float> all, one;
    P->threads.resize(passes.size());
    for (size_t i = 0; i < passes.size(); ++i) {
        srcs[i] = gen_source_tc(passes[i]);
        smem[i] = tc_smem(passes[i]);
        P->threads[i] = 1 << (passes[i].k - kRegBits);
        P->ntiles.push_back(dim(s) >> passes[i].k);
        pack_tc_mats(passes[i], one);
        P->mat_off.push_back(all.size() * sizeof(float));
        all.insert(all.end(), one.begin(), one.end());
        P->args.emplace_back();
    }
    QV_TRY(get_kernels(s, srcs, "qv_tc", smem, P->threads, P->fns));
    for (const auto &f : P->fns) {
        // at most as many CTAs per SM as tensor memory serves
        const int cap = 512 / tc_cols(passes[size_t(&f - &P->fns[0])].k);
        if (f->per_sm > cap) return fail(QV_ERR_UNSUPPORTED, "tensor-core pass: %d CTAs per SM exceed tensor memory", f->per_sm);
    }
    QV_CUDA(cudaSetDevice(s->device));
    if (!all.empty()) {
        QV_CUDA(cudaMalloc(&P->mats, all.size() * sizeof(float)));
        QV_TRY(copy_h2d(s, P->mats, all.data(), all.size() * sizeof(float)));
    }
    out = P;
    return QV_OK;
}
}  // namespace

qv_status jit_prepare(qv_state *s, const std::vector<plan::Pass> &passes, std::shared_ptr<JitProgram> &out)
{
    if (!passes.empty() && passes.front().tc) return jit_prepare_tc(s, passes, out);
    const bool c64 = s->dt == QV_C64;
    auto P = std::make_shared<JitProgram>();
    std::vector<std::string> srcs(passes.size());
    std::vector<size_t> smem(passes.size());
    P->threads.resize(passes.size());
    for (size_t i = 0; i < passes.size(); ++i) {
        srcs[i] = gen_source(passes[i], c64);
        smem[i] = (c64 ? 8 : 16) * (size_t(1) << passes[i].k);
        P->threads[i] = 1 << (passes[i].k - kRegBits);
        P->ntiles.push_back(dim(s) >> passes[i].k);
    }
    QV_TRY(get_kernels(s, srcs, "qv_pass", smem, P->threads, P->fns));
    for (const plan::Pass &p : passes) {
        size_t total = 0;
        for (const plan::Op &op : p.ops) total += c64 ? size_t(coef_slots_c64(op)) : 16;
        std::vector<uint64_t> coef(std::max<size_t>(1, total), 0);
        size_t off = 0;
        for (const plan::Op &op : p.ops) {
            if (c64) op_coeffs_c64(op, coef.data() + off);
            else op_coeffs_c128(op, reinterpret_cast<double *>(coef.data() + off));
            off += c64 ? size_t(coef_slots_c64(op)) : 16;
        }
        P->args.push_back(std::move(coef));
    }
    out = P;
    return QV_OK;
}

qv_status jit_launch(qv_state *s, const JitProgram &P, cudaStream_t on)
{
    QV_CUDA(cudaSetDevice(s->device));
    // on a stream of the caller's (a batch graph being captured): no counters, no events
    const bool count = on == nullptr;
    CUstream cs = reinterpret_cast<CUstream>(count ? s->stream : on);
    if (P.tc) {
        int *status = nullptr;
        QV_TRY(status_word(s, &status));
        uint32_t spin = 1u << 22;
        for (size_t i = 0; i < P.fns.size(); ++i) {
            const Compiled &c = *P.fns[i];
            uint64_t ntiles = P.ntiles[i];
            const unsigned grid = unsigned(std::min<uint64_t>(ntiles, uint64_t(c.per_sm) * s->num_sms));
            void *amp = s->amp;
            void *mats = static_cast<char *>(P.mats) + P.mat_off[i];
            void *args[] = {&amp, &ntiles, &mats, &status, &spin};
            if (count) {
                prof_bytes(s, QV_K_FUSED, 2.0 * double(dim(s)) * amp_bytes(s->dt));
                prof_begin(s, QV_K_FUSED);
            }
            const CUresult r =
                api().launch(c.fn, grid, 1, 1, unsigned(P.threads[i]), 1, 1, unsigned(c.smem), cs, args, nullptr);
            if (count) prof_end(s, QV_K_FUSED);
            if (r != CUDA_SUCCESS) return cu_fail(r, "cuLaunchKernel");
        }
        return QV_OK;
    }
    for (size_t i = 0; i < P.fns.size(); ++i) {
        const Compiled &c = *P.fns[i];
        uint64_t ntiles = P.ntiles[i];
        const unsigned grid = unsigned(std::min<uint64_t>(ntiles, uint64_t(c.per_sm) * s->num_sms));
        void *amp = s->amp;
        void *args[] = {&amp, &ntiles, const_cast<uint64_t *>(P.args[i].data())};
        if (count) {
            prof_bytes(s, QV_K_FUSED, 2.0 * double(dim(s)) * amp_bytes(s->dt));
            prof_begin(s, QV_K_FUSED);
        }
        const CUresult r =
            api().launch(c.fn, grid, 1, 1, unsigned(P.threads[i]), 1, 1, unsigned(c.smem), cs, args, nullptr);
        if (count) prof_end(s, QV_K_FUSED);
        if (r != CUDA_SUCCESS) return cu_fail(r, "cuLaunchKernel");
        if (count) s->prof.h2d += P.args[i].size() * sizeof(uint64_t);
    }
    return QV_OK;
}

qv_status jit_run_plan(qv_state *s, const std::vector<plan::Pass> &passes)
{
    std::shared_ptr<JitProgram> P;
    QV_TRY(jit_prepare(s, passes, P));
    return jit_launch(s, *P);
}

qv_status jit_prepare_adjoint(qv_state *s, const std::vector<plan::Pass> &passes, std::shared_ptr<JitProgram> &out)
{
    if (s->dt != QV_C64) return fail(QV_ERR_UNSUPPORTED, "compiled adjoint passes are complex64 only");
    auto P = std::make_shared<JitProgram>();
    std::vector<std::string> srcs(passes.size());
    std::vector<size_t> smem(passes.size());
    std::vector<int> nslots(passes.size(), 0);
    P->threads.resize(passes.size());
    for (size_t i = 0; i < passes.size(); ++i) {
        for (const plan::Op &op : passes[i].ops) nslots[i] += op.nd;
        srcs[i] = gen_source_adj(passes[i], nslots[i]);
        P->threads[i] = 1 << (passes[i].k - kRegBits);
        smem[i] = 24 * (size_t(1) << passes[i].k) + size_t(2 * sizeof(float)) * nslots[i] * (P->threads[i] / 32);
        P->ntiles.push_back(dim(s) >> passes[i].k);
    }
    QV_TRY(get_kernels(s, srcs, "qv_adj", smem, P->threads, P->fns));
    for (size_t i = 0; i < passes.size(); ++i) {
        const plan::Pass &p = passes[i];
        size_t total = 0;
        for (const plan::Op &op : p.ops) total += size_t(coef_slots_adj(op));
        total = std::max<size_t>(1, total);
        const size_t ns = std::max(1, nslots[i]);
        std::vector<uint64_t> buf(total + (ns + 1) / 2, 0);  // QvAdjArgs: u64 c[total]; int gslot[ns]
        size_t off = 0;
        int32_t *gslot = reinterpret_cast<int32_t *>(buf.data() + total);
        int lsl = 0;
        for (const plan::Op &op : p.ops) {
            op_coeffs_c64(op, buf.data() + off);
            for (int d = 0; d < op.nd; ++d) {
                for (int e = 0; e < 4; ++e)
                    lane_triple(buf.data() + off + 24 + 12 * d + 3 * e, op.sreg == 3 ? cd(0.0) : op.D[d][e],
                                op.D[d][e]);
                gslot[lsl++] = op.slot + d;
            }
            off += size_t(coef_slots_adj(op));
        }
        P->args.push_back(std::move(buf));
    }
    out = P;
    return QV_OK;
}

qv_status jit_launch_adjoint(qv_state *s, const JitProgram &P, void *lam, double *part, int G)
{
    QV_CUDA(cudaSetDevice(s->device));
    for (size_t i = 0; i < P.fns.size(); ++i) {
        const Compiled &c = *P.fns[i];
        uint64_t ntiles = P.ntiles[i];
        const unsigned grid = unsigned(std::min<uint64_t>({ntiles, uint64_t(c.per_sm) * s->num_sms, uint64_t(G)}));
        void *amp = s->amp;
        void *args[] = {&amp, &lam, &ntiles, &part, &G, const_cast<uint64_t *>(P.args[i].data())};
        prof_bytes(s, QV_K_ADJOINT, 4.0 * double(dim(s)) * amp_bytes(s->dt));
        prof_begin(s, QV_K_ADJOINT);
        const CUresult r = api().launch(c.fn, grid, 1, 1, unsigned(P.threads[i]), 1, 1, unsigned(c.smem),
                                          reinterpret_cast<CUstream>(s->stream), args, nullptr);
        prof_end(s, QV_K_ADJOINT);
        if (r != CUDA_SUCCESS) return cu_fail(r, "cuLaunchKernel");
        s->prof.h2d += P.args[i].size() * sizeof(uint64_t);
    }
    return QV_OK;
}

qv_status jit_run_adjoint(qv_state *s, const std::vector<plan::Pass> &passes, void *lam, double *part, int G)
{
    std::shared_ptr<JitProgram> P;
    QV_TRY(jit_prepare_adjoint(s, passes, P));
    return jit_launch_adjoint(s, *P, lam, part, G);
}

qv_status jit_prepare_batch(qv_state *s, const std::vector<std::vector<plan::Pass> *> &plans, int chunk_tiles,
                            JitBatch &out)
{
    const std::vector<plan::Pass> &P0 = *plans.front();
    out.npasses = int(P0.size());
    out.stride = 1;
    for (const plan::Pass &p : P0) {
        int t = 0;
        for (const plan::Op &op : p.ops) t += coef_slots_c64(op);
        out.stride = std::max(out.stride, t);
    }
    out.coefs.assign(plans.size() * P0.size() * size_t(out.stride), 0);
    for (size_t c = 0; c < plans.size(); ++c)
        for (size_t p = 0; p < P0.size(); ++p) {
            uint64_t *dst = out.coefs.data() + (c * P0.size() + p) * size_t(out.stride);
            size_t off = 0;
            for (const plan::Op &op : (*plans[c])[p].ops) {
                op_coeffs_c64(op, dst + off);
                off += size_t(coef_slots_c64(op));
            }
        }
    const std::string src = gen_source_batch(P0, out.stride, chunk_tiles);
    out.threads = 1 << (P0.front().k - kRegBits);
    out.smem = 8 * (size_t(1) << P0.front().k);
    std::vector<std::shared_ptr<Compiled>> fns;
    QV_TRY(get_kernels(s, {src}, "qv_batch", {out.smem}, {out.threads}, fns));
    out.fn = fns[0];
    out.per_sm = fns[0]->per_sm;
    return QV_OK;
}

qv_status jit_launch_batch(const JitBatch &jb, cudaStream_t stream, unsigned grid, void **args)
{
    const CUresult r = api().launch(jb.fn->fn, grid, 1, 1, unsigned(jb.threads), 1, 1, unsigned(jb.smem),
                                    reinterpret_cast<CUstream>(stream), args, nullptr);
    if (r != CUDA_SUCCESS) return cu_fail(r, "cuLaunchKernel");
    return QV_OK;
}

bool jit_same_structure(const std::vector<plan::Pass> &a, const std::vector<plan::Pass> &b)
{
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
        if (!same_structure(a[i], b[i])) return false;
    return true;
}

}  // namespace qv
