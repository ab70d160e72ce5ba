// Adjoint differentiation of <psi|H|psi> with respect to the gate angles, and
// the Pauli-sum apply it needs. Not in the paper; it reuses the paper's pair
// update (Sec. III-A, Eq. 5) on two state buffers at once.
//
// psi_L = U_L ... U_1 psi_0 and E = <psi_L|H|psi_L>. With lambda = H psi_L and
// the reverse sweep l = L..1:
//     psi    <- U_l^dagger psi                    (now psi = psi_{l-1})
//     g[p]   += 2 Re <lambda | dU_l/dtheta_p | psi>  for each trainable angle
//     lambda <- U_l^dagger lambda
// every derivative uses one pass over both buffers and no stored states
// (Jones and Gacon, "Efficient calculation of gradients in classical
// simulations of variational quantum algorithms", arXiv:2009.02823).
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "planner.h"
#include "qv_device.cuh"
#include "qv_internal.h"
#include "qv_jit.h"
#include "qv_plan.h"

namespace qv {

struct AdjointBuffers {
    void *lam = nullptr;       // second state buffer (lambda)
    size_t lam_bytes = 0;
    double *part = nullptr;    // per-block partial sums
    size_t part_count = 0;
    // compiled reverse sweep of the last gate list (same bytes: no re-planning)
    std::vector<qv_gate> key;
    std::shared_ptr<JitProgram> sweep;
};

namespace {

constexpr int kThreads = 256;
constexpr int kMaxD = 3;  // trainable angles per gate (U3)

// ---------------------------------------------------------------- H|psi>
constexpr int kMaxTerms = 64;
// Terms sharing one X mask; coefficients coeff * i^{ny} in the state's
// precision (the sum over terms is per amplitude, not a reduction over the
// state, and FP64 runs at a small fraction of the FP32 rate on this GPU).
template <typename R> struct PauliGroupA {
    uint64_t x;
    int32_t nt;
    int32_t zero_z;       // every z mask is 0: c is the constant (c0re, c0im)
    int32_t has_im;       // some coefficient has an imaginary part
    int32_t tab;          // chunks of Z-term tables (pure-Z group), 0: none
    R c0re, c0im;
    uint64_t z[kMaxTerms];
    R cre[kMaxTerms], cim[kMaxTerms];
};

// out_j = sum over groups sum_t c_t i^{ny_t} (-1)^{popcount(src & z_t)} psi_src, src = j ^ x
template <typename R>
__global__ void __launch_bounds__(kThreads) pauli_apply_kernel(const R *__restrict__ psi, R *__restrict__ out,
                                                               uint64_t N, const PauliGroupA<R> *groups, int ng,
                                                               const R *ztab, int tab_words)
{
    extern __shared__ unsigned char smem_raw[];
    PauliGroupA<R> *g = reinterpret_cast<PauliGroupA<R> *>(smem_raw);
    R *tab = reinterpret_cast<R *>(smem_raw + size_t(ng) * sizeof(PauliGroupA<R>));
    static_assert(sizeof(PauliGroupA<R>) % 8 == 0, "copied as 8-byte words");
    for (int k = threadIdx.x; k < ng * int(sizeof(PauliGroupA<R>) / 8); k += kThreads)
        reinterpret_cast<uint64_t *>(g)[k] = reinterpret_cast<const uint64_t *>(groups)[k];
    for (int k = threadIdx.x; k < tab_words; k += kThreads) tab[k] = ztab[k];
    __syncthreads();
    // NA outputs j0 + k * S a thread at a time: each group's fields and Z terms are
    // read once for them, and the partner loads of four groups for all of them are
    // issued before any is used (the far partners come from DRAM; the kernel is
    // bound by their latency)
    using V = typename Cplx<R>::V;
    const uint64_t S = uint64_t(gridDim.x) * kThreads;
    uint64_t j0 = uint64_t(blockIdx.x) * kThreads + threadIdx.x;
    auto outputs = [&](auto na) {
        constexpr int NA = decltype(na)::value;
        R ar[NA], ai[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) ar[k] = ai[k] = R(0);
        for (int q0 = 0; q0 < ng; q0 += 4) {
            V v[4][NA];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int k = 0; k < NA; ++k)
                    if (q0 + u < ng) v[u][k] = load_amp(psi, (j0 + k * S) ^ g[q0 + u].x);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + u;
                if (q >= ng) break;
                R cr[NA], ci[NA];
#pragma unroll
                for (int k = 0; k < NA; ++k) {
                    cr[k] = g[q].zero_z ? g[q].c0re : R(0);
                    ci[k] = g[q].zero_z ? g[q].c0im : R(0);
                }
                if (!g[q].zero_z) {
                    const bool him = g[q].has_im != 0;
                    for (int t = 0; t < g[q].nt; ++t) {
                        const uint64_t zk = g[q].z[t];
                        const R fr = g[q].cre[t], fi = g[q].cim[t];
#pragma unroll
                        for (int k = 0; k < NA; ++k) {
                            const uint64_t src = (j0 + k * S) ^ g[q].x;
                            const uint32_t par =
                                (__popc(uint32_t(src) & uint32_t(zk)) ^ __popc(uint32_t(src >> 32) & uint32_t(zk >> 32))) & 1u;
                            const R sg = par ? R(-1) : R(1);
                            cr[k] += sg * fr;
                            if (him) ci[k] += sg * fi;
                        }
                    }
                    if (g[q].tab) {
#pragma unroll
                        for (int k = 0; k < NA; ++k) ztab_add(tab, g[q].tab, (j0 + k * S) ^ g[q].x, him, cr[k], ci[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < NA; ++k) {
                    ar[k] += cr[k] * v[u][k].x - ci[k] * v[u][k].y;
                    ai[k] += cr[k] * v[u][k].y + ci[k] * v[u][k].x;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NA; ++k) reinterpret_cast<V *>(out)[j0 + k * S] = V{ar[k], ai[k]};
    };
    for (; j0 + 3 * S < N; j0 += 4 * S) outputs(std::integral_constant<int, 4>{});
    for (; j0 < N; j0 += S) outputs(std::integral_constant<int, 1>{});
}

// ---------------------------------------------------------------- Re <a|b>
__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int V> __device__ __forceinline__ void block_sum_to(double (&x)[V], double *out, int stride)
{
    __shared__ double sm[kThreads / 32][kMaxD + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = warp_sum(x[v]);
    if (lane == 0)
#pragma unroll
        for (int v = 0; v < V; ++v) sm[warp][v] = x[v];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int v = 0; v < V; ++v) {
            double s = 0;
            for (int w = 0; w < kThreads / 32; ++w) s += sm[w][v];
            out[v * stride + blockIdx.x] = s;
        }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) inner_re_kernel(const R *__restrict__ a, const R *__restrict__ b,
                                                            uint64_t N, double *part)
{
    CompSum<R> acc;
    for (uint64_t j = uint64_t(blockIdx.x) * kThreads + threadIdx.x; j < N; j += uint64_t(gridDim.x) * kThreads)
        acc.add(a[2 * j] * b[2 * j] + a[2 * j + 1] * b[2 * j + 1]);
    double x[1] = {acc.value()};
    block_sum_to<1>(x, part, gridDim.x);
}

// Neumaier sum of each of `rows` rows of `cols` partials; one block per row.
__global__ void __launch_bounds__(kThreads) rows_sum_kernel(const double *part, int cols, double *out)
{
    __shared__ double ss[kThreads], cc[kThreads];
    Neumaier acc;
    for (int k = threadIdx.x; k < cols; k += kThreads) acc.add(part[size_t(blockIdx.x) * cols + k]);
    ss[threadIdx.x] = acc.s;
    cc[threadIdx.x] = acc.c;
    __syncthreads();
    if (threadIdx.x == 0) {
        Neumaier f;
        double c = 0;
        for (int k = 0; k < kThreads; ++k) {
            f.add(ss[k]);
            c += cc[k];
        }
        out[blockIdx.x] = f.value() + c;
    }
}

// ---------------------------------------------------------------- reverse step
// One gate of the reverse sweep on both buffers. Pairs (i0, i0 | 2^t) with bit
// t = 0 (and the control bit = 1 when ctrl >= 0):
//   psi'   = Ud psi,  g_d += 2 Re( conj(lam) . dU_d psi' ),  lam' = Ud lam
// Ud = U^dagger. Partial sums of g_d go to part[d * gridDim.x + block].
template <typename R, int ND>
__global__ void __launch_bounds__(kThreads) adjoint_step_kernel(R *__restrict__ psi, R *__restrict__ lam,
                                                                uint64_t pairs, int t, int ctrl, Mat2<R> Ud,
                                                                Mat2<R> d0, Mat2<R> d1, Mat2<R> d2, double *part)
{
    const uint64_t tb = uint64_t(1) << t;
    const int lo = ctrl >= 0 ? min(t, ctrl) : t, hi = ctrl >= 0 ? max(t, ctrl) : -1;
    const uint64_t cset = ctrl >= 0 ? uint64_t(1) << ctrl : 0;
    CompSum<R> g[ND > 0 ? ND : 1];
    for (uint64_t p = uint64_t(blockIdx.x) * kThreads + threadIdx.x; p < pairs; p += uint64_t(gridDim.x) * kThreads) {
        uint64_t i0 = insert_zero(p, lo);
        if (hi >= 0) i0 = insert_zero(i0, hi);
        i0 |= cset;
        const uint64_t i1 = i0 | tb;
        R ar = psi[2 * i0], ai = psi[2 * i0 + 1], br = psi[2 * i1], bi = psi[2 * i1 + 1];
        R lr = lam[2 * i0], li = lam[2 * i0 + 1], mr = lam[2 * i1], mi = lam[2 * i1 + 1];
        apply2(Ud, ar, ai, br, bi);
        psi[2 * i0] = ar;
        psi[2 * i0 + 1] = ai;
        psi[2 * i1] = br;
        psi[2 * i1 + 1] = bi;
        if constexpr (ND > 0) {
            const Mat2<R> *dd[3] = {&d0, &d1, &d2};
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                R xr = ar, xi = ai, yr = br, yi = bi;
                apply2(*dd[d], xr, xi, yr, yi);
                // Re( conj(l) x + conj(m) y )
                g[d].add(R(2) * (lr * xr + li * xi + mr * yr + mi * yi));
            }
        }
        apply2(Ud, lr, li, mr, mi);
        lam[2 * i0] = lr;
        lam[2 * i0 + 1] = li;
        lam[2 * i1] = mr;
        lam[2 * i1 + 1] = mi;
    }
    if constexpr (ND > 0) {
        double x[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) x[d] = g[d].value();
        block_sum_to<ND>(x, part, gridDim.x);
    }
}

template <typename R> __global__ void swap2_kernel(R *a, R *b, uint64_t units, int p, int q)
{
    using V = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const int lo = min(p, q), hi = max(p, q);
    for (uint64_t u = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < units; u += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t i = insert_zero(insert_zero(u, lo), hi);
        const uint64_t i1 = i | (uint64_t(1) << p), i2 = i | (uint64_t(1) << q);
        V *va = reinterpret_cast<V *>(a), *vb = reinterpret_cast<V *>(b);
        V x = va[i1];
        va[i1] = va[i2];
        va[i2] = x;
        x = vb[i1];
        vb[i1] = vb[i2];
        vb[i2] = x;
    }
}

// ---------------------------------------------------------------- host helpers
template <typename R> Mat2<R> to_mat(const cd U[4])
{
    Mat2<R> m;
    for (int e = 0; e < 4; ++e) {
        m.r[e] = R(U[e].real());
        m.i[e] = R(U[e].imag());
    }
    return m;
}

// Derivatives of the gate matrix with respect to each trainable angle (the
// matrices of qv.h differentiated in closed form). Returns how many.
int gate_derivs(const qv_gate &g, cd dU[3][4], int slot[3])
{
    const double th = g.theta[0], ph = g.theta[1], la = g.theta[2];
    const cd I(0, 1);
    const double c = std::cos(th / 2), s = std::sin(th / 2);
    int nd = 0;
    auto put = [&](int sl, cd a, cd b, cd cc, cd d) {
        dU[nd][0] = a; dU[nd][1] = b; dU[nd][2] = cc; dU[nd][3] = d;
        slot[nd] = sl;
        ++nd;
    };
    switch (g.kind) {
    case QV_G_RX:
        if (g.param[0] >= 0) put(0, -0.5 * s, -0.5 * I * c, -0.5 * I * c, -0.5 * s);
        break;
    case QV_G_RY:
        if (g.param[0] >= 0) put(0, -0.5 * s, -0.5 * c, 0.5 * c, -0.5 * s);
        break;
    case QV_G_RZ:
        if (g.param[0] >= 0) put(0, -0.5 * I * std::polar(1.0, -th / 2), 0, 0, 0.5 * I * std::polar(1.0, th / 2));
        break;
    case QV_G_P:
        if (g.param[0] >= 0) put(0, 0, 0, 0, I * std::polar(1.0, th));
        break;
    case QV_G_U3:
        if (g.param[0] >= 0)
            put(0, -0.5 * s, -0.5 * std::polar(1.0, la) * c, 0.5 * std::polar(1.0, ph) * c,
                -0.5 * std::polar(1.0, ph + la) * s);
        if (g.param[1] >= 0) put(1, 0, 0, I * std::polar(1.0, ph) * s, I * std::polar(1.0, ph + la) * c);
        if (g.param[2] >= 0) put(2, 0, -I * std::polar(1.0, la) * s, 0, I * std::polar(1.0, ph + la) * c);
        break;
    default: break;
    }
    return nd;
}

unsigned grid_of(const qv_state *s, uint64_t work)
{
    const uint64_t want = (work + kThreads - 1) / kThreads;
    return unsigned(std::max<uint64_t>(1, std::min<uint64_t>(want, uint64_t(s->num_sms) * 4)));
}

template <typename R>
qv_status pauli_apply_impl(qv_state *s, const void *src, void *dst, const qv_pauli_term *terms, size_t nt)
{
    std::vector<PauliGroupA<R>> groups;
    for (size_t k = 0; k < nt; ++k) {
        const uint64_t x = terms[k].xmask, z = terms[k].zmask;
        const int ny = __builtin_popcountll(x & z);
        static const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, 1, 0, -1};
        PauliGroupA<R> *g = nullptr;
        for (auto &gg : groups)
            if (gg.x == x && gg.nt < kMaxTerms) { g = &gg; break; }
        if (!g) {
            groups.emplace_back();
            g = &groups.back();
            std::memset(g, 0, sizeof *g);
            g->x = x;
        }
        g->z[g->nt] = z;
        g->cre[g->nt] = R(terms[k].coeff * pr[ny & 3]);
        g->cim[g->nt] = R(terms[k].coeff * pi[ny & 3]);
        g->nt++;
    }
    for (PauliGroupA<R> &gg : groups) {
        gg.zero_z = 1;
        gg.has_im = 0;
        double c0r = 0, c0i = 0;
        for (int k = 0; k < gg.nt; ++k) {
            gg.zero_z &= gg.z[k] == 0;
            gg.has_im |= gg.cim[k] != R(0);
            c0r += double(gg.cre[k]);
            c0i += double(gg.cim[k]);
        }
        gg.c0re = R(c0r);
        gg.c0im = R(c0i);
    }
    // the pure-Z group's terms that lie inside one 8-bit chunk of the index go into tables
    // (only when the tables fit in shared memory beside the groups)
    const std::vector<R> htab = groups.size() * sizeof(PauliGroupA<R>) + kZTabWords * sizeof(R) <= 200 * 1024
                                    ? ztab_for_group<R>(s->n, groups)
                                    : std::vector<R>();
    const size_t gbytes = groups.size() * sizeof(PauliGroupA<R>), tbytes = htab.size() * sizeof(R);
    if (gbytes + tbytes > 200 * 1024)
        return fail(QV_ERR_UNSUPPORTED, "Hamiltonian too large (%zu X-mask groups)", groups.size());
    QV_TRY(ensure_scratch(s, std::max<size_t>(gbytes + tbytes, 8)));
    if (!groups.empty()) QV_TRY(copy_h2d(s, s->scratch.ptr, groups.data(), gbytes));
    R *dtab = reinterpret_cast<R *>(static_cast<char *>(s->scratch.ptr) + gbytes);
    if (tbytes) QV_TRY(copy_h2d(s, dtab, htab.data(), tbytes));
    QV_TRY(allow_smem(reinterpret_cast<const void *>(pauli_apply_kernel<R>), 200 * 1024));
    prof_bytes(s, QV_K_PAULI, double(dim(s)) * 2 * sizeof(R) * (2 + groups.size()));
    QV_LAUNCH(s, QV_K_PAULI,
              pauli_apply_kernel<R><<<grid_of(s, dim(s)), kThreads, gbytes + tbytes, s->stream>>>(
                  static_cast<const R *>(src), static_cast<R *>(dst), dim(s),
                  static_cast<const PauliGroupA<R> *>(s->scratch.ptr), int(groups.size()), dtab, int(htab.size())));
    return QV_OK;
}

// ---------------------------------------------------------------- tiled reverse sweep
// The reverse sweep in tiles, as the forward pass does it (Sec. III-B/C/E
// blocking applied to both buffers): a pass loads a tile of 2^K amplitudes of
// psi and of lambda into shared memory (the 5 lowest qubits plus K - 5 chosen
// ones), runs a run of consecutive reverse-order gates whose targets lie in
// the tile (controls and diagonal targets may lie outside, where they are
// uniform per tile), and stores both tiles once. Each derivative is summed per
// thread over its pairs of one tile (at most 16 terms, plain sum), per warp
// with two-sum compensation in the state's precision, per CTA across tiles in
// shared memory (compensated), then in FP64 across warps and CTAs.
namespace tiles {

constexpr int kT = 256;          // threads per CTA
constexpr int kLow = 5;          // contiguous low qubits of every tile
constexpr int kMaxSlots = 96;    // derivative slots per pass
constexpr int kMaxKt = 12;

enum : int32_t { AG_PAIR = 0, AG_DIAG = 1, AG_SWAP = 2, AG_SIGN = 3, AG_PAIR_REAL = 4 };
// AG_SIGN: diagonal, entries +-1, no trainable angle (Z, CZ); AG_PAIR_REAL: a
// 2x2 whose matrix and derivatives are real (RY, H, X), no control.

template <typename R> struct AGate {
    int32_t kind;       // AG_*
    int32_t t, t2;      // tile positions: target (PAIR; DIAG, -1 if outside), both qubits (SWAP)
    int32_t cpos;       // control tile position, -1 if none in the tile
    uint64_t cext;      // control outside the tile (physical mask), 0 if none
    uint64_t text;      // AG_DIAG with the target outside the tile (physical mask)
    int32_t nd, lslot;  // trainable angles, first local slot
    R ud[8];            // U^dagger, (re, im) row-major
    R du[3][8];         // dU / d angle
};

struct AHead {
    int32_t ngates, nslots, nseg, pad;
    int32_t s_high[kMaxKt - kLow];
    int32_t seg_src[kMaxKt + 1], seg_w[kMaxKt + 1], seg_dst[kMaxKt + 1];
    int32_t gslot[kMaxSlots];  // global slot of each local slot
};

template <typename R> struct MaxG { static constexpr int v = 160; };
template <> struct MaxG<double> { static constexpr int v = 96; };

// One pass, passed by value (kernel parameter space, read through the constant bank).
template <typename R> struct AProg {
    AHead h;
    AGate<R> g[MaxG<R>::v];
};
static_assert(sizeof(AProg<float>) < 32000 && sizeof(AProg<double>) < 32000, "kernel parameter limit");

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

// Compensated warp sum in precision R: (hi, lo) of every lane -> the warp's
// total, two-sum on the high parts, low parts added (no FP64 per tile: FP64
// runs at a small fraction of the FP32 rate on this GPU).
template <typename R> __device__ __forceinline__ void warp_comp_sum(R &hi, R &lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const R h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        R sum, err;
        two_sum(hi, h2, sum, err);
        hi = sum;
        lo += l2 + err;
    }
}

template <typename R> __device__ __forceinline__ Mat2<R> mat_of(const R (&m)[8])
{
    Mat2<R> u;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        u.r[e] = m[2 * e];
        u.i[e] = m[2 * e + 1];
    }
    return u;
}

// x with a 0 inserted at bit b (32-bit tile indices)
__device__ __forceinline__ int ins0(int x, int b) { return ((x >> b) << (b + 1)) | (x & ((1 << b) - 1)); }

// One 2x2 gate of the reverse sweep on the tile (pairs along tile position
// A.t; with CTRL only pairs whose control bit is 1): psi <- Ud psi, then
// g[d] += 2 Re <lambda | dU_d psi> over this thread's pairs, lambda <- Ud lambda.
template <typename R, int NT, int ND, bool CTRL>
__device__ __forceinline__ void tile_pair(typename V2<R>::T *sp, typename V2<R>::T *sl, const AGate<R> &A,
                                          R (&g)[3], int tid)
{
    using V = typename V2<R>::T;
    const Mat2<R> ud = mat_of<R>(A.ud);
    Mat2<R> dm[ND > 0 ? ND : 1];
#pragma unroll
    for (int d = 0; d < ND; ++d) dm[d] = mat_of<R>(A.du[d]);
    const int tq = A.t;
    const int lo = CTRL ? min(tq, A.cpos) : tq, hi = CTRL ? max(tq, A.cpos) : 0;
    const int cset = CTRL ? (1 << A.cpos) : 0;
    constexpr int NP = CTRL ? NT / 4 : NT / 2;
#pragma unroll
    for (int j0 = 0; j0 < NP; j0 += kT) {
        const int j = j0 + tid;
        int i0 = ins0(j, lo);
        if (CTRL) i0 = ins0(i0, hi) | cset;
        const int i1 = i0 | (1 << tq);
        V a0 = sp[i0], a1 = sp[i1], l0 = sl[i0], l1 = sl[i1];
        apply2(ud, a0.x, a0.y, a1.x, a1.y);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            R xr = a0.x, xi = a0.y, yr = a1.x, yi = a1.y;
            apply2(dm[d], xr, xi, yr, yi);
            g[d] += R(2) * (l0.x * xr + l0.y * xi + l1.x * yr + l1.y * yi);
        }
        apply2(ud, l0.x, l0.y, l1.x, l1.y);
        sp[i0] = a0;
        sp[i1] = a1;
        sl[i0] = l0;
        sl[i1] = l1;
    }
}

// apply2 for a real matrix (imaginary parts zero): half the multiplications
template <typename R>
__device__ __forceinline__ void apply2_real(const Mat2<R> &U, R &ar, R &ai, R &br, R &bi)
{
    const R xr = ar, xi = ai, yr = br, yi = bi;
    ar = U.r[0] * xr + U.r[1] * yr;
    ai = U.r[0] * xi + U.r[1] * yi;
    br = U.r[2] * xr + U.r[3] * yr;
    bi = U.r[2] * xi + U.r[3] * yi;
}

// tile_pair for a real, uncontrolled gate
template <typename R, int NT, int ND>
__device__ __forceinline__ void tile_pair_real(typename V2<R>::T *sp, typename V2<R>::T *sl, const AGate<R> &A,
                                               R (&g)[3], int tid)
{
    using V = typename V2<R>::T;
    const Mat2<R> ud = mat_of<R>(A.ud);
    Mat2<R> dm[ND > 0 ? ND : 1];
#pragma unroll
    for (int d = 0; d < ND; ++d) dm[d] = mat_of<R>(A.du[d]);
    const int tq = A.t;
#pragma unroll
    for (int j0 = 0; j0 < NT / 2; j0 += kT) {
        const int i0 = ins0(j0 + tid, tq), i1 = i0 | (1 << tq);
        V a0 = sp[i0], a1 = sp[i1], l0 = sl[i0], l1 = sl[i1];
        apply2_real(ud, a0.x, a0.y, a1.x, a1.y);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            R xr = a0.x, xi = a0.y, yr = a1.x, yi = a1.y;
            apply2_real(dm[d], xr, xi, yr, yi);
            g[d] += R(2) * (l0.x * xr + l0.y * xi + l1.x * yr + l1.y * yi);
        }
        apply2_real(ud, l0.x, l0.y, l1.x, l1.y);
        sp[i0] = a0;
        sp[i1] = a1;
        sl[i0] = l0;
        sl[i1] = l1;
    }
}

// A diagonal gate with entries +-1 and nothing to differentiate: sign flips.
template <typename R, int NT>
__device__ __forceinline__ void tile_sign(typename V2<R>::T *sp, typename V2<R>::T *sl, const AGate<R> &A, bool up,
                                          int tid)
{
    using V = typename V2<R>::T;
    const R s0 = A.ud[0], s3 = A.ud[6];
    const int t = A.t, c = A.cpos;
#pragma unroll
    for (int l0 = 0; l0 < NT; l0 += kT) {
        const int l = l0 + tid;
        if (c >= 0 && !((l >> c) & 1)) continue;
        const R f = (t >= 0 ? ((l >> t) & 1) != 0 : up) ? s3 : s0;
        V x = sp[l], y = sl[l];
        x.x *= f;
        x.y *= f;
        y.x *= f;
        y.y *= f;
        sp[l] = x;
        sl[l] = y;
    }
}

// A diagonal gate: one complex factor per amplitude, chosen by the target bit
// (tile position A.t, or `up` for a target outside the tile).
template <typename R, int NT, int ND>
__device__ __forceinline__ void tile_diag(typename V2<R>::T *sp, typename V2<R>::T *sl, const AGate<R> &A, bool up,
                                          R (&g)[3], int tid)
{
    using V = typename V2<R>::T;
    const R u0r = A.ud[0], u0i = A.ud[1], u3r = A.ud[6], u3i = A.ud[7];
    R d0r[ND > 0 ? ND : 1], d0i[ND > 0 ? ND : 1], d3r[ND > 0 ? ND : 1], d3i[ND > 0 ? ND : 1];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        d0r[d] = A.du[d][0];
        d0i[d] = A.du[d][1];
        d3r[d] = A.du[d][6];
        d3i[d] = A.du[d][7];
    }
    const int t = A.t, c = A.cpos;
#pragma unroll
    for (int l0 = 0; l0 < NT; l0 += kT) {
        const int l = l0 + tid;
        if (c >= 0 && !((l >> c) & 1)) continue;
        const bool one = t >= 0 ? ((l >> t) & 1) != 0 : up;
        V x = sp[l], y = sl[l];
        cmul(one ? u3r : u0r, one ? u3i : u0i, x.x, x.y);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            R zr = x.x, zi = x.y;
            cmul(one ? d3r[d] : d0r[d], one ? d3i[d] : d0i[d], zr, zi);
            g[d] += R(2) * (y.x * zr + y.y * zi);
        }
        cmul(one ? u3r : u0r, one ? u3i : u0i, y.x, y.y);
        sp[l] = x;
        sl[l] = y;
    }
}

template <typename R> constexpr size_t smem_bytes(int K)
{
    return 2 * (size_t(1) << K) * sizeof(typename V2<R>::T) + (size_t(1) << (K - kLow)) * 8 +
           size_t(kMaxSlots) * (kT / 32) * sizeof(CompSum<R>);
}

// part[gslot * G + blockIdx.x] = this CTA's sum of each derivative of the pass.
template <typename R, int K>
__global__ void __launch_bounds__(kT) adj_tile_kernel(R *__restrict__ psi, R *__restrict__ lam, uint64_t ntiles,
                                                      const __grid_constant__ AProg<R> P, double *part, int G)
{
    using V = typename V2<R>::T;
    constexpr int NT = 1 << K;
    extern __shared__ __align__(16) unsigned char smem[];
    V *sp = reinterpret_cast<V *>(smem);
    V *sl = sp + NT;
    uint64_t *phys_hi = reinterpret_cast<uint64_t *>(sl + NT);
    CompSum<R> *acc = reinterpret_cast<CompSum<R> *>(phys_hi + (NT >> kLow));  // [slot][warp]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const AHead &h = P.h;
    for (int i = tid; i < (NT >> kLow); i += kT) {
        uint64_t v = 0;
        for (int j = 0; j < K - kLow; ++j)
            if ((i >> j) & 1) v |= uint64_t(1) << h.s_high[j];
        phys_hi[i] = v;
    }
    for (int i = tid; i < h.nslots * (kT / 32); i += kT) acc[i] = CompSum<R>();
    __syncthreads();
    V *gp = reinterpret_cast<V *>(psi), *gl = reinterpret_cast<V *>(lam);
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint64_t base = 0;
        for (int q = 0; q < h.nseg; ++q)
            base |= ((t >> h.seg_src[q]) & ((uint64_t(1) << h.seg_w[q]) - 1)) << h.seg_dst[q];
        for (int l = tid; l < NT; l += kT) {
            const uint64_t gi = base | uint64_t(l & 31) | phys_hi[l >> kLow];
            sp[l] = gp[gi];
            sl[l] = gl[gi];
        }
        __syncthreads();
        for (int a = 0; a < h.ngates; ++a) {
            const AGate<R> &A = P.g[a];
            if (A.cext && !(base & A.cext)) continue;  // control outside the tile is 0: uniform skip
            if (A.kind == AG_SWAP) {
                const int lo = min(A.t, A.t2), hi = max(A.t, A.t2);
                for (int u = tid; u < NT / 4; u += kT) {
                    const int i = int(insert_zero(insert_zero(uint64_t(u), lo), hi));
                    const int i1 = i | (1 << A.t), i2 = i | (1 << A.t2);
                    V x = sp[i1];
                    sp[i1] = sp[i2];
                    sp[i2] = x;
                    x = sl[i1];
                    sl[i1] = sl[i2];
                    sl[i2] = x;
                }
                __syncthreads();
                continue;
            }
            R gs[3] = {R(0), R(0), R(0)};
            if (A.kind == AG_SIGN) {
                tile_sign<R, NT>(sp, sl, A, (base & A.text) != 0, tid);
            } else if (A.kind == AG_PAIR_REAL) {
                switch (A.nd) {
                case 0: tile_pair_real<R, NT, 0>(sp, sl, A, gs, tid); break;
                case 1: tile_pair_real<R, NT, 1>(sp, sl, A, gs, tid); break;
                case 2: tile_pair_real<R, NT, 2>(sp, sl, A, gs, tid); break;
                default: tile_pair_real<R, NT, 3>(sp, sl, A, gs, tid); break;
                }
            } else if (A.kind == AG_DIAG) {
                const bool up = (base & A.text) != 0;  // target bit when the target lies outside
                switch (A.nd) {
                case 0: tile_diag<R, NT, 0>(sp, sl, A, up, gs, tid); break;
                case 1: tile_diag<R, NT, 1>(sp, sl, A, up, gs, tid); break;
                case 2: tile_diag<R, NT, 2>(sp, sl, A, up, gs, tid); break;
                default: tile_diag<R, NT, 3>(sp, sl, A, up, gs, tid); break;
                }
            } else if (A.cpos >= 0) {
                switch (A.nd) {
                case 0: tile_pair<R, NT, 0, true>(sp, sl, A, gs, tid); break;
                case 1: tile_pair<R, NT, 1, true>(sp, sl, A, gs, tid); break;
                case 2: tile_pair<R, NT, 2, true>(sp, sl, A, gs, tid); break;
                default: tile_pair<R, NT, 3, true>(sp, sl, A, gs, tid); break;
                }
            } else {
                switch (A.nd) {
                case 0: tile_pair<R, NT, 0, false>(sp, sl, A, gs, tid); break;
                case 1: tile_pair<R, NT, 1, false>(sp, sl, A, gs, tid); break;
                case 2: tile_pair<R, NT, 2, false>(sp, sl, A, gs, tid); break;
                default: tile_pair<R, NT, 3, false>(sp, sl, A, gs, tid); break;
                }
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d >= A.nd) break;
                R hi = gs[d], lo = R(0);
                warp_comp_sum(hi, lo);
                if (lane == 0) {
                    CompSum<R> &c = acc[(A.lslot + d) * (kT / 32) + warp];
                    c.add(hi);
                    c.lo += lo;
                }
            }
            __syncthreads();
        }
        for (int l = tid; l < NT; l += kT) {
            const uint64_t gi = base | uint64_t(l & 31) | phys_hi[l >> kLow];
            gp[gi] = sp[l];
            gl[gi] = sl[l];
        }
        __syncthreads();
    }
    for (int sidx = tid; sidx < h.nslots; sidx += kT) {
        double v = 0;
        for (int w = 0; w < kT / 32; ++w) v += acc[sidx * (kT / 32) + w].value();
        part[size_t(h.gslot[sidx]) * G + blockIdx.x] = v;
    }
}

}  // namespace tiles

// Reverse sweep in tiled passes. gate_slot[l] = global slot of gate l's first
// trainable angle. part has G columns per slot and must be zero beforehand
// (a pass writes only the columns of the CTAs it launches).
template <typename R>
qv_status adjoint_sweep_tiled(qv_state *s, const qv_gate *g, size_t ng, const std::vector<int> &gate_slot,
                              double *part, int G)
{
    using namespace tiles;
    const int n = s->n;
    const int K = std::min(n, sizeof(R) == 4 ? 12 : 11);
    const int maxg = MaxG<R>::v;
    auto kern = K == 12 ? adj_tile_kernel<R, 12> : K == 11 ? adj_tile_kernel<R, 11> : adj_tile_kernel<R, 10>;
    const size_t smem = smem_bytes<R>(K);
    QV_TRY(allow_smem(reinterpret_cast<const void *>(kern), int(smem)));
    int per_sm = 0;
    QV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, smem));
    if (per_sm < 1) return fail(QV_ERR_UNSUPPORTED, "tiled reverse sweep does not fit on an SM");
    const uint64_t ntiles = dim(s) >> K;
    const unsigned grid = unsigned(std::min<uint64_t>({ntiles, uint64_t(per_sm) * s->num_sms, uint64_t(G)}));
    R *psi = static_cast<R *>(s->amp), *lam = static_cast<R *>(s->adj->lam);

    // A gate is applied as diagonal (target may lie outside the tile) when its
    // matrix and every derivative matrix are diagonal: RX(0) is the identity,
    // but its derivative is not.
    auto diagonal = [&](const qv_gate &G1) {
        cd U[4], dU[3][4];
        int sl[3];
        gate_matrix(G1, U);
        bool d = U[1] == 0.0 && U[2] == 0.0;
        const int nd = gate_derivs(G1, dU, sl);
        for (int k = 0; k < nd; ++k) d &= dU[k][1] == 0.0 && dU[k][2] == 0.0;
        return d;
    };
    std::vector<size_t> rem;  // gates still to sweep, in reverse order
    for (size_t l = ng; l-- > 0;) rem.push_back(l);
    auto prog = std::make_unique<AProg<R>>();
    while (!rem.empty()) {
        std::vector<char> inS(n, 0), blocked(n, 0);
        for (int q = 0; q < kLow; ++q) inS[q] = 1;
        int room = K - kLow, nslots = 0;
        std::vector<size_t> taken, left;
        for (size_t l : rem) {
            const qv_gate &G1 = g[l];
            int qs[3], nq = 0;
            qs[nq++] = G1.target;
            if (G1.kind == QV_G_SWAP) qs[nq++] = G1.target2;
            if (G1.ctrl >= 0) qs[nq++] = G1.ctrl;
            bool blk = false;
            for (int i = 0; i < nq; ++i) blk |= blocked[qs[i]] != 0;
            bool ok = !blk && int(taken.size()) < maxg;
            int need[2], nn = 0;
            int nd = 0;
            if (ok) {
                if (G1.kind == QV_G_SWAP) {
                    need[nn++] = G1.target;
                    need[nn++] = G1.target2;
                } else {
                    if (!diagonal(G1)) need[nn++] = G1.target;
                    for (int a = 0; a < 3; ++a) nd += G1.param[a] >= 0;
                }
                int add = 0;
                for (int i = 0; i < nn; ++i) add += !inS[need[i]];
                ok = add <= room && nslots + nd <= kMaxSlots;
            }
            if (ok) {
                for (int i = 0; i < nn; ++i)
                    if (!inS[need[i]]) {
                        inS[need[i]] = 1;
                        --room;
                    }
                nslots += nd;
                taken.push_back(l);
            } else {
                for (int i = 0; i < nq; ++i) blocked[qs[i]] = 1;
                left.push_back(l);
            }
        }
        if (taken.empty()) return fail(QV_ERR_UNSUPPORTED, "tiled reverse sweep made no progress");
        for (int q = kLow; q < n && room > 0; ++q)
            if (!inS[q]) {
                inS[q] = 1;
                --room;
            }
        AHead &hd = prog->h;
        std::memset(&hd, 0, sizeof hd);
        std::vector<int> pos_of(n, -1);
        for (int q = 0; q < kLow; ++q) pos_of[q] = q;
        int j = 0;
        for (int q = kLow; q < n; ++q)
            if (inS[q]) {
                hd.s_high[j] = q;
                pos_of[q] = kLow + j;
                ++j;
            }
        int src = 0;
        for (int q = 0; q < n;) {
            if (inS[q]) {
                ++q;
                continue;
            }
            int w = 0;
            while (q + w < n && !inS[q + w]) ++w;
            hd.seg_src[hd.nseg] = src;
            hd.seg_w[hd.nseg] = w;
            hd.seg_dst[hd.nseg] = q;
            hd.nseg++;
            src += w;
            q += w;
        }
        hd.ngates = int(taken.size());
        for (size_t a = 0; a < taken.size(); ++a) {
            const qv_gate &G1 = g[taken[a]];
            AGate<R> &A = prog->g[a];
            std::memset(&A, 0, sizeof A);
            A.cpos = -1;
            if (G1.ctrl >= 0) {
                if (pos_of[G1.ctrl] >= 0) A.cpos = pos_of[G1.ctrl];
                else A.cext = uint64_t(1) << G1.ctrl;
            }
            if (G1.kind == QV_G_SWAP) {
                A.kind = AG_SWAP;
                A.t = pos_of[G1.target];
                A.t2 = pos_of[G1.target2];
                continue;
            }
            cd U[4], dU[3][4];
            gate_matrix(G1, U);
            const cd Ud[4] = {std::conj(U[0]), std::conj(U[2]), std::conj(U[1]), std::conj(U[3])};
            for (int e = 0; e < 4; ++e) {
                A.ud[2 * e] = R(Ud[e].real());
                A.ud[2 * e + 1] = R(Ud[e].imag());
            }
            int sl[3];
            A.nd = gate_derivs(G1, dU, sl);
            for (int d = 0; d < A.nd; ++d)
                for (int e = 0; e < 4; ++e) {
                    A.du[d][2 * e] = R(dU[d][e].real());
                    A.du[d][2 * e + 1] = R(dU[d][e].imag());
                }
            if (A.nd) {
                A.lslot = hd.nslots;
                for (int d = 0; d < A.nd; ++d) hd.gslot[hd.nslots++] = gate_slot[taken[a]] + d;
            }
            A.kind = diagonal(G1) ? AG_DIAG : AG_PAIR;
            bool real = true;  // matrix and derivatives real
            for (int e = 0; e < 4; ++e) {
                real &= U[e].imag() == 0.0;
                for (int d = 0; d < A.nd; ++d) real &= dU[d][e].imag() == 0.0;
            }
            if (A.kind == AG_DIAG && real && A.nd == 0 && std::abs(U[0].real()) == 1.0 && std::abs(U[3].real()) == 1.0)
                A.kind = AG_SIGN;
            if (A.kind == AG_PAIR && real && G1.ctrl < 0) A.kind = AG_PAIR_REAL;
            A.t = pos_of[G1.target];  // -1 (outside the tile) only for a diagonal gate
            if (A.t < 0) A.text = uint64_t(1) << G1.target;
        }
        prof_bytes(s, QV_K_ADJOINT, 4.0 * double(dim(s)) * amp_bytes(s->dt));
        QV_LAUNCH(s, QV_K_ADJOINT, kern<<<grid, kT, smem, s->stream>>>(psi, lam, ntiles, *prog, part, G));
        rem.swap(left);
    }
    return QV_OK;
}

// Reverse sweep as compiled passes (complex64): the daggered gates in reverse
// order, planned like a forward circuit; each gate with trainable angles
// carries its derivative matrices and gets an op of its own.
qv_status adjoint_sweep_compiled(qv_state *s, const qv_gate *g, size_t ng, const std::vector<int> &gate_slot,
                                 double *part, int G)
{
    AdjointBuffers &B = *s->adj;
    if (B.sweep && B.key.size() == ng && std::memcmp(B.key.data(), g, ng * sizeof(qv_gate)) == 0)
        return jit_launch_adjoint(s, *B.sweep, B.lam, part, G);
    B.key.clear();
    B.sweep.reset();
    std::vector<plan::PGate> pg;
    pg.reserve(ng);
    for (size_t l = ng; l-- > 0;) {
        const qv_gate &G1 = g[l];
        plan::PGate p{};
        p.t = G1.target;
        p.t2 = -1;
        p.c = G1.ctrl;
        if (G1.kind == QV_G_SWAP) {
            p.cls = plan::G_SWAP;
            p.t2 = G1.target2;
            pg.push_back(p);
            continue;
        }
        cd U[4], dU[3][4];
        gate_matrix(G1, U);
        p.U[0] = std::conj(U[0]);
        p.U[1] = std::conj(U[2]);
        p.U[2] = std::conj(U[1]);
        p.U[3] = std::conj(U[3]);
        int sl[3];
        p.nd = gate_derivs(G1, dU, sl);
        p.slot = p.nd ? gate_slot[l] : -1;
        for (int d = 0; d < p.nd; ++d)
            for (int e = 0; e < 4; ++e) p.dU[d][e] = dU[d][e];
        p.cls = p.nd > 0 ? plan::G_GEN : plan::classify(p.U);
        if (p.nd == 1 && G1.param[0] >= 0)
            p.gen = G1.kind == QV_G_RX ? 1 : G1.kind == QV_G_RY ? 2 : G1.kind == QV_G_RZ ? 3 : G1.kind == QV_G_P ? 4 : 0;
        pg.push_back(p);
    }
    std::vector<plan::Pass> passes;
    plan::PlanStats st;
    std::string err;
    const int K = std::min(s->n, plan::kMaxK);
    if (!plan::make_plan(s->n, K, true, true, false, pg, passes, st, err))
        return fail(QV_ERR_UNSUPPORTED, "planner: %s", err.c_str());
    QV_TRY(jit_prepare_adjoint(s, passes, B.sweep));
    B.key.assign(g, g + ng);
    return jit_launch_adjoint(s, *B.sweep, B.lam, part, G);
}

template <typename R>
qv_status adjoint_impl(qv_state *s, const qv_gate *g, size_t ng, const qv_pauli_term *H, size_t nt, size_t nparams,
                       double *grad_out, double *expval_out, int sweep)
{
    if (!s->adj) s->adj = new AdjointBuffers;
    AdjointBuffers &B = *s->adj;
    const size_t bytes = dim(s) * amp_bytes(s->dt);
    if (B.lam_bytes < bytes) {
        if (B.lam) {
            QV_TRY(sync_and_check(s));
            QV_CUDA(cudaFree(B.lam));
            B.lam = nullptr;
            B.lam_bytes = 0;
        }
        QV_CUDA(cudaMalloc(&B.lam, bytes));
        B.lam_bytes = bytes;
    }
    // derivative slots: (gate, angle) pairs with a parameter index
    struct Slot {
        size_t gate;
        int angle;
    };
    std::vector<Slot> slots;
    for (size_t l = 0; l < ng; ++l)
        for (int a = 0; a < 3; ++a)
            if (g[l].param[a] >= 0) {
                if (size_t(g[l].param[a]) >= nparams)
                    return fail(QV_ERR_ARG, "gate %zu: parameter index %d >= nparams %zu", l, g[l].param[a], nparams);
                slots.push_back({l, a});
            }
    const unsigned grid = unsigned(s->num_sms) * 4;
    const size_t need = (slots.size() + 1) * size_t(grid) + slots.size() + 1;
    if (B.part_count < need) {
        if (B.part) {
            QV_TRY(sync_and_check(s));
            QV_CUDA(cudaFree(B.part));
            B.part = nullptr;
        }
        QV_CUDA(cudaMalloc(&B.part, need * sizeof(double)));
        B.part_count = need;
    }
    double *part = B.part;                                // [slot][grid], then [grid] for the energy
    double *sums = B.part + (slots.size() + 1) * grid;    // slot sums, then the energy

    // 1. forward: psi <- U_L ... U_1 psi
    qv_plan_opts po{};
    po.mode = QV_MODE_AUTO;
    if (fused_supported(s, &po)) QV_TRY(apply_fused(s, g, ng, &po));
    else
        for (size_t l = 0; l < ng; ++l) QV_TRY(apply_gate_plain(s, g[l]));
    // 2. lambda = H psi, E = Re <psi|lambda>
    QV_TRY(pauli_apply_impl<R>(s, s->amp, B.lam, H, nt));
    prof_bytes(s, QV_K_ADJOINT, double(bytes) * 2);
    QV_LAUNCH(s, QV_K_ADJOINT,
              inner_re_kernel<R><<<grid, kThreads, 0, s->stream>>>(static_cast<const R *>(s->amp),
                                                                    static_cast<const R *>(B.lam), dim(s),
                                                                    part + slots.size() * grid));
    // 3. reverse sweep
    R *psi = static_cast<R *>(s->amp), *lam = static_cast<R *>(B.lam);
    size_t slot_next = slots.size();
    const bool use_tiles = sweep != QV_SWEEP_PER_GATE && s->n >= 10;
    if (use_tiles) {
        std::vector<int> gate_slot(ng, -1);
        for (size_t k = slots.size(); k-- > 0;) gate_slot[slots[k].gate] = int(k);
        if (!slots.empty()) QV_CUDA(cudaMemsetAsync(part, 0, slots.size() * grid * sizeof(double), s->stream));
        const bool compiled = sweep != QV_SWEEP_TILES && sizeof(R) == 4 && jit_available(nullptr);
        if (compiled) QV_TRY(adjoint_sweep_compiled(s, g, ng, gate_slot, part, int(grid)));
        else QV_TRY(adjoint_sweep_tiled<R>(s, g, ng, gate_slot, part, int(grid)));
    }
    for (size_t l = use_tiles ? 0 : ng; l-- > 0;) {
        const qv_gate &G = g[l];
        if (G.kind == QV_G_SWAP) {
            const uint64_t units = dim(s) >> 2;
            prof_bytes(s, QV_K_ADJOINT, double(units) * 8 * sizeof(R) * 2);
            QV_LAUNCH(s, QV_K_ADJOINT, swap2_kernel<R><<<grid_of(s, units), kThreads, 0, s->stream>>>(
                                           psi, lam, units, G.target, G.target2));
            continue;
        }
        cd U[4], Ud[4], dU[3][4];
        gate_matrix(G, U);
        Ud[0] = std::conj(U[0]);
        Ud[1] = std::conj(U[2]);
        Ud[2] = std::conj(U[1]);
        Ud[3] = std::conj(U[3]);
        int sl[3];
        const int nd = gate_derivs(G, dU, sl);
        const uint64_t pairs = dim(s) >> (G.ctrl >= 0 ? 2 : 1);
        const Mat2<R> m0 = to_mat<R>(nd > 0 ? dU[0] : U), m1 = to_mat<R>(nd > 1 ? dU[1] : U),
                      m2 = to_mat<R>(nd > 2 ? dU[2] : U);
        slot_next -= nd;
        double *pp = part + slot_next * grid;
        prof_bytes(s, QV_K_ADJOINT, double(pairs) * 8 * sizeof(R) * 2);
        const Mat2<R> ud = to_mat<R>(Ud);
        switch (nd) {
        case 0:
            QV_LAUNCH(s, QV_K_ADJOINT, adjoint_step_kernel<R, 0><<<grid, kThreads, 0, s->stream>>>(
                                           psi, lam, pairs, G.target, G.ctrl, ud, m0, m1, m2, pp));
            break;
        case 1:
            QV_LAUNCH(s, QV_K_ADJOINT, adjoint_step_kernel<R, 1><<<grid, kThreads, 0, s->stream>>>(
                                           psi, lam, pairs, G.target, G.ctrl, ud, m0, m1, m2, pp));
            break;
        case 2:
            QV_LAUNCH(s, QV_K_ADJOINT, adjoint_step_kernel<R, 2><<<grid, kThreads, 0, s->stream>>>(
                                           psi, lam, pairs, G.target, G.ctrl, ud, m0, m1, m2, pp));
            break;
        default:
            QV_LAUNCH(s, QV_K_ADJOINT, adjoint_step_kernel<R, 3><<<grid, kThreads, 0, s->stream>>>(
                                           psi, lam, pairs, G.target, G.ctrl, ud, m0, m1, m2, pp));
            break;
        }
    }
    // 4. reduce the partials: one row per slot, plus the energy row
    const int rows = int(slots.size()) + 1;
    QV_LAUNCH(s, QV_K_ADJOINT, rows_sum_kernel<<<rows, kThreads, 0, s->stream>>>(part, int(grid), sums));
    QV_TRY(ensure_host_out(s, rows));
    QV_TRY(copy_d2h(s, s->host_out, sums, sizeof(double) * rows));
    QV_TRY(sync_and_check(s));
    std::vector<Neumaier> acc(nparams);
    for (size_t k = 0; k < slots.size(); ++k) acc[g[slots[k].gate].param[slots[k].angle]].add(s->host_out[k]);
    if (grad_out)
        for (size_t p = 0; p < nparams; ++p) grad_out[p] = acc[p].value();
    if (expval_out) *expval_out = s->host_out[slots.size()];
    return QV_OK;
}

}  // namespace

qv_status pauli_apply(qv_state *s, const void *src, void *dst, const qv_pauli_term *terms, size_t nt)
{
    return s->dt == QV_C64 ? pauli_apply_impl<float>(s, src, dst, terms, nt)
                           : pauli_apply_impl<double>(s, src, dst, terms, nt);
}

qv_status adjoint_grad(qv_state *s, const qv_gate *g, size_t ng, const qv_pauli_term *H, size_t nt, size_t nparams,
                       double *grad_out, double *expval_out, int sweep)
{
    return s->dt == QV_C64 ? adjoint_impl<float>(s, g, ng, H, nt, nparams, grad_out, expval_out, sweep)
                           : adjoint_impl<double>(s, g, ng, H, nt, nparams, grad_out, expval_out, sweep);
}

void adjoint_release(qv_state *s)
{
    if (s->adj) {
        if (s->adj->lam) cudaFree(s->adj->lam);
        if (s->adj->part) cudaFree(s->adj->part);
        delete s->adj;
        s->adj = nullptr;
    }
}

}  // namespace qv
