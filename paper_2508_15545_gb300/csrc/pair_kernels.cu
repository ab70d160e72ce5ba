// Per-gate kernels: the amplitude-pairing update of Sec. III-A (Eq. 5), one
// pass over the state per gate, plus basis-state set-up, diagonal gates and
// qubit swaps.
//
// Work is split into "units". A unit of the high-target kernel is a group of W
// consecutive pairs: W amplitudes with bit t = 0 starting at `base` and their
// partners at base + 2^t, each loaded with 16-byte vector accesses (C64: W = 4,
// 32 bytes per half; C128: W = 2). Lanes of a warp take consecutive units, so
// both halves are read as contiguous runs. Low targets (t < log2 W) take units
// of 2W contiguous amplitudes and pair inside a thread's registers.
#include <algorithm>

#include "qv_device.cuh"
#include "qv_internal.h"

namespace qv {
namespace {

template <typename R> struct Traits;
template <> struct Traits<float> { static constexpr int W = 4, LOGW = 2; };
template <> struct Traits<double> { static constexpr int W = 2, LOGW = 1; };

constexpr int kThreads = 256;

template <typename R> Mat2<R> to_mat(const cd U[4])
{
    Mat2<R> m;
    for (int e = 0; e < 4; ++e) {
        m.r[e] = R(U[e].real());
        m.i[e] = R(U[e].imag());
    }
    return m;
}

unsigned grid_for(const qv_state *s, uint64_t units)
{
    const uint64_t want = (units + kThreads - 1) / kThreads;
    const uint64_t cap = uint64_t(s->num_sms) * 8;
    return unsigned(std::max<uint64_t>(1, std::min(want, cap)));
}

// ---------------------------------------------------------------- Eq. 5, t >= log2 W
// c_ins: control bit >= log2 W folded into the unit index (only control-1
// units exist); c_pred: control bit < log2 W tested per element; -1 = none.
template <typename R>
__global__ void __launch_bounds__(kThreads) pair_high_kernel(R *__restrict__ amp, uint64_t units, int t,
                                                             int c_ins, int c_pred, Mat2<R> U)
{
    constexpr int W = Traits<R>::W;
    const uint64_t tb = uint64_t(1) << t;
    const int lo = c_ins >= 0 ? min(t, c_ins) : t;
    const int hi = c_ins >= 0 ? max(t, c_ins) : -1;
    const uint64_t cset = c_ins >= 0 ? uint64_t(1) << c_ins : 0;
    for (uint64_t u = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < units;
         u += uint64_t(gridDim.x) * blockDim.x) {
        uint64_t base = insert_zero(u * W, lo);
        if (hi >= 0) base = insert_zero(base, hi);
        base |= cset;
        AmpGroup<R, W> a, b;
        load_group(amp, base, a);
        load_group(amp, base | tb, b);
#pragma unroll
        for (int e = 0; e < W; ++e)
            if (c_pred < 0 || ((e >> c_pred) & 1)) apply2(U, a.re[e], a.im[e], b.re[e], b.im[e]);
        store_group(amp, base, a);
        store_group(amp, base | tb, b);
    }
}

// ---------------------------------------------------------------- Eq. 5, t < log2 W
template <typename R, int T>
__global__ void __launch_bounds__(kThreads) pair_low_kernel(R *__restrict__ amp, uint64_t units, int c_ins,
                                                            int c_pred, Mat2<R> U)
{
    constexpr int W2 = 2 * Traits<R>::W;
    const uint64_t cset = c_ins >= 0 ? uint64_t(1) << c_ins : 0;
    for (uint64_t u = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < units;
         u += uint64_t(gridDim.x) * blockDim.x) {
        uint64_t base = u * W2;
        if (c_ins >= 0) base = insert_zero(base, c_ins);
        base |= cset;
        AmpGroup<R, W2> a;
        load_group(amp, base, a);
#pragma unroll
        for (int e = 0; e < W2; ++e) {
            if ((e >> T) & 1) continue;
            if (c_pred >= 0 && !((e >> c_pred) & 1)) continue;
            apply2(U, a.re[e], a.im[e], a.re[e + (1 << T)], a.im[e + (1 << T)]);
        }
        store_group(amp, base, a);
    }
}

// ---------------------------------------------------------------- diagonal gates
// Visits the W-groups whose bits ins0 / ins1 (>= log2 W, -1 = unused) are 1;
// inside a group only elements whose bits in pred_mask (< log2 W) are all 1
// change. Each changed amplitude is multiplied by d1 if bit `sel` of its index
// is 1, else by d0 (sel = -1: always d0).
template <typename R>
__global__ void __launch_bounds__(kThreads) diag_kernel(R *__restrict__ amp, uint64_t units, int ins0, int ins1,
                                                        unsigned pred_mask, int sel, R d0r, R d0i, R d1r, R d1i)
{
    constexpr int W = Traits<R>::W;
    uint64_t setbits = 0;
    if (ins0 >= 0) setbits |= uint64_t(1) << ins0;
    if (ins1 >= 0) setbits |= uint64_t(1) << ins1;
    for (uint64_t u = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < units;
         u += uint64_t(gridDim.x) * blockDim.x) {
        uint64_t base = u * W;
        if (ins0 >= 0) base = insert_zero(base, ins0);
        if (ins1 >= 0) base = insert_zero(base, ins1);
        base |= setbits;
        AmpGroup<R, W> a;
        load_group(amp, base, a);
#pragma unroll
        for (int e = 0; e < W; ++e) {
            if ((unsigned(e) & pred_mask) != pred_mask) continue;
            const bool one = sel >= 0 && (((base + e) >> sel) & 1);
            cmul(one ? d1r : d0r, one ? d1i : d0i, a.re[e], a.im[e]);
        }
        store_group(amp, base, a);
    }
}

// ---------------------------------------------------------------- swap / basis
template <typename R>
__global__ void __launch_bounds__(kThreads) swap_kernel(R *__restrict__ amp, uint64_t units, int a, int b)
{
    using V = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    V *v = reinterpret_cast<V *>(amp);
    const int lo = min(a, b), hi = max(a, b);
    for (uint64_t u = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < units;
         u += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t i = insert_zero(insert_zero(u, lo), hi);
        const uint64_t i1 = i | (uint64_t(1) << a), i2 = i | (uint64_t(1) << b);
        const V x = v[i1];
        v[i1] = v[i2];
        v[i2] = x;
    }
}

// States with fewer amplitudes than two register groups (C64: n <= 2, C128:
// n = 1): one thread walks Eq. 5 directly.
template <typename R>
__global__ void tiny_gate_kernel(R *amp, int n, int t, int ctrl, Mat2<R> U)
{
    const uint64_t N = uint64_t(1) << n, tb = uint64_t(1) << t;
    for (uint64_t i = 0; i < N; ++i) {
        if (i & tb) continue;
        if (ctrl >= 0 && !((i >> ctrl) & 1)) continue;
        const uint64_t j = i | tb;
        apply2(U, amp[2 * i], amp[2 * i + 1], amp[2 * j], amp[2 * j + 1]);
    }
}

template <typename R> __global__ void set_one_kernel(R *amp, uint64_t j)
{
    amp[2 * j] = R(1);
    amp[2 * j + 1] = R(0);
}

template <typename R> qv_status pair_impl(qv_state *s, int t, int ctrl, const cd Ud[4])
{
    constexpr int W = Traits<R>::W, LOGW = Traits<R>::LOGW;
    const int n = s->n;
    R *amp = static_cast<R *>(s->amp);
    const Mat2<R> U = to_mat<R>(Ud);
    if (dim(s) < uint64_t(2 * W)) {
        prof_bytes(s, QV_K_PAIR, 2.0 * double(dim(s)) * sizeof(R) * 2);
        QV_LAUNCH(s, QV_K_PAIR, tiny_gate_kernel<R><<<1, 1, 0, s->stream>>>(amp, n, t, ctrl, U));
    } else if (t >= LOGW) {
        // High target: units of W pairs. A control >= log2 W is folded into the index.
        const int c_ins = ctrl >= LOGW ? ctrl : -1;
        const int c_pred = (ctrl >= 0 && ctrl < LOGW) ? ctrl : -1;
        const uint64_t units = (dim(s) >> (c_ins >= 0 ? 2 : 1)) / W;
        if (units == 0) return QV_OK;
        prof_bytes(s, QV_K_PAIR, double(units) * 2 * W * sizeof(R) * 2 * 2);
        QV_LAUNCH(s, QV_K_PAIR,
                  pair_high_kernel<R><<<grid_for(s, units), kThreads, 0, s->stream>>>(amp, units, t, c_ins, c_pred, U));
    } else {
        constexpr int W2 = 2 * W;
        const int c_ins = ctrl >= LOGW + 1 ? ctrl : -1;
        const int c_pred = (ctrl >= 0 && ctrl < LOGW + 1) ? ctrl : -1;
        const uint64_t units = (dim(s) >> (c_ins >= 0 ? 1 : 0)) / W2;
        if (units == 0) return QV_OK;
        prof_bytes(s, QV_K_PAIR, double(units) * W2 * sizeof(R) * 2 * 2);
        const unsigned grid = grid_for(s, units);
        switch (t) {
        case 0:
            QV_LAUNCH(s, QV_K_PAIR, pair_low_kernel<R, 0><<<grid, kThreads, 0, s->stream>>>(amp, units, c_ins, c_pred, U));
            break;
        case 1:
            if constexpr (LOGW > 1) {
                QV_LAUNCH(s, QV_K_PAIR,
                          pair_low_kernel<R, 1><<<grid, kThreads, 0, s->stream>>>(amp, units, c_ins, c_pred, U));
                break;
            }
            // fallthrough for C128 is impossible: t < LOGW = 1
        default: return fail(QV_ERR_ARG, "internal: low target out of range");
        }
    }
    QV_CUDA(cudaGetLastError());
    return QV_OK;
}

template <typename R> qv_status diag_impl(qv_state *s, int t, int ctrl, cd d0, cd d1)
{
    constexpr int W = Traits<R>::W, LOGW = Traits<R>::LOGW;
    R *amp = static_cast<R *>(s->amp);
    if (dim(s) < uint64_t(2 * W)) {
        const cd U[4] = {d0, 0, 0, d1};
        return pair_impl<R>(s, t, ctrl, U);
    }
    int bits[2];
    int nb = 0;
    int sel = -1;
    cd p0 = d0, p1 = d1;
    if (d0 == cd(1, 0)) {
        // Only amplitudes with bit t = 1 (and control = 1) change, by d1.
        bits[nb++] = t;
        if (ctrl >= 0) bits[nb++] = ctrl;
        p0 = d1;
    } else {
        if (ctrl >= 0) bits[nb++] = ctrl;
        sel = t;
    }
    int ins[2] = {-1, -1};
    int ni = 0;
    unsigned pred = 0;
    for (int k = 0; k < nb; ++k) {
        if (bits[k] >= LOGW) ins[ni++] = bits[k];
        else pred |= 1u << bits[k];
    }
    if (ni == 2 && ins[0] > ins[1]) std::swap(ins[0], ins[1]);
    const uint64_t units = (dim(s) >> ni) / W;
    if (units == 0) return QV_OK;
    prof_bytes(s, QV_K_DIAG, double(units) * W * sizeof(R) * 2 * 2);
    QV_LAUNCH(s, QV_K_DIAG,
              diag_kernel<R><<<grid_for(s, units), kThreads, 0, s->stream>>>(
                  amp, units, ins[0], ins[1], pred, sel, R(p0.real()), R(p0.imag()), R(p1.real()), R(p1.imag())));
    QV_CUDA(cudaGetLastError());
    return QV_OK;
}

}  // namespace

qv_status launch_pair(qv_state *s, int t, int ctrl, const cd U[4])
{
    return s->dt == QV_C64 ? pair_impl<float>(s, t, ctrl, U) : pair_impl<double>(s, t, ctrl, U);
}

qv_status launch_diag(qv_state *s, int t, int ctrl, cd d0, cd d1)
{
    return s->dt == QV_C64 ? diag_impl<float>(s, t, ctrl, d0, d1) : diag_impl<double>(s, t, ctrl, d0, d1);
}

qv_status launch_swap(qv_state *s, int a, int b)
{
    const uint64_t units = dim(s) >> 2;
    if (units == 0) return QV_OK;
    prof_bytes(s, QV_K_SWAP, double(units) * 2 * amp_bytes(s->dt) * 2);
    if (s->dt == QV_C64)
        QV_LAUNCH(s, QV_K_SWAP, swap_kernel<float><<<grid_for(s, units), kThreads, 0, s->stream>>>(
                                    static_cast<float *>(s->amp), units, a, b));
    else
        QV_LAUNCH(s, QV_K_SWAP, swap_kernel<double><<<grid_for(s, units), kThreads, 0, s->stream>>>(
                                    static_cast<double *>(s->amp), units, a, b));
    QV_CUDA(cudaGetLastError());
    return QV_OK;
}

qv_status launch_set_basis(qv_state *s, uint64_t j)
{
    QV_CUDA(cudaMemsetAsync(s->amp, 0, dim(s) * amp_bytes(s->dt), s->stream));
    prof_bytes(s, QV_K_BASIS, double(dim(s)) * amp_bytes(s->dt));
    if (s->dt == QV_C64)
        QV_LAUNCH(s, QV_K_BASIS, set_one_kernel<float><<<1, 1, 0, s->stream>>>(static_cast<float *>(s->amp), j));
    else
        QV_LAUNCH(s, QV_K_BASIS, set_one_kernel<double><<<1, 1, 0, s->stream>>>(static_cast<double *>(s->amp), j));
    QV_CUDA(cudaGetLastError());
    return QV_OK;
}

}  // namespace qv
