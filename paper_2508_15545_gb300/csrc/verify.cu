// Closed-form verification on the GPU: distance of the state to QFT|j>,
// sum_k |a_k - exp(2 pi i (j k mod 2^n) / 2^n) / 2^(n/2)|^2, for states too
// large for a host reference (a 33-qubit complex64 state is 64 GiB).
//
// The phase index m = j k mod 2^n is exact in 64-bit integer arithmetic (the
// low 64 bits of the product hold it since 2^n divides 2^64). exp(2 pi i m /
// 2^n) is the product of two FP64 table entries, T_hi[m >> L] * T_lo[m & (2^L
// - 1)], each filled with sincospi on an exactly representable argument, so a
// reference amplitude is within a few FP64 ulp. Squares and sums are FP64.
#include <algorithm>
#include <cmath>

#include "qv_device.cuh"
#include "qv_internal.h"

namespace qv {
namespace {

constexpr int kThreads = 256;

// T[i] = exp(2 pi i * (i << shift) / 2^n) for i < count
__global__ void phase_table_kernel(double2 *T, uint64_t count, int shift, int n)
{
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += uint64_t(gridDim.x) * blockDim.x) {
        // angle / pi = 2 (i << shift) / 2^n, exact in double for n <= 52
        const double x = std::ldexp(double(i << shift), 1 - n);
        double s, c;
        sincospi(x, &s, &c);
        T[i] = make_double2(c, s);
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) qft_dist_kernel(const R *__restrict__ amp, int n, uint64_t j,
                                                            const double2 *__restrict__ Thi,
                                                            const double2 *__restrict__ Tlo, int L, double scale,
                                                            double *part)
{
    const uint64_t N = uint64_t(1) << n, mask = N - 1, lmask = (uint64_t(1) << L) - 1;
    double acc = 0;
    for (uint64_t k = uint64_t(blockIdx.x) * kThreads + threadIdx.x; k < N; k += uint64_t(gridDim.x) * kThreads) {
        const uint64_t m = (j * k) & mask;
        const double2 a = __ldg(&Thi[m >> L]), b = __ldg(&Tlo[m & lmask]);
        const double er = (a.x * b.x - a.y * b.y) * scale, ei = (a.x * b.y + a.y * b.x) * scale;
        const double dr = double(amp[2 * k]) - er, di = double(amp[2 * k + 1]) - ei;
        acc += dr * dr + di * di;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < kThreads / 32; ++w) s += ws[w];
        part[blockIdx.x] = s;
    }
}

__global__ void sum_kernel(const double *part, int np, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        Neumaier a;
        for (int k = 0; k < np; ++k) a.add(part[k]);
        *out = a.value();
    }
}

template <typename A, typename B>
__global__ void __launch_bounds__(kThreads) dist_kernel(const A *__restrict__ a, const B *__restrict__ b, uint64_t N,
                                                        double *part)
{
    double acc = 0;
    for (uint64_t k = uint64_t(blockIdx.x) * kThreads + threadIdx.x; k < N; k += uint64_t(gridDim.x) * kThreads) {
        const double dr = double(a[2 * k]) - double(b[2 * k]), di = double(a[2 * k + 1]) - double(b[2 * k + 1]);
        acc += dr * dr + di * di;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < kThreads / 32; ++w) s += ws[w];
        part[blockIdx.x] = s;
    }
}

}  // namespace

qv_status distance(qv_state *a, qv_state *b, double *out)
{
    QV_CUDA(cudaStreamSynchronize(b->stream));
    const unsigned grid = unsigned(a->num_sms) * 8;
    QV_TRY(ensure_scratch(a, (grid + 1) * sizeof(double)));
    double *part = static_cast<double *>(a->scratch.ptr), *res = part + grid;
    prof_bytes(a, QV_K_VERIFY, double(dim(a)) * (amp_bytes(a->dt) + amp_bytes(b->dt)));
    const uint64_t N = dim(a);
    if (a->dt == QV_C64 && b->dt == QV_C64)
        QV_LAUNCH(a, QV_K_VERIFY, dist_kernel<float, float><<<grid, kThreads, 0, a->stream>>>(
                                      static_cast<const float *>(a->amp), static_cast<const float *>(b->amp), N, part));
    else if (a->dt == QV_C64)
        QV_LAUNCH(a, QV_K_VERIFY, dist_kernel<float, double><<<grid, kThreads, 0, a->stream>>>(
                                      static_cast<const float *>(a->amp), static_cast<const double *>(b->amp), N, part));
    else if (b->dt == QV_C64)
        QV_LAUNCH(a, QV_K_VERIFY, dist_kernel<double, float><<<grid, kThreads, 0, a->stream>>>(
                                      static_cast<const double *>(a->amp), static_cast<const float *>(b->amp), N, part));
    else
        QV_LAUNCH(a, QV_K_VERIFY, dist_kernel<double, double><<<grid, kThreads, 0, a->stream>>>(
                                      static_cast<const double *>(a->amp), static_cast<const double *>(b->amp), N, part));
    QV_LAUNCH(a, QV_K_VERIFY, sum_kernel<<<1, 32, 0, a->stream>>>(part, int(grid), res));
    QV_TRY(ensure_host_out(a, 1));
    QV_TRY(copy_d2h(a, a->host_out, res, sizeof(double)));
    QV_TRY(sync_and_check(a));
    *out = std::sqrt(std::max(0.0, a->host_out[0]));
    return QV_OK;
}

qv_status verify_qft(qv_state *s, uint64_t j, double *dist)
{
    const int n = s->n;
    const int L = (n + 1) / 2;
    const uint64_t nlo = uint64_t(1) << L, nhi = uint64_t(1) << (n - L);
    const unsigned grid = unsigned(s->num_sms) * 8;
    const size_t bytes = (nlo + nhi) * sizeof(double2) + (grid + 1) * sizeof(double);
    QV_TRY(ensure_scratch(s, bytes));
    double2 *Tlo = static_cast<double2 *>(s->scratch.ptr), *Thi = Tlo + nlo;
    double *part = reinterpret_cast<double *>(Thi + nhi), *res = part + grid;
    QV_LAUNCH(s, QV_K_VERIFY, phase_table_kernel<<<256, 256, 0, s->stream>>>(Tlo, nlo, 0, n));
    QV_LAUNCH(s, QV_K_VERIFY, phase_table_kernel<<<256, 256, 0, s->stream>>>(Thi, nhi, L, n));
    const double scale = std::ldexp(1.0, -n / 2) * ((n & 1) ? std::sqrt(0.5) : 1.0);
    prof_bytes(s, QV_K_VERIFY, double(dim(s)) * amp_bytes(s->dt));
    if (s->dt == QV_C64)
        QV_LAUNCH(s, QV_K_VERIFY, qft_dist_kernel<float><<<grid, kThreads, 0, s->stream>>>(
                                      static_cast<const float *>(s->amp), n, j, Thi, Tlo, L, scale, part));
    else
        QV_LAUNCH(s, QV_K_VERIFY, qft_dist_kernel<double><<<grid, kThreads, 0, s->stream>>>(
                                      static_cast<const double *>(s->amp), n, j, Thi, Tlo, L, scale, part));
    QV_LAUNCH(s, QV_K_VERIFY, sum_kernel<<<1, 32, 0, s->stream>>>(part, int(grid), res));
    QV_TRY(ensure_host_out(s, 1));
    QV_TRY(copy_d2h(s, s->host_out, res, sizeof(double)));
    QV_TRY(sync_and_check(s));
    *dist = std::sqrt(std::max(0.0, s->host_out[0]));
    return QV_OK;
}

}  // namespace qv
