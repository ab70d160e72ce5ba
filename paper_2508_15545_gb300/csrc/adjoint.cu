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
#include <cmath>
#include <cstring>
#include <vector>

#include "qv_device.cuh"
#include "qv_internal.h"
#include "qv_plan.h"

namespace qv {

struct AdjointBuffers {
    void *lam = nullptr;       // second state buffer (lambda)
    size_t lam_bytes = 0;
    double *part = nullptr;    // per-block partial sums
    size_t part_count = 0;
};

namespace {

constexpr int kThreads = 256;
constexpr int kMaxD = 3;  // trainable angles per gate (U3)

// ---------------------------------------------------------------- H|psi>
constexpr int kMaxTerms = 64;
struct PauliGroupA {
    uint64_t x;
    int nt;
    uint64_t z[kMaxTerms];
    double cre[kMaxTerms], cim[kMaxTerms];
};

// out_j = sum over groups sum_t c_t i^{ny_t} (-1)^{popcount(src & z_t)} psi_src, src = j ^ x
template <typename R>
__global__ void __launch_bounds__(kThreads) pauli_apply_kernel(const R *__restrict__ psi, R *__restrict__ out,
                                                               uint64_t N, const PauliGroupA *groups, int ng)
{
    extern __shared__ unsigned char smem_raw[];
    PauliGroupA *g = reinterpret_cast<PauliGroupA *>(smem_raw);
    for (int k = threadIdx.x; k < ng * int(sizeof(PauliGroupA) / 8); k += kThreads)
        reinterpret_cast<uint64_t *>(g)[k] = reinterpret_cast<const uint64_t *>(groups)[k];
    __syncthreads();
    for (uint64_t j = uint64_t(blockIdx.x) * kThreads + threadIdx.x; j < N; j += uint64_t(gridDim.x) * kThreads) {
        double ar = 0, ai = 0;
        for (int q = 0; q < ng; ++q) {
            const uint64_t src = j ^ g[q].x;
            double cr = 0, ci = 0;
            for (int k = 0; k < g[q].nt; ++k) {
                const double sg = (__popcll(src & g[q].z[k]) & 1) ? -1.0 : 1.0;
                cr += sg * g[q].cre[k];
                ci += sg * g[q].cim[k];
            }
            const double vr = psi[2 * src], vi = psi[2 * src + 1];
            ar += cr * vr - ci * vi;
            ai += cr * vi + ci * vr;
        }
        out[2 * j] = R(ar);
        out[2 * j + 1] = R(ai);
    }
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
    std::vector<PauliGroupA> groups;
    for (size_t k = 0; k < nt; ++k) {
        const uint64_t x = terms[k].xmask, z = terms[k].zmask;
        const int ny = __builtin_popcountll(x & z);
        static const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, 1, 0, -1};
        PauliGroupA *g = nullptr;
        for (auto &gg : groups)
            if (gg.x == x && gg.nt < kMaxTerms) { g = &gg; break; }
        if (!g) {
            groups.emplace_back();
            g = &groups.back();
            std::memset(g, 0, sizeof *g);
            g->x = x;
        }
        g->z[g->nt] = z;
        g->cre[g->nt] = terms[k].coeff * pr[ny & 3];
        g->cim[g->nt] = terms[k].coeff * pi[ny & 3];
        g->nt++;
    }
    const size_t gbytes = groups.size() * sizeof(PauliGroupA);
    if (gbytes > 200 * 1024) return fail(QV_ERR_UNSUPPORTED, "Hamiltonian too large (%zu X-mask groups)", groups.size());
    QV_TRY(ensure_scratch(s, std::max<size_t>(gbytes, 8)));
    if (!groups.empty()) QV_TRY(copy_h2d(s, s->scratch.ptr, groups.data(), gbytes));
    static bool attr = false;
    if (!attr) {
        QV_CUDA(cudaFuncSetAttribute(pauli_apply_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    prof_bytes(s, QV_K_PAULI, double(dim(s)) * 2 * sizeof(R) * (2 + groups.size()));
    QV_LAUNCH(s, QV_K_PAULI,
              pauli_apply_kernel<R><<<grid_of(s, dim(s)), kThreads, gbytes, s->stream>>>(
                  static_cast<const R *>(src), static_cast<R *>(dst), dim(s),
                  static_cast<const PauliGroupA *>(s->scratch.ptr), int(groups.size())));
    return QV_OK;
}

template <typename R>
qv_status adjoint_impl(qv_state *s, const qv_gate *g, size_t ng, const qv_pauli_term *H, size_t nt, size_t nparams,
                       double *grad_out, double *expval_out)
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
    for (size_t l = ng; l-- > 0;) {
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
                       double *grad_out, double *expval_out)
{
    return s->dt == QV_C64 ? adjoint_impl<float>(s, g, ng, H, nt, nparams, grad_out, expval_out)
                           : adjoint_impl<double>(s, g, ng, H, nt, nparams, grad_out, expval_out);
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
