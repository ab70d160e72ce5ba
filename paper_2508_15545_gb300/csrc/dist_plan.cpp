// Schedule of a circuit on a state split over 2^g ranks (host only, no CUDA).
//
// The paper's parallel strategy (Sec. III-D, Eq. 9) gives rank r the
// contiguous index range [r 2^n / C, (r + 1) 2^n / C - 1] of the 2^n
// amplitudes, C = 2^g: the top g bits of an index name its rank ("global"
// qubits), the low L = n - g bits its place in the rank's shard ("local"
// qubits). A gate whose amplitude pairs (i, i XOR 2^t) stay inside a shard
// (t local) runs on every rank independently. A pair that crosses ranks
// (Sec. III-D, Fig. 4) needs data from the partner rank; here the global
// physical qubit is first exchanged with the top local one:
//
//   physical SWAP(p_g, L - 1) moves the amplitudes whose bits p_g and L - 1
//   differ. On rank r with b = bit (p_g - L) of r, those are the local half
//   with bit L - 1 = !b; it goes to rank r XOR 2^(p_g - L) at the same
//   offsets of that rank's half with bit L - 1 = b. So the two ranks trade
//   one contiguous half of their shards (the upper half on the rank whose bit
//   is 0, the lower half on the other) and the circuit continues with the two
//   logical qubits' positions exchanged.
//
// What needs no data from another rank: a control on a global qubit is a
// constant on each rank (the gate runs without it where the rank's bit is 1
// and not at all elsewhere); a diagonal gate on a global qubit multiplies the
// shard by one of its two diagonal entries; a SWAP of two qubits only
// exchanges their logical labels. The local qubit sent away at an exchange is
// the one whose logical qubit is next needed as a non-diagonal target
// furthest in the future; it is first moved to position L - 1 by a local SWAP
// (a relabel in the fused passes).
#include <algorithm>
#include <complex>
#include <vector>

#include "qv_internal.h"

namespace qv {

qv_status dist_plan(int n, int g, int rank, const qv_gate *gates, size_t ng, std::vector<qv_dist_step> &steps,
                    std::vector<qv_gate> &lg, std::vector<int32_t> &final_perm, bool restore)
{
    const int L = n - g;
    std::vector<int> perm(n), inv(n);  // logical -> physical, physical -> logical
    for (int q = 0; q < n; ++q) perm[q] = inv[q] = q;
    steps.clear();
    lg.clear();
    size_t seg_begin = 0;
    // gates of the circuit in the current segment, counted the same way on every
    // rank: a segment whose gates all fall away on this rank (controls that are 0
    // here) still gives an (empty) step, so every rank has the same steps
    size_t pending = 0;
    auto flush = [&]() {
        if (pending > 0 || lg.size() > seg_begin) {
            qv_dist_step s{};
            s.kind = QV_DIST_LOCAL;
            s.gate_begin = seg_begin;
            s.gate_end = lg.size();
            steps.push_back(s);
        }
        seg_begin = lg.size();
        pending = 0;
    };
    auto needs_local = [&](const qv_gate &x, cd U[4]) {
        if (x.kind == QV_G_SWAP) return false;
        return !is_diagonal(U);
    };
    // next position after `from` at which logical qubit q is the target of a
    // gate that must run locally (non-diagonal); ng when never
    auto next_use = [&](int q, size_t from) {
        for (size_t k = from; k < ng; ++k) {
            if (gates[k].target != q || gates[k].kind == QV_G_SWAP) continue;
            cd U[4];
            if (gate_matrix(gates[k], U) && !is_diagonal(U)) return k;
        }
        return ng;
    };
    auto swap_labels = [&](int pa, int pb) {
        const int qa = inv[pa], qb = inv[pb];
        std::swap(perm[qa], perm[qb]);
        inv[pa] = qb;
        inv[pb] = qa;
    };
    auto bit_of_rank = [&](int p) { return (rank >> (p - L)) & 1; };
    auto local_swap = [&](int pa, int pb) {  // data moves: labels follow
        qv_gate s{};
        s.kind = QV_G_SWAP;
        s.target = pa;
        s.target2 = pb;
        s.ctrl = -1;
        s.param[0] = s.param[1] = s.param[2] = -1;
        lg.push_back(s);
        ++pending;
        swap_labels(pa, pb);
    };
    auto exchange = [&](int pg) {  // global position pg <-> local position L - 1
        flush();
        qv_dist_step e{};
        e.kind = QV_DIST_EXCHANGE;
        e.global_bit = pg - L;
        e.peer = rank ^ (1 << (pg - L));
        e.send_upper = bit_of_rank(pg) == 0 ? 1 : 0;
        steps.push_back(e);
        swap_labels(pg, L - 1);
    };
    for (size_t k = 0; k < ng; ++k) {
        const qv_gate &x = gates[k];
        if (x.kind == QV_G_SWAP) {  // exchange the two logical labels; no data moves
            swap_labels(perm[x.target], perm[x.target2]);
            continue;
        }
        cd U[4];
        if (!gate_matrix(x, U)) return fail(QV_ERR_ARG, "gate %zu: unknown kind", k);
        if (needs_local(x, U) && perm[x.target] >= L) {
            // bring the target to local position L - 1 through one half-shard exchange
            const int pg = perm[x.target];
            int victim = -1;
            size_t far = 0;
            for (int p = 0; p < L; ++p) {
                if (x.ctrl >= 0 && perm[x.ctrl] == p) continue;  // keep the gate's control local
                const size_t u = next_use(inv[p], k);
                if (victim < 0 || u > far) {
                    victim = p;
                    far = u;
                }
            }
            if (victim < 0) return fail(QV_ERR_UNSUPPORTED, "no local qubit to exchange (n = %d, g = %d)", n, g);
            if (victim != L - 1) local_swap(victim, L - 1);
            exchange(pg);
        }
        // the gate on this rank
        ++pending;
        qv_gate y = x;
        const int pt = perm[x.target];
        int pc = x.ctrl >= 0 ? perm[x.ctrl] : -1;
        if (pc >= L) {
            if (!bit_of_rank(pc)) continue;  // control 0 on this rank: the gate does nothing here
            pc = -1;
            y.ctrl = -1;
        }
        if (pt >= L) {
            // diagonal gate on a global qubit: the shard (or, with a local control
            // c, its half with bit c = 1) times one diagonal entry d: diag(d, d) on
            // local qubit 0, or diag(1, d) on c
            const cd d = bit_of_rank(pt) ? U[3] : U[0];
            if (d == cd(1.0)) continue;
            qv_gate z{};
            z.kind = QV_G_MATRIX;
            z.target = pc >= 0 ? pc : 0;
            z.target2 = -1;
            z.ctrl = -1;
            z.param[0] = z.param[1] = z.param[2] = -1;
            z.u[0].re = pc >= 0 ? 1.0 : d.real();
            z.u[0].im = pc >= 0 ? 0.0 : d.imag();
            z.u[3].re = d.real();
            z.u[3].im = d.imag();
            lg.push_back(z);
            continue;
        }
        y.target = pt;
        y.ctrl = pc;
        lg.push_back(y);
    }
    if (restore) {
        // back to the natural order: every global position gets its own logical
        // qubit through local position L - 1, then one local permutation (SWAPs,
        // relabels in the fused passes) orders the local positions
        for (int pg = n - 1; pg >= L; --pg) {
            if (inv[pg] == pg) continue;
            if (perm[pg] >= L) exchange(perm[pg]);  // logical pg sits at another global position
            if (perm[pg] != L - 1) local_swap(perm[pg], L - 1);
            exchange(pg);
        }
        for (int p = 0; p < L; ++p)
            if (inv[p] != p) local_swap(perm[p], p);
    }
    flush();
    final_perm.assign(perm.begin(), perm.end());
    return QV_OK;
}

}  // namespace qv
