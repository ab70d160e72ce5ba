// Pass planner for the fused tiled kernel; see planner.h for the model.
#include "planner.h"

#include <algorithm>
#include <cstdio>

namespace qv {
namespace plan {

namespace {

constexpr int kMaxOpsPerPass = 384;
constexpr int kMaxStagesPerPass = 48;
constexpr int kLookahead = 96;  // gates scanned when ranking candidate tile qubits

// Tile qubits a gate needs: the target of a non-diagonal 2x2, both qubits of a
// SWAP; diagonal gates and controls need none (their bits may lie outside).
inline int needs(const PGate &g, int out[2])
{
    switch (g.cls) {
    case G_GEN:
    case G_X: out[0] = g.t; return 1;
    case G_SWAP: out[0] = g.t; out[1] = g.t2; return 2;
    default: return 0;
    }
}

inline int qubits(const PGate &g, int out[3])
{
    int k = 0;
    out[k++] = g.t;
    if (g.t2 >= 0) out[k++] = g.t2;
    if (g.c >= 0) out[k++] = g.c;
    return k;
}

// In-order scan with blocking: a gate is taken when none of its qubits is
// blocked by an earlier gate left behind and `ok(g)` holds; a gate left behind
// blocks all of its qubits. Returns the taken gate indices (into `rem`).
template <typename Ok>
int scan(const std::vector<PGate> &gates, const std::vector<int> &rem, int n, Ok ok, std::vector<int> *taken,
         int limit = 1 << 30)
{
    std::vector<char> blocked(n, 0);
    int cnt = 0, seen = 0;
    for (size_t r = 0; r < rem.size() && seen < limit; ++r, ++seen) {
        const PGate &g = gates[rem[r]];
        int qs[3];
        const int nq = qubits(g, qs);
        bool blk = false;
        for (int i = 0; i < nq; ++i) blk |= blocked[qs[i]] != 0;
        if (!blk && ok(g)) {
            ++cnt;
            if (taken) taken->push_back(int(r));
        } else {
            for (int i = 0; i < nq; ++i) blocked[qs[i]] = 1;
        }
    }
    return cnt;
}

struct LayoutState {
    int k;
    bool lane0;      // 8-byte amplitudes: two per 16-byte access, tile position 0 on register bit 0
    Layout L;
    int nq() const { return k - kRegBits; }
    int reg_of(int pos) const
    {
        for (int j = 0; j < kRegBits; ++j)
            if (L.P[j] == pos) return j;
        return -1;
    }
    int thr_of(int pos) const
    {
        for (int b = 0; b < nq(); ++b)
            if (L.Q[b] == pos) return b;
        return -1;
    }
};

bool is_canonical(const Layout &L, int k, bool lane0)
{
    if (lane0) {
        if (L.P[0] != 0) return false;
        for (int b = 0; b < 5; ++b)
            if (L.Q[b] != b + 1) return false;
    } else {
        for (int b = 0; b < 5; ++b)
            if (L.Q[b] != b) return false;
    }
    (void)k;
    return true;
}

// Builds a layout with register positions `regs`. Thread bits: the first few
// lanes take positions of distinct residue classes so the swizzled
// shared-memory transpose stays free of bank conflicts (8-byte amplitudes: a
// half warp, 4 lane bits, residues mod 4; 16-byte: a quarter warp, mod 3).
Layout make_layout(int k, bool lane0, const int regs[kRegBits])
{
    Layout L;
    for (int j = 0; j < kRegBits; ++j) L.P[j] = int8_t(regs[j]);
    std::vector<int> rest;
    for (int p = 0; p < k; ++p) {
        bool r = false;
        for (int j = 0; j < kRegBits; ++j) r |= regs[j] == p;
        if (!r) rest.push_back(p);
    }
    const int nl = lane0 ? 4 : 3, mod = lane0 ? 4 : 3;
    std::vector<int> q;
    std::vector<char> used(rest.size(), 0);
    for (int res = 0; res < mod && int(q.size()) < nl; ++res)
        for (size_t i = 0; i < rest.size(); ++i)
            if (!used[i] && rest[i] % mod == res) {
                q.push_back(rest[i]);
                used[i] = 1;
                break;
            }
    for (size_t i = 0; i < rest.size(); ++i)
        if (!used[i]) q.push_back(rest[i]);
    for (int b = 0; b < k - kRegBits; ++b) L.Q[b] = int8_t(q[b]);
    for (int b = k - kRegBits; b < kMaxK - kRegBits; ++b) L.Q[b] = -1;
    return L;
}

Layout canonical_layout(int k, bool lane0, const int extra[kRegBits])
{
    // 8-byte: P = {0, e0, e1, e2} (e >= 6), Q = 1..5 then the rest ascending.
    // 16-byte: P = {e0..e3} (e >= 5), Q = 0..4 then the rest ascending.
    Layout L;
    int regs[kRegBits];
    if (lane0) {
        regs[0] = 0;
        for (int j = 1; j < kRegBits; ++j) regs[j] = extra[j - 1];
    } else {
        for (int j = 0; j < kRegBits; ++j) regs[j] = extra[j];
    }
    for (int j = 0; j < kRegBits; ++j) L.P[j] = int8_t(regs[j]);
    int b = 0;
    const int first = lane0 ? 1 : 0;
    for (int p = first; p < first + 5; ++p) L.Q[b++] = int8_t(p);
    for (int p = 0; p < k; ++p) {
        bool used = (p >= first && p < first + 5);
        for (int j = 0; j < kRegBits; ++j) used |= regs[j] == p;
        if (!used) L.Q[b++] = int8_t(p);
    }
    for (; b < kMaxK - kRegBits; ++b) L.Q[b] = -1;
    return L;
}

}  // namespace

int classify(const std::complex<double> U[4])
{
    if (U[1] == 0.0 && U[2] == 0.0) return G_DIAG;
    if (U[0] == 0.0 && U[3] == 0.0 && U[1] == 1.0 && U[2] == 1.0) return G_X;
    return G_GEN;
}

bool make_plan(int n, int k, bool lane0, const std::vector<PGate> &gates, std::vector<Pass> &out, PlanStats &stats,
               std::string &err)
{
    out.clear();
    stats = PlanStats{};
    if (k < kMinK || k > kMaxK || k > n) {
        err = "tile size out of range";
        return false;
    }
    const int nh = k - kChunkBits;
    std::vector<int> rem(gates.size());
    for (size_t i = 0; i < gates.size(); ++i) rem[i] = int(i);

    while (!rem.empty()) {
        // ---- choose the tile's high qubits greedily
        std::vector<char> inS(n, 0);
        for (int q = 0; q < kChunkBits; ++q) inS[q] = 1;
        for (int step = 0; step < nh; ++step) {
            int best = -1;
            long long best_score = -1;
            for (int q = kChunkBits; q < n; ++q) {
                if (inS[q]) continue;
                inS[q] = 1;
                const int cnt = scan(gates, rem, n, [&](const PGate &g) {
                    int need[2];
                    const int nn = needs(g, need);
                    for (int i = 0; i < nn; ++i)
                        if (!inS[need[i]]) return false;
                    return true;
                }, nullptr);
                inS[q] = 0;
                // tie-break: gates needing q soon
                int soon = 0;
                for (size_t r = 0; r < rem.size() && r < size_t(kLookahead); ++r) {
                    int need[2];
                    const int nn = needs(gates[rem[r]], need);
                    for (int i = 0; i < nn; ++i) soon += need[i] == q;
                }
                const long long score = (long long)cnt * 4096 + soon * 16 + (n - q);
                if (score > best_score) {
                    best_score = score;
                    best = q;
                }
            }
            inS[best] = 1;
        }
        Pass P;
        P.k = k;
        int pos_of[64];
        for (int q = 0; q < n; ++q) pos_of[q] = -1;
        for (int q = 0; q < kChunkBits; ++q) pos_of[q] = q;
        {
            int j = 0;
            for (int q = kChunkBits; q < n; ++q)
                if (inS[q]) {
                    P.s_high[j] = q;
                    pos_of[q] = kChunkBits + j;
                    ++j;
                }
        }
        // tile id bits -> runs of physical bits outside the tile
        {
            int src = 0;
            for (int q = 0; q < n;) {
                if (inS[q]) {
                    ++q;
                    continue;
                }
                int w = 0;
                while (q + w < n && !inS[q + w]) ++w;
                P.seg_src[P.nseg] = src;
                P.seg_w[P.nseg] = w;
                P.seg_dst[P.nseg] = q;
                P.nseg++;
                src += w;
                q += w;
            }
        }
        // ---- gates of this pass (in order with blocking)
        std::vector<int> taken;
        scan(gates, rem, n, [&](const PGate &g) {
            int need[2];
            const int nn = needs(g, need);
            for (int i = 0; i < nn; ++i)
                if (!inS[need[i]]) return false;
            return true;
        }, &taken);
        if (taken.empty()) {
            err = "planner made no progress";
            return false;
        }
        std::vector<int> pg;  // gate indices of this pass, in order
        for (int r : taken) pg.push_back(rem[r]);

        // ---- stages: run gates whose target is a register bit; transpose otherwise
        LayoutState ls{k, lane0, {}};
        auto frontier_targets = [&](const std::vector<int> &left, std::vector<int> &pos, bool restrict_canon) {
            // targets (tile positions) of non-diagonal gates in frontier order, then any later ones
            std::vector<char> blocked(n, 0);
            auto consider = [&](int p) {
                if (p < 0) return;
                if (restrict_canon) {
                    if (lane0 && p < 6) return;
                    if (!lane0 && p < 5) return;
                }
                if (std::find(pos.begin(), pos.end(), p) == pos.end()) pos.push_back(p);
            };
            for (int pass2 = 0; pass2 < 2 && int(pos.size()) < kRegBits; ++pass2) {
                std::fill(blocked.begin(), blocked.end(), 0);
                for (int gi : left) {
                    const PGate &g = gates[gi];
                    int qs[3];
                    const int nq = qubits(g, qs);
                    bool blk = false;
                    for (int i = 0; i < nq; ++i) blk |= blocked[qs[i]] != 0;
                    if ((g.cls == G_GEN || g.cls == G_X) && (pass2 == 1 || !blk)) consider(pos_of[g.t]);
                    for (int i = 0; i < nq; ++i) blocked[qs[i]] = 1;
                    if (int(pos.size()) >= kRegBits) break;
                }
            }
        };
        std::vector<int> left = pg;
        std::vector<Stage> stages;
        std::vector<Op> ops;
        {
            std::vector<int> pos;
            frontier_targets(left, pos, true);
            const int lo = lane0 ? 6 : 5;
            for (int p = k - 1; p >= lo && int(pos.size()) < kRegBits; --p)
                if (std::find(pos.begin(), pos.end(), p) == pos.end()) pos.push_back(p);
            int extra[kRegBits] = {0, 0, 0, 0};
            for (int j = 0; j < (lane0 ? 3 : 4); ++j) extra[j] = pos[j];
            ls.L = canonical_layout(k, lane0, extra);
        }
        Stage cur{ls.L, ls.L, 0, 0};
        auto emit = [&](const PGate &g) {
            Op o{};
            o.treg = o.creg = -1;
            if (g.c >= 0) {
                const int pc = pos_of[g.c];
                if (pc < 0) o.cext = uint64_t(1) << g.c;
                else if (ls.reg_of(pc) >= 0) o.creg = int8_t(ls.reg_of(pc));
                else o.cthr = 1u << ls.thr_of(pc);
            }
            if (g.cls == G_DIAG) {
                o.type = OP_DIAG;
                const int pt = pos_of[g.t];
                if (pt < 0) o.text = uint64_t(1) << g.t;
                else if (ls.reg_of(pt) >= 0) o.treg = int8_t(ls.reg_of(pt));
                else o.tthr = 1u << ls.thr_of(pt);
                o.m[0] = g.U[0].real(); o.m[1] = g.U[0].imag();
                o.m[2] = g.U[3].real(); o.m[3] = g.U[3].imag();
            } else {
                o.type = g.cls == G_X ? OP_X : OP_GEN;
                o.treg = int8_t(ls.reg_of(pos_of[g.t]));
                for (int e = 0; e < 4; ++e) {
                    o.m[2 * e] = g.U[e].real();
                    o.m[2 * e + 1] = g.U[e].imag();
                }
            }
            ops.push_back(o);
        };
        while (!left.empty()) {
            // run every executable gate in order (with blocking)
            std::vector<int> still;
            std::vector<char> blocked(n, 0);
            int ran = 0;
            for (int gi : left) {
                const PGate &g = gates[gi];
                int qs[3];
                const int nq = qubits(g, qs);
                bool blk = false;
                for (int i = 0; i < nq; ++i) blk |= blocked[qs[i]] != 0;
                bool exec = false;
                if (!blk && int(ops.size()) < kMaxOpsPerPass) {
                    if (g.cls == G_DIAG || g.cls == G_SWAP) exec = true;
                    else exec = ls.reg_of(pos_of[g.t]) >= 0;
                }
                if (exec) {
                    if (g.cls == G_SWAP) {
                        const int a = pos_of[g.t], b = pos_of[g.t2];
                        for (int j = 0; j < kRegBits; ++j)
                            ls.L.P[j] = int8_t(ls.L.P[j] == a ? b : ls.L.P[j] == b ? a : ls.L.P[j]);
                        for (int q = 0; q < ls.nq(); ++q)
                            ls.L.Q[q] = int8_t(ls.L.Q[q] == a ? b : ls.L.Q[q] == b ? a : ls.L.Q[q]);
                    } else {
                        emit(g);
                    }
                    ++ran;
                } else {
                    still.push_back(gi);
                    for (int i = 0; i < nq; ++i) blocked[qs[i]] = 1;
                }
            }
            left.swap(still);
            if (left.empty()) break;
            (void)ran;
            if (int(ops.size()) >= kMaxOpsPerPass || int(stages.size()) + 2 >= kMaxStagesPerPass) {
                // pass is full: give the rest back to later passes
                break;
            }
            {
                // the first gate left needs a register bit it lacks: new register set
                cur.out = ls.L;
                cur.op_end = int(ops.size());
                stages.push_back(cur);
                std::vector<int> pos;
                frontier_targets(left, pos, false);
                for (int j = 0; j < kRegBits && int(pos.size()) < kRegBits; ++j)
                    if (std::find(pos.begin(), pos.end(), ls.L.P[j]) == pos.end()) pos.push_back(ls.L.P[j]);
                int regs[kRegBits];
                for (int j = 0; j < kRegBits; ++j) regs[j] = pos[j];
                ls.L = make_layout(k, lane0, regs);
                cur = Stage{ls.L, ls.L, int(ops.size()), int(ops.size())};
            }
        }
        cur.out = ls.L;
        cur.op_end = int(ops.size());
        stages.push_back(cur);
        if (!is_canonical(ls.L, k, lane0)) {
            int extra[kRegBits];
            int ne = 0;
            const int lo = lane0 ? 6 : 5;
            for (int j = 0; j < kRegBits && ne < kRegBits; ++j)
                if (ls.L.P[j] >= lo) extra[ne++] = ls.L.P[j];
            for (int p = k - 1; p >= lo && ne < kRegBits; --p) {
                bool have = false;
                for (int e = 0; e < ne; ++e) have |= extra[e] == p;
                if (!have) extra[ne++] = p;
            }
            Layout C = canonical_layout(k, lane0, extra);
            stages.push_back(Stage{C, C, int(ops.size()), int(ops.size())});
        }
        // gates handed to this pass but not run go back to the front of `rem`
        std::vector<char> ran_mask(gates.size(), 0);
        for (int gi : pg) ran_mask[gi] = 1;
        for (int gi : left) ran_mask[gi] = 0;
        std::vector<int> nrem;
        for (int gi : rem)
            if (!ran_mask[gi]) nrem.push_back(gi);
        P.ngates = int(pg.size() - left.size());
        P.stages = std::move(stages);
        P.ops = std::move(ops);
        stats.passes++;
        stats.stages += int(P.stages.size());
        stats.transposes += int(P.stages.size()) - 1;
        stats.gates += P.ngates;
        stats.ops += int(P.ops.size());
        out.push_back(std::move(P));
        rem.swap(nrem);
    }
    return true;
}

}  // namespace plan
}  // namespace qv
