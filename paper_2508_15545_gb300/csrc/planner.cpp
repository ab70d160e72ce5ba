// Pass planner for the fused tiled kernel; see planner.h for the model.
#include "planner.h"

#include <algorithm>

namespace qv {
namespace plan {

namespace {

constexpr int kMaxOpsPerPass = 160;
constexpr int kMaxOpsAdjoint = 60;  // adjoint plans: ops carry derivatives (coefficient space)
constexpr int kMaxStagesPerPass = 40;
constexpr int kLookahead = 96;  // gates scanned when ranking candidate tile qubits

using cd = std::complex<double>;

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
// blocks all of its qubits. Returns the number taken; `taken` gets indices into rem.
template <typename Ok>
int scan(const std::vector<PGate> &gates, const std::vector<int> &rem, int n, Ok ok, std::vector<int> *taken)
{
    std::vector<char> blocked(n, 0);
    int cnt = 0;
    for (size_t r = 0; r < rem.size(); ++r) {
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

// Layout constraints. With pin0, register bit 3 is tile position 0 and the
// shared-memory word index is l >> 1; otherwise the word index is l.
inline int lane_first(bool pin0) { return pin0 ? 1 : 0; }

bool is_canonical(const Layout &L, bool pin0)
{
    if (pin0 && L.P[3] != 0) return false;
    for (int b = 0; b < 5; ++b)
        if (L.Q[b] != b + lane_first(pin0)) return false;
    return true;
}

// Thread bits for register positions `regs`: the first lanes take positions
// whose word-index bit falls in distinct residue classes, so the swizzled
// transpose is free of bank conflicts (8-byte words: a half warp = 4 lane
// bits, residues mod 4; 16-byte words: a quarter warp = 3 lane bits, mod 3).
Layout make_layout(int k, bool pin0, const int regs[kRegBits])
{
    Layout L;
    for (int j = 0; j < kRegBits; ++j) L.P[j] = int8_t(regs[j]);
    std::vector<int> rest;
    for (int p = 0; p < k; ++p) {
        bool r = false;
        for (int j = 0; j < kRegBits; ++j) r |= regs[j] == p;
        if (!r) rest.push_back(p);
    }
    const int nl = pin0 ? 4 : 3, mod = pin0 ? 4 : 3, sh = pin0 ? 1 : 0;
    std::vector<int> q;
    std::vector<char> used(rest.size(), 0);
    for (int res = 0; res < mod && int(q.size()) < nl; ++res)
        for (size_t i = 0; i < rest.size(); ++i)
            if (!used[i] && (rest[i] - sh) % mod == res) {
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

// Load/store layout: lanes on positions f..f+4 (f = 1 with pin0, else 0);
// register bits on `extra` (positions >= f + 5) plus position 0 with pin0.
Layout canonical_layout(int k, bool pin0, const int extra[kRegBits])
{
    Layout L;
    int regs[kRegBits];
    if (pin0) {
        for (int j = 0; j < 3; ++j) regs[j] = extra[j];
        regs[3] = 0;
    } else {
        for (int j = 0; j < kRegBits; ++j) regs[j] = extra[j];
    }
    for (int j = 0; j < kRegBits; ++j) L.P[j] = int8_t(regs[j]);
    int b = 0;
    const int first = lane_first(pin0);
    for (int p = first; p < first + 5; ++p) L.Q[b++] = int8_t(p);
    for (int p = 0; p < k; ++p) {
        bool used = (p >= first && p < first + 5);
        for (int j = 0; j < kRegBits; ++j) used |= regs[j] == p;
        if (!used) L.Q[b++] = int8_t(p);
    }
    for (; b < kMaxK - kRegBits; ++b) L.Q[b] = -1;
    return L;
}

void matmul(const cd A[4], const cd B[4], cd out[4])  // out = A B
{
    const cd r0 = A[0] * B[0] + A[1] * B[2], r1 = A[0] * B[1] + A[1] * B[3];
    const cd r2 = A[2] * B[0] + A[3] * B[2], r3 = A[2] * B[1] + A[3] * B[3];
    out[0] = r0; out[1] = r1; out[2] = r2; out[3] = r3;
}

// ---------------------------------------------------------------- pair fusion
// A 4x4 over up to two register bits q[0], q[1] (index bit j <-> q[j]; nq = 1
// leaves index bit 1 as an identity slot).
struct PairBlock {
    int q[2] = {-1, -1};
    int nq = 0;
    cd M[16];
    std::vector<int> ops;  // indices of the ops it holds, ascending
};

// dst (over register bits dq) = src (over sq, nsq used slots) acting as the
// identity on every bit of dq it does not hold.
void embed4(const cd src[16], const int sq[2], int nsq, const int dq[2], cd dst[16])
{
    int slot[2];  // dst slot j -> src slot or -1
    for (int j = 0; j < 2; ++j) {
        slot[j] = -1;
        for (int i = 0; i < nsq; ++i)
            if (sq[i] == dq[j] && dq[j] >= 0) slot[j] = i;
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            int rs = 0, cs = 0;
            bool eq = true;
            for (int j = 0; j < 2; ++j) {
                const int rb = (r >> j) & 1, cb = (c >> j) & 1;
                if (slot[j] < 0) eq &= rb == cb;
                else {
                    rs |= rb << slot[j];
                    cs |= cb << slot[j];
                }
            }
            // src slots not mapped (the identity slot of a one-bit source) stay 0
            dst[4 * r + c] = eq ? src[4 * rs + cs] : cd(0.0);
        }
}

void mul4(const cd A[16], const cd B[16], cd out[16])  // out = A B
{
    cd t[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            cd a = 0.0;
            for (int k = 0; k < 4; ++k) a += A[4 * r + k] * B[4 * k + c];
            t[4 * r + c] = a;
        }
    std::copy(t, t + 16, out);
}

void ident4(cd M[16])
{
    for (int e = 0; e < 16; ++e) M[e] = (e % 5 == 0) ? cd(1.0) : cd(0.0);
}

// 4x4 of a fusable op (target and select on register bits among q) over q.
void op_matrix4(const Op &op, const int q[2], cd out[16])
{
    auto bit = [&](int idx, int reg) {
        for (int j = 0; j < 2; ++j)
            if (q[j] == reg) return (idx >> j) & 1;
        return 0;
    };
    int tj = 0;
    for (int j = 0; j < 2; ++j)
        if (q[j] == op.treg) tj = j;
    for (int e = 0; e < 16; ++e) out[e] = 0.0;
    for (int c = 0; c < 4; ++c) {
        const int sel = op.sreg >= 0 ? bit(c, op.sreg) : 0;
        const int xt = (c >> tj) & 1;
        if (op.type == OP_DIAG) {
            out[4 * c + c] = op.M[sel][xt ? 3 : 0];
            continue;
        }
        for (int rt = 0; rt < 2; ++rt) {
            const int r = (c & ~(1 << tj)) | (rt << tj);
            out[4 * r + c] += op.M[sel][2 * rt + xt];
        }
    }
}

// Merges, inside each stage, runs of ops on at most two register bits into
// GEN2 ops when the 4x4 takes fewer FP32 operations than the ops it replaces.
// An op on other bits commutes with a run, so the run is emitted when it
// closes (a later op touches one of its bits and cannot join it).
void fuse_pair_blocks(Pass &P, bool pin0, int &pair_ops)
{
    std::vector<Op> nops;
    std::vector<Stage> nst = P.stages;
    for (Stage &st : nst) {
        const int b0 = int(nops.size());
        std::vector<PairBlock> blocks;
        std::vector<char> open;
        int owner[kRegBits] = {-1, -1, -1, -1};
        auto close = [&](int bi) {
            PairBlock &B = blocks[bi];
            double c = 0;
            for (int o : B.ops) c += fma_per_amp_c64(P.ops[o]);
            if (B.nq == 2 && c > 16.0 + 1e-9) {
                Op g{};
                g.type = OP_GEN2;
                g.treg = int8_t(B.q[0]);
                g.treg2 = int8_t(B.q[1]);
                g.sreg = -1;
                std::copy(B.M, B.M + 16, g.M4);
                nops.push_back(g);
                ++pair_ops;
            } else {
                for (int o : B.ops) nops.push_back(P.ops[o]);
            }
            for (int j = 0; j < B.nq; ++j) owner[B.q[j]] = -1;
            open[bi] = 0;
        };
        for (int k = st.op_begin; k < st.op_end; ++k) {
            const Op &op = P.ops[k];
            int R[2], nr = 0;
            if (op.treg >= 0) R[nr++] = op.treg;
            if (op.sreg >= 0 && op.sreg != op.treg) R[nr++] = op.sreg;
            bool fusable = (op.type == OP_GEN || op.type == OP_X || op.type == OP_DIAG) && op.treg >= 0 && !op.sthr &&
                           !op.sext && !op.tthr && !op.text;
            for (int i = 0; i < nr; ++i) fusable &= !(pin0 && R[i] == 3);
            if (!fusable) {
                for (int i = 0; i < nr; ++i)
                    if (owner[R[i]] >= 0) close(owner[R[i]]);
                nops.push_back(op);
                continue;
            }
            std::vector<int> S;
            for (int i = 0; i < nr; ++i)
                if (owner[R[i]] >= 0 && std::find(S.begin(), S.end(), owner[R[i]]) == S.end()) S.push_back(owner[R[i]]);
            std::vector<int> U;
            for (int bi : S)
                for (int j = 0; j < blocks[bi].nq; ++j) U.push_back(blocks[bi].q[j]);
            for (int i = 0; i < nr; ++i)
                if (std::find(U.begin(), U.end(), R[i]) == U.end()) U.push_back(R[i]);
            if (U.size() > 2) {
                for (int bi : S) close(bi);
                S.clear();
                U.assign(R, R + nr);
            }
            PairBlock NB;
            NB.nq = int(U.size());
            for (int j = 0; j < NB.nq; ++j) NB.q[j] = U[j];
            ident4(NB.M);
            for (int bi : S) {
                cd e[16];
                embed4(blocks[bi].M, blocks[bi].q, blocks[bi].nq, NB.q, e);
                mul4(e, NB.M, NB.M);
                NB.ops.insert(NB.ops.end(), blocks[bi].ops.begin(), blocks[bi].ops.end());
                open[bi] = 0;
            }
            std::sort(NB.ops.begin(), NB.ops.end());
            cd om[16];
            op_matrix4(op, NB.q, om);
            mul4(om, NB.M, NB.M);
            NB.ops.push_back(k);
            blocks.push_back(NB);
            open.push_back(1);
            for (int j = 0; j < NB.nq; ++j) owner[NB.q[j]] = int(blocks.size()) - 1;
        }
        for (size_t bi = 0; bi < blocks.size(); ++bi)
            if (open[bi]) close(int(bi));
        st.op_begin = b0;
        st.op_end = int(nops.size());
    }
    P.ops = std::move(nops);
    P.stages = std::move(nst);
}


// ---------------------------------------------------------------- tensor-core stages
// A stage's register set is a bitmask R over tile positions. A gate runs when
// its non-diagonal target is a register position and its control (and a
// diagonal target) is a register position or lies outside the tile; at most
// one qubit outside the tile per stage (`ext`), whose value picks one of two
// matrices for the whole tile.
bool tc_exec(const PGate &g, const std::vector<int> &pos_of, uint32_t R, int &ext)
{
    if (g.cls == G_SWAP) return true;  // both qubits are tile positions (pass selection)
    auto in_reg = [&](int q) { return pos_of[q] >= 0 && ((R >> pos_of[q]) & 1u); };
    int need = -1;
    if (!in_reg(g.t)) {
        if (g.cls != G_DIAG || pos_of[g.t] >= 0) return false;
        need = g.t;
    }
    if (g.c >= 0 && !in_reg(g.c)) {
        if (pos_of[g.c] >= 0 || need >= 0) return false;
        need = g.c;
    }
    if (need >= 0) {
        if (ext == -2 || (ext >= 0 && ext != need)) return false;  // -2: no qubit outside allowed
        ext = need;
    }
    return true;
}

inline uint32_t swap_bits(uint32_t R, int a, int b)
{
    const uint32_t x = ((R >> a) ^ (R >> b)) & 1u;
    return R ^ ((x << a) | (x << b));
}

// Gates of `left` that would run (in order, with blocking) with register set R;
// `ext_used` reports whether one needs a qubit outside the tile.
int tc_count(const std::vector<PGate> &gates, const std::vector<int> &left, const std::vector<int> &pos_of, int n,
             uint32_t R, size_t max_scan, bool *ext_used)
{
    std::vector<char> blocked(n, 0);
    int cnt = 0, ext = -1;
    for (size_t i = 0; i < left.size() && i < max_scan; ++i) {
        const PGate &g = gates[left[i]];
        int qs[3];
        const int nq = qubits(g, qs);
        bool blk = false;
        for (int j = 0; j < nq; ++j) blk |= blocked[qs[j]] != 0;
        if (!blk && tc_exec(g, pos_of, R, ext)) {
            ++cnt;
            if (g.cls == G_SWAP) R = swap_bits(R, pos_of[g.t], pos_of[g.t2]);
        } else {
            for (int j = 0; j < nq; ++j) blocked[qs[j]] = 1;
        }
    }
    if (ext_used) *ext_used = ext >= 0;
    return cnt;
}

// Layout with register bit j on the j-th set bit of R. Lanes: positions 0..4
// when R holds none of them (the load/store layout); otherwise the first four
// lanes take positions of distinct residues mod 4, so that a half warp's 8-byte
// shared-memory words (word = swizzled position) fall in distinct banks.
Layout tc_layout(int k, uint32_t R)
{
    Layout L;
    int j = 0;
    for (int p = 0; p < k; ++p)
        if ((R >> p) & 1u) L.P[j++] = int8_t(p);
    std::vector<int> rest;
    for (int p = 0; p < k; ++p)
        if (!((R >> p) & 1u)) rest.push_back(p);
    std::vector<int> q;
    if ((R & ((1u << kTcLanes) - 1)) == 0) {
        q = rest;  // ascending: lanes on 0..4
    } else {
        std::vector<char> used(rest.size(), 0);
        for (int res = 0; res < 4; ++res)
            for (size_t i = 0; i < rest.size(); ++i)
                if (!used[i] && rest[i] % 4 == res) {
                    q.push_back(rest[i]);
                    used[i] = 1;
                    break;
                }
        for (size_t i = 0; i < rest.size(); ++i)
            if (!used[i]) q.push_back(rest[i]);
    }
    for (int b = 0; b < k - kRegBits; ++b) L.Q[b] = int8_t(q[b]);
    for (int b = k - kRegBits; b < kMaxK - kRegBits; ++b) L.Q[b] = -1;
    return L;
}

bool tc_canonical(const Layout &L, int k)
{
    for (int b = 0; b < kTcLanes; ++b)
        if (L.Q[b] != b) return false;
    for (int j = 0; j < kRegBits; ++j)
        if (L.P[j] < kTcLanes) return false;
    (void)k;
    return true;
}

int reg_bit(const Layout &L, int pos)
{
    for (int j = 0; j < kRegBits; ++j)
        if (L.P[j] == pos) return j;
    return -1;
}

// G <- M G for the 16x16 embedding M of gate g in register coordinates (target
// register bit jt, control register bit jc, or -1). `v` is the value of the
// stage's qubit outside the tile for this matrix variant; `ext` that qubit.
void tc_mul_gate(cd G[kTcSlot], const PGate &g, int jt, int jc, int v, int ext)
{
    cd M[kTcSlot];
    for (int e = 0; e < kTcSlot; ++e) M[e] = 0.0;
    for (int c = 0; c < 16; ++c) {
        bool on = true;
        if (g.c >= 0) on = jc >= 0 ? ((c >> jc) & 1) != 0 : (g.c == ext && v == 1);
        if (!on) {
            M[16 * c + c] = 1.0;
            continue;
        }
        if (jt < 0) {  // diagonal gate on the qubit outside the tile
            M[16 * c + c] = g.U[(g.t == ext && v == 1) ? 3 : 0];
            continue;
        }
        const int xt = (c >> jt) & 1;
        for (int rt = 0; rt < 2; ++rt) {
            const int r = (c & ~(1 << jt)) | (rt << jt);
            M[16 * r + c] += g.U[2 * rt + xt];
        }
    }
    cd T[kTcSlot];
    for (int r = 0; r < 16; ++r)
        for (int c = 0; c < 16; ++c) {
            cd a = 0.0;
            for (int m = 0; m < 16; ++m) a += M[16 * r + m] * G[16 * m + c];
            T[16 * r + c] = a;
        }
    std::copy(T, T + kTcSlot, G);
}

uint32_t mask_of(const int8_t P[kRegBits])
{
    uint32_t m = 0;
    for (int j = 0; j < kRegBits; ++j) m |= 1u << P[j];
    return m;
}

// Stages of one tensor-core pass over the gates `left` (tile positions
// pos_of). Runs gates until `left` is empty or the matrix slots are used up;
// `left` keeps the gates that did not run.
void build_tc_pass(const std::vector<PGate> &gates, std::vector<int> &left, const std::vector<int> &pos_of, int n, int k,
                   Pass &P)
{
    const size_t scan_max = 2 * kLookahead;
    const uint32_t low = (1u << kTcLanes) - 1;
    const int max_slots = tc_max_slots(k);
    auto best_set = [&](bool prefer_high, bool *ext_used) {
        uint32_t best = 0, best_high = 0;
        int bc = -1, bch = -1;
        bool be = false, beh = false;
        for (uint32_t R = 0; R < (1u << k); ++R) {
            if (__builtin_popcount(R) != kRegBits) continue;
            bool e = false;
            const int c = tc_count(gates, left, pos_of, n, R, scan_max, &e);
            if (c > bc) {
                bc = c;
                best = R;
                be = e;
            }
            if (!(R & low) && c > bch) {
                bch = c;
                best_high = R;
                beh = e;
            }
        }
        // a first stage without lanes among its registers needs no transpose after the load
        if (prefer_high && bch > 0 && 4 * bch >= 3 * bc) {
            *ext_used = beh;
            return best_high;
        }
        *ext_used = be;
        return best;
    };
    std::vector<Stage> stages;
    int slots = 0;
    bool ext_used = false;
    uint32_t R = best_set(true, &ext_used);
    Layout L;
    if (R & low) {  // load in a canonical layout, then transpose to R
        uint32_t H = 0;
        for (int p = k - 1, c = 0; p >= kTcLanes && c < kRegBits; --p, ++c) H |= 1u << p;
        const Layout C = tc_layout(k, H);
        stages.push_back(Stage{C, C, 0, 0, -1, -1});
    }
    L = tc_layout(k, R);
    while (!left.empty()) {
        if (slots + 1 > max_slots) break;
        const bool allow_ext = slots + 2 <= max_slots;
        Stage st{L, L, 0, 0, slots, -1};
        cd G[2][kTcSlot];
        for (int v = 0; v < 2; ++v)
            for (int e = 0; e < kTcSlot; ++e) G[v][e] = (e % 17 == 0) ? cd(1.0) : cd(0.0);
        std::vector<int> still;
        std::vector<char> blocked(n, 0);
        int ext = allow_ext ? -1 : -2, ran = 0;
        for (int gi : left) {
            const PGate &g = gates[gi];
            int qs[3];
            const int nq = qubits(g, qs);
            bool blk = false;
            for (int j = 0; j < nq; ++j) blk |= blocked[qs[j]] != 0;
            if (!blk && tc_exec(g, pos_of, mask_of(L.P), ext)) {
                ++ran;
                if (g.cls == G_SWAP) {
                    const int a = pos_of[g.t], b = pos_of[g.t2];
                    for (int j = 0; j < kRegBits; ++j) L.P[j] = int8_t(L.P[j] == a ? b : L.P[j] == b ? a : L.P[j]);
                    for (int q = 0; q < k - kRegBits; ++q) L.Q[q] = int8_t(L.Q[q] == a ? b : L.Q[q] == b ? a : L.Q[q]);
                    continue;
                }
                const int jt = pos_of[g.t] >= 0 ? reg_bit(L, pos_of[g.t]) : -1;
                const int jc = (g.c >= 0 && pos_of[g.c] >= 0) ? reg_bit(L, pos_of[g.c]) : -1;
                for (int v = 0; v < 2; ++v) tc_mul_gate(G[v], g, jt, jc, v, ext);
            } else {
                still.push_back(gi);
                for (int j = 0; j < nq; ++j) blocked[qs[j]] = 1;
            }
        }
        left.swap(still);
        st.out = L;
        if (ran == 0) break;  // the frontier needs a qubit outside the tile and no slot is left for it
        st.ext = ext >= 0 ? ext : -1;
        const int nv = ext >= 0 ? 2 : 1;
        for (int v = 0; v < nv; ++v) P.tcm.insert(P.tcm.end(), G[v], G[v] + kTcSlot);
        slots += nv;
        stages.push_back(st);
        if (left.empty()) break;
        R = best_set(false, &ext_used);
        L = tc_layout(k, R);
    }
    L = stages.back().out;
    if (!tc_canonical(L, k)) {
        uint32_t H = 0;
        int c = 0;
        for (int j = 0; j < kRegBits; ++j)
            if (L.P[j] >= kTcLanes) {
                H |= 1u << L.P[j];
                ++c;
            }
        for (int p = k - 1; p >= kTcLanes && c < kRegBits; --p)
            if (!((H >> p) & 1u)) {
                H |= 1u << p;
                ++c;
            }
        const Layout C = tc_layout(k, H);
        stages.push_back(Stage{C, C, 0, 0, -1, -1});
    }
    P.stages = std::move(stages);
    P.tc = true;
    P.tc_unitary = true;
    for (size_t sl = 0; sl < P.tcm.size() / kTcSlot; ++sl) {
        const cd *G = P.tcm.data() + sl * kTcSlot;
        for (int r = 0; r < 16; ++r)
            for (int c = 0; c < 16; ++c) {
                cd a = 0.0;
                for (int m = 0; m < 16; ++m) a += std::conj(G[16 * m + r]) * G[16 * m + c];
                if (std::abs(a - (r == c ? 1.0 : 0.0)) > 1e-12) P.tc_unitary = false;
            }
    }
}

}  // namespace

double fma_per_amp_c64(const Op &op)
{
    const bool reg_sel = op.sreg >= 0 && op.sreg != 3;
    switch (op.type) {
    case OP_X: return 0.0;
    case OP_DIAG: return reg_sel && op.m0id ? 2.0 : 4.0;
    case OP_GEN2: return 16.0;
    default: return reg_sel && op.m0id ? 4.0 : 8.0;
    }
}

int classify(const std::complex<double> U[4])
{
    if (U[1] == 0.0 && U[2] == 0.0) return G_DIAG;
    if (U[0] == 0.0 && U[3] == 0.0 && U[1] == 1.0 && U[2] == 1.0) return G_X;
    return G_GEN;
}

bool make_plan(int n, int k, bool pin0, bool fuse, bool pairs, const std::vector<PGate> &gates,
               std::vector<Pass> &out, PlanStats &stats, std::string &err, bool tc)
{
    out.clear();
    stats = PlanStats{};
    if (k < kMinK || k > kMaxK || k > n) {
        err = "tile size out of range";
        return false;
    }
    if (tc) {
        if (k < 11) {
            err = "tensor-core passes need tiles of 2^11 or 2^12 amplitudes";
            return false;
        }
        pin0 = false;
    }
    const int nh = k - kChunkBits;
    if (pin0) {
        // Qubit 0 never leaves register bit 3, so a SWAP touching it cannot be
        // a relabeling: expand it into CNOT(0->x) CNOT(x->0) CNOT(0->x).
        bool any = false;
        for (const PGate &g : gates) any |= g.cls == G_SWAP && (g.t == 0 || g.t2 == 0);
        if (any) {
            std::vector<PGate> ex;
            ex.reserve(gates.size() + 8);
            for (const PGate &g : gates) {
                if (g.cls == G_SWAP && (g.t == 0 || g.t2 == 0)) {
                    const int x = g.t == 0 ? g.t2 : g.t;
                    PGate c{};
                    c.cls = G_X;
                    c.t2 = -1;
                    c.U[0] = 0.0; c.U[1] = 1.0; c.U[2] = 1.0; c.U[3] = 0.0;
                    c.t = x; c.c = 0; ex.push_back(c);
                    c.t = 0; c.c = x; ex.push_back(c);
                    c.t = x; c.c = 0; ex.push_back(c);
                } else {
                    ex.push_back(g);
                }
            }
            return make_plan(n, k, pin0, fuse, pairs, ex, out, stats, err, tc);
        }
    }
    std::vector<int> rem(gates.size());
    for (size_t i = 0; i < gates.size(); ++i) rem[i] = int(i);
    bool adjoint = false;
    for (const PGate &g : gates) adjoint |= g.nd > 0;
    const int max_ops = adjoint ? kMaxOpsAdjoint : kMaxOpsPerPass;
    const int first_free = pin0 ? 6 : 5;  // lowest position a canonical register bit may take

    while (!rem.empty()) {
        // ---- choose the tile's high qubits greedily
        std::vector<char> inS(n, 0);
        // tensor-core stages take one qubit outside the tile per gate at most: a
        // controlled diagonal gate needs its target in the tile
        auto need_of = [&](const PGate &g, int need[2]) {
            const int nn = needs(g, need);
            if (tc && nn == 0 && g.cls == G_DIAG && g.c >= 0) {
                need[0] = g.t;
                return 1;
            }
            return nn;
        };
        auto fits = [&](const PGate &g) {
            int need[2];
            const int nn = need_of(g, need);
            for (int i = 0; i < nn; ++i)
                if (!inS[need[i]]) return false;
            return true;
        };
        // Adding one qubit at a time can miss a gate that needs two (a SWAP of two
        // qubits outside the tile that everything else waits behind); then the
        // first gate's qubits are put in first, which always makes progress.
        for (int attempt = 0; attempt < 2; ++attempt) {
            std::fill(inS.begin(), inS.end(), 0);
            for (int q = 0; q < kChunkBits; ++q) inS[q] = 1;
            int steps = nh;
            if (attempt == 1) {
                int need[2];
                const int nn = need_of(gates[rem[0]], need);
                for (int i = 0; i < nn; ++i)
                    if (!inS[need[i]]) {
                        inS[need[i]] = 1;
                        --steps;
                    }
            }
            for (int step = 0; step < steps; ++step) {
                int best = -1;
                long long best_score = -1;
                for (int q = kChunkBits; q < n; ++q) {
                    if (inS[q]) continue;
                    inS[q] = 1;
                    const int cnt = scan(gates, rem, n, fits, nullptr);
                    inS[q] = 0;
                    int soon = 0;  // tie-break: gates needing q soon
                    for (size_t r = 0; r < rem.size() && r < size_t(kLookahead); ++r) {
                        int need[2];
                        const int nn = need_of(gates[rem[r]], need);
                        for (int i = 0; i < nn; ++i) soon += need[i] == q;
                    }
                    const long long score = (long long)cnt * 4096 + soon * 16 + (n - q);
                    if (score > best_score) {
                        best_score = score;
                        best = q;
                    }
                }
                if (best < 0) {
                    err = "no qubit left to add to the tile";
                    return false;
                }
                inS[best] = 1;
            }
            if (scan(gates, rem, n, fits, nullptr) > 0) break;
        }
        Pass P;
        P.k = k;
        std::vector<int> pos_of(n, -1);
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
        {  // tile id bits -> runs of physical bits outside the tile
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
        std::vector<int> taken;
        scan(gates, rem, n, fits, &taken);
        if (taken.empty()) {
            err = "planner made no progress";
            return false;
        }
        std::vector<int> pg;
        for (int r : taken) pg.push_back(rem[r]);
        if (tc) {
            std::vector<int> left = pg;
            build_tc_pass(gates, left, pos_of, n, k, P);
            if (left.size() == pg.size()) {
                err = "planner made no progress";
                return false;
            }
            std::vector<char> done(gates.size(), 0);
            for (int gi : pg) done[gi] = 1;
            for (int gi : left) done[gi] = 0;
            std::vector<int> nrem;
            for (int gi : rem)
                if (!done[gi]) nrem.push_back(gi);
            P.ngates = int(pg.size() - left.size());
            stats.passes++;
            stats.stages += int(P.stages.size());
            stats.transposes += int(P.stages.size()) - 1;
            stats.gates += P.ngates;
            for (const Stage &st : P.stages)
                if (st.mat >= 0) {
                    stats.tc_mats++;
                    // 16 complex multiply-adds per amplitude and stage (8 real operations each)
                    stats.flops_per_amp += 128.0;
                }
            out.push_back(std::move(P));
            rem.swap(nrem);
            continue;
        }

        // ---- stages: run gates whose target is a register bit; transpose otherwise
        LayoutState ls{k, {}};
        // targets (tile positions) of non-diagonal gates in frontier order, then later ones
        auto frontier_targets = [&](const std::vector<int> &left, std::vector<int> &pos, int lo, int want) {
            std::vector<char> blocked(n, 0);
            auto consider = [&](int p) {
                if (p < lo || (pin0 && p == 0)) return;
                if (std::find(pos.begin(), pos.end(), p) == pos.end()) pos.push_back(p);
            };
            for (int round = 0; round < 2 && int(pos.size()) < want; ++round) {
                std::fill(blocked.begin(), blocked.end(), 0);
                for (int gi : left) {
                    const PGate &g = gates[gi];
                    int qs[3];
                    const int nq = qubits(g, qs);
                    bool blk = false;
                    for (int i = 0; i < nq; ++i) blk |= blocked[qs[i]] != 0;
                    if ((g.cls == G_GEN || g.cls == G_X) && (round == 1 || !blk) && pos_of[g.t] >= 0)
                        consider(pos_of[g.t]);
                    for (int i = 0; i < nq; ++i) blocked[qs[i]] = 1;
                    if (int(pos.size()) >= want) break;
                }
            }
        };
        const int nfree = pin0 ? 3 : 4;  // register bits the planner chooses
        std::vector<int> left = pg;
        std::vector<Stage> stages;
        std::vector<Op> ops;
        {
            std::vector<int> pos;
            frontier_targets(left, pos, first_free, nfree);
            for (int p = k - 1; p >= first_free && int(pos.size()) < nfree; --p)
                if (std::find(pos.begin(), pos.end(), p) == pos.end()) pos.push_back(p);
            int extra[kRegBits] = {0, 0, 0, 0};
            for (int j = 0; j < nfree; ++j) extra[j] = pos[j];
            ls.L = canonical_layout(k, pin0, extra);
        }
        Stage cur{ls.L, ls.L, 0, 0};

        // ---- gate fusion bookkeeping (reset at every layout change)
        std::vector<int> open_op(n, -1);   // op open for fusion on this target qubit
        std::vector<int> op_sel, op_time;  // per op: select qubit, gate time it was created
        std::vector<int> last_mod(n, -1);  // gate time of the last non-diagonal gate per qubit
        int gtime = 0;
        auto close_all = [&]() { std::fill(open_op.begin(), open_op.end(), -1); };
        auto coord = [&](int q, int8_t &reg, uint32_t &thr, uint64_t &ext) {
            const int p = pos_of[q];
            if (p < 0) ext = uint64_t(1) << q;
            else if (ls.reg_of(p) >= 0) reg = int8_t(ls.reg_of(p));
            else thr = 1u << ls.thr_of(p);
        };
        auto process = [&](const PGate &g) {
            const int t = g.t, c = g.c;
            const bool nondiag = g.cls != G_DIAG;
            const int o = (fuse && g.nd == 0) ? open_op[t] : -1;
            bool fused = false;
            if (o >= 0) {
                Op &op = ops[o];
                const int so = op_sel[o];
                if (c < 0) {
                    for (int s = 0; s < 2; ++s) {
                        if (s == 0 && op.m0id) {
                            for (int e = 0; e < 4; ++e) op.M[0][e] = g.U[e];
                        } else {
                            matmul(g.U, op.M[s], op.M[s]);
                        }
                    }
                    op.m0id = 0;
                    fused = true;
                } else if ((so < 0 || so == c) && last_mod[c] < op_time[o]) {
                    if (so < 0) {
                        for (int e = 0; e < 4; ++e) op.M[1][e] = op.M[0][e];
                        coord(c, op.sreg, op.sthr, op.sext);
                        op_sel[o] = c;
                    }
                    matmul(g.U, op.M[1], op.M[1]);
                    fused = true;
                }
                if (fused) {
                    // X or diagonal ops absorbing anything but diagonals become general
                    // 2x2 ops (a non-diagonal gate on t is only run when t is a register bit)
                    if (nondiag || op.type != OP_DIAG) op.type = OP_GEN;
                } else {
                    open_op[t] = -1;
                }
            }
            if (!fused) {
                Op op{};
                op.treg = op.sreg = op.treg2 = -1;
                op.type = g.cls == G_DIAG ? OP_DIAG : g.cls == G_X ? OP_X : OP_GEN;
                if (op.type == OP_DIAG) coord(t, op.treg, op.tthr, op.text);
                else op.treg = int8_t(ls.reg_of(pos_of[t]));
                const cd I[4] = {1.0, 0.0, 0.0, 1.0};
                for (int e = 0; e < 4; ++e) {
                    op.M[0][e] = c >= 0 ? I[e] : g.U[e];
                    op.M[1][e] = g.U[e];
                }
                op.m0id = c >= 0 ? 1 : 0;
                if (c >= 0) coord(c, op.sreg, op.sthr, op.sext);
                op.nd = g.nd;
                op.slot = g.slot;
                op.gen = g.gen;
                for (int d = 0; d < g.nd; ++d)
                    for (int e = 0; e < 4; ++e) op.D[d][e] = g.dU[d][e];
                open_op[t] = g.nd > 0 ? -1 : int(ops.size());  // nothing merges into a differentiated op
                op_sel.push_back(c);
                op_time.push_back(gtime);
                ops.push_back(op);
            }
            if (nondiag) {
                last_mod[t] = gtime;
                for (int q = 0; q < n; ++q)
                    if (open_op[q] >= 0 && op_sel[open_op[q]] == t) open_op[q] = -1;
            }
            if (c >= 0) open_op[c] = -1;
            ++gtime;
        };

        while (!left.empty()) {
            // run every executable gate in order (with blocking)
            std::vector<int> still;
            std::vector<char> blocked(n, 0);
            for (int gi : left) {
                const PGate &g = gates[gi];
                int qs[3];
                const int nq = qubits(g, qs);
                bool blk = false;
                for (int i = 0; i < nq; ++i) blk |= blocked[qs[i]] != 0;
                bool exec = false;
                if (!blk && int(ops.size()) < max_ops) {
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
                        close_all();
                    } else {
                        process(g);
                    }
                } else {
                    still.push_back(gi);
                    for (int i = 0; i < nq; ++i) blocked[qs[i]] = 1;
                }
            }
            left.swap(still);
            if (left.empty()) break;
            if (int(ops.size()) >= max_ops || int(stages.size()) + 2 >= kMaxStagesPerPass) break;
            // the first gate left needs a register bit it lacks: new register set
            cur.out = ls.L;
            cur.op_end = int(ops.size());
            stages.push_back(cur);
            std::vector<int> pos;
            frontier_targets(left, pos, 0, nfree);
            for (int j = 0; j < kRegBits && int(pos.size()) < nfree; ++j) {
                const int p = ls.L.P[j];
                if (!(pin0 && p == 0) && std::find(pos.begin(), pos.end(), p) == pos.end()) pos.push_back(p);
            }
            int regs[kRegBits];
            for (int j = 0; j < nfree; ++j) regs[j] = pos[j];
            if (pin0) regs[3] = 0;
            ls.L = make_layout(k, pin0, regs);
            cur = Stage{ls.L, ls.L, int(ops.size()), int(ops.size())};
            close_all();
        }
        cur.out = ls.L;
        cur.op_end = int(ops.size());
        stages.push_back(cur);
        if (!is_canonical(ls.L, pin0)) {
            int extra[kRegBits];
            int ne = 0;
            for (int j = 0; j < kRegBits && ne < nfree; ++j)
                if (ls.L.P[j] >= first_free) extra[ne++] = ls.L.P[j];
            for (int p = k - 1; p >= first_free && ne < nfree; --p) {
                bool have = false;
                for (int e = 0; e < ne; ++e) have |= extra[e] == p;
                if (!have) extra[ne++] = p;
            }
            Layout C = canonical_layout(k, pin0, extra);
            stages.push_back(Stage{C, C, int(ops.size()), int(ops.size())});
        }
        // gates of this pass that did not run go back to `rem`, in order
        std::vector<char> done(gates.size(), 0);
        for (int gi : pg) done[gi] = 1;
        for (int gi : left) done[gi] = 0;
        std::vector<int> nrem;
        for (int gi : rem)
            if (!done[gi]) nrem.push_back(gi);
        P.ngates = int(pg.size() - left.size());
        P.stages = std::move(stages);
        P.ops = std::move(ops);
        if (fuse && pairs) fuse_pair_blocks(P, pin0, stats.pair_ops);
        stats.passes++;
        stats.stages += int(P.stages.size());
        stats.transposes += int(P.stages.size()) - 1;
        stats.gates += P.ngates;
        stats.ops += int(P.ops.size());
        for (const Op &op : P.ops) {
            const double f = op.type == OP_GEN    ? 14.0
                             : op.type == OP_DIAG ? (sign_only(op) ? 0.0 : 6.0)
                             : op.type == OP_GEN2 ? 30.0
                                                  : 0.0;
            stats.flops_per_amp += op.m0id ? 0.5 * f : f;
        }
        out.push_back(std::move(P));
        rem.swap(nrem);
    }
    return true;
}

}  // namespace plan
}  // namespace qv
