// Pass planner for the fused tiled kernel (pure host C++, no CUDA).
//
// The paper's block storage (Sec. III-C, Eq. 7-8) loads only the blocks a gate
// touches and aligns each amplitude pair (i, i XOR 2^k) inside one block
// (Sec. III-E); its sliding window (Sec. III-B, Eq. 6) keeps a block on fast
// memory while every pending update is applied. On the GPU a block is a tile
// of 2^K amplitudes whose index bits are the low kChunkBits physical qubits
// (one contiguous run of 2^kChunkBits amplitudes) plus K - kChunkBits freely
// chosen higher qubits: every pair of a gate whose target is among the tile's
// qubits lies inside the tile. One pass loads every tile once, applies all
// gates assigned to the pass on chip, and stores the tile once.
//
// Inside a tile, thread t holds 2^kRegBits amplitudes in registers. A layout
// says which tile positions are register bits (P) and which are thread-index
// bits (Q, lanes first). A gate can be applied in registers when its target is
// a register bit; controls and diagonal gates may sit anywhere (register bit,
// thread bit, or a qubit outside the tile, which is uniform per tile). Changing
// the layout is a shared-memory transpose. A SWAP of two tile qubits moves no
// data: it exchanges the positions two layout bits refer to.
#pragma once

#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

namespace qv {
namespace plan {

constexpr int kRegBits = 4;    // amplitudes per thread = 16
constexpr int kChunkBits = 5;  // contiguous low qubits always in the tile
constexpr int kMaxK = 12;
constexpr int kMinK = 10;

enum GateClass : int { G_GEN = 0, G_X = 1, G_DIAG = 2, G_SWAP = 3 };

// A validated gate in planner form.
struct PGate {
    int cls;          // GateClass
    int t, t2, c;     // target, swap partner (-1), control (-1)
    std::complex<double> U[4];
    // Adjoint plans only: nd > 0 marks a gate whose derivatives dU[0..nd) are
    // evaluated where it runs (first gradient slot `slot`). Such a gate gets an
    // op of its own (class G_GEN), never merged with other gates.
    int nd = 0, slot = -1;
    std::complex<double> dU[3][4];
    // Adjoint plans: the gate is exp(-i theta G / 2) (gen 1, 2, 3: G = X, Y, Z on
    // the target) or P(theta) (gen 4: dP = i |1><1| P) in its one trainable angle, so
    // its derivative term can be taken from psi before the gate is undone; 0: use dU
    int gen = 0;
};

enum OpType : int8_t { OP_GEN = 0, OP_X = 1, OP_DIAG = 2, OP_GEN2 = 3 };

// One on-chip operation in the coordinates of the layout of its stage. It
// applies M[s] to the target qubit, where s is the value of one "select" bit
// (a register bit, a thread-index bit, a physical qubit outside the tile, or
// none: s = 0). A controlled gate is M[0] = I, M[1] = U (m0id = 1); the
// planner multiplies later gates on the same target into an open op (both
// branches, or only the s = 1 branch for a gate controlled by the select bit).
// GEN2 is a dense 4x4 on two register bits (treg, treg2) that replaces a run
// of ops acting only on those two bits: M4 row-major, index bit 0 <-> treg,
// bit 1 <-> treg2.
struct Op {
    int8_t type;      // OpType: GEN (any 2x2), X (the bit flip, unfused), DIAG (diagonal), GEN2 (4x4)
    int8_t treg;      // target register bit (GEN, X, GEN2; DIAG with a register target), else -1
    int8_t treg2;     // GEN2: second register bit, else -1
    int8_t sreg;      // select register bit, else -1
    int8_t m0id;      // M[0] is the identity
    uint32_t sthr;    // select = this thread-index bit (0: none)
    uint32_t tthr;    // DIAG: target on this thread-index bit (0: none)
    uint64_t sext;    // select = this physical qubit outside the tile (0: none)
    uint64_t text;    // DIAG: target physical qubit outside the tile (0: none)
    std::complex<double> M[2][4];   // row-major 2x2 for s = 0 / 1 (DIAG: entries [0], [3])
    std::complex<double> M4[16];    // GEN2 only
    int nd = 0, slot = -1;          // adjoint plans: derivatives of this op's gate (see PGate)
    std::complex<double> D[3][4];   // derivative matrices, applied where M[1] applies
    int gen = 0;                    // adjoint plans: generator form of the derivative (see PGate)
};

// A diagonal op whose entries are all +1 or -1 (Z, CZ and products of them):
// it only flips signs, so the compiled engine applies it with sign-bit XORs
// and the cost model counts no floating-point operations for it.
inline bool sign_only(const Op &op)
{
    if (op.type != OP_DIAG) return false;
    for (int s = 0; s < 2; ++s)
        for (int e : {0, 3}) {
            const std::complex<double> d = op.M[s][e];
            if (d.imag() != 0.0 || (d.real() != 1.0 && d.real() != -1.0)) return false;
        }
    return true;
}

struct Layout {
    int8_t P[kRegBits];          // register bit j -> tile position
    int8_t Q[kMaxK - kRegBits];  // thread bit b -> tile position (lanes are b < 5)
};

struct Stage {
    Layout in;        // layout the registers are read in (after the transpose)
    Layout out;       // layout at the end of the stage (SWAPs relabel positions)
    int op_begin, op_end;
    // Tensor-core plans only: first slot of this stage's 16x16 matrix in
    // Pass::tcm (-1: a transpose-only stage) and the physical qubit outside the
    // tile whose value selects slot mat + 1 instead of mat (-1: none).
    int mat = -1, ext = -1;
};

struct Pass {
    int k = 0;
    int s_high[kMaxK - kChunkBits];  // physical qubit of tile position kChunkBits + j (ascending)
    // tile id -> base index: runs of consecutive physical bits outside the tile
    int nseg = 0;
    int seg_src[kMaxK], seg_w[kMaxK], seg_dst[kMaxK];
    std::vector<Stage> stages;
    std::vector<Op> ops;
    int ngates = 0;
    // Tensor-core plans: every stage applies one dense 16x16 complex matrix to
    // the 16 amplitudes that differ in its four register positions (register
    // bit j <-> index bit j, row-major, out = M in); tcm holds kTcSlot entries
    // per matrix slot.
    bool tc = false;
    std::vector<std::complex<double>> tcm;
    // every matrix of the pass is unitary (to 1e-12): the pass then keeps the
    // norm of every tile, since it acts inside tiles
    bool tc_unitary = false;
};

constexpr int kTcSlot = 256;
constexpr int kTcLanes = 5;  // tensor-core load/store layouts: lane b <-> tile position b
// Matrix slots a tensor-core pass may hold (shared memory: 8 KB each).
inline int tc_max_slots(int k) { return k >= 12 ? 8 : 7; }

struct PlanStats {
    int passes = 0, stages = 0, transposes = 0, gates = 0, ops = 0, pair_ops = 0;
    int tc_mats = 0;  // tensor-core plans: stages that apply a matrix
    // algorithmic floating-point operations per amplitude of the state, summed
    // over all ops: a 2x2 complex matrix on a pair is 28 real operations (14 per
    // amplitude), a diagonal one 6 per amplitude, X none, a 4x4 on a group of
    // four 30 per amplitude (4 complex products, 3 sums); a controlled op
    // (identity when its select bit is 0) updates half the amplitudes
    double flops_per_amp = 0;
};

// Plans gates[0..ng) for an n-qubit state with tiles of 2^k amplitudes
// (kMinK <= k <= min(kMaxK, n)). `pin0` is set for 8-byte amplitudes: tile
// position 0 stays on register bit 3 in every layout (the kernel packs the two
// amplitudes that differ in qubit 0 into one f32x2 register and moves them as
// one 8-byte unit), and the load/store layout puts lanes on positions 1..5
// (one 16-byte access = the two amplitudes of one packed pair). Without pin0
// (16-byte amplitudes) lanes of the load/store layout sit on positions 0..4.
// Returns false with `err` set on failure.
// `fuse` = false keeps one op per gate. `pairs` (with `fuse`) then merges runs
// of ops that act only on two register bits (targets and register selects; not
// the packed lane bit) into GEN2 ops where that takes fewer FP32 operations.
//
// `tc` plans for the tensor-core kernel instead (k >= 11, 8-byte amplitudes;
// pin0, fuse and pairs are ignored): a stage holds any four tile positions in
// registers and runs, in order, every gate whose qubits are all register
// positions, except that a control or a diagonal target may lie outside the
// tile (one such qubit per stage: it selects one of two matrices per tile).
// The stage's gates multiply into one 16x16 matrix. Load and store layouts put
// lanes on tile positions 0..4 and registers on positions >= 5.
bool make_plan(int n, int k, bool pin0, bool fuse, bool pairs, const std::vector<PGate> &gates,
               std::vector<Pass> &out, PlanStats &stats, std::string &err, bool tc = false);

// FP32 fused multiply-adds per amplitude the compiled complex64 kernel spends
// on `op` (the cost model of the pair fusion).
double fma_per_amp_c64(const Op &op);

// Classifies a 2x2 matrix: G_DIAG if off-diagonal entries are 0, G_X if it is
// exactly [[0,1],[1,0]], else G_GEN.
int classify(const std::complex<double> U[4]);

}  // namespace plan
}  // namespace qv
