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
};

enum OpType : int8_t { OP_GEN = 0, OP_X = 1, OP_DIAG = 2 };

// One on-chip operation in the coordinates of the current layout.
struct Op {
    int8_t type;      // OpType
    int8_t treg;      // target register bit (GEN, X, DIAG on a register bit), else -1
    int8_t creg;      // control register bit, else -1
    int8_t pad0;
    uint32_t cthr;    // thread-index bits that must all be 1 (controls on thread bits)
    uint32_t tthr;    // DIAG: thread-index bit selecting d1
    uint32_t pad1;
    uint64_t cext;    // physical bits outside the tile that must all be 1
    uint64_t text;    // DIAG: physical bit outside the tile selecting d1
    double m[8];      // GEN/X: U00 U01 U10 U11 (re, im); DIAG: d0, d1 (re, im)
};

struct Layout {
    int8_t P[kRegBits];          // register bit j -> tile position
    int8_t Q[kMaxK - kRegBits];  // thread bit b -> tile position (lanes are b < 5)
};

struct Stage {
    Layout in;        // layout the registers are read in (after the transpose)
    Layout out;       // layout at the end of the stage (SWAPs relabel positions)
    int op_begin, op_end;
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
};

struct PlanStats {
    int passes = 0, stages = 0, transposes = 0, gates = 0, ops = 0;
};

// Plans gates[0..ng) for an n-qubit state with tiles of 2^k amplitudes
// (kMinK <= k <= min(kMaxK, n)). `canonical_lane0` selects the load/store
// layout: true for 8-byte amplitudes (register bit 0 = tile position 0, lanes =
// positions 1..5, two amplitudes per 16-byte access), false for 16-byte ones
// (lanes = positions 0..4). Returns false with `err` set on failure.
bool make_plan(int n, int k, bool canonical_lane0, const std::vector<PGate> &gates, std::vector<Pass> &out,
               PlanStats &stats, std::string &err);

// Classifies a 2x2 matrix: G_DIAG if off-diagonal entries are 0, G_X if it is
// exactly [[0,1],[1,0]], else G_GEN.
int classify(const std::complex<double> U[4]);

}  // namespace plan
}  // namespace qv
