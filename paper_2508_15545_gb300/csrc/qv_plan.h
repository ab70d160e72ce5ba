// Fused-pass planning and execution (the on-chip form of the paper's
// sliding-window cache and block storage, Sec. III-B/C/E) and qubit
// permutations.
#pragma once

#include <string>
#include <vector>

#include "planner.h"
#include "qv_internal.h"

namespace qv {

// True when qv_apply_circuit in QV_MODE_AUTO should take the fused path.
bool fused_supported(const qv_state *s, const qv_plan_opts *opts);
qv_status apply_fused(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts);
// Plan statistics (out, may be NULL) and algorithmic cost (cost, may be NULL:
// cost[0] = HBM bytes, cost[1] = floating-point operations) of the fused plan.
qv_status plan_info(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t out[4],
                    double cost[2]);
// Host only: the generated CUDA source of compiled pass `pass` of that plan,
// and NVRTC compilation of all its passes (out as jit_compile_host).
qv_status plan_source(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int pass,
                      std::string &src);
qv_status plan_compile(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int64_t out[4]);
// Host only: one stage of a tensor-core plan (qv_plan_tc_stage).
qv_status plan_tc_stage(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int pass,
                        int stage, qv_tc_stage *out);

// A state in host memory: the circuit runs in device windows (window.cu).
qv_status apply_windowed(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts);
void window_release(qv_state *s);
// The window a host-memory state takes without window_bits: the whole state
// when it fits in half of the free device memory, else 0 (passes in place).
int default_window_bits(const qv_state *s);

// Bit q of every index moves to bit perm[q].
qv_status apply_permutation(qv_state *s, const int32_t *perm);
// Frees per-handle planning buffers.
void plan_cache_release(qv_state *s);
// qv_gate list -> planner gates (matrices in FP64, classified).
qv_status to_pgates(const qv_gate *g, size_t ng, std::vector<plan::PGate> &out);

// ---- autotuner (autotune.cu)
// Tile bits to use by default: the autotuned value for (n, dtype, engine) when
// one was measured, else min(n, 12).
int tuned_tile_bits(int n, qv_dtype dt, bool interpreting = true);
// Engine flags (QV_PLAN_NO_PAIRS, QV_PLAN_TENSOR) the autotuner chose with that
// tile size, 0 when untuned; whether (n, dtype, engine) was tuned at all.
int tuned_flags(int n, qv_dtype dt, bool interpreting);
bool tile_bits_tuned(int n, qv_dtype dt, bool interpreting);
// Times the fused path with every tile size (and, with `variants`, the
// schedule variants: 4x4 pair operations on or off, tensor-core stages) on the
// caller's circuit and keeps the fastest for (n, dtype, engine).
qv_status autotune(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t *best_k,
                   int32_t *best_flags, bool variants = true);

// ---- batched circuits (batch.cu)
qv_status batch_create(const qv_batch_item *items, size_t count, const qv_pauli_term *H, size_t nt,
                       const qv_plan_opts *opts, qv_batch **out);
qv_status batch_run(qv_batch *b, double *expvals);
// Per launch group: tile bits, circuits, qubits of its first circuit, compiled
// (1) or interpreting (0), L2 group size and tiles per work item (6 values each).
size_t batch_info(const qv_batch *b, int32_t *out, size_t cap);
// Launches one bounded wait on a counter nothing increments (`limit` polls).
qv_status wait_selftest(qv_state *s, uint32_t limit);
void batch_release(qv_batch *b);

}  // namespace qv
