/*
 * qv.h -- C ABI of libqv.so, a GB300 (sm_103a) state-vector simulator built on
 * the amplitude-pairing rule of QVecOpt (arXiv 2508.15545).
 *
 * Problem statement (Sec. II, Eq. 1-2): an n-qubit state is a dense vector of
 * 2^n complex amplitudes, 8 bytes each in single precision (QV_C64: float re,
 * float im) or 16 bytes in double precision (QV_C128: double re, double im),
 * stored interleaved (re, im) in index order on the GPU. Qubit q is bit q of
 * the amplitude index (little-endian): a gate on qubit k pairs amplitude i with
 * amplitude i XOR 2^k (Sec. III-A, Eq. 5).
 *
 * Conventions for every entry point:
 *   - Every call returns a qv_status; QV_OK is 0. On failure qv_last_error()
 *     returns a message for the calling thread. No call aborts the process or
 *     traps the GPU; a failed call leaves the state's contents unspecified but
 *     the handle valid (destroy it or overwrite it).
 *   - Work is enqueued on the handle's CUDA stream (the one given at creation
 *     or by qv_set_stream) and the call returns without synchronising, except
 *     calls that write host memory (qv_get_state, reductions, gradients), which
 *     synchronise that stream before returning.
 *   - Host arrays passed in are owned by the caller and only read during the
 *     call; the library copies gate lists. Host outputs are written before the
 *     call returns.
 *   - One handle must not be used from two host threads at once.
 */
#ifndef QV_H
#define QV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qv_state qv_state;   /* opaque handle */

typedef enum { QV_C64 = 0, QV_C128 = 1 } qv_dtype;

typedef enum {
    QV_OK = 0,
    QV_ERR_ARG = 1,          /* bad argument: qubit out of range, ctrl == target, NULL, non-finite matrix ... */
    QV_ERR_OOM = 2,          /* device allocation failed or the state would not fit */
    QV_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error string) */
    QV_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up (status word set by a kernel) */
    QV_ERR_UNSUPPORTED = 5   /* valid request this build does not handle */
} qv_status;

typedef struct { double re, im; } qv_c128;

/* Gate kinds. Matrices follow OpenQASM: RX/RY/RZ(t) = exp(-i t sigma / 2),
 * P(l) = diag(1, e^{il}), U3(t,p,l) = [[cos t/2, -e^{il} sin t/2],
 * [e^{ip} sin t/2, e^{i(p+l)} cos t/2]], H = [[1,1],[1,-1]]/sqrt 2. */
typedef enum {
    QV_G_H = 0, QV_G_X = 1, QV_G_Y = 2, QV_G_Z = 3, QV_G_S = 4, QV_G_SDG = 5,
    QV_G_T = 6, QV_G_TDG = 7, QV_G_RX = 8, QV_G_RY = 9, QV_G_RZ = 10, QV_G_P = 11,
    QV_G_U3 = 12, QV_G_MATRIX = 13, QV_G_SWAP = 14
} qv_gate_kind;

/* One gate of a circuit. target: the qubit the 2x2 matrix acts on; target2:
 * second qubit of QV_G_SWAP (else -1); ctrl: control qubit (the gate acts on
 * the amplitudes whose control bit is 1) or -1; theta: angles (RX/RY/RZ/P use
 * theta[0]; U3 uses theta, phi, lambda); param: index of the trainable
 * parameter behind each angle, or -1 (used by qv_adjoint_grad only);
 * u: row-major matrix for QV_G_MATRIX (row/column 0 = target bit 0). */
typedef struct {
    int32_t kind;
    int32_t target;
    int32_t target2;
    int32_t ctrl;
    int32_t param[3];
    int32_t reserved;
    double  theta[3];
    qv_c128 u[4];
} qv_gate;

/* How qv_apply_circuit runs a gate list. */
typedef enum {
    QV_MODE_AUTO = 0,    /* fused passes when n >= the tile size, else per gate */
    QV_MODE_PLAIN = 1,   /* one strided pair-update kernel per gate (Eq. 5 per gate) */
    QV_MODE_FUSED = 2    /* tiled passes: many gates per HBM round trip */
} qv_mode;

/* qv_plan_opts.flags */
#define QV_PLAN_NO_FUSION 1  /* fused mode: one on-chip operation per gate (no 2x2 products) */
#define QV_PLAN_INTERPRET 2  /* fused mode: run the planner's program with the precompiled
                                interpreting kernel instead of compiling each pass (NVRTC);
                                also used when NVRTC cannot be loaded */
#define QV_PLAN_NO_PAIRS 4   /* fused mode: no 4x4 operations on two register qubits (the
                                compiled complex64 kernel merges runs of operations on two
                                qubits into one 4x4 when that takes fewer FP32 operations) */
#define QV_PLAN_HOST_IN_PLACE 32  /* fused mode, state in host memory: every pass reads and writes
                                the host memory in place over the host link instead of running in
                                a device window */
#define QV_PLAN_AUTOTUNE 16  /* qv_batch_create: run the autotuner once for every qubit count of
                                the batch that has no tuned tile size yet (on the first state of
                                that size with its circuit; the batch run resets the states) */
#define QV_PLAN_TENSOR 8     /* fused mode, complex64, tiles of 2^11 or 2^12: every stage of a
                                pass multiplies its gates into one 16x16 complex matrix and
                                applies it on the tensor cores (tcgen05, TF32 operands split
                                in three products for FP32 accuracy) */

typedef struct {
    int32_t mode;        /* qv_mode */
    int32_t tile_bits;   /* fused: log2 of the tile size in amplitudes (0 = default) */
    int32_t flags;       /* QV_PLAN_* bits */
    int32_t window_bits; /* fused, state in host memory (QV_ALLOC_HOST): log2 of the amplitudes of
                            the device windows it is staged through; below n the state streams
                            through two windows in chunks (the split schedule of qv_dist_plan).
                            0 = default: the whole state as one window when it takes at most half
                            of the free device memory, else passes in place */
    int32_t reserved[4]; /* set to 0 */
} qv_plan_opts;

/* One Pauli string times a real coefficient: X on the qubits set only in
 * xmask, Z on those set only in zmask, Y on those set in both. */
typedef struct {
    double   coeff;
    uint64_t xmask;
    uint64_t zmask;
} qv_pauli_term;

/* ------------------------------------------------------------------------ */
/* State lifetime (Sec. II, Eq. 1-2)                                          */
/* ------------------------------------------------------------------------ */

/* Allocates a 2^n-amplitude state of dtype dt on the current CUDA device
 * (1 <= n <= 40) and sets it to |0...0> (amplitude 0 = 1) on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream). The library owns the
 * device buffer. QV_ERR_OOM if it does not fit. */
qv_status qv_create(int n, qv_dtype dt, void *cuda_stream, qv_state **out);

/* qv_create with placement flags. QV_ALLOC_HOST puts the amplitudes in
 * page-locked host memory mapped into the device's address space: the paper
 * keeps states larger than fast memory in a slower tier (Sec. III-B/C, the
 * disk and its RAM cache); here that tier is the host memory behind
 * NVLink-C2C, and every kernel reads and writes it there. QV_ERR_OOM when
 * the allocation would take more than 3/4 of the host's free memory. */
#define QV_ALLOC_HOST 1
qv_status qv_create_ex(int n, qv_dtype dt, void *cuda_stream, int32_t flags, qv_state **out);

/* Wraps a caller-owned device buffer of 2^n amplitudes (interleaved re, im;
 * 16-byte aligned) without copying or initialising it. The buffer must stay
 * valid until qv_destroy; the library never frees it. */
qv_status qv_wrap(void *dev_ptr, int n, qv_dtype dt, void *cuda_stream, qv_state **out);

/* Frees the handle (and the device buffer if the library allocated it) after
 * synchronising its stream. NULL is accepted. */
qv_status qv_destroy(qv_state *s);

/* Changes the stream later calls enqueue on. */
qv_status qv_set_stream(qv_state *s, void *cuda_stream);

/* Reports n, dtype and the device pointer of the amplitudes (any may be NULL). */
qv_status qv_info(const qv_state *s, int *n, qv_dtype *dt, void **dev_ptr);

/* Sets the state to the basis state |j> (amplitude j = 1, all others 0). */
qv_status qv_set_basis(qv_state *s, uint64_t j);

/* Copies the whole state to / from host memory. `bytes` must equal
 * 2^n * (8 or 16). qv_get_state synchronises. */
qv_status qv_get_state(qv_state *s, void *host, size_t bytes);
qv_status qv_set_state(qv_state *s, const void *host, size_t bytes);

/* ------------------------------------------------------------------------ */
/* Gates                                                                      */
/* ------------------------------------------------------------------------ */

/* Eq. 5: (a_i, a_{i^2^t}) <- U (a_i, a_{i^2^t}) for every i with bit t = 0,
 * one pass over the state. U is row-major (U[0] = U00, U[1] = U01, U[2] = U10,
 * U[3] = U11), given in double precision and rounded once to the state's
 * precision. Any 2x2 matrix is accepted (unitarity is not checked); non-finite
 * entries give QV_ERR_ARG. */
qv_status qv_apply_1q(qv_state *s, int target, const qv_c128 U[4]);

/* Controlled U: Eq. 5 restricted to the pairs whose bit `ctrl` is 1 (the paper
 * names CNOT in Sec. II without printing a rule; this is |0><0| (x) I +
 * |1><1| (x) U). ctrl == target gives QV_ERR_ARG. */
qv_status qv_apply_controlled(qv_state *s, int ctrl, int target, const qv_c128 U[4]);

/* Applies gates g[0..ng-1] in order (Eq. 3 per gate). The gate list is copied
 * and validated first; on QV_ERR_ARG nothing has been applied. `opts` may be
 * NULL (QV_MODE_AUTO). In fused mode the paper's sliding window and block
 * storage (Sec. III-B/C, Eq. 6-8) become 2^k-amplitude tiles held on chip, and
 * consecutive gates whose pairs fall inside a tile share one pass over HBM
 * (Sec. III-E). The result equals per-gate application up to rounding order. */
qv_status qv_apply_circuit(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts);

/* Plans g[0..ng) for an n-qubit state of dtype dt as qv_apply_circuit would in
 * QV_MODE_FUSED, without touching a GPU, and reports out[0] = HBM passes,
 * out[1] = on-chip stages, out[2] = shared-memory transposes, out[3] = on-chip
 * operations. Host only. */
qv_status qv_plan_info(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t out[4]);

/* The CUDA source that the compiled fused engine generates for pass `pass`
 * (0-based) of the plan qv_plan_info describes, for inspection: *len = its
 * length; when cap > 0, up to cap - 1 bytes and a terminating NUL are written
 * to buf. QV_ERR_ARG for a pass outside the plan or with QV_PLAN_INTERPRET
 * (the interpreting engine compiles nothing). Host only. */
qv_status qv_plan_source(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t pass,
                         char *buf, size_t cap, size_t *len);

/* Compiles every pass of that plan with NVRTC for sm_103a without a GPU or a
 * driver, as the compiled engine would before launching them: out[0] = passes
 * compiled, out[1] = generated source bytes, out[2] = the most registers a
 * thread of any pass uses (ptxas report), out[3] = passes whose registers
 * spill to local memory. QV_ERR_UNSUPPORTED when NVRTC cannot be loaded,
 * QV_ERR_CUDA (with the start of the compiler log in qv_last_error) when a
 * pass does not compile. Host only. */
qv_status qv_plan_compile(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int64_t out[4]);

/* One stage of a tensor-core plan (QV_PLAN_TENSOR), for inspection. A pass
 * loads every tile of 2^k amplitudes; tile position p is physical qubit
 * tile_qubit[p]. In a stage, thread t of a tile holds the 16 amplitudes whose
 * tile positions are deposit(t; in_thr) | deposit(r; in_reg), r = 0..15 (bit j
 * of r at position in_reg[j], bit b of t at in_thr[b]); the stage replaces that
 * vector by M r-vector (M row-major 16x16, variant 1 where the physical qubit
 * ext is 1 in the tile's index, else variant 0) and writes it back through the
 * positions of out_reg / out_thr (which differ from the input positions only
 * after SWAP gates, exchanges of position labels). A stage without a matrix
 * only changes the layout. */
typedef struct {
    int32_t k;             /* tile bits */
    int32_t nstages;       /* stages of this pass */
    int32_t tile_qubit[12];
    int32_t in_reg[4];
    int32_t in_thr[8];     /* k - 4 entries used */
    int32_t out_reg[4];
    int32_t out_thr[8];
    int32_t has_matrix;
    int32_t ext;           /* -1: one matrix for every tile */
    qv_c128 m[2][256];
} qv_tc_stage;

/* Stage `stage` of pass `pass` of the tensor-core plan of g[0..ng) (opts must
 * carry QV_PLAN_TENSOR; complex64). QV_ERR_ARG for a pass or stage outside the
 * plan. Host only: the planner's output, not an execution of it. */
qv_status qv_plan_tc_stage(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t pass,
                           int32_t stage, qv_tc_stage *out);

/* Algorithmic cost of the fused plan of g[0..ng) (host only, as qv_plan_info):
 * out[0] = HBM bytes, one read and one write of the state per pass;
 * out[1] = floating-point operations: per amplitude and on-chip operation,
 * 14 for a 2x2 complex matrix (Eq. 5: 4 complex products and 2 sums per
 * pair), 6 for a diagonal one, 0 for X, half of that when the operation is
 * controlled (only the amplitudes with the control set change). The
 * roofline of a fused pass is the larger of bytes / HBM bandwidth and
 * operations / arithmetic peak. */
qv_status qv_plan_cost(int n, qv_dtype dt, const qv_gate *g, size_t ng, const qv_plan_opts *opts, double out[2]);

/* The tile size (log2 amplitudes) fused mode uses for an n-qubit state of
 * dtype dt when qv_plan_opts.tile_bits is 0: the autotuner's choice for
 * (n, dt, engine) if it ran in this process, else a measured default
 * (2^11 for the compiled complex64 pass, 2^12 otherwise), at most n. A state
 * created with QV_ALLOC_HOST always takes 2^12 (at most n): its passes are bound
 * by the host link, so the fewest passes win. Host only. */
int32_t qv_default_tile_bits(int n, qv_dtype dt, int32_t flags);

/* Autotuner: runs g[0..ng) in fused mode with every supported tile size
 * (2^10 .. 2^12 amplitudes, at most 2^n) and, for the compiled complex64
 * engine, every schedule variant (FP32 passes with 4x4 pair operations,
 * without them, and tensor-core stages, whose register sets and transposes
 * differ), times each with CUDA events after a warm-up run, and remembers the
 * fastest for this (n, dtype, engine) -- later fused calls, batches and plans
 * with tile_bits = 0 and no engine flags use it. opts selects the engine
 * (QV_PLAN_INTERPRET) and fusion flags; *best_tile_bits gets the winning tile
 * size. Overwrites the state (it is |0...0> on return). Synchronises. */
qv_status qv_autotune(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t *best_tile_bits);

/* The same; out[0] = the winning tile bits, out[1] = the winning schedule
 * variant as plan flags (0, QV_PLAN_NO_PAIRS or QV_PLAN_TENSOR). Not in the
 * paper. */
qv_status qv_autotune_ex(qv_state *s, const qv_gate *g, size_t ng, const qv_plan_opts *opts, int32_t out[2]);

/* Reorders qubits: bit q of every amplitude index moves to bit perm[q]
 * (out[pi(i)] = in[i]). perm is a permutation of 0..n-1. In place. */
qv_status qv_permute_qubits(qv_state *s, const int32_t *perm);

/* ------------------------------------------------------------------------ */
/* Reductions (not in the paper). Squares and short runs are summed in the   */
/* state's precision with error-free (two-sum) compensation; everything       */
/* beyond a thread is summed in FP64 with Neumaier compensation.             */
/* ------------------------------------------------------------------------ */

/* <psi|psi>. Synchronises. */
qv_status qv_norm2(qv_state *s, double *out);

/* <Z_q> = sum_i |a_i|^2 (1 - 2 bit_q(i)) for q = 0..n-1 into per_qubit[n]
 * (may be NULL) and sum_q weights[q] <Z_q> into *total (weights NULL = all 1;
 * total may be NULL). Synchronises. */
qv_status qv_expect_z(qv_state *s, const double *weights, double *per_qubit, double *total);

/* <psi|H|psi> for H = sum_t terms[t].coeff * P_t. Synchronises. */
qv_status qv_expect_pauli(qv_state *s, const qv_pauli_term *terms, size_t nt, double *out);

/* out = H |psi> for H = sum_t terms[t].coeff * P_t; `out` is another state of
 * the same n, dtype and stream (its previous contents are overwritten). */
qv_status qv_apply_pauli(qv_state *s, const qv_pauli_term *terms, size_t nt, qv_state *out);

/* ------------------------------------------------------------------------ */
/* Gradients (not in the paper)                                               */
/* ------------------------------------------------------------------------ */

/* Gradient of E = <psi|H|psi>, psi = U_L ... U_1 psi_0, with respect to the
 * trainable angles (qv_gate.param) by the adjoint method (Jones and Gacon,
 * arXiv:2009.02823): a forward pass (fused), lambda = H psi, then a reverse
 * sweep that per gate un-computes psi <- U^dagger psi, adds 2 Re <lambda|
 * dU/dtheta psi> for each trainable angle and updates lambda <- U^dagger
 * lambda, in one pass over both buffers; no intermediate state is stored.
 * psi_0 is the handle's current state; when the call returns the handle
 * holds psi_0 again (up to rounding). grad_out[p] sums the derivatives of
 * every angle with param == p (0 <= p < nparams); trainable angles are
 * theta[0] of RX, RY, RZ, P and all three of U3. *expval_out (may be NULL)
 * gets E. Needs one extra state buffer on the device. Synchronises. */
qv_status qv_adjoint_grad(qv_state *s, const qv_gate *g, size_t ng, const qv_pauli_term *H, size_t nt,
                          size_t nparams, double *grad_out, double *expval_out);

/* Reverse sweeps of qv_adjoint_grad_ex. QV_SWEEP_PER_GATE: one pass over psi
 * and lambda per gate. QV_SWEEP_TILES (n >= 10): a pass loads 2^k-amplitude
 * tiles of both buffers into shared memory, runs consecutive reverse-order
 * gates whose targets lie in the tile (the blocking of Sec. III-B/C, Eq. 6-8,
 * applied to both buffers) and accumulates their derivatives, then stores
 * both tiles once. QV_SWEEP_COMPILED (complex64, n >= 10, NVRTC present;
 * otherwise as QV_SWEEP_TILES): the same passes planned and compiled like the
 * forward passes, both tiles held in registers. QV_SWEEP_AUTO picks the
 * compiled sweep where it applies, else the tiled one. All give the same
 * result up to rounding order. */
#define QV_SWEEP_AUTO 0
#define QV_SWEEP_PER_GATE 1
#define QV_SWEEP_TILES 2
#define QV_SWEEP_COMPILED 3

/* qv_adjoint_grad with a choice of reverse sweep (QV_SWEEP_*). */
qv_status qv_adjoint_grad_ex(qv_state *s, const qv_gate *g, size_t ng, const qv_pauli_term *H, size_t nt,
                             size_t nparams, double *grad_out, double *expval_out, int32_t sweep_mode);

/* ------------------------------------------------------------------------ */
/* Measurement and partial amplitudes (not in the paper; Sec. III-E notes     */
/* that its strategies carry over to partial-amplitude simulation)            */
/* ------------------------------------------------------------------------ */

/* Samples computational-basis outcomes from p_i = |a_i|^2 / sum |a|^2 by
 * inverse CDF: out[k] = the smallest i with p_0 + ... + p_i > u[k]. The
 * uniforms u[k] in [0, 1) are inputs (the caller's random numbers); a target
 * that rounds to the total takes the last outcome of nonzero probability.
 * Probabilities and sums are FP64. One read of the state plus one read of
 * each segment of 4096 amplitudes that holds a shot. Synchronises. */
qv_status qv_sample(qv_state *s, const double *u, size_t nshots, uint64_t *out);

/* Copies amplitudes idx[0..k) to host (interleaved re, im in the state's
 * precision: 8 or 16 bytes each). Synchronises. */
qv_status qv_get_amplitudes(qv_state *s, const uint64_t *idx, size_t k, void *host);

/* Distance of the state to the closed form of the quantum Fourier transform
 * of the basis state |j> (the paper's workloads have no QFT; this checks large
 * runs on the GPU): *dist = sqrt( sum_k |a_k - exp(2 pi i (j k mod 2^n) / 2^n)
 * / 2^(n/2)|^2 ). The phase index is exact integer arithmetic; the reference
 * amplitudes come from FP64 sincospi tables; sums are FP64. Synchronises. */
qv_status qv_verify_qft(qv_state *s, uint64_t j, double *dist);

/* ||psi_a - psi_b||_2 in FP64 for two states of the same n (either dtype;
 * e.g. a complex64 run against its complex128 rerun). Runs on a's stream
 * after synchronising b's. Synchronises. */
qv_status qv_distance(qv_state *a, qv_state *b, double *out);

/* Allocation-free Z sums (the paper has no counterpart; this exists for
 * callers that cannot allocate device memory). Some callers cannot call
 * cudaMalloc at the point where they need a result: code recording a CUDA
 * graph, where a cudaMalloc/cudaFree would not be captured and may
 * synchronise the device; latency-critical loops, where those calls block
 * and can serialise unrelated streams; processes whose device memory is
 * carved out by a pool or quota they do not own. This call needs no handle
 * and allocates nothing: it runs the same kernels as qv_expect_z on a
 * caller-owned state and writes, on the device,
 *     dev_out[0]     = sum_i |a_i|^2
 *     dev_out[1 + q] = sum over i with bit q set of |a_i|^2   (q < n)
 * (so <Z_q> = dev_out[0] - 2 dev_out[1 + q]). dev_amp: 2^n amplitudes of dtype
 * dt, 16-byte aligned; dev_out: n + 1 doubles of device memory, 8-byte
 * aligned, owned by the caller. Work is enqueued on cuda_stream; the call
 * returns without synchronising and without any host<->device copy.
 * Limit: 1 <= n <= 30 (QV_ERR_ARG beyond). The partial sums of states with
 * n >= 14 live in one fixed 7,864,320-byte device array inside the library,
 * present on every device that loads it until the process exits. The first
 * call on a device looks that array's address up (cudaGetSymbolAddress, which
 * may load the library's device code); make that first call before any stream
 * capture. The address is kept for the life of the process: after a
 * cudaDeviceReset of that device it is stale, so do not call this entry point
 * on a device that was reset. dev_amp, dev_out and the stream must belong to
 * the current device (QV_ERR_ARG otherwise). Every call shares the array, so
 * calls that can overlap on the GPU (different streams without ordering) race
 * and give wrong sums; calls on one stream are safe. Nothing in the array needs
 * to start at zero: every call overwrites the part it reads. */
qv_status qv_zsums_noalloc(const void *dev_amp, int n, qv_dtype dt, void *cuda_stream, double *dev_out);

/* ------------------------------------------------------------------------ */
/* Instrumentation (not in the paper)                                         */
/* ------------------------------------------------------------------------ */

/* Kernel classes the library launches. */
typedef enum {
    QV_K_BASIS = 0,    /* state set-up */
    QV_K_PAIR = 1,     /* per-gate pair update (Eq. 5), plain and controlled */
    QV_K_DIAG = 2,     /* per-gate diagonal gate */
    QV_K_SWAP = 3,     /* per-gate qubit swap */
    QV_K_FUSED = 4,    /* tiled multi-gate pass */
    QV_K_REDUCE = 5,   /* norm / Z reductions */
    QV_K_PAULI = 6,    /* Pauli-string expectation and H|psi> */
    QV_K_ADJOINT = 7,  /* adjoint reverse sweep */
    QV_K_BATCH = 8,    /* batched persistent launch */
    QV_K_VERIFY = 9,   /* closed-form verification */
    QV_K_COUNT = 10
} qv_kernel_class;

typedef struct {
    uint64_t launches;   /* kernels of this class launched since the last reset */
    double ms;           /* summed device time (CUDA events around each launch) when timing is on */
    double bytes;        /* algorithmic HBM bytes: one read and one write of every amplitude the
                            launches had to change, one read of those they only read */
} qv_kernel_stat;

/* Resets the handle's counters; with timing != 0 every later launch is
 * bracketed by CUDA events on the handle's stream (small overhead per launch). */
qv_status qv_profile(qv_state *s, int timing);

/* Synchronises, then writes min(count, QV_K_COUNT) per-class stats. */
qv_status qv_profile_read(qv_state *s, qv_kernel_stat *out, int count);

/* Bytes the library copied host->device and device->host since the last
 * qv_profile reset (gate programs, results; not qv_get/set_state). */
qv_status qv_transfer_bytes(qv_state *s, uint64_t *h2d, uint64_t *d2h);

/* ------------------------------------------------------------------------ */
/* Batches (not in the paper)                                                 */
/* ------------------------------------------------------------------------ */

typedef struct qv_batch qv_batch;   /* opaque */

/* One member of a batch: a state and the circuit to run on it. */
typedef struct {
    qv_state *state;
    const qv_gate *gates;
    size_t ngates;
} qv_batch_item;

/* Plans every circuit (fused passes; tile size per qubit count from the
 * autotuner unless opts->tile_bits is set; all states must have the same
 * dtype, n >= 10, and be distinct), uploads the pass programs, and captures
 * one CUDA graph that sets every state to |0...0>, runs all circuits in one
 * persistent launch per tile size -- CTAs claim (circuit, pass, tile chunk)
 * work items from an atomic counter in round order and wait (bounded) on a
 * per-pass completion counter before a circuit's next pass -- and, when nt > 0,
 * reduces <H> for every state. The gate lists are copied; the states must
 * outlive the batch. */
qv_status qv_batch_create(const qv_batch_item *items, size_t count, const qv_pauli_term *H, size_t nt,
                          const qv_plan_opts *opts, qv_batch **out);

/* Replays the batch's graph on its own stream (after synchronising the
 * states' streams) and waits for it. expvals[count] (may be NULL) gets <H>
 * per state when the batch has a Hamiltonian. QV_ERR_TIMEOUT if a
 * dependency wait in the persistent launch gave up. */
qv_status qv_batch_run(qv_batch *b, double *expvals);

/* How a batch runs, for inspection (host only): per persistent launch group, 6
 * values -- tile bits, circuits, qubits of its first circuit, 1 for the
 * compiled kernel (circuits of one plan structure), 0 for the interpreting
 * one, 2 for a circuit large enough to fill the GPU alone (at least 2^12
 * tiles per pass: its own compiled fused passes, in the same graph), then the
 * circuits whose passes of one round are queued together (compiled kernel; 0
 * otherwise) and tiles per work item (0 for a circuit of its own). Writes at most cap groups to
 * out; returns the number of groups, or -1 for a NULL batch. Not in the paper. */
int32_t qv_batch_info(const qv_batch *b, int32_t *out, size_t cap);

qv_status qv_batch_destroy(qv_batch *b);

/* One-shot batch: qv_batch_create, one qv_batch_run and qv_batch_destroy in a
 * single call, with the same arguments and rules (expvals[count] may be NULL).
 * For repeated runs of the same circuits keep a qv_batch instead: creating it
 * plans, compiles and captures the graph. */
qv_status qv_apply_batch(const qv_batch_item *items, size_t count, const qv_pauli_term *H, size_t nt,
                         const qv_plan_opts *opts, double *expvals);

/* Waits for the handle's stream and reports device-side failures: kernels
 * whose waits are bounded (the compiled fused passes' tile copies, the batch
 * dependencies) write a status word instead of hanging; this call (and every
 * call that synchronises) returns QV_ERR_TIMEOUT once when it is set. */
qv_status qv_sync(qv_state *s);

/* Self-test of the bounded device wait (the one the batch kernel uses for
 * its pass dependencies): one thread waits on a zeroed counter that nothing
 * increments and gives up after `limit` polls (128 ns apart; limit <= 2^24).
 * Returns QV_ERR_TIMEOUT on a healthy device, with the handle and its stream
 * still usable; QV_ERR_ARG for a larger limit. */
qv_status qv_wait_selftest(qv_state *s, uint32_t limit);

/* Message describing the last failure on the calling thread ("" if none). */
const char *qv_last_error(void);

/* ------------------------------------------------------------------------ */
/* A state split over 2^g ranks (Sec. III-D, Eq. 9): schedule, host only.     */
/* ------------------------------------------------------------------------ */

/* Rank r of C = 2^g holds amplitudes [r 2^n / C, (r + 1) 2^n / C - 1] (Eq. 9):
 * the top g physical qubits name the rank ("global"), the low L = n - g the
 * position in its shard ("local"). qv_dist_plan turns a circuit into this
 * rank's steps:
 *   QV_DIST_LOCAL     run local_gates[gate_begin, gate_end) on the shard (an
 *                     L-qubit state; qubit indices are local physical ones);
 *   QV_DIST_EXCHANGE  trade one half of the shard with rank `peer` = rank XOR
 *                     2^global_bit: the upper half (local bit L - 1 = 1) when
 *                     send_upper, else the lower half; the partner's half
 *                     replaces it at the same offsets.
 * An exchange swaps the global qubit with local qubit L - 1 (Sec. III-D,
 * Fig. 4: pairs (i, i XOR 2^t) that cross ranks become local). Controls and
 * diagonal gates on global qubits need no exchange (each rank knows its own
 * bits) and SWAP gates only relabel qubits, so final_perm[q] (n entries) is
 * the physical qubit holding logical qubit q at the end. */
typedef enum { QV_DIST_LOCAL = 0, QV_DIST_EXCHANGE = 1 } qv_dist_kind;
typedef struct {
    int32_t  kind;        /* qv_dist_kind */
    int32_t  global_bit;  /* exchange: j, the rank bit of the global qubit */
    int32_t  peer;        /* exchange: rank XOR 2^j */
    int32_t  send_upper;  /* exchange: 1 = the half with local bit L - 1 = 1 */
    uint64_t gate_begin;  /* local: first gate of the step in local_gates */
    uint64_t gate_end;    /* local: one past the last */
} qv_dist_step;

/* qv_dist_plan flags: QV_DIST_RESTORE appends the steps that bring every
 * logical qubit back to its own physical position (final_perm = identity). */
#define QV_DIST_RESTORE 1

/* Schedule of g[0..ng) on rank `rank` of 2^global_bits ranks (1 <= global_bits
 * < n, 0 <= rank < 2^global_bits). With steps or local_gates NULL only the
 * counts *nsteps and *ngates are written; otherwise steps_cap and gates_cap
 * must hold them (QV_ERR_ARG if not). final_perm (n int32) may be NULL. Every
 * rank calls it with the same gates and gets the same sequence of step kinds
 * and exchange partners in matching order. Not in the paper beyond Eq. 9 and
 * Fig. 4: the exchange rule is this library's reading of Sec. III-D. */
qv_status qv_dist_plan(int n, int global_bits, int rank, const qv_gate *g, size_t ng, int32_t flags,
                       qv_dist_step *steps, size_t steps_cap, size_t *nsteps, qv_gate *local_gates, size_t gates_cap,
                       size_t *ngates, int32_t *final_perm);

#ifdef __cplusplus
}
#endif

#endif /* QV_H */
