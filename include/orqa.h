/*
 * orqa.h -- C ABI of the GB300 sparse Pauli dynamics library (liborqa.so).
 *
 * The library propagates a real Pauli sum O = sum_I O_I sigma_I (Eq. define_O
 * of arXiv 2506.13241) through rotation gates exp(-i theta/2 sigma_J) in the
 * Heisenberg picture (Eq. update_rule), merging duplicate strings and
 * truncating small coefficients after every non-Clifford gate (Algorithm 1),
 * and evaluates <0|O|0> (Eq. magnetization).  Every step runs in CUDA kernels
 * on the caller's stream; the host code only orchestrates.
 *
 * Pauli strings.  A string on n <= 128 qubits is a pair of bit planes
 * (x, z) of W = (n <= 64 ? 1 : 2) little-endian uint64 words each; bit q of
 * word q/64 belongs to qubit q.  (x_q, z_q) = (0,0) identity, (1,0) sigma_x,
 * (1,1) sigma_y, (0,1) sigma_z.  This is a linear re-coding of the paper's
 * two-bit local index (Sec. II: 00 = id, 01 = x, 10 = y, 11 = z):
 * z = high bit, x = high xor low; it keeps the XOR product of Eq. orqaproduct.
 * Host arrays of strings are string-major: word w of string i is at
 * x[i * W + w].
 *
 * Memory.  The library allocates no device memory.  The caller passes one
 * device buffer of at least orqa_workspace_bytes(n_qubits, capacity) bytes
 * (for example a torch uint8 tensor) and keeps it alive until orqa_destroy.
 * Host-side bookkeeping (the context) is allocated with malloc.
 *
 * Errors.  Every call returns an orqa_status; on failure the context keeps a
 * message (orqa_last_error) and the operator held before the call is left
 * unchanged (all layer work goes to scratch buffers that are committed only
 * on success).
 *
 * Synchronisation.  Calls enqueue work on the context's stream.  Calls that
 * return a host value (a live count, an expectation value, an export) wait
 * for the stream.
 */
#ifndef ORQA_H
#define ORQA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ORQA_OK = 0,
    ORQA_EINVAL = 1,     /* bad argument: null pointer, size, qubit index, gate kind */
    ORQA_ENOMEM = 2,     /* workspace smaller than orqa_workspace_bytes() */
    ORQA_ECAPACITY = 3,  /* a result would exceed the capacity; operator unchanged */
    ORQA_ECUDA = 4,      /* a CUDA runtime call failed (message holds its text) */
    ORQA_ETIMEOUT = 5,   /* a bounded device-side wait ran out; operator unchanged */
    ORQA_ESTATE = 6      /* call not valid in the current state */
} orqa_status;

/* Gate kinds.  Each gate is exp(-i theta/2 sigma_J) (App. A).
 *   ORQA_RX : sigma_J = sigma_x on qubit q0 (any theta).
 *   ORQA_RZZ: sigma_J = sigma_z on q0 times sigma_z on q1 (q0 != q1); theta
 *             must be a multiple of pi/2 (Clifford), the only case of the
 *             kicked Ising circuit (theta_zz = -pi/2, Eq. eq:u).
 * An angle within 1e-12 of a multiple of pi/2 is applied as an exact
 * Clifford rotation: (cos, sin) in {0, +1, -1}. */
enum { ORQA_RX = 1, ORQA_RZZ = 2 };

typedef struct {
    int32_t kind;   /* ORQA_RX or ORQA_RZZ */
    int32_t q0;     /* qubit (0-based) */
    int32_t q1;     /* second qubit of ORQA_RZZ, ignored otherwise */
    int32_t pad;    /* must be 0 */
    double theta;   /* rotation angle */
} orqa_gate;

/* orqa_config.flags */
enum {
    ORQA_FLAG_PROFILE = 1,   /* time every kernel launch with CUDA events on the
                                context's stream (see orqa_profile) */
    ORQA_FLAG_RELATIVE = 2,  /* relative truncation (Eq. truncation1): the
                                `delta` of apply_layer / merge_truncate is eps0
                                and a string is dropped when c == 0 or
                                |c| <= eps0 * max|c|, the max taken over the
                                operator after each gate's updates */
    ORQA_FLAG_FP32 = 4       /* precision form: coefficients stored and
                                multiplied in FP32, with cos and sin carried
                                as float pairs hi + lo; two-member pair
                                updates (the merges of Algorithm 1) evaluated
                                with the compensated Dot2 scheme; duplicate
                                merging of input and <0|O|0> accumulate in
                                FP64.  The ABI still takes and returns FP64
                                arrays. */
};

/* Most problems one batched context may hold. */
#define ORQA_MAX_PROBLEMS 4096

typedef struct {
    int32_t n_qubits;        /* 1..128 */
    int32_t flags;           /* ORQA_FLAG_PROFILE | ORQA_FLAG_RELATIVE | ORQA_FLAG_FP32, or 0 */
    int64_t capacity;        /* most strings any intermediate set may hold (all problems together) */
    void* workspace;         /* device buffer, 256-byte aligned */
    uint64_t workspace_bytes;
    void* stream;            /* cudaStream_t, or NULL for the default stream */
    int32_t n_problems;      /* 0 or 1: one operator.  2..ORQA_MAX_PROBLEMS: a batched
                                context holding that many independent operators
                                (see "Batched contexts" below); not with
                                ORQA_FLAG_RELATIVE */
    int32_t reserved;        /* must be 0 */
} orqa_config;

typedef struct {
    int64_t n_strings;        /* |O|: live strings */
    int64_t last_layer_in;    /* strings entering the last apply_layer */
    int64_t last_layer_peak;  /* largest intermediate set inside it */
    int64_t string_gate_updates; /* sum over its gates of |O| before the gate */
    int64_t branch_events;    /* anticommuting (string, gate) pairs in it */
    int64_t dropped;          /* strings removed by truncation in it */
    int64_t pair_updates_one; /* (pair, gate) updates with one member present */
    int64_t pair_updates_two; /* (pair, gate) updates with both members present */
    int32_t chunk_passes;     /* device passes its rotation layer took */
    int32_t pad;
    double sum_sq;            /* sum of c^2 over the live strings (FP64, fixed summation
                                 order): 1 for a normalised Pauli-string observable, kept by
                                 every rotation (Eq. update_rule is an orthogonal 2x2 map on
                                 each pair) and lowered only by truncation */
    double max_abs;           /* max |c| over the live strings (exact) */
    double dropped_sum_sq;    /* sum of c^2 of the strings the last call's truncation
                                 removed (Eq. truncation1), so that sum_sq before minus
                                 sum_sq after equals it up to rounding; NaN for a call whose
                                 X layers ran without orqa_set_norm_tracking */
} orqa_stats_t;

/* Per-kernel launch profile (ORQA_FLAG_PROFILE).
 *   bytes: the kernel's algorithmic DRAM traffic in this implementation's
 *     pass structure: the bytes its inputs and outputs must move at least
 *     once (not counting hash-probe misses or cache effects).
 *   floor_bytes: the kernel's share of the method's own traffic floor, the
 *     same for any implementation: per X gate 8 bytes of z per string tested
 *     and, per anticommuting string, its record read, the child record and
 *     the parent's coefficient written and a merge that meets and writes
 *     both once (4R + sizeof(c) bytes per branch event, R the bytes of one
 *     string, charged to the unit kernel, which does all branching); per ZZ
 *     layer R read plus the z planes and c written per string; per
 *     expectation the x planes and c read.  0 for kernels without one. */
typedef struct {
    char name[32];
    int64_t launches;
    double ms;               /* summed CUDA-event durations */
    double bytes;            /* summed algorithmic bytes (pass structure) */
    double floor_bytes;      /* summed floor bytes (method) */
} orqa_kernel_profile;

typedef struct orqa_ctx orqa_ctx;

/* Bytes of device workspace needed for n_qubits and capacity (one
 * operator), or 0 for invalid sizes. */
uint64_t orqa_workspace_bytes(int32_t n_qubits, int64_t capacity);

/* The same for a context of n_problems operators (orqa_config.n_problems). */
uint64_t orqa_workspace_bytes_batch(int32_t n_qubits, int64_t capacity, int32_t n_problems);

/* Creates a context holding the empty operator.  The workspace and the
 * stream stay owned by the caller.  EINVAL on bad sizes, ENOMEM if the
 * workspace is too small. */
orqa_status orqa_create(const orqa_config* cfg, orqa_ctx** out);

/* Replaces the operator by the n strings in the HOST arrays x, z (n*W words
 * each) and c (n doubles); the arrays are copied.  Duplicate strings are
 * summed and exact zeros dropped (the insert-or-add of Algorithm 1).
 * ECAPACITY if n > capacity. */
orqa_status orqa_set_operator(orqa_ctx* ctx, int64_t n, const uint64_t* x,
                              const uint64_t* z, const double* c);

/* As orqa_set_operator, but x, z, c are DEVICE arrays in the same
 * string-major layout, read on the context's stream. */
orqa_status orqa_set_operator_device(orqa_ctx* ctx, int64_t n, const uint64_t* x,
                                     const uint64_t* z, const double* c);

/* Applies n_gates mutually commuting gates in array order (Eq. update_rule,
 * one gate at a time as in Algorithm 1).  All gates must be of one kind.
 *   ORQA_RZZ (Clifford): each string maps to exactly one string with an
 *     exact sign; nothing merges and |c| is unchanged.  Strings with
 *     |c| < delta are then dropped.  The library may hold such a layer
 *     back and apply it inside the next ORQA_RX layer's first pass over the
 *     operator, which saves a pass; every other call that reads or changes
 *     the operator applies it first, so no result differs.
 *   ORQA_RX: after every gate, duplicates are merged and strings with
 *     c == 0 or |c| < delta are dropped (the truncation loop of Algorithm 1
 *     with the absolute threshold); the result is the one of that per-gate
 *     schedule, bit for bit.
 * With ORQA_FLAG_RELATIVE, delta is eps0 and the truncation after every gate
 * is the relative one (an X layer is then applied one gate at a time, since
 * the threshold depends on the whole operator after each gate).
 * n_live_out (may be NULL) receives |O| after the layer.  ECAPACITY if an
 * intermediate set would exceed the capacity (operator unchanged). */
orqa_status orqa_apply_layer(orqa_ctx* ctx, const orqa_gate* gates, int32_t n_gates,
                             double delta, int64_t* n_live_out);

/* Applies one rotation exp(-i theta/2 sigma_J) about a general Pauli string
 * J given as HOST planes xj, zj (W words each, the string encoding above;
 * not the identity, no qubit >= n_qubits), then merges duplicates and drops
 * c == 0 and |c| < delta (relative: |c| <= delta * max|c|): one gate of
 * Algorithm 1 for any sigma_J (Eq. update_rule).  A string P that
 * anticommutes with J becomes cos(theta) P plus i^(1+B(J,P)) sin(theta)
 * sigma_{J xor P}, where sigma_J sigma_P = i^B(J,P) sigma_{J xor P}.
 * Generators need not commute with each other, so this call takes one gate. */
orqa_status orqa_apply_pauli_rotation(orqa_ctx* ctx, const uint64_t* xj, const uint64_t* zj,
                                      double theta, double delta, int64_t* n_live_out);

/* Merges duplicate strings (sums their coefficients) and drops c == 0 and
 * |c| < delta (with ORQA_FLAG_RELATIVE: |c| <= delta * max|c|, the max over
 * the merged operator): the insert-or-add and truncate loops of Algorithm 1
 * applied to the whole operator.  n_live_out (may be NULL) receives |O|. */
orqa_status orqa_merge_truncate(orqa_ctx* ctx, double delta, int64_t* n_live_out);

/* <0|O|0> = sum of O_I over strings with no sigma_x / sigma_y factor
 * (x plane all zero), in FP64 (Eq. magnetization). */
orqa_status orqa_expect(orqa_ctx* ctx, double* out);

/* Copies the operator to HOST arrays (cap strings at most; x, z: cap*W
 * words, c: cap doubles) in canonical order: ascending by the 256-bit key
 * of the string, x words from the highest to the lowest, then z words
 * likewise (batched contexts: by problem index first).  The order is made
 * on the device (a radix sort in the context's free buffers; the operator
 * is not modified).  *n_out receives |O|.  ECAPACITY (nothing copied) if
 * |O| > cap. */
orqa_status orqa_export(orqa_ctx* ctx, int64_t cap, uint64_t* x, uint64_t* z, double* c,
                        int64_t* n_out);

/* Pauli-string density D_t(x) of App. D: counts of the live strings (all
 * problems of a batched context) by sign and by bin of |x| = |c| / max|c|.
 * The n_bins bins are uniform in log10|x| over [log10_lo, 0]: with
 * w = -log10_lo / n_bins, edge k is t_k = max|c| * 10^(log10_lo + k w)
 * (formed in FP64; t_n_bins = max|c|), bin k holds t_k <= |c| < t_{k+1}
 * (the last bin also |c| = max|c|), and an extra bin n_bins counts
 * |c| < t_0.  counts (HOST, 2 * (n_bins + 1) int64): counts[s * (n_bins + 1)
 * + k], s = 0 for c > 0 and 1 for c < 0.  max_abs_out (may be NULL)
 * receives max|c|.  1 <= n_bins <= 256, -300 <= log10_lo < 0.
 * Normalising counts by |O| and the bin width gives D_t. */
orqa_status orqa_histogram(orqa_ctx* ctx, int32_t n_bins, double log10_lo, int64_t* counts,
                           double* max_abs_out);

/* Counters of the operator (|O|, sum c^2, max |c|) and of the last
 * apply_layer, apply_pauli_rotation, merge_truncate or run_program call
 * (updates, branch events, dropped strings and their sum of c^2).  The
 * first call after the operator changed reduces its coefficients on the
 * device (8 bytes per string) and waits for the stream; later calls return
 * the cached values. */
orqa_status orqa_stats(orqa_ctx* ctx, orqa_stats_t* out);

/* orqa_stats without the device reduction: the counters of the last call,
 * with sum_sq and max_abs as cached (NaN if the operator changed since the
 * last orqa_stats).  For per-layer bookkeeping inside timed loops. */
orqa_status orqa_counters(orqa_ctx* ctx, orqa_stats_t* out);

/* on = 1: the X-layer kernels also add up the c^2 of every string their
 * truncation removes (orqa_stats_t.dropped_sum_sq), the bookkeeping that
 * checks sum_sq_before - sum_sq_after = dropped_sum_sq layer by layer.  It
 * costs FP64 work in the hot kernels, so it is off (0) by default; no
 * result changes with it.  Other truncations (ZZ layers, merges, relative
 * truncation) always report it. */
orqa_status orqa_set_norm_tracking(orqa_ctx* ctx, int32_t on);

/* Profile of kernel kind `index` (0 <= index < orqa_profile_count()) since
 * the last reset; zeros unless the context was created with
 * ORQA_FLAG_PROFILE.  EINVAL for an index out of range. */
int32_t orqa_profile_count(void);
orqa_status orqa_profile(orqa_ctx* ctx, int32_t index, orqa_kernel_profile* out);
orqa_status orqa_profile_reset(orqa_ctx* ctx);

/* Message of the last failed call on ctx ("" if none).  Valid until the next
 * call on ctx. */
const char* orqa_last_error(const orqa_ctx* ctx);

/* Releases the host context (the caller's workspace is not freed). */
void orqa_destroy(orqa_ctx* ctx);

/* Batched contexts.  A context created with n_problems = P > 1 holds P
 * independent operators O_0 .. O_{P-1} (for example one per observable and
 * angle of a parameter sweep) in one set of buffers: every string carries
 * its problem index, strings of different problems never merge, and each
 * kernel launch processes all problems together whatever their sizes.  The
 * plain calls apply to every problem (orqa_apply_layer with the gates'
 * own angles, orqa_merge_truncate, orqa_stats over all strings); the calls
 * below add per-problem inputs and outputs.  orqa_expect and
 * orqa_set_operator(_device) return ORQA_ESTATE / ORQA_EINVAL on a batched
 * context. */

/* Replaces all operators by the n strings of the HOST arrays x, z, c (as in
 * orqa_set_operator); problem[i] in [0, P) is the operator string i belongs
 * to.  Duplicates within one problem are summed. */
orqa_status orqa_set_operator_batch(orqa_ctx* ctx, int64_t n, const uint64_t* x,
                                    const uint64_t* z, const double* c,
                                    const int32_t* problem);

/* orqa_apply_layer with per-problem angles: theta is a HOST array of
 * P rows of n_gates angles (row p holds problem p's angle for each gate, in
 * gate order) and replaces the gates' theta.  ORQA_RX layers only (ZZ
 * layers are the same Clifford layer for every problem: use
 * orqa_apply_layer). */
orqa_status orqa_apply_layer_batch(orqa_ctx* ctx, const orqa_gate* gates, int32_t n_gates,
                                   const double* theta, double delta, int64_t* n_live_out);

/* <0|O_p|0> for every problem: out is a HOST array of P doubles (P = 1 for
 * a plain context, where it equals orqa_expect). */
orqa_status orqa_expect_batch(orqa_ctx* ctx, double* out);

/* Live strings per problem: out is a HOST array of P int64. */
orqa_status orqa_problem_sizes(orqa_ctx* ctx, int64_t* out);

/* orqa_export plus each string's problem index (problem: cap int32, may be
 * NULL; all 0 for a plain context), in the same canonical order (problem
 * index, then key). */
orqa_status orqa_export_batch(orqa_ctx* ctx, int64_t cap, uint64_t* x, uint64_t* z, double* c,
                              int32_t* problem, int64_t* n_out);

/* Captured programs.  A program is a sequence of layers repeated `repeat`
 * times, for example the two layers of one kicked-Ising Trotter step
 * repeated for t steps.  orqa_run_program applies it as ONE CUDA graph
 * launch on the context's stream: every layer, every chunk pass of an X
 * layer (a device-side loop: a conditional graph node re-runs the pass
 * while strings remain active) and every requested expectation runs on the
 * device with no host round trip.  The result is the one of the same layers
 * applied with orqa_apply_layer(_batch), bit for bit.  The graph is captured
 * on the first run and replayed while the program, delta, the tuning and the
 * operator's buffer are unchanged.  Not available with ORQA_FLAG_RELATIVE. */
typedef struct {
    const orqa_gate* gates;   /* one layer, as for orqa_apply_layer */
    int32_t n_gates;
    int32_t expect_after;     /* 1: evaluate <0|O|0> (every problem) after this layer */
    const double* theta;      /* batched ORQA_RX layers: n_problems rows of n_gates
                                 angles (as for orqa_apply_layer_batch), or NULL */
} orqa_layer_desc;

/* Runs the program.  expect_out: HOST array of n_expect_out doubles that
 * receives, in order, the P values of every expect_after layer of every
 * repetition (P = n_problems, 1 for a plain context); EINVAL if it is too
 * short or the program asks for more than 65536 values.  On an error inside
 * the graph (capacity, a bounded wait) the call returns that status, the
 * context holds the operator after the last completed layer, and the
 * values not yet computed are NaN. */
orqa_status orqa_run_program(orqa_ctx* ctx, const orqa_layer_desc* layers, int32_t n_layers,
                             int32_t repeat, double delta, double* expect_out, int64_t n_expect_out);

/* Launch parameters of the X-layer pipeline.  Every setting gives the same
 * result; they trade occupancy, scatter locality and shared-memory hash
 * load.
 *   range_target   strings per unit-kernel CTA range (tile), 128..4096
 *   sub_max        most strings one shared-memory sub-range holds, 128..256;
 *                  the shared hash table has 512 slots, so its load is at
 *                  most sub_max / 512
 *   bucket_density most strings per fine bucket on average at full capacity,
 *                  8..128 and at most sub_max / 3 (a bucket must fit one
 *                  sub-range with margin; default 80): the bucket count is
 *                  the power of two at or above capacity / bucket_density,
 *                  i.e. the number of hash bits that partition the strings
 *   grid_per_sm    CTAs per SM of the streaming kernels, 1..32 */
typedef struct {
    int32_t range_target;
    int32_t sub_max;
    int32_t bucket_density;
    int32_t grid_per_sm;
} orqa_tuning;

orqa_status orqa_get_tuning(orqa_ctx* ctx, orqa_tuning* out);
orqa_status orqa_set_tuning(orqa_ctx* ctx, const orqa_tuning* in);

/* Picks the tuning for a program by measurement: starting from the current
 * tuning, each parameter in turn is set to each of its candidate values
 * (the others held), the program is run `trials` times from the current
 * operator (restored before every run) and timed with CUDA events around
 * the graph launch, and the fastest value is kept.  The best tuning is left
 * set, *best_ms (may be NULL) receives its time, and the operator is
 * restored.  If a run fails (for example a capacity overflow under one of
 * the candidate settings), the call returns that run's status and message
 * with the starting tuning and the starting operator put back.  The
 * operator must fit the host memory of one export. */
orqa_status orqa_autotune(orqa_ctx* ctx, const orqa_layer_desc* layers, int32_t n_layers,
                          int32_t repeat, double delta, int32_t trials, orqa_tuning* best,
                          double* best_ms);

/* Sharding one operator over R ranks (one GPU each) by a hash of the z
 * plane: the multi-device partition of the ORQA method (Sec. II, the
 * partial operators O^(m) of Eq. eq:Om), with the owner map of Eq.
 * distributor taken as owner(z), a fixed 64-bit mix of the z words reduced
 * mod R.  An X rotation flips only x bits, so the strings an X layer can
 * merge share their z plane and every X layer (branching, merging,
 * truncation) runs on each rank with no data from another.  A ZZ layer maps
 * each string to exactly one string with a new z: after it each rank calls
 * orqa_shard_split, the ranks exchange the records (one all-to-all), and
 * each calls orqa_shard_append on what it received.  <0|O|0> is the sum of
 * the ranks' orqa_expect values.  Plain (not batched) contexts only. */
#define ORQA_SHARD_MAX_RANKS 512

/* owner(z) of n strings: z is a HOST array of n*W words (string-major);
 * out[i] in [0, n_ranks).  Host-only; the device uses the same function. */
orqa_status orqa_shard_owner(int32_t n_qubits, int64_t n, const uint64_t* z, int32_t n_ranks, int32_t* out);

/* Moves the strings of the operator whose owner is not `rank` to the DEVICE
 * buffer `send` (send_cap records of 2W + 1 uint64 words: the x words, the z
 * words, then the coefficient's bit pattern -- a float in the low 32 bits
 * in the FP32 form), grouped by destination rank in ascending order;
 * send_counts (HOST, n_ranks int64) receives the records per destination
 * (0 for `rank` itself).  The operator keeps its own strings.  ECAPACITY
 * (nothing moved) if more than send_cap strings leave. */
orqa_status orqa_shard_split(orqa_ctx* ctx, int32_t n_ranks, int32_t rank, int64_t send_cap, uint64_t* send,
                             int64_t* send_counts);

/* Appends n records (the format of orqa_shard_split) from the DEVICE buffer
 * recv to the operator, without merging: the caller guarantees that they
 * are distinct from each other and from the operator's strings, as the
 * strings arriving after a ZZ layer are (the layer is a bijection), and
 * that they were truncated at the same threshold as the operator.
 * ECAPACITY (nothing appended) if |O| + n exceeds the capacity. */
orqa_status orqa_shard_append(orqa_ctx* ctx, int64_t n, const uint64_t* recv);

/* Test hooks of the failure paths (not for production use).  Each makes a
 * bounded device-side condition fire without faulting or hanging the GPU,
 * so that tests can check the status it returns and that the operator held
 * before the failing call is unchanged.  value 0 restores the default.
 *   ORQA_DEBUG_SPIN_LIMIT         iterations of the merge hash table's
 *                                 bounded wait, 1..2^22 (default 2^22)
 *   ORQA_DEBUG_POISON_MERGE_TABLE 1: later merges start with every table slot
 *                                 marked as being published by another
 *                                 thread, so each insertion waits until the
 *                                 spin limit and the call returns
 *                                 ORQA_ETIMEOUT
 *   ORQA_DEBUG_MERGE_TABLE_SLOTS  most hash-table slots a merge may use (a
 *                                 power of two >= 16): more distinct strings
 *                                 than slots return ORQA_ECAPACITY
 *   ORQA_DEBUG_PASS_LIMIT         most chunk passes of an X layer, 1..32 (a
 *                                 layer needing more returns ORQA_ETIMEOUT)
 *   ORQA_DEBUG_BUCKET_SHIFT       fine bucket = hash >> shift, from the
 *                                 default up to 63 (fewer, fuller buckets:
 *                                 one above the shared-memory range size
 *                                 returns ORQA_ECAPACITY); orqa_set_tuning
 *                                 restores the default
 *   ORQA_DEBUG_NO_ZZ_FUSION       1: every ORQA_RZZ layer is applied by a
 *                                 pass of its own at once, never held back
 *                                 for the next X layer's entry split (the
 *                                 results are the same bit for bit; the
 *                                 tests compare the two) */
enum {
    ORQA_DEBUG_SPIN_LIMIT = 1,
    ORQA_DEBUG_POISON_MERGE_TABLE = 2,
    ORQA_DEBUG_MERGE_TABLE_SLOTS = 3,
    ORQA_DEBUG_PASS_LIMIT = 4,
    ORQA_DEBUG_BUCKET_SHIFT = 5,
    ORQA_DEBUG_NO_ZZ_FUSION = 6
};
orqa_status orqa_debug_set(orqa_ctx* ctx, int32_t knob, int64_t value);

/* Largest operator orqa_expect_noalloc accepts (2^27 strings). */
#define ORQA_NOALLOC_MAX_STRINGS 134217728LL

/* <0|O|0> of an operator held in caller-owned DEVICE arrays, without a
 * context and without allocating any device memory.  This entry point has
 * no counterpart in the paper; it exists for callers that cannot call
 * cudaMalloc: code embedded in a host framework whose allocator owns the
 * device memory pool, and latency-critical paths that cannot accept the
 * device-wide synchronisation an allocation may imply.
 *   x: n*W words (string-major, as in orqa_set_operator), c: n doubles, both
 *      device (or managed) memory of the current device, 8-byte aligned;
 *      out: HOST pointer receiving the sum of c over strings whose x plane is
 *      zero, in FP64.
 * The call waits for `stream` (it copies the result to the host), so it
 * cannot be used inside stream capture.
 * Scratch is a fixed file-scope device array (65537 doubles) that every GPU
 * loading the library holds until exit; the first call on a device looks up
 * that array's device address.  All calls share the array: calls whose
 * kernels overlap on the GPU race and must be serialised by the caller.
 * Returns ORQA_ECAPACITY (nothing launched) if n > ORQA_NOALLOC_MAX_STRINGS,
 * ORQA_EINVAL for bad arguments (including host or misaligned pointers,
 * checked before any launch), ORQA_ECUDA if a CUDA call fails. */
orqa_status orqa_expect_noalloc(int32_t n_qubits, int64_t n, const uint64_t* x, const double* c,
                                double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ORQA_H */
