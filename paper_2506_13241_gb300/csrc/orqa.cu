// liborqa: C ABI (include/orqa.h) and host orchestration of the kernels in
// orqa_kernels.cuh and orqa_layer.cuh.  The host side validates arguments, carves the caller's
// workspace, computes cos/sin of each gate once, launches kernels on the
// caller's stream and reads back small counters; every per-string step runs
// on the device.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "orqa.h"
#include "orqa_kernels.cuh"
#include "orqa_layer.cuh"
#include "orqa_sort.cuh"
#include "orqa_shard.cuh"

using namespace orqa;

namespace {
enum KernelKind {
    K_RZZ, K_TRUNCATE, K_SPLIT, K_SCAN, K_BUCKET_SCATTER, K_LOCAL,
    K_MERGE_ASSIGN, K_MERGE_OFFSETS, K_MERGE_SCATTER, K_MERGE_REDUCE, K_EXPECT, K_COUNT
};
const char* const KERNEL_NAMES[K_COUNT] = {
    "rzz_layer", "truncate", "rx_split", "fine_scan", "bucket_scatter", "unit_local",
    "merge_assign", "merge_offsets", "merge_scatter", "merge_reduce", "expect"};

constexpr int ROT_SLOTS_HOST = 16;  // equals ROT_SLOTS below

struct PendingLaunch {
    int kind;
    cudaEvent_t a, b;
    double bytes;
    double floor_bytes;
};
}  // namespace

struct orqa_ctx {
    int n_qubits = 0;
    int W = 1;
    int P = 1;              // problems sharing the context (batched if > 1)
    long long cap = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 1;

    StrList buf[3];
    int cur = 0;            // buffer holding the operator
    long long n = 0;        // |O|
    double clean_delta = 0; // no live coefficient is below this

    // duplicate merge (global hash table)
    int32_t* uid = nullptr;
    int32_t* rank = nullptr;
    uint64_t* unit_z = nullptr;
    uint64_t* unit_xb = nullptr;
    uint16_t* unit_pid = nullptr;
    int32_t* unit_count = nullptr;
    long long* unit_off = nullptr;
    double* sorted_c = nullptr;
    int32_t* table = nullptr;
    long long table_cap = 0;
    // X-layer passes (fine buckets)
    int n_fine = 0;
    int fshift = 0;
    uint32_t* fcount = nullptr;     // 16-bit counts, two per word
    int range_target = LB_TARGET;  // strings per unit-kernel range
    int sub_max = LB_MAX;          // most strings of one shared-memory sub-range
    int bucket_density = 80;       // strings per fine bucket at full capacity (at most)
    int n_fine_max = 0;            // fine-bucket arrays are sized for this many
    int grid_per_sm = 32;          // CTAs per SM of the streaming kernels
    // captured programs (one per starting buffer) and their device results
    cudaStream_t cap_stream = nullptr;
    cudaStream_t body_stream = nullptr;
    struct CachedProgram {
        uint64_t key;
        int start_cur;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
    };
    std::vector<CachedProgram> programs;
    double* prog_results = nullptr;
    ProgramStats* prog_stats = nullptr;
    uint32_t* foffsets = nullptr;
    long long* tile_sums = nullptr;
    int32_t* range_start = nullptr;    // first bucket of each unit-kernel range
    uint64_t* hash_active = nullptr;   // unit-key hashes of the active list
    int32_t* rank_active = nullptr;    // ranks inside their fine buckets
    void* records = nullptr;           // bucket-ordered copy of the active list
    size_t shared_bytes = 0;           // size of the layer / merge scratch region
    size_t local_smem = 0;
    Counters* ctr = nullptr;
    double* partials = nullptr;
    double* scalar = nullptr;
    // batched contexts: per-problem rotation tables, expectation partials,
    // per-problem outputs
    double2* rot64 = nullptr;      // ROT_SLOTS tables of P * MAX_QUBITS (cos, sin)
    float4* rot32 = nullptr;
    double* batch_partials = nullptr;
    double* batch_out = nullptr;   // P doubles
    unsigned long long* sizes_out = nullptr;  // P counters
    std::vector<double2> rot_host[ROT_SLOTS_HOST];  // host staging, one per table slot
    std::vector<float4> rot_host32[ROT_SLOTS_HOST];

    orqa_stats_t stats{};
    std::string err;
    // norms of the committed operator (orqa_stats), valid until it changes
    bool norms_valid = false;
    double norm_sq = 0.0, norm_max = 0.0;
    bool track_norm = false;   // orqa_set_norm_tracking
    // failure-path test hooks (orqa_debug_set)
    long long spin_limit = SPIN_LIMIT;
    bool poison_table = false;
    long long dbg_table_slots = 0;
    int pass_limit = MAX_PASSES;
    // A ZZ layer held back to be applied by the entry split of the next X
    // layer (k_rx_split<.., ZZ = true>), which saves the layer's own pass
    // over the operator.  Every other operation on the operator applies it
    // first (settle_zz).  zz_fuse = false (orqa_debug_set) applies every ZZ
    // layer at once.
    bool zz_pending = false;
    ZZGroups zz_pend{};
    bool zz_fuse = true;

    // ORQA_FLAG_PROFILE: CUDA events around every launch, resolved at the
    // next stream synchronisation.
    bool profile = false;
    bool relative = false;   // ORQA_FLAG_RELATIVE
    bool fp32 = false;       // ORQA_FLAG_FP32: coefficients stored as float
    std::vector<PendingLaunch> pending;
    std::vector<cudaEvent_t> event_pool;
    long long prof_launches[K_COUNT] = {};
    double prof_ms[K_COUNT] = {};
    double prof_bytes[K_COUNT] = {};
    double prof_floor[K_COUNT] = {};

    void drop_programs() {
        for (auto& p : programs) {
            cudaGraphExecDestroy(p.exec);
            cudaGraphDestroy(p.graph);
        }
        programs.clear();
    }

    ~orqa_ctx() {
        drop_programs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (body_stream) cudaStreamDestroy(body_stream);
        for (auto& p : pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : event_pool) cudaEventDestroy(e);
    }
};

namespace {

constexpr size_t ALIGN = 256;

// The ZZ stage of an entry split that has none (the kernel never reads it).
const ZZGroups kNoZZ{};

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

long long pow2_at_least(long long v) {
    long long p = 1024;
    while (p < v) p <<= 1;
    return p;
}

struct Layout {
    size_t str_x, str_c;  // per string buffer: x and z planes, c
    size_t str_pid;       // per string buffer: problem indices (batched contexts)
    size_t shared;        // region shared by the layer scratch and the merge scratch
    size_t total;
    long long table_cap;  // merge hash table slots
    long long n_fine;
};

// Rotation tables a batched context holds: one per distinct X layer of a
// captured program (host-driven layers use slot 0).
constexpr int ROT_SLOTS = ROT_SLOTS_HOST;
// Smallest range target the unit kernel may be tuned to (sizes range_start).
constexpr int MIN_RANGE_TARGET = 128;

// Fine buckets: about `density` strings each at full capacity, a power of
// two and a multiple of the scan tile, at most SCAN_TILE tiles.
long long fine_buckets(long long cap, int density = 16) {
    long long f = SCAN_TILE;
    while (f < cap / density && f < (long long)SCAN_TILE * SCAN_TILE) f <<= 1;
    return f;
}

// Densest bucket setting a context may be tuned to (sizes the bucket arrays).
constexpr int MIN_BUCKET_DENSITY = 8;
// Results a captured program may return (expectation values).
constexpr size_t PROGRAM_RESULTS = 65536;

// The X-layer scratch (bucket records, hashes and ranks of the active list)
// and the duplicate-merge scratch (entry tables, coefficients, hash table)
// are never live at the same time, so they share one region.
size_t layer_scratch_bytes(int W, size_t C) {
    return align_up(C * (size_t)record_bytes(W)) + align_up(C * 8) + align_up(C * 4);
}

size_t merge_scratch_bytes(int W, size_t C, long long table_cap, int P) {
    return 2 * align_up(C * 4) + 2 * align_up(C * W * 8) + (P > 1 ? align_up(C * 2) : 0) + align_up(C * 4) +
           2 * align_up(C * 8) + align_up((size_t)table_cap * 4);
}

// Offsets are computed in the same order by orqa_workspace_bytes and
// orqa_create.
Layout layout(int n_qubits, long long cap, int P) {
    Layout L{};
    const int W = n_qubits <= 64 ? 1 : 2;
    const size_t C = (size_t)cap;
    L.str_x = align_up(C * W * 8);
    L.str_c = align_up(C * 8);
    L.str_pid = P > 1 ? align_up(C * 2) : 0;
    // merge table at load factor <= 0.75; the shared region covers both uses
    L.table_cap = pow2_at_least((4 * cap + 2) / 3);
    L.shared = std::max(layer_scratch_bytes(W, C), merge_scratch_bytes(W, C, L.table_cap, P));
    L.n_fine = fine_buckets(cap, MIN_BUCKET_DENSITY);
    const size_t F = (size_t)L.n_fine;
    size_t t = 0;
    t += 3 * (2 * L.str_x + L.str_c + L.str_pid);  // three string buffers
    t += L.shared;                         // layer / merge scratch
    t += align_up(F * 2);                  // fine counts (16 bits each)
    t += align_up((F + 1) * 4);            // fine offsets (32-bit)
    t += align_up(((size_t)SCAN_TILE + 1) * 8);  // scan tile sums
    t += align_up(((size_t)(cap / MIN_RANGE_TARGET) + 2) * 4);  // unit-kernel range starts
    t += align_up(sizeof(Counters));
    t += align_up(EXPECT_BLOCKS * 8);
    t += align_up(64);
    t += align_up(PROGRAM_RESULTS * 8) + align_up(sizeof(ProgramStats));
    if (P > 1) {
        const size_t tab = (size_t)P * MAX_QUBITS;
        t += 2 * align_up(ROT_SLOTS * tab * 16);  // rotation tables
        t += align_up((size_t)EXPECT_BATCH_BLOCKS * P * 8);                    // expectation partials
        t += align_up((size_t)P * 8) + align_up((size_t)P * 8);                // outputs, sizes
    }
    L.total = t;
    return L;
}

orqa_status fail(orqa_ctx* ctx, orqa_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

#define CUDA_TRY(ctx, expr)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, ORQA_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define LAUNCH_CHECK(ctx)                                                               \
    do {                                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, ORQA_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

// Calls FN<W, T>(args) for the context's plane width and coefficient type.
#define ORQA_DISPATCH(ctx, FN, ...)                                                          \
    ((ctx)->W == 1 ? ((ctx)->fp32 ? FN<1, float>(__VA_ARGS__) : FN<1, double>(__VA_ARGS__)) \
                   : ((ctx)->fp32 ? FN<2, float>(__VA_ARGS__) : FN<2, double>(__VA_ARGS__)))

// cos and sin of a rotation angle, exact (0, +-1) within 1e-12 of a
// multiple of pi/2.
void cos_sin(double theta, double* c, double* s, bool* clifford) {
    const double half_pi = 1.57079632679489661923;
    const double k = std::nearbyint(theta / half_pi);
    if (std::fabs(theta - k * half_pi) <= 1e-12) {
        const long long m = (((long long)k % 4) + 4) % 4;
        static const double tab[4][2] = {{1.0, 0.0}, {0.0, 1.0}, {-1.0, 0.0}, {0.0, -1.0}};
        *c = tab[m][0];
        *s = tab[m][1];
        *clifford = true;
        return;
    }
    *c = std::cos(theta);
    *s = std::sin(theta);
    *clifford = false;
}

// Threshold bits for the integer truncation tests of the stored type T:
// ge_bits<T>(d): |c| >= d  <=>  mag(c) >= ge_bits;  gt_bits<T>(d): |c| > d
// <=> mag(c) > gt_bits.  For FP32 the threshold is rounded up (resp. down)
// to a float, so the test on the float value equals the test against d.
unsigned long long mag64(double d) {
    unsigned long long b;
    memcpy(&b, &d, 8);
    return b & 0x7fffffffffffffffull;
}

unsigned long long mag32(float f) {
    unsigned b;
    memcpy(&b, &f, 4);
    return (unsigned long long)(b & 0x7fffffffu);
}

template <typename T>
unsigned long long ge_bits(double d);
template <>
unsigned long long ge_bits<double>(double d) { return mag64(d); }
template <>
unsigned long long ge_bits<float>(double d) {
    float f = (float)d;
    if ((double)f < d) f = std::nextafter(f, INFINITY);
    return mag32(f);
}

template <typename T>
unsigned long long gt_bits(double d);
template <>
unsigned long long gt_bits<double>(double d) { return mag64(d); }
template <>
unsigned long long gt_bits<float>(double d) {
    float f = (float)d;
    if ((double)f > d) f = std::nextafter(f, 0.0f);
    return mag32(f);
}

// Magnitude bits of type T back to a double.
template <typename T>
double from_mag(unsigned long long b);
template <>
double from_mag<double>(unsigned long long b) {
    double d;
    memcpy(&d, &b, 8);
    return d;
}
template <>
double from_mag<float>(unsigned long long b) {
    const unsigned u = (unsigned)b;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

int grid_for(const orqa_ctx* ctx, long long n, int block = 256) {
    long long b = (n + block - 1) / block;
    long long cap = (long long)ctx->sm_count * ctx->grid_per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaEvent_t take_event(orqa_ctx* ctx) {
    cudaEvent_t e = nullptr;
    if (!ctx->event_pool.empty()) {
        e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
    } else {
        cudaEventCreate(&e);
    }
    return e;
}

// Returns the index of the pending record (or -1) so that the byte count can
// be filled in once the counters are known.
int prof_begin(orqa_ctx* ctx, int kind, double bytes) {
    if (!ctx->profile) return -1;
    PendingLaunch p{kind, take_event(ctx), take_event(ctx), bytes, 0.0};
    cudaEventRecord(p.a, ctx->stream);
    ctx->pending.push_back(p);
    return (int)ctx->pending.size() - 1;
}

void prof_end(orqa_ctx* ctx, int rec) {
    if (rec >= 0) cudaEventRecord(ctx->pending[rec].b, ctx->stream);
}

void prof_set_bytes(orqa_ctx* ctx, int rec, double bytes) {
    if (rec >= 0) ctx->pending[rec].bytes = bytes;
}

// The launch's share of the method's per-gate traffic floor (see
// orqa_kernel_profile.floor_bytes).
void prof_set_floor(orqa_ctx* ctx, int rec, double bytes) {
    if (rec >= 0) ctx->pending[rec].floor_bytes = bytes;
}

// Call only after the stream has been synchronised.
void prof_resolve(orqa_ctx* ctx) {
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ctx->prof_ms[p.kind] += ms;
            ctx->prof_bytes[p.kind] += p.bytes;
            ctx->prof_floor[p.kind] += p.floor_bytes;
            ctx->prof_launches[p.kind] += 1;
        }
        ctx->event_pool.push_back(p.a);
        ctx->event_pool.push_back(p.b);
    }
    ctx->pending.clear();
}

orqa_status sync_counters(orqa_ctx* ctx, Counters* h) {
    CUDA_TRY(ctx, cudaMemcpyAsync(h, ctx->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return ORQA_OK;
}

// Clears the layer counters and the error bits (the committed operator's
// size and buffer, n_live and cur, are kept).
orqa_status reset_counters(orqa_ctx* ctx) {
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->ctr, 0, offsetof(Counters, n_live), ctx->stream));
    return ORQA_OK;
}

// Makes buffer `cur` with n strings the committed operator, on the host and
// on the device.
orqa_status host_commit(orqa_ctx* ctx, int cur, long long n) {
    ctx->cur = cur;
    ctx->n = n;
    ctx->norms_valid = false;
    k_set_live<<<1, 32, 0, ctx->stream>>>(ctx->ctr, n, cur);
    LAUNCH_CHECK(ctx);
    return ORQA_OK;
}

orqa_status check_flags(orqa_ctx* ctx, const Counters& h, const char* what) {
    if (h.err & ERR_TIMEOUT)
        return fail(ctx, ORQA_ETIMEOUT, std::string(what) + ": a bounded hash-table wait ran out");
    if (h.err & ERR_TABLE_FULL) return fail(ctx, ORQA_ECAPACITY, std::string(what) + ": hash table full");
    if (h.err & ERR_PASS_LIMIT)
        return fail(ctx, ORQA_ETIMEOUT, std::string(what) + ": chunk-pass limit reached");
    if (h.err & ERR_BUCKET_OVERFLOW)
        return fail(ctx, ORQA_ECAPACITY, std::string(what) + ": a bucket range exceeded the shared-memory capacity");
    if (h.err & ERR_OVERFLOW) {
        char b[256];
        snprintf(b, sizeof b, "%s: result exceeds capacity %lld (needed at least %llu + %llu)", what,
                 ctx->cap, (unsigned long long)h.n_done, (unsigned long long)h.n_next);
        return fail(ctx, ORQA_ECAPACITY, b);
    }
    return ORQA_OK;
}

// Bytes of one string in the SoA buffers: x and z planes plus the coefficient.
template <int W, typename T>
constexpr double string_bytes() {
    return 16.0 * W + (double)sizeof(T);
}

template <int W, typename Tin, typename Tout>
orqa_status merge_into(orqa_ctx* ctx, StrList src, long long n, int dst_buf, double delta,
                       long long* n_out) {
    long long tcap = std::min(pow2_at_least(2 * (n > 0 ? n : 1)), ctx->table_cap);
    if (4 * n > 3 * tcap) return fail(ctx, ORQA_ECAPACITY, "merge: hash table too small");
    if (ctx->dbg_table_slots > 0) tcap = std::min(tcap, ctx->dbg_table_slots);  // test hook
    if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;
    int r_as = -1, r_off = -1, r_sc = -1, r_red = -1;
    if (n > 0) {
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->table, 0xff, (size_t)tcap * 4, ctx->stream));
        if (ctx->poison_table) {  // test hook: every slot looks busy
            k_fill_busy<<<grid_for(ctx, tcap), 256, 0, ctx->stream>>>(ctx->table, tcap);
            LAUNCH_CHECK(ctx);
        }
        const int g = grid_for(ctx, n);
        r_as = prof_begin(ctx, K_MERGE_ASSIGN, 0);
        k_merge_assign<W><<<g, 256, 0, ctx->stream>>>(src, n, ctx->table, tcap - 1, ctx->unit_z, ctx->unit_xb,
                                                       ctx->unit_pid, ctx->unit_count, ctx->uid, ctx->rank, ctx->ctr,
                                                       ctx->spin_limit);
        prof_end(ctx, r_as);
        LAUNCH_CHECK(ctx);
        r_off = prof_begin(ctx, K_MERGE_OFFSETS, 0);
        k_merge_offsets<<<g, 256, 0, ctx->stream>>>(ctx->unit_count, ctx->unit_off, ctx->ctr);
        prof_end(ctx, r_off);
        LAUNCH_CHECK(ctx);
        r_sc = prof_begin(ctx, K_MERGE_SCATTER, (double)n * 32.0);
        k_merge_scatter<Tin><<<g, 256, 0, ctx->stream>>>(reinterpret_cast<const Tin*>(src.c), n, ctx->uid, ctx->rank,
                                                          ctx->unit_off, ctx->sorted_c);
        prof_end(ctx, r_sc);
        LAUNCH_CHECK(ctx);
        r_red = prof_begin(ctx, K_MERGE_REDUCE, 0);
        k_merge_reduce<W, Tout><<<g, 256, 0, ctx->stream>>>(ctx->unit_z, ctx->unit_xb, ctx->unit_pid, ctx->unit_count,
                                                             ctx->unit_off, ctx->sorted_c, ge_bits<Tout>(delta),
                                                             ctx->buf[dst_buf], ctx->cap, ctx->ctr);
        prof_end(ctx, r_red);
        LAUNCH_CHECK(ctx);
    }
    Counters h{};
    orqa_status st = sync_counters(ctx, &h);
    if (st != ORQA_OK) return st;
    {
        const double R = string_bytes<W, Tout>(), nu = (double)h.n_units, nn = (double)n;
        prof_set_bytes(ctx, r_as, nn * (32.0 * W + 12.0) + nu * (16.0 * W + 4.0));
        prof_set_bytes(ctx, r_off, nu * 12.0);
        prof_set_bytes(ctx, r_red, nu * (16.0 * W + 12.0) + nn * 8.0 + (double)h.n_done * R);
        prof_resolve(ctx);
    }
    st = check_flags(ctx, h, "merge");
    if (st != ORQA_OK) return st;
    *n_out = (long long)h.n_done;
    ctx->stats.dropped = (int64_t)h.dropped;
    ctx->stats.dropped_sum_sq = h.dropped_sq;
    return ORQA_OK;
}

// Groups the edges of a ZZ layer for k_rzz_layer: one set per Clifford mode
// (a repeated edge opens a new set), each set split by offset d = j - i into
// masks of left endpoints.  Launches are cut at MAX_ZZ_SETS / MAX_ZZ_GROUPS;
// all gates commute, so any such order is the array order's result.
orqa_status build_zz_groups(orqa_ctx* ctx, const orqa_gate* g, int ng, std::vector<ZZGroups>& launches) {
    struct Edge { int i, j, mode; };
    std::vector<std::vector<Edge>> sets;   // edges per set
    std::vector<int> set_mode;
    for (int k = 0; k < ng; ++k) {
        double c, s;
        bool cl;
        cos_sin(g[k].theta, &c, &s, &cl);
        if (!cl) return fail(ctx, ORQA_EINVAL, "ORQA_RZZ angle must be a multiple of pi/2");
        int mode;
        if (s == 0.0)
            mode = (c > 0) ? 0 : 1;
        else
            mode = (s < 0) ? 2 : 3;
        if (mode == 0) continue;
        const int i = std::min(g[k].q0, g[k].q1), j = std::max(g[k].q0, g[k].q1);
        int target = -1;
        for (int t = 0; t < (int)sets.size() && target < 0; ++t) {
            if (set_mode[t] != mode) continue;
            bool dup = false;
            for (const Edge& e : sets[t]) dup = dup || (e.i == i && e.j == j);
            if (!dup) target = t;
        }
        if (target < 0) {
            sets.push_back({});
            set_mode.push_back(mode);
            target = (int)sets.size() - 1;
        }
        sets[target].push_back({i, j, mode});
    }
    ZZGroups cur{};
    for (size_t t = 0; t < sets.size(); ++t) {
        // offset groups of this set
        std::vector<int> ds;
        for (const Edge& e : sets[t])
            if (std::find(ds.begin(), ds.end(), e.j - e.i) == ds.end()) ds.push_back(e.j - e.i);
        std::sort(ds.begin(), ds.end());
        if (cur.n_sets == MAX_ZZ_SETS || cur.n_groups + (int)ds.size() > MAX_ZZ_GROUPS) {
            launches.push_back(cur);
            cur = ZZGroups{};
        }
        for (int d : ds) {
            const int gi = cur.n_groups++;
            cur.d[gi] = d;
            cur.mask[gi][0] = cur.mask[gi][1] = 0;
            for (const Edge& e : sets[t])
                if (e.j - e.i == d) cur.mask[gi][e.i >> 6] |= 1ull << (e.i & 63);
        }
        cur.set_mode[cur.n_sets] = set_mode[t];
        cur.set_end[cur.n_sets] = cur.n_groups;
        ++cur.n_sets;
    }
    if (cur.n_sets) launches.push_back(cur);
    return ORQA_OK;
}

// Drops c == 0 and |c| < delta from the committed operator (the truncation
// loop of Algorithm 1 on its own) into the next buffer.
template <int W, typename T>
orqa_status truncate_abs(orqa_ctx* ctx, double delta, long long* dropped, double* dropped_sq = nullptr) {
    const int dst = (ctx->cur + 1) % 3;
    if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;
    const int r = prof_begin(ctx, K_TRUNCATE, 0);
    k_truncate<W, T, false><<<grid_for(ctx, ctx->n), 256, 0, ctx->stream>>>(ctx->buf[ctx->cur], ctx->n, ctx->buf[dst],
                                                                           ctx->cap, ge_bits<T>(delta), ctx->ctr);
    prof_end(ctx, r);
    LAUNCH_CHECK(ctx);
    Counters h{};
    orqa_status st = sync_counters(ctx, &h);
    if (st != ORQA_OK) return st;
    prof_set_bytes(ctx, r, (double)ctx->n * sizeof(T) + (double)h.n_done * (16.0 * W + string_bytes<W, T>()));
    prof_resolve(ctx);
    if ((st = check_flags(ctx, h, "truncate")) != ORQA_OK) return st;
    *dropped = ctx->n - (long long)h.n_done;
    if (dropped_sq) *dropped_sq = h.dropped_sq;
    if ((st = host_commit(ctx, dst, (long long)h.n_done)) != ORQA_OK) return st;
    ctx->clean_delta = delta;
    return ORQA_OK;
}

// Applies the ZZ layer G to the committed operator in place.
template <int W, typename T>
orqa_status launch_rzz(orqa_ctx* ctx, const ZZGroups& G) {
    if (ctx->n == 0) return ORQA_OK;
    // error bits that a failed earlier call left would make the kernel skip
    if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;
    const double b = (double)ctx->n * (string_bytes<W, T>() + 8.0 * W + sizeof(T));
    const int r = prof_begin(ctx, K_RZZ, b);
    k_rzz_layer<W, T><<<grid_for(ctx, ctx->n), 256, 0, ctx->stream>>>(ctx->buf[ctx->cur], ctx->cap, ctx->ctr, G);
    prof_end(ctx, r);
    prof_set_floor(ctx, r, b);
    LAUNCH_CHECK(ctx);
    return ORQA_OK;
}

template <int W, typename T>
orqa_status settle_zz_t(orqa_ctx* ctx) {
    const orqa_status st = launch_rzz<W, T>(ctx, ctx->zz_pend);
    if (st == ORQA_OK) ctx->zz_pending = false;
    return st;
}

// Applies a held-back ZZ layer, if any, to the committed operator.
orqa_status settle_zz(orqa_ctx* ctx) {
    return ctx->zz_pending ? ORQA_DISPATCH(ctx, settle_zz_t, ctx) : ORQA_OK;
}

// A ZZ layer of one launch is held back for the next X layer's entry split
// (the operator it leaves is the same; an X layer that fails leaves it
// held back over the unchanged operator).
template <int W, typename T>
orqa_status apply_rzz(orqa_ctx* ctx, const orqa_gate* g, int ng, double delta) {
    std::vector<ZZGroups> launches;
    orqa_status st = build_zz_groups(ctx, g, ng, launches);
    if (st != ORQA_OK) return st;
    if (ctx->zz_pending && (st = settle_zz_t<W, T>(ctx)) != ORQA_OK) return st;
    if (ctx->zz_fuse && launches.size() == 1 && ctx->n > 0) {
        ctx->zz_pend = launches[0];
        ctx->zz_pending = true;
    } else {
        for (const ZZGroups& l : launches)
            if ((st = launch_rzz<W, T>(ctx, l)) != ORQA_OK) return st;
    }
    ctx->stats.last_layer_in = ctx->n;
    ctx->stats.last_layer_peak = ctx->n;
    ctx->stats.string_gate_updates = (int64_t)ctx->n * ng;
    ctx->stats.branch_events = 0;
    ctx->stats.dropped = 0;
    ctx->stats.pair_updates_one = 0;
    ctx->stats.pair_updates_two = 0;
    ctx->stats.chunk_passes = 0;
    ctx->stats.dropped_sum_sq = 0.0;
    // |c| is unchanged by the layer and strings map one to one, so the
    // truncation may run before the held-back layer is applied
    if (delta > ctx->clean_delta && ctx->n > 0) {
        long long dropped = 0;
        double dsq = 0.0;
        st = truncate_abs<W, T>(ctx, delta, &dropped, &dsq);
        if (st != ORQA_OK) return st;
        ctx->stats.dropped = dropped;
        ctx->stats.dropped_sum_sq = dsq;
    }
    return ORQA_OK;
}

// Exclusive scan of fine-bucket counts fcount[k] into foffsets.
orqa_status fine_scan(orqa_ctx* ctx) {
    const int tiles = ctx->n_fine / SCAN_TILE;
    const int r = prof_begin(ctx, K_SCAN, (double)ctx->n_fine * 20.0);
    k_scan_tiles<<<tiles, SCAN_THREADS, 0, ctx->stream>>>(ctx->fcount, ctx->foffsets, ctx->tile_sums, ctx->ctr);
    k_scan_top<<<1, SCAN_THREADS, 0, ctx->stream>>>(ctx->tile_sums, tiles, ctx->ctr);
    k_scan_add<<<tiles, SCAN_THREADS, 0, ctx->stream>>>(ctx->foffsets, ctx->tile_sums, ctx->fcount, ctx->n_fine,
                                                         ctx->range_start, ctx->range_target, ctx->ctr);
    prof_end(ctx, r);
    LAUNCH_CHECK(ctx);
    return ORQA_OK;
}

// Fills the parameters of an X layer (strictly ascending qubits).  For a
// batched context with per-problem angles (theta: n_problems rows of ng
// angles), the (cos, sin) table of every problem is written to rotation
// table `slot`; otherwise every problem uses the gates' own angles.
orqa_status build_rx_run(orqa_ctx* ctx, const orqa_gate* g, int ng, double delta, const double* theta, int slot,
                         RxRun& run) {
    run = RxRun{};
    run.delta = delta;
    run.track_norm = ctx->track_norm ? 1 : 0;
    run.dbits64 = ge_bits<double>(delta);
    run.dbits32 = (uint32_t)ge_bits<float>(delta);
    run.q_first = g[0].q0;
    for (int k = 0; k < ng; ++k) {
        const int q = g[k].q0;
        if (k > 0 && q <= g[k - 1].q0)
            return fail(ctx, ORQA_EINVAL, "ORQA_RX gates of one layer must have strictly ascending qubits");
        run.mask[q >> 6] |= 1ull << (q & 63);
        bool cl;
        cos_sin(g[k].theta, &run.cs[q], &run.sn[q], &cl);
        run.csf[q] = (float)run.cs[q];
        run.snf[q] = (float)run.sn[q];
        run.cslf[q] = (float)(run.cs[q] - (double)run.csf[q]);
        run.snlf[q] = (float)(run.sn[q] - (double)run.snf[q]);
    }
    run.uniform = ctx->P == 1 ? 1 : 0;
    for (int k = 1; k < ng; ++k)
        if (g[k].theta != g[0].theta) run.uniform = 0;
    if (ctx->P > 1) {
        const size_t tab = (size_t)ctx->P * MAX_QUBITS;
        std::vector<double2>& h64 = ctx->rot_host[slot];
        std::vector<float4>& h32 = ctx->rot_host32[slot];
        h64.assign(tab, make_double2(0.0, 0.0));
        h32.assign(tab, make_float4(0.f, 0.f, 0.f, 0.f));
        for (int p = 0; p < ctx->P; ++p)
            for (int k = 0; k < ng; ++k) {
                const int q = g[k].q0;
                double c = run.cs[q], sn = run.sn[q];
                if (theta) {
                    const double th = theta[(size_t)p * ng + k];
                    if (!std::isfinite(th)) return fail(ctx, ORQA_EINVAL, "apply_layer_batch: angle not finite");
                    bool cl;
                    cos_sin(th, &c, &sn, &cl);
                }
                h64[(size_t)p * MAX_QUBITS + q] = make_double2(c, sn);
                const float ch = (float)c, sh = (float)sn;
                h32[(size_t)p * MAX_QUBITS + q] =
                    make_float4(ch, sh, (float)(c - (double)ch), (float)(sn - (double)sh));
            }
        double2* d64 = ctx->rot64 + (size_t)slot * tab;
        float4* d32 = ctx->rot32 + (size_t)slot * tab;
        CUDA_TRY(ctx, cudaMemcpyAsync(d64, h64.data(), tab * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(d32, h32.data(), tab * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
        run.tab.f64 = d64;
        run.tab.f32 = d32;
    }
    return ORQA_OK;
}

// String lists of an X layer applied to the operator in buffer S: the
// output goes to buffer (S + 1) % 3 and the active list of the passes lives
// in buffer (S + 2) % 3 with the hash and rank arrays.
struct RxLists {
    StrList src, done, act;
    int D;
};

RxLists rx_lists(orqa_ctx* ctx, int S) {
    RxLists L;
    L.src = ctx->buf[S];
    L.D = (S + 1) % 3;
    L.done = ctx->buf[L.D];
    L.act = ctx->buf[(S + 2) % 3];
    L.act.h = ctx->hash_active;
    L.act.rank = ctx->rank_active;
    return L;
}

int local_grid(const orqa_ctx* ctx, long long n_active) {
    const long long ranges = (n_active + ctx->range_target - 1) / ctx->range_target;
    const long long cap = (long long)ctx->sm_count * (ctx->fp32 ? lb_ctas<float>() : lb_ctas<double>());  // resident CTAs of the unit kernel
    return (int)std::max(1ll, std::min(ranges, cap));
}

// One chunk pass (scan, scatter, unit kernel, bookkeeping) on the device;
// the counts are read on the device, so the grids may be upper bounds.
template <int W, typename T>
orqa_status enqueue_pass(orqa_ctx* ctx, const RxLists& L, const RxRun& run, int scatter_grid, int local_grid_n,
                         cudaGraphConditionalHandle cond, int use_cond, int* r_sc, int* r_lo) {
    orqa_status st = fine_scan(ctx);
    if (st != ORQA_OK) return st;
    *r_sc = prof_begin(ctx, K_BUCKET_SCATTER, 0);
    k_bucket_scatter<W, T><<<scatter_grid, 256, 0, ctx->stream>>>(L.act, ctx->cap, ctx->fshift, ctx->foffsets,
                                                                   ctx->records, ctx->fcount, ctx->n_fine, ctx->ctr);
    prof_end(ctx, *r_sc);
    LAUNCH_CHECK(ctx);
    *r_lo = prof_begin(ctx, K_LOCAL, 0);
    if (run.track_norm)
        k_bucket_local<W, T, true><<<local_grid_n, LB_THREADS, ctx->local_smem, ctx->stream>>>(
            ctx->records, ctx->foffsets, ctx->range_start, ctx->n_fine, ctx->range_target, ctx->sub_max, run, L.done,
            L.act, ctx->cap, ctx->ctr, ctx->fcount, ctx->fshift);
    else
        k_bucket_local<W, T, false><<<local_grid_n, LB_THREADS, ctx->local_smem, ctx->stream>>>(
            ctx->records, ctx->foffsets, ctx->range_start, ctx->n_fine, ctx->range_target, ctx->sub_max, run, L.done,
            L.act, ctx->cap, ctx->ctr, ctx->fcount, ctx->fshift);
    prof_end(ctx, *r_lo);
    LAUNCH_CHECK(ctx);
    k_pass_advance<<<1, 32, 0, ctx->stream>>>(ctx->ctr, 0, cond, use_cond, ctx->pass_limit);
    LAUNCH_CHECK(ctx);
    return ORQA_OK;
}

template <int W, typename T>
orqa_status apply_rx(orqa_ctx* ctx, const orqa_gate* g, int ng, double delta, const double* theta) {
    RxRun run;
    orqa_status st = build_rx_run(ctx, g, ng, delta, theta, 0, run);
    if (st != ORQA_OK) return st;
    const double R = string_bytes<W, T>();
    const RxLists L = rx_lists(ctx, ctx->cur);
    const long long n_in = ctx->n;
    if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->fcount, 0, (size_t)ctx->n_fine * 2, ctx->stream));
    int r_split = -1;
    const bool fused = ctx->zz_pending;  // a held-back ZZ layer is applied by the split
    if (n_in > 0) {
        r_split = prof_begin(ctx, K_SPLIT, 0);
        if (fused)
            k_rx_split<W, T, true><<<grid_for(ctx, n_in), 256, 0, ctx->stream>>>(
                L.src, L.done, L.act, ctx->cap, run, ctx->ctr, ctx->fcount, ctx->fshift, ctx->zz_pend);
        else
            k_rx_split<W, T, false><<<grid_for(ctx, n_in), 256, 0, ctx->stream>>>(
                L.src, L.done, L.act, ctx->cap, run, ctx->ctr, ctx->fcount, ctx->fshift, kNoZZ);
        prof_end(ctx, r_split);
        LAUNCH_CHECK(ctx);
    }
    k_pass_advance<<<1, 32, 0, ctx->stream>>>(ctx->ctr, 1, 0, 0, ctx->pass_limit);
    LAUNCH_CHECK(ctx);
    Counters h{};
    if ((st = sync_counters(ctx, &h)) != ORQA_OK) return st;
    // z and c of every string, x of every routed one (of every string when
    // fused), the routed string written, hash and rank of the active ones
    prof_set_bytes(ctx, r_split, (double)n_in * (8.0 * W + sizeof(T) + (fused ? 8.0 * W : 0.0)) +
                                     (double)(h.n_done + h.n_active) * ((fused ? 0.0 : 8.0 * W) + R) +
                                     (double)h.n_active * 12.0);
    // the fused ZZ layer's floor (R read, z and c written per string)
    if (fused) prof_set_floor(ctx, r_split, (double)n_in * (R + 8.0 * W + sizeof(T)));
    prof_resolve(ctx);
    if ((st = check_flags(ctx, h, "rotation layer")) != ORQA_OK) return st;
    int pass = 0;
    // per-gate floor of an X gate (8 bytes of z per string tested, then per
    // anticommuting string its x, z, c read, the child record and the
    // parent's c written, and a merge that meets and writes both once):
    // 8 + (R - 8) + R + sizeof(T) + 2R bytes per branch event, charged to the
    // unit kernel, which does all branching
    const double floor_per_branch = 4.0 * R + (double)sizeof(T);
    while (h.n_active > 0) {  // ends: k_pass_advance flags an error beyond pass_limit passes
        const long long n_active = (long long)h.n_active;
        const unsigned long long done_before = h.n_done;
        const unsigned long long branch_before = h.branch_events;
        int r_sc = -1, r_lo = -1;
        // the scatter also clears the bucket counts: its grid covers both
        const long long scatter_work = std::max((n_active + SCATTER_ILP - 1) / SCATTER_ILP, (long long)ctx->n_fine);
        st = enqueue_pass<W, T>(ctx, L, run, grid_for(ctx, scatter_work), local_grid(ctx, n_active), 0, 0, &r_sc,
                                &r_lo);
        if (st != ORQA_OK) return st;
        if ((st = sync_counters(ctx, &h)) != ORQA_OK) return st;
        const double outs = (double)(h.n_done - done_before) + (double)h.n_active;
        prof_set_bytes(ctx, r_sc, (double)n_active * (R + 12.0 + record_bytes(W)));
        prof_set_bytes(ctx, r_lo, (double)n_active * record_bytes(W) + outs * R + (double)h.n_active * 12.0);
        prof_set_floor(ctx, r_lo, (double)(h.branch_events - branch_before) * floor_per_branch);
        prof_resolve(ctx);
        if ((st = check_flags(ctx, h, "rotation layer")) != ORQA_OK) return st;
        ++pass;
    }
    // Sum over the gates of |O| before each gate (Counters::upd_w)
    const long long updates = (long long)ng * n_in - (long long)h.split_dropped * (ng - 1) + (long long)h.upd_w;
    if ((st = host_commit(ctx, L.D, (long long)h.n_done)) != ORQA_OK) return st;
    ctx->zz_pending = false;
    ctx->clean_delta = delta;
    ctx->stats.last_layer_in = n_in;
    ctx->stats.last_layer_peak = (long long)h.peak;
    ctx->stats.string_gate_updates = updates;
    ctx->stats.branch_events = (int64_t)h.branch_events;
    ctx->stats.dropped = (int64_t)h.dropped;
    ctx->stats.pair_updates_one = (int64_t)h.pairs_one;
    ctx->stats.pair_updates_two = (int64_t)h.pairs_two;
    ctx->stats.chunk_passes = pass;
    ctx->stats.dropped_sum_sq = run.track_norm ? h.dropped_sq : std::nan("");
    return ORQA_OK;
}

// Relative truncation of Eq. (truncation1): drop c == 0 and |c| <= eps0 *
// max|c|.  The threshold is eps0 * max formed on the host in FP64, the same
// product the CPU oracle forms.
template <int W, typename T>
orqa_status truncate_relative(orqa_ctx* ctx, double eps0, long long* dropped, double* dropped_sq = nullptr) {
    *dropped = 0;
    if (dropped_sq) *dropped_sq = 0.0;
    if (ctx->n == 0) return ORQA_OK;
    unsigned long long* mx = (unsigned long long*)ctx->scalar;
    CUDA_TRY(ctx, cudaMemsetAsync(mx, 0, 8, ctx->stream));
    k_absmax<T><<<grid_for(ctx, ctx->n), 256, 0, ctx->stream>>>(reinterpret_cast<const T*>(ctx->buf[ctx->cur].c),
                                                                ctx->n, mx);
    LAUNCH_CHECK(ctx);
    unsigned long long mb = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&mb, mx, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    const double mval = from_mag<T>(mb);
    const double thr = eps0 * mval;
    const int dst = (ctx->cur + 1) % 3;
    if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;
    const int r = prof_begin(ctx, K_TRUNCATE, 0);
    k_truncate<W, T, true><<<grid_for(ctx, ctx->n), 256, 0, ctx->stream>>>(ctx->buf[ctx->cur], ctx->n, ctx->buf[dst],
                                                                          ctx->cap, gt_bits<T>(thr), ctx->ctr);
    prof_end(ctx, r);
    LAUNCH_CHECK(ctx);
    Counters h{};
    orqa_status st = sync_counters(ctx, &h);
    if (st != ORQA_OK) return st;
    prof_set_bytes(ctx, r, (double)ctx->n * sizeof(T) + (double)h.n_done * (16.0 * W + string_bytes<W, T>()));
    prof_resolve(ctx);
    if ((st = check_flags(ctx, h, "relative truncation")) != ORQA_OK) return st;
    *dropped = ctx->n - (long long)h.n_done;
    if (dropped_sq) *dropped_sq = h.dropped_sq;
    return host_commit(ctx, dst, (long long)h.n_done);
}

// One rotation about a general Pauli string (see k_pauli_expand), then the
// duplicate merge with truncation: the per-gate loop of Algorithm 1.
template <int W, typename T>
orqa_status apply_pauli_impl(orqa_ctx* ctx, const uint64_t* xj, const uint64_t* zj, double theta, double delta) {
    PauliGen J{};
    for (int w = 0; w < W; ++w) {
        J.x[w] = xj[w];
        J.z[w] = zj[w];
    }
    bool cl;
    cos_sin(theta, &J.c, &J.s, &cl);
    J.ch = (float)J.c;
    J.sh = (float)J.s;
    J.cl = (float)(J.c - (double)J.ch);
    J.sl = (float)(J.s - (double)J.sh);
    const long long n_in = ctx->n;
    const int stage = (ctx->cur + 1) % 3, out = (ctx->cur + 2) % 3;
    if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;
    if (n_in > 0) {
        k_pauli_expand<W, T><<<grid_for(ctx, n_in), 256, 0, ctx->stream>>>(ctx->buf[ctx->cur], n_in, ctx->buf[stage],
                                                                           ctx->cap, J, ctx->ctr);
        LAUNCH_CHECK(ctx);
    }
    Counters h{};
    orqa_status st = sync_counters(ctx, &h);
    if (st != ORQA_OK) return st;
    if ((st = check_flags(ctx, h, "pauli rotation")) != ORQA_OK) return st;
    const unsigned long long branches = h.branch_events;
    long long m = 0;
    const double dabs = ctx->relative ? 0.0 : delta;
    if ((st = merge_into<W, T, T>(ctx, ctx->buf[stage], (long long)h.n_done, out, dabs, &m)) != ORQA_OK) return st;
    const long long dropped_merge = ctx->stats.dropped;
    const double dsq_merge = ctx->stats.dropped_sum_sq;
    if ((st = host_commit(ctx, out, m)) != ORQA_OK) return st;
    long long dropped_rel = 0;
    double dsq_rel = 0.0;
    if (ctx->relative) {
        if ((st = truncate_relative<W, T>(ctx, delta, &dropped_rel, &dsq_rel)) != ORQA_OK) return st;
        ctx->clean_delta = 0.0;
    } else {
        ctx->clean_delta = delta;
    }
    ctx->stats.last_layer_in = n_in;
    ctx->stats.last_layer_peak = std::max(n_in, (long long)h.n_done);
    ctx->stats.string_gate_updates = n_in;
    ctx->stats.branch_events = (int64_t)branches;
    ctx->stats.dropped = dropped_merge + dropped_rel;
    ctx->stats.dropped_sum_sq = dsq_merge + dsq_rel;
    ctx->stats.pair_updates_one = 0;
    ctx->stats.pair_updates_two = 0;
    ctx->stats.chunk_passes = 0;
    return ORQA_OK;
}

// D_t(x) of the committed operator (k_histogram): the edges are
// t_k = max|c| * 10^(log10_lo + k * w), w = -log10_lo / n_bins, formed on the
// host in FP64, with t_n_bins = max|c|.
template <int W, typename T>
orqa_status histogram_impl(orqa_ctx* ctx, int n_bins, double log10_lo, int64_t* counts, double* max_out) {
    const int nb2 = 2 * (n_bins + 1);
    std::vector<unsigned long long> hc((size_t)nb2, 0ull);
    double mval = 0.0;
    if (ctx->n > 0) {
        unsigned long long* mx = (unsigned long long*)ctx->scalar;
        CUDA_TRY(ctx, cudaMemsetAsync(mx, 0, 8, ctx->stream));
        k_absmax<T><<<grid_for(ctx, ctx->n), 256, 0, ctx->stream>>>(reinterpret_cast<const T*>(ctx->buf[ctx->cur].c),
                                                                    ctx->n, mx);
        LAUNCH_CHECK(ctx);
        unsigned long long mb = 0;
        CUDA_TRY(ctx, cudaMemcpyAsync(&mb, mx, 8, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        mval = from_mag<T>(mb);
        const double w = -log10_lo / n_bins;
        std::vector<unsigned long long> tb((size_t)n_bins + 1);
        for (int k = 0; k < n_bins; ++k) tb[(size_t)k] = ge_bits<T>(mval * std::pow(10.0, log10_lo + k * w));
        tb[(size_t)n_bins] = ge_bits<T>(mval);
        // scratch: thresholds then counts, in the expectation partials
        if ((size_t)(n_bins + 1 + nb2) > (size_t)EXPECT_BLOCKS) return fail(ctx, ORQA_EINVAL, "histogram: too many bins");
        unsigned long long* d_tb = reinterpret_cast<unsigned long long*>(ctx->partials);
        unsigned long long* d_cnt = d_tb + n_bins + 1;
        CUDA_TRY(ctx, cudaMemcpyAsync(d_tb, tb.data(), tb.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        CUDA_TRY(ctx, cudaMemsetAsync(d_cnt, 0, (size_t)nb2 * 8, ctx->stream));
        if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;
        k_histogram<T><<<grid_for(ctx, ctx->n), 256, (size_t)nb2 * 4, ctx->stream>>>(
            reinterpret_cast<const T*>(ctx->buf[ctx->cur].c), ctx->cap, ctx->ctr, d_tb, n_bins, d_cnt);
        LAUNCH_CHECK(ctx);
        CUDA_TRY(ctx, cudaMemcpyAsync(hc.data(), d_cnt, (size_t)nb2 * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    }
    for (int k = 0; k < nb2; ++k) counts[k] = (int64_t)hc[(size_t)k];
    if (max_out) *max_out = mval;
    return ORQA_OK;
}

// A layer with relative truncation.  ZZ gates keep every |c|, so the max is
// unchanged through a ZZ layer and one truncation after it equals one after
// every gate.  X gates are applied one at a time: the gate with exact zeros
// dropped, then the truncation with the max of the resulting operator.
template <int W, typename T>
orqa_status apply_layer_relative(orqa_ctx* ctx, const orqa_gate* g, int ng, double eps0) {
    orqa_stats_t acc{};
    long long dropped = 0;
    double dsq = 0.0;
    orqa_status st;
    if (g[0].kind == ORQA_RZZ) {
        if ((st = apply_rzz<W, T>(ctx, g, ng, 0.0)) != ORQA_OK) return st;
        acc = ctx->stats;
        if ((st = truncate_relative<W, T>(ctx, eps0, &dropped, &dsq)) != ORQA_OK) return st;
        acc.dropped += dropped;
        acc.dropped_sum_sq += dsq;
    } else {
        for (int k = 0; k < ng; ++k) {
            if (k > 0 && g[k].q0 <= g[k - 1].q0)
                return fail(ctx, ORQA_EINVAL, "ORQA_RX gates of one layer must have strictly ascending qubits");
            if ((st = apply_rx<W, T>(ctx, &g[k], 1, 0.0, nullptr)) != ORQA_OK) return st;
            if ((st = truncate_relative<W, T>(ctx, eps0, &dropped, &dsq)) != ORQA_OK) return st;
            const orqa_stats_t& s = ctx->stats;
            if (k == 0) acc.last_layer_in = s.last_layer_in;
            acc.last_layer_peak = std::max(acc.last_layer_peak, s.last_layer_peak);
            acc.string_gate_updates += s.string_gate_updates;
            acc.branch_events += s.branch_events;
            acc.dropped += s.dropped + dropped;
            acc.dropped_sum_sq += s.dropped_sum_sq + dsq;
            acc.pair_updates_one += s.pair_updates_one;
            acc.pair_updates_two += s.pair_updates_two;
            acc.chunk_passes += s.chunk_passes;
        }
    }
    ctx->stats = acc;
    ctx->clean_delta = 0.0;
    return ORQA_OK;
}

// <0|O|0> of the committed operator in buffer `cur` into device memory: one
// double (plain context) or one per problem (batched context).
template <int W, typename T>
orqa_status enqueue_expect(orqa_ctx* ctx, int cur, long long n_hint, double* dev_out) {
    const StrList s = ctx->buf[cur];
    if (ctx->P > 1) {
        const size_t sm = (size_t)ctx->P * 8;
        k_expect_batch_partial<W, T><<<EXPECT_BATCH_BLOCKS, 256, sm, ctx->stream>>>(s, ctx->cap, ctx->ctr, ctx->P,
                                                                                     ctx->batch_partials);
        k_expect_batch_final<<<(ctx->P + 255) / 256, 256, 0, ctx->stream>>>(ctx->batch_partials, EXPECT_BATCH_BLOCKS,
                                                                           ctx->P, dev_out, ctx->ctr);
    } else {
        const int r = prof_begin(ctx, K_EXPECT, (double)n_hint * (8.0 * W + sizeof(T)));
        k_expect_partial<W, T><<<EXPECT_BLOCKS, 256, 0, ctx->stream>>>(s, ctx->cap, ctx->ctr, ctx->partials);
        k_expect_final<<<1, 32, 0, ctx->stream>>>(ctx->partials, EXPECT_BLOCKS, dev_out, ctx->ctr);
        prof_end(ctx, r);
        prof_set_floor(ctx, r, (double)n_hint * (8.0 * W + sizeof(T)));
    }
    LAUNCH_CHECK(ctx);
    return ORQA_OK;
}

template <int W, typename T>
orqa_status expect_impl(orqa_ctx* ctx, double* out) {
    if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;  // error bits of an earlier failed call
    double* dev = ctx->P > 1 ? ctx->batch_out : ctx->scalar;
    orqa_status st = enqueue_expect<W, T>(ctx, ctx->cur, ctx->n, dev);
    if (st != ORQA_OK) return st;
    CUDA_TRY(ctx, cudaMemcpyAsync(out, dev, (size_t)ctx->P * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_resolve(ctx);
    return ORQA_OK;
}

// Sum of c^2 and max |c| of the committed operator (k_norms_partial, then
// the block partials added in a fixed order), cached until it changes.
template <int W, typename T>
orqa_status norms_impl(orqa_ctx* ctx) {
    double sq = 0.0, mx = 0.0;
    if (ctx->n > 0) {
        if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;  // error bits of an earlier failed call
        unsigned long long* mbits = reinterpret_cast<unsigned long long*>(ctx->scalar) + 1;
        CUDA_TRY(ctx, cudaMemsetAsync(mbits, 0, 8, ctx->stream));
        k_norms_partial<T><<<EXPECT_BLOCKS, 256, 0, ctx->stream>>>(reinterpret_cast<const T*>(ctx->buf[ctx->cur].c),
                                                                    ctx->cap, ctx->ctr, ctx->partials, mbits);
        k_expect_final<<<1, 32, 0, ctx->stream>>>(ctx->partials, EXPECT_BLOCKS, ctx->scalar + 2, ctx->ctr);
        LAUNCH_CHECK(ctx);
        double hv[3] = {0.0, 0.0, 0.0};
        CUDA_TRY(ctx, cudaMemcpyAsync(hv, ctx->scalar, sizeof hv, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        unsigned long long mb;
        memcpy(&mb, &hv[1], 8);
        sq = hv[2];
        mx = from_mag<T>(mb);
    }
    ctx->norm_sq = sq;
    ctx->norm_max = mx;
    ctx->norms_valid = true;
    return ORQA_OK;
}

// Merge of caller input (FP64 coefficients) into the stored type T, and of
// the operator itself.
template <int W, typename T>
orqa_status merge_input(orqa_ctx* ctx, StrList src, long long n, int dst, double delta, long long* m) {
    return merge_into<W, double, T>(ctx, src, n, dst, delta, m);
}

template <int W, typename T>
orqa_status merge_state(orqa_ctx* ctx, StrList src, long long n, int dst, double delta, long long* m) {
    return merge_into<W, T, T>(ctx, src, n, dst, delta, m);
}

// problem: HOST array of n problem indices (batched contexts), else null.
orqa_status set_from(orqa_ctx* ctx, int64_t n, const uint64_t* x, const uint64_t* z, const double* c,
                     const int32_t* problem, cudaMemcpyKind kind) {
    if (!ctx) return ORQA_EINVAL;
    if (n < 0 || (n > 0 && (!x || !z || !c))) return fail(ctx, ORQA_EINVAL, "set_operator: bad arguments");
    if (n > ctx->cap) return fail(ctx, ORQA_ECAPACITY, "set_operator: n exceeds capacity");
    if (ctx->P > 1 && n > 0 && !problem)
        return fail(ctx, ORQA_EINVAL, "set_operator: a batched context takes problem indices (orqa_set_operator_batch)");
    std::vector<uint16_t> pid16;
    if (problem) {
        if (ctx->P > 1) pid16.resize((size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            if (problem[i] < 0 || problem[i] >= ctx->P)
                return fail(ctx, ORQA_EINVAL, "set_operator_batch: problem index out of range");
            if (ctx->P > 1) pid16[(size_t)i] = (uint16_t)problem[i];
        }
    }
    const int W = ctx->W;
    const int stage = (ctx->cur + 1) % 3, dst = (ctx->cur + 2) % 3;
    StrList s = ctx->buf[stage];
    if (n > 0) {
        CUDA_TRY(ctx, cudaMemcpyAsync(s.x, x, (size_t)n * W * 8, kind, ctx->stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.z, z, (size_t)n * W * 8, kind, ctx->stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.c, c, (size_t)n * 8, kind, ctx->stream));
        if (!pid16.empty())
            CUDA_TRY(ctx, cudaMemcpyAsync(s.pid, pid16.data(), (size_t)n * 2, cudaMemcpyHostToDevice, ctx->stream));
    }
    long long m = 0;
    orqa_status st = ORQA_DISPATCH(ctx, merge_input, ctx, s, n, dst, 0.0, &m);  // waits for the stream
    if (st != ORQA_OK) return st;
    if ((st = host_commit(ctx, dst, m)) != ORQA_OK) return st;
    ctx->zz_pending = false;  // it belonged to the replaced operator
    ctx->clean_delta = 0.0;
    ctx->stats = orqa_stats_t{};
    ctx->err.clear();
    return ORQA_OK;
}

// The committed operator in canonical order (orqa_sort.cuh): *out_buf
// receives the string buffer holding it, which is the committed buffer
// itself when no digit varies (at most one string, or one key).
template <int W, typename T>
orqa_status sorted_buffer(orqa_ctx* ctx, int* out_buf) {
    *out_buf = ctx->cur;
    const long long n = ctx->n;
    if (n <= 1) return ORQA_OK;
    const int K = 2 * W + (ctx->P > 1 ? 1 : 0);
    unsigned long long init[2 * (2 * 2 + 1)];
    for (int k = 0; k < K; ++k) {
        init[2 * k] = 0ull;
        init[2 * k + 1] = ~0ull;
    }
    unsigned long long* d_oa = reinterpret_cast<unsigned long long*>(ctx->partials);
    CUDA_TRY(ctx, cudaMemcpyAsync(d_oa, init, (size_t)2 * K * 8, cudaMemcpyHostToDevice, ctx->stream));
    k_sort_bits<W><<<grid_for(ctx, n), SORT_THREADS, 0, ctx->stream>>>(ctx->buf[ctx->cur], n, K, d_oa);
    LAUNCH_CHECK(ctx);
    unsigned long long oa[2 * (2 * 2 + 1)];
    CUDA_TRY(ctx, cudaMemcpyAsync(oa, d_oa, (size_t)2 * K * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    // blocks: one chunk each; their digit counts must fit the scratch region
    long long G = std::min<long long>(4ll * ctx->sm_count, (n + 2047) / 2048);
    G = std::max(1ll, std::min<long long>(G, (long long)(ctx->shared_bytes / (SORT_DIGITS * 4)) - 1));
    const long long chunk = (n + G - 1) / G;
    unsigned* hist = reinterpret_cast<unsigned*>(ctx->records);
    const int free_bufs[2] = {(ctx->cur + 1) % 3, (ctx->cur + 2) % 3};
    int src = ctx->cur, nxt = 0;
    for (int k = 0; k < K; ++k) {
        const unsigned long long vary = oa[2 * k] ^ oa[2 * k + 1];
        for (int shift = 0; shift < 64; shift += 8) {
            if (((vary >> shift) & 255ull) == 0) continue;
            const int dst = free_bufs[nxt];
            k_sort_hist<W><<<(int)G, SORT_THREADS, 0, ctx->stream>>>(ctx->buf[src], n, chunk, k, shift, hist, (int)G);
            k_sort_scan<<<1, 1024, 0, ctx->stream>>>(hist, (int)(SORT_DIGITS * G));
            k_sort_scatter<W, T><<<(int)G, SORT_THREADS, 0, ctx->stream>>>(ctx->buf[src], ctx->buf[dst], n, chunk, k,
                                                                            shift, hist, (int)G);
            LAUNCH_CHECK(ctx);
            src = dst;
            nxt ^= 1;
        }
    }
    *out_buf = src;
    return ORQA_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Dynamic shared memory of the unit kernel (both instantiations).
template <int W, typename T>
cudaError_t set_local_smem(orqa_ctx* ctx) {
    ctx->local_smem = sizeof(LocalSmem<W, T>);
    // all of the SM's unified memory that can be shared memory: the unit
    // kernel's occupancy is bound by it
    for (const void* f : {(const void*)k_bucket_local<W, T, false>, (const void*)k_bucket_local<W, T, true>}) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctx->local_smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

uint64_t orqa_workspace_bytes_batch(int32_t n_qubits, int64_t capacity, int32_t n_problems) {
    if (n_qubits < 1 || n_qubits > 128 || capacity < 1 || capacity > 0x7fffffffLL || n_problems < 0 ||
        n_problems > ORQA_MAX_PROBLEMS)
        return 0;
    return (uint64_t)layout(n_qubits, capacity, std::max(1, (int)n_problems)).total;
}

uint64_t orqa_workspace_bytes(int32_t n_qubits, int64_t capacity) {
    return orqa_workspace_bytes_batch(n_qubits, capacity, 1);
}

orqa_status orqa_create(const orqa_config* cfg, orqa_ctx** out) {
    if (!cfg || !out) return ORQA_EINVAL;
    *out = nullptr;
    if (cfg->n_qubits < 1 || cfg->n_qubits > 128 || cfg->capacity < 1 || cfg->capacity > 0x7fffffffLL ||
        (cfg->flags & ~(ORQA_FLAG_PROFILE | ORQA_FLAG_RELATIVE | ORQA_FLAG_FP32)) != 0 || !cfg->workspace ||
        ((uintptr_t)cfg->workspace % ALIGN) != 0 || cfg->n_problems < 0 || cfg->n_problems > ORQA_MAX_PROBLEMS ||
        cfg->reserved != 0)
        return ORQA_EINVAL;
    const int P = std::max(1, (int)cfg->n_problems);
    // relative truncation takes the max over the whole operator: one problem only
    if (P > 1 && (cfg->flags & ORQA_FLAG_RELATIVE)) return ORQA_EINVAL;
    const Layout L = layout(cfg->n_qubits, cfg->capacity, P);
    if (cfg->workspace_bytes < L.total) return ORQA_ENOMEM;
    orqa_ctx* ctx = new orqa_ctx();
    ctx->P = P;
    ctx->n_qubits = cfg->n_qubits;
    ctx->W = cfg->n_qubits <= 64 ? 1 : 2;
    ctx->cap = cfg->capacity;
    ctx->stream = (cudaStream_t)cfg->stream;
    ctx->profile = (cfg->flags & ORQA_FLAG_PROFILE) != 0;
    ctx->relative = (cfg->flags & ORQA_FLAG_RELATIVE) != 0;
    ctx->fp32 = (cfg->flags & ORQA_FLAG_FP32) != 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete ctx;
        return ORQA_ECUDA;
    }
    char* p = (char*)cfg->workspace;
    const size_t C = (size_t)cfg->capacity;
    for (int b = 0; b < 3; ++b) {
        ctx->buf[b].x = (uint64_t*)p; p += L.str_x;
        ctx->buf[b].z = (uint64_t*)p; p += L.str_x;
        ctx->buf[b].c = (double*)p;   p += L.str_c;
        ctx->buf[b].h = nullptr;
        ctx->buf[b].rank = nullptr;
        ctx->buf[b].pid = nullptr;
        if (P > 1) {
            ctx->buf[b].pid = (uint16_t*)p;
            p += L.str_pid;
        }
    }
    {
        // layer scratch and merge scratch: two views of one region
        char* q = p;
        ctx->records = (void*)q; q += align_up(C * (size_t)record_bytes(ctx->W));
        ctx->hash_active = (uint64_t*)q; q += align_up(C * 8);
        ctx->rank_active = (int32_t*)q;
        q = p;
        ctx->uid = (int32_t*)q; q += align_up(C * 4);
        ctx->rank = (int32_t*)q; q += align_up(C * 4);
        ctx->unit_z = (uint64_t*)q; q += align_up(C * ctx->W * 8);
        ctx->unit_xb = (uint64_t*)q; q += align_up(C * ctx->W * 8);
        if (P > 1) {
            ctx->unit_pid = (uint16_t*)q;
            q += align_up(C * 2);
        }
        ctx->unit_count = (int32_t*)q; q += align_up(C * 4);
        ctx->unit_off = (long long*)q; q += align_up(C * 8);
        ctx->sorted_c = (double*)q; q += align_up(C * 8);
        ctx->table = (int32_t*)q;
        ctx->table_cap = L.table_cap;
        ctx->shared_bytes = L.shared;
        p += L.shared;
    }
    const size_t F = (size_t)L.n_fine;
    ctx->n_fine_max = (int)L.n_fine;
    ctx->n_fine = (int)fine_buckets(cfg->capacity, ctx->bucket_density);
    ctx->fshift = 64 - __builtin_ctzll((unsigned long long)ctx->n_fine);
    ctx->fcount = (uint32_t*)p; p += align_up(F * 2);
    ctx->foffsets = (uint32_t*)p; p += align_up((F + 1) * 4);
    ctx->tile_sums = (long long*)p; p += align_up(((size_t)SCAN_TILE + 1) * 8);
    ctx->range_start = (int32_t*)p; p += align_up(((size_t)(cfg->capacity / MIN_RANGE_TARGET) + 2) * 4);
    ctx->ctr = (Counters*)p; p += align_up(sizeof(Counters));
    ctx->partials = (double*)p; p += align_up(EXPECT_BLOCKS * 8);
    ctx->scalar = (double*)p; p += align_up(64);
    ctx->prog_results = (double*)p; p += align_up(PROGRAM_RESULTS * 8);
    ctx->prog_stats = (ProgramStats*)p; p += align_up(sizeof(ProgramStats));
    if (P > 1) {
        const size_t tab = (size_t)P * MAX_QUBITS;
        ctx->rot64 = (double2*)p; p += align_up(ROT_SLOTS * tab * 16);
        ctx->rot32 = (float4*)p; p += align_up(ROT_SLOTS * tab * 16);
        ctx->batch_partials = (double*)p; p += align_up((size_t)EXPECT_BATCH_BLOCKS * P * 8);
        ctx->batch_out = (double*)p; p += align_up((size_t)P * 8);
        ctx->sizes_out = (unsigned long long*)p; p += align_up((size_t)P * 8);
    }
    if ((size_t)(p - (char*)cfg->workspace) != L.total) {  // the carve-up must match the layout
        delete ctx;
        return ORQA_EINVAL;
    }
    cudaError_t fe;
    if (ctx->W == 1 && !ctx->fp32)
        fe = set_local_smem<1, double>(ctx);
    else if (ctx->W == 1)
        fe = set_local_smem<1, float>(ctx);
    else if (!ctx->fp32)
        fe = set_local_smem<2, double>(ctx);
    else
        fe = set_local_smem<2, float>(ctx);
    // the empty operator, committed in buffer 0
    if (fe != cudaSuccess || cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        delete ctx;
        return ORQA_ECUDA;
    }
    *out = ctx;
    return ORQA_OK;
}

orqa_status orqa_set_operator(orqa_ctx* ctx, int64_t n, const uint64_t* x, const uint64_t* z,
                              const double* c) {
    return set_from(ctx, n, x, z, c, nullptr, cudaMemcpyHostToDevice);
}

orqa_status orqa_set_operator_device(orqa_ctx* ctx, int64_t n, const uint64_t* x, const uint64_t* z,
                                     const double* c) {
    return set_from(ctx, n, x, z, c, nullptr, cudaMemcpyDeviceToDevice);
}

orqa_status orqa_set_operator_batch(orqa_ctx* ctx, int64_t n, const uint64_t* x, const uint64_t* z,
                                    const double* c, const int32_t* problem) {
    if (!ctx) return ORQA_EINVAL;
    if (n > 0 && !problem) return fail(ctx, ORQA_EINVAL, "set_operator_batch: null problem array");
    return set_from(ctx, n, x, z, c, problem, cudaMemcpyHostToDevice);
}

}  // extern "C"

namespace {

orqa_status apply_layer_impl(orqa_ctx* ctx, const orqa_gate* gates, int32_t n_gates, const double* theta,
                             double delta, int64_t* n_live_out) {
    if (!ctx) return ORQA_EINVAL;
    if (n_gates < 0 || (n_gates > 0 && !gates)) return fail(ctx, ORQA_EINVAL, "apply_layer: bad gate array");
    if (!(delta >= 0.0) || std::isinf(delta)) return fail(ctx, ORQA_EINVAL, "apply_layer: delta must be finite and >= 0");
    if (n_gates == 0) {
        if (n_live_out) *n_live_out = ctx->n;
        return ORQA_OK;
    }
    const int kind = gates[0].kind;
    for (int k = 0; k < n_gates; ++k) {
        const orqa_gate& g = gates[k];
        if (g.kind != kind) return fail(ctx, ORQA_EINVAL, "apply_layer: all gates of a layer must be of one kind");
        if (g.pad != 0 || !std::isfinite(g.theta)) return fail(ctx, ORQA_EINVAL, "apply_layer: bad gate field");
        if (g.q0 < 0 || g.q0 >= ctx->n_qubits) return fail(ctx, ORQA_EINVAL, "apply_layer: qubit out of range");
        if (kind == ORQA_RZZ && (g.q1 < 0 || g.q1 >= ctx->n_qubits || g.q1 == g.q0))
            return fail(ctx, ORQA_EINVAL, "apply_layer: bad second qubit");
        if (kind != ORQA_RX && kind != ORQA_RZZ) return fail(ctx, ORQA_EINVAL, "apply_layer: unknown gate kind");
    }
    if (theta && kind != ORQA_RX)
        return fail(ctx, ORQA_EINVAL, "apply_layer_batch: per-problem angles are for ORQA_RX layers only");
    orqa_status st = ORQA_OK;
    if (ctx->relative)
        st = settle_zz(ctx);
    if (st != ORQA_OK) return st;
    if (ctx->relative)
        st = ORQA_DISPATCH(ctx, apply_layer_relative, ctx, gates, n_gates, delta);
    else if (kind == ORQA_RZZ)
        st = ORQA_DISPATCH(ctx, apply_rzz, ctx, gates, n_gates, delta);
    else
        st = ORQA_DISPATCH(ctx, apply_rx, ctx, gates, n_gates, delta, theta);
    if (st != ORQA_OK) return st;
    ctx->stats.n_strings = ctx->n;
    if (n_live_out) *n_live_out = ctx->n;
    ctx->err.clear();
    return ORQA_OK;
}

}  // namespace

extern "C" {

orqa_status orqa_apply_layer(orqa_ctx* ctx, const orqa_gate* gates, int32_t n_gates, double delta,
                             int64_t* n_live_out) {
    return apply_layer_impl(ctx, gates, n_gates, nullptr, delta, n_live_out);
}

orqa_status orqa_apply_layer_batch(orqa_ctx* ctx, const orqa_gate* gates, int32_t n_gates, const double* theta,
                                   double delta, int64_t* n_live_out) {
    return apply_layer_impl(ctx, gates, n_gates, theta, delta, n_live_out);
}

orqa_status orqa_apply_pauli_rotation(orqa_ctx* ctx, const uint64_t* xj, const uint64_t* zj, double theta,
                                      double delta, int64_t* n_live_out) {
    if (!ctx) return ORQA_EINVAL;
    if (!xj || !zj || !std::isfinite(theta) || !(delta >= 0.0) || std::isinf(delta))
        return fail(ctx, ORQA_EINVAL, "apply_pauli_rotation: bad arguments");
    uint64_t any = 0;
    for (int w = 0; w < ctx->W; ++w) {
        any |= xj[w] | zj[w];
        const int hi = ctx->n_qubits - 64 * w;  // qubits held by word w
        if (hi < 64) {
            const uint64_t outside = hi <= 0 ? ~0ull : ~((1ull << hi) - 1ull);
            if ((xj[w] | zj[w]) & outside) return fail(ctx, ORQA_EINVAL, "apply_pauli_rotation: J acts beyond n_qubits");
        }
    }
    if (!any) return fail(ctx, ORQA_EINVAL, "apply_pauli_rotation: J is the identity");
    orqa_status st = settle_zz(ctx);
    if (st != ORQA_OK) return st;
    st = ORQA_DISPATCH(ctx, apply_pauli_impl, ctx, xj, zj, theta, delta);
    if (st != ORQA_OK) return st;
    ctx->stats.n_strings = ctx->n;
    if (n_live_out) *n_live_out = ctx->n;
    ctx->err.clear();
    return ORQA_OK;
}

orqa_status orqa_merge_truncate(orqa_ctx* ctx, double delta, int64_t* n_live_out) {
    if (!ctx) return ORQA_EINVAL;
    if (!(delta >= 0.0) || std::isinf(delta)) return fail(ctx, ORQA_EINVAL, "merge_truncate: bad delta");
    orqa_status st = settle_zz(ctx);
    if (st != ORQA_OK) return st;
    const int dst = (ctx->cur + 1) % 3;
    long long m = 0;
    const double dabs = ctx->relative ? 0.0 : delta;
    st = ORQA_DISPATCH(ctx, merge_state, ctx, ctx->buf[ctx->cur], ctx->n, dst, dabs, &m);
    if (st != ORQA_OK) return st;
    if ((st = host_commit(ctx, dst, m)) != ORQA_OK) return st;
    if (ctx->relative) {
        long long dropped = 0;
        st = ORQA_DISPATCH(ctx, truncate_relative, ctx, delta, &dropped);
        if (st != ORQA_OK) return st;
        m = ctx->n;
        delta = 0.0;
    }
    if (delta > ctx->clean_delta) ctx->clean_delta = delta;
    ctx->stats.n_strings = m;
    if (n_live_out) *n_live_out = m;
    ctx->err.clear();
    return ORQA_OK;
}

orqa_status orqa_expect(orqa_ctx* ctx, double* out) {
    if (!ctx || !out) return ORQA_EINVAL;
    if (ctx->P > 1) return fail(ctx, ORQA_ESTATE, "expect: batched context (use orqa_expect_batch)");
    const orqa_status st = settle_zz(ctx);
    if (st != ORQA_OK) return st;
    return ORQA_DISPATCH(ctx, expect_impl, ctx, out);
}

orqa_status orqa_expect_batch(orqa_ctx* ctx, double* out) {
    if (!ctx || !out) return ORQA_EINVAL;
    const orqa_status st = settle_zz(ctx);
    if (st != ORQA_OK) return st;
    return ORQA_DISPATCH(ctx, expect_impl, ctx, out);
}

orqa_status orqa_histogram(orqa_ctx* ctx, int32_t n_bins, double log10_lo, int64_t* counts, double* max_abs_out) {
    if (!ctx || !counts) return ORQA_EINVAL;
    if (n_bins < 1 || n_bins > 256 || !(log10_lo < 0.0) || !std::isfinite(log10_lo) || log10_lo < -300.0)
        return fail(ctx, ORQA_EINVAL, "histogram: need 1 <= n_bins <= 256 and -300 <= log10_lo < 0");
    const orqa_status st = settle_zz(ctx);
    if (st != ORQA_OK) return st;
    return ORQA_DISPATCH(ctx, histogram_impl, ctx, n_bins, log10_lo, counts, max_abs_out);
}

orqa_status orqa_problem_sizes(orqa_ctx* ctx, int64_t* out) {
    if (!ctx || !out) return ORQA_EINVAL;
    if (ctx->P == 1) {
        out[0] = ctx->n;
        return ORQA_OK;
    }
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->sizes_out, 0, (size_t)ctx->P * 8, ctx->stream));
    k_problem_sizes<<<grid_for(ctx, ctx->n), 256, (size_t)ctx->P * 4, ctx->stream>>>(
        ctx->buf[ctx->cur].pid, ctx->cap, ctx->ctr, ctx->P, ctx->sizes_out);
    LAUNCH_CHECK(ctx);
    CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->sizes_out, (size_t)ctx->P * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return ORQA_OK;
}

orqa_status orqa_export_batch(orqa_ctx* ctx, int64_t cap, uint64_t* x, uint64_t* z, double* c, int32_t* problem,
                              int64_t* n_out) {
    if (!ctx || !n_out) return ORQA_EINVAL;
    *n_out = ctx->n;
    if (ctx->n > cap) return fail(ctx, ORQA_ECAPACITY, "export: operator larger than cap");
    if (ctx->n > 0 && (!x || !z || !c)) return fail(ctx, ORQA_EINVAL, "export: null array");
    const orqa_status zst = settle_zz(ctx);
    if (zst != ORQA_OK) return zst;
    int sb = ctx->cur;
    const orqa_status sst = ORQA_DISPATCH(ctx, sorted_buffer, ctx, &sb);
    if (sst != ORQA_OK) return sst;
    const StrList s = ctx->buf[sb];
    const size_t n = (size_t)ctx->n;
    std::vector<float> cf(ctx->fp32 ? n : 0);
    std::vector<uint16_t> pid16(problem && ctx->P > 1 ? n : 0);
    if (n > 0) {
        CUDA_TRY(ctx, cudaMemcpyAsync(x, s.x, n * ctx->W * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(z, s.z, n * ctx->W * 8, cudaMemcpyDeviceToHost, ctx->stream));
        if (ctx->fp32)
            CUDA_TRY(ctx, cudaMemcpyAsync(cf.data(), s.c, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
        else
            CUDA_TRY(ctx, cudaMemcpyAsync(c, s.c, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        if (!pid16.empty())
            CUDA_TRY(ctx, cudaMemcpyAsync(pid16.data(), s.pid, n * 2, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < cf.size(); ++i) c[i] = (double)cf[i];
    if (problem)
        for (size_t i = 0; i < n; ++i) problem[i] = pid16.empty() ? 0 : (int32_t)pid16[i];
    return ORQA_OK;
}

orqa_status orqa_export(orqa_ctx* ctx, int64_t cap, uint64_t* x, uint64_t* z, double* c, int64_t* n_out) {
    return orqa_export_batch(ctx, cap, x, z, c, nullptr, n_out);
}

orqa_status orqa_stats(orqa_ctx* ctx, orqa_stats_t* out) {
    if (!ctx || !out) return ORQA_EINVAL;
    if (!ctx->norms_valid) {
        const orqa_status st = ORQA_DISPATCH(ctx, norms_impl, ctx);
        if (st != ORQA_OK) return st;
    }
    ctx->stats.n_strings = ctx->n;
    ctx->stats.sum_sq = ctx->norm_sq;
    ctx->stats.max_abs = ctx->norm_max;
    *out = ctx->stats;
    return ORQA_OK;
}

orqa_status orqa_counters(orqa_ctx* ctx, orqa_stats_t* out) {
    if (!ctx || !out) return ORQA_EINVAL;
    ctx->stats.n_strings = ctx->n;
    ctx->stats.sum_sq = ctx->norms_valid ? ctx->norm_sq : std::nan("");
    ctx->stats.max_abs = ctx->norms_valid ? ctx->norm_max : std::nan("");
    *out = ctx->stats;
    return ORQA_OK;
}

orqa_status orqa_set_norm_tracking(orqa_ctx* ctx, int32_t on) {
    if (!ctx || (on != 0 && on != 1)) return ORQA_EINVAL;
    ctx->track_norm = on != 0;
    return ORQA_OK;
}

orqa_status orqa_debug_set(orqa_ctx* ctx, int32_t knob, int64_t value) {
    if (!ctx) return ORQA_EINVAL;
    switch (knob) {
    case ORQA_DEBUG_SPIN_LIMIT:
        if (value < 0 || value > SPIN_LIMIT) return fail(ctx, ORQA_EINVAL, "debug_set: spin limit out of range");
        ctx->spin_limit = value ? value : SPIN_LIMIT;
        return ORQA_OK;
    case ORQA_DEBUG_POISON_MERGE_TABLE:
        if (value != 0 && value != 1) return fail(ctx, ORQA_EINVAL, "debug_set: poison is 0 or 1");
        ctx->poison_table = value != 0;
        return ORQA_OK;
    case ORQA_DEBUG_MERGE_TABLE_SLOTS:
        if (value != 0 && (value < 16 || (value & (value - 1)) != 0 || value > ctx->table_cap))
            return fail(ctx, ORQA_EINVAL, "debug_set: table slots must be 0 or a power of two in [16, table size]");
        ctx->dbg_table_slots = value;
        return ORQA_OK;
    case ORQA_DEBUG_PASS_LIMIT:
        if (value < 0 || value > MAX_PASSES) return fail(ctx, ORQA_EINVAL, "debug_set: pass limit out of range");
        ctx->pass_limit = value ? (int)value : MAX_PASSES;
        return ORQA_OK;
    case ORQA_DEBUG_BUCKET_SHIFT: {
        const int base = 64 - __builtin_ctzll((unsigned long long)ctx->n_fine);
        if (value != 0 && (value < base || value > 63))
            return fail(ctx, ORQA_EINVAL, "debug_set: bucket shift must be 0 or in [default, 63]");
        ctx->fshift = value ? (int)value : base;
        return ORQA_OK;
    }
    case ORQA_DEBUG_NO_ZZ_FUSION: {
        if (value != 0 && value != 1) return fail(ctx, ORQA_EINVAL, "debug_set: no-fusion is 0 or 1");
        const orqa_status st = settle_zz(ctx);
        if (st != ORQA_OK) return st;
        ctx->zz_fuse = value == 0;
        return ORQA_OK;
    }
    default:
        return fail(ctx, ORQA_EINVAL, "debug_set: unknown knob");
    }
}

int32_t orqa_profile_count(void) { return K_COUNT; }

orqa_status orqa_profile(orqa_ctx* ctx, int32_t index, orqa_kernel_profile* out) {
    if (!ctx || !out || index < 0 || index >= K_COUNT) return ORQA_EINVAL;
    memset(out, 0, sizeof(*out));
    strncpy(out->name, KERNEL_NAMES[index], sizeof(out->name) - 1);
    out->launches = ctx->prof_launches[index];
    out->ms = ctx->prof_ms[index];
    out->bytes = ctx->prof_bytes[index];
    out->floor_bytes = ctx->prof_floor[index];
    return ORQA_OK;
}

orqa_status orqa_profile_reset(orqa_ctx* ctx) {
    if (!ctx) return ORQA_EINVAL;
    for (int k = 0; k < K_COUNT; ++k) {
        ctx->prof_launches[k] = 0;
        ctx->prof_ms[k] = 0.0;
        ctx->prof_bytes[k] = 0.0;
        ctx->prof_floor[k] = 0.0;
    }
    return ORQA_OK;
}

const char* orqa_last_error(const orqa_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void orqa_destroy(orqa_ctx* ctx) { delete ctx; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Captured programs: a layer sequence applied as one CUDA graph.  The graph
// holds the same kernels as the host-driven calls; the chunk passes of an X
// layer form a conditional WHILE node whose body (scan, scatter, unit
// kernel, pass bookkeeping) re-runs while strings remain active, and all
// counts are read on the device, so the grids are fixed upper bounds (the
// unit kernel is persistent).
// ---------------------------------------------------------------------------
namespace {

struct ProgLayer {
    int kind = 0;
    int ng = 0;
    int expect_after = 0;
    std::vector<ZZGroups> zz;
    RxRun rx{};
};

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

// Validates the layers, builds their launch parameters (uploading batched
// rotation tables, one slot per X layer of the sequence) and hashes
// everything that the captured graph depends on.
orqa_status prepare_program(orqa_ctx* ctx, const orqa_layer_desc* d, int nl, int repeat, double delta,
                            std::vector<ProgLayer>& pl, int* n_expect) {
    if (nl < 1 || !d || repeat < 1) return fail(ctx, ORQA_EINVAL, "run_program: empty program");
    if (!(delta >= 0.0) || std::isinf(delta)) return fail(ctx, ORQA_EINVAL, "run_program: bad delta");
    if (ctx->relative) return fail(ctx, ORQA_ESTATE, "run_program: not available with relative truncation");
    pl.assign(nl, ProgLayer{});
    int slot = 0;
    long long per_rep = 0;
    for (int l = 0; l < nl; ++l) {
        const orqa_layer_desc& L = d[l];
        if (L.n_gates < 1 || !L.gates) return fail(ctx, ORQA_EINVAL, "run_program: empty layer");
        const int kind = L.gates[0].kind;
        for (int k = 0; k < L.n_gates; ++k) {
            const orqa_gate& g = L.gates[k];
            if (g.kind != kind || g.pad != 0 || !std::isfinite(g.theta) || g.q0 < 0 || g.q0 >= ctx->n_qubits ||
                (kind != ORQA_RX && kind != ORQA_RZZ) ||
                (kind == ORQA_RZZ && (g.q1 < 0 || g.q1 >= ctx->n_qubits || g.q1 == g.q0)))
                return fail(ctx, ORQA_EINVAL, "run_program: bad gate");
        }
        if (L.theta && (kind != ORQA_RX || ctx->P == 1))
            return fail(ctx, ORQA_EINVAL, "run_program: per-problem angles are for ORQA_RX layers of a batched context");
        pl[l].kind = kind;
        pl[l].ng = L.n_gates;
        pl[l].expect_after = L.expect_after ? 1 : 0;
        per_rep += pl[l].expect_after;
        orqa_status st;
        if (kind == ORQA_RZZ) {
            st = build_zz_groups(ctx, L.gates, L.n_gates, pl[l].zz);
        } else {
            if (slot >= ROT_SLOTS) return fail(ctx, ORQA_EINVAL, "run_program: more than 16 X layers in the sequence");
            st = build_rx_run(ctx, L.gates, L.n_gates, delta, L.theta, slot++, pl[l].rx);
        }
        if (st != ORQA_OK) return st;
    }
    const long long total = per_rep * repeat * ctx->P;
    if (total > (long long)PROGRAM_RESULTS) return fail(ctx, ORQA_EINVAL, "run_program: more than 65536 results");
    *n_expect = (int)total;
    return ORQA_OK;
}

uint64_t program_key(const orqa_ctx* ctx, const orqa_layer_desc* d, int nl, int repeat, double delta) {
    uint64_t h = 0xcbf29ce484222325ull;
    const int head[13] = {ctx->W, ctx->P, ctx->fp32 ? 1 : 0, ctx->cur, repeat, ctx->range_target, ctx->sub_max,
                          ctx->n_fine, ctx->grid_per_sm, ctx->fshift, ctx->pass_limit, ctx->track_norm ? 1 : 0,
                          ctx->zz_fuse ? 1 : 0};
    h = fnv(h, head, sizeof head);
    h = fnv(h, &delta, sizeof delta);
    for (int l = 0; l < nl; ++l) {
        h = fnv(h, &d[l].n_gates, 4);
        h = fnv(h, &d[l].expect_after, 4);
        h = fnv(h, d[l].gates, sizeof(orqa_gate) * (size_t)d[l].n_gates);
        if (d[l].theta) h = fnv(h, d[l].theta, sizeof(double) * (size_t)d[l].n_gates * (size_t)ctx->P);
    }
    return h;
}

// Whether the ZZ layer li of repetition r is held back for the entry split
// of the X layer that follows it at once (no expectation between them).
bool program_holds_zz(const orqa_ctx* ctx, const std::vector<ProgLayer>& pl, size_t li, int r, int repeat) {
    const ProgLayer& L = pl[li];
    const ProgLayer* nx = li + 1 < pl.size() ? &pl[li + 1] : (r + 1 < repeat ? &pl[0] : nullptr);
    return L.kind == ORQA_RZZ && ctx->zz_fuse && !L.expect_after && L.zz.size() == 1 && nx && nx->kind == ORQA_RX;
}

#define CAPTURE_TRY(expr)                                                           \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            err = std::string(#expr) + ": " + cudaGetErrorString(e_);              \
            goto abort_capture;                                                     \
        }                                                                           \
    } while (0)

template <int W, typename T>
orqa_status capture_program(orqa_ctx* ctx, const std::vector<ProgLayer>& pl, int repeat, cudaGraph_t* out) {
    cudaStream_t saved = ctx->stream;
    const bool prof = ctx->profile;
    cudaStream_t cs = ctx->cap_stream;
    std::string err;
    int cur = ctx->cur;
    size_t off = 0;
    const int g_stream = ctx->sm_count * ctx->grid_per_sm;
    const int g_local = ctx->sm_count * lb_ctas<T>();
    cudaGraph_t graph = nullptr;
    const ZZGroups* held = nullptr;  // a ZZ layer left to the next entry split
    ctx->profile = false;
    ctx->stream = cs;
    CAPTURE_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < repeat; ++r) {
        for (size_t li = 0; li < pl.size(); ++li) {
            const ProgLayer& L = pl[li];
            if (L.kind == ORQA_RZZ) {
                if (program_holds_zz(ctx, pl, li, r, repeat))
                    held = &L.zz[0];
                else
                    for (const ZZGroups& gz : L.zz)
                        k_rzz_layer<W, T><<<g_stream, 256, 0, cs>>>(ctx->buf[cur], ctx->cap, ctx->ctr, gz);
                k_layer_end_zz<<<1, 32, 0, cs>>>(ctx->ctr, L.ng, ctx->prog_stats);
                CAPTURE_TRY(cudaGetLastError());
            } else {
                const RxLists X = rx_lists(ctx, cur);
                k_layer_begin<<<1, 32, 0, cs>>>(ctx->ctr);
                CAPTURE_TRY(cudaMemsetAsync(ctx->fcount, 0, (size_t)ctx->n_fine * 2, cs));
                if (held)
                    k_rx_split<W, T, true><<<g_stream, 256, 0, cs>>>(X.src, X.done, X.act, ctx->cap, L.rx, ctx->ctr,
                                                                     ctx->fcount, ctx->fshift, *held);
                else
                    k_rx_split<W, T, false><<<g_stream, 256, 0, cs>>>(X.src, X.done, X.act, ctx->cap, L.rx,
                                                                      ctx->ctr, ctx->fcount, ctx->fshift, kNoZZ);
                held = nullptr;
                CAPTURE_TRY(cudaGetLastError());
                cudaStreamCaptureStatus cst;
                cudaGraph_t g = nullptr;
                CAPTURE_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr));
                cudaGraphConditionalHandle h;
                CAPTURE_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
                k_pass_advance<<<1, 32, 0, cs>>>(ctx->ctr, 1, h, 1, ctx->pass_limit);
                CAPTURE_TRY(cudaGetLastError());
                const cudaGraphNode_t* deps = nullptr;
                size_t nd = 0;
                CAPTURE_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd));
                cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
                cp.conditional.handle = h;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                cudaGraphNode_t node;
                CAPTURE_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                CAPTURE_TRY(cudaStreamBeginCaptureToGraph(ctx->body_stream, body, nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeThreadLocal));
                ctx->stream = ctx->body_stream;
                int r_sc = -1, r_lo = -1;
                const orqa_status pst = enqueue_pass<W, T>(ctx, X, L.rx, g_stream, g_local, h, 1, &r_sc, &r_lo);
                ctx->stream = cs;
                cudaGraph_t body_out = nullptr;
                const cudaError_t be = cudaStreamEndCapture(ctx->body_stream, &body_out);
                if (pst != ORQA_OK || be != cudaSuccess) {
                    err = "chunk-pass capture failed: " + ctx->err + " " + cudaGetErrorString(be);
                    goto abort_capture;
                }
                CAPTURE_TRY(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1,
                                                                cudaStreamSetCaptureDependencies));
                k_layer_end_x<<<1, 32, 0, cs>>>(ctx->ctr, X.D, L.ng, ctx->prog_stats);
                CAPTURE_TRY(cudaGetLastError());
                cur = X.D;
            }
            if (L.expect_after) {
                if (enqueue_expect<W, T>(ctx, cur, 0, ctx->prog_results + off) != ORQA_OK) {
                    err = "expectation capture failed: " + ctx->err;
                    goto abort_capture;
                }
                off += (size_t)ctx->P;
            }
        }
    }
    CAPTURE_TRY(cudaStreamEndCapture(cs, &graph));
    ctx->stream = saved;
    ctx->profile = prof;
    *out = graph;
    return ORQA_OK;
abort_capture : {
    cudaGraph_t partial = nullptr;
    cudaStreamEndCapture(cs, &partial);
    if (partial) cudaGraphDestroy(partial);
    cudaGetLastError();
    ctx->stream = saved;
    ctx->profile = prof;
    return fail(ctx, ORQA_ECUDA, "run_program: " + err);
}
}

// Runs a prepared program; graph_ms (may be NULL) receives the duration of
// the graph launch measured with CUDA events on the context's stream.
template <int W, typename T>
orqa_status run_program_impl(orqa_ctx* ctx, const orqa_layer_desc* d, int nl, int repeat, double delta,
                             double* out, int64_t n_out, float* graph_ms) {
    std::vector<ProgLayer> pl;
    int n_expect = 0;
    orqa_status st = prepare_program(ctx, d, nl, repeat, delta, pl, &n_expect);
    if (st != ORQA_OK) return st;
    if (n_expect > 0 && (!out || n_out < n_expect))
        return fail(ctx, ORQA_EINVAL, "run_program: expect_out too short");
    if ((st = settle_zz(ctx)) != ORQA_OK) return st;
    // A first ZZ layer meets strings below delta only if the operator was
    // never truncated at delta; dropping them before the layer is the same
    // as after it (a ZZ layer maps strings one to one with |c| unchanged).
    if (pl[0].kind == ORQA_RZZ && delta > ctx->clean_delta && ctx->n > 0) {
        long long dropped = 0;
        if ((st = truncate_abs<W, T>(ctx, delta, &dropped)) != ORQA_OK) return st;
    }
    if (!ctx->cap_stream) {
        CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->body_stream, cudaStreamNonBlocking));
    }
    const uint64_t key = program_key(ctx, d, nl, repeat, delta);
    cudaGraphExec_t exec = nullptr;
    for (auto& p : ctx->programs)
        if (p.key == key && p.start_cur == ctx->cur) exec = p.exec;
    if (!exec) {
        // a rotation-table upload above must not overlap the capture stream's work
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        cudaGraph_t graph = nullptr;
        if ((st = capture_program<W, T>(ctx, pl, repeat, &graph)) != ORQA_OK) return st;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        if (ie != cudaSuccess) {
            cudaGraphDestroy(graph);
            return fail(ctx, ORQA_ECUDA, std::string("run_program: cudaGraphInstantiate: ") + cudaGetErrorString(ie));
        }
        for (size_t i = 0; i < ctx->programs.size(); ++i)
            if (ctx->programs[i].start_cur == ctx->cur) {
                cudaGraphExecDestroy(ctx->programs[i].exec);
                cudaGraphDestroy(ctx->programs[i].graph);
                ctx->programs.erase(ctx->programs.begin() + (long)i);
                break;
            }
        ctx->programs.push_back({key, ctx->cur, graph, exec});
    }
    const long long n_in = ctx->n;
    if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->prog_stats, 0, sizeof(ProgramStats), ctx->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (graph_ms) {
        CUDA_TRY(ctx, cudaEventCreate(&e0));
        CUDA_TRY(ctx, cudaEventCreate(&e1));
        CUDA_TRY(ctx, cudaEventRecord(e0, ctx->stream));
    }
    CUDA_TRY(ctx, cudaGraphLaunch(exec, ctx->stream));
    if (graph_ms) CUDA_TRY(ctx, cudaEventRecord(e1, ctx->stream));
    Counters h{};
    ProgramStats ps{};
    CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->ctr, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaMemcpyAsync(&ps, ctx->prog_stats, sizeof ps, cudaMemcpyDeviceToHost, ctx->stream));
    if (n_expect > 0)
        CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->prog_results, (size_t)n_expect * 8, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (graph_ms) {
        cudaEventElapsedTime(graph_ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    // the committed operator (after the last completed layer)
    ctx->cur = h.cur;
    ctx->n = (long long)h.n_live;
    ctx->norms_valid = false;
    bool any_x = false;
    for (const ProgLayer& L : pl) any_x = any_x || L.kind == ORQA_RX;
    if (any_x && ps.x_layers > 0) ctx->clean_delta = delta;
    ctx->stats.last_layer_in = n_in;
    ctx->stats.last_layer_peak = (int64_t)ps.peak;
    ctx->stats.string_gate_updates = (int64_t)ps.updates;
    ctx->stats.branch_events = (int64_t)ps.branch_events;
    ctx->stats.dropped = (int64_t)ps.dropped;
    ctx->stats.pair_updates_one = (int64_t)ps.pairs_one;
    ctx->stats.pair_updates_two = (int64_t)ps.pairs_two;
    ctx->stats.chunk_passes = (int32_t)ps.passes;
    ctx->stats.dropped_sum_sq = ctx->track_norm ? ps.dropped_sq : std::nan("");
    ctx->stats.n_strings = ctx->n;
    if (h.err) {
        // an X layer that stopped after a ZZ layer held back for it: that
        // layer is complete but not yet applied to the committed buffer
        const long long k = (long long)h.n_layers, nlay = (long long)pl.size();
        if (k >= 1 && k < nlay * repeat && program_holds_zz(ctx, pl, (size_t)((k - 1) % nlay), (int)((k - 1) / nlay),
                                                           repeat)) {
            ctx->zz_pend = pl[(size_t)((k - 1) % nlay)].zz[0];
            ctx->zz_pending = true;
        }
        char where[96];
        snprintf(where, sizeof where, "program (stopped after %u of %lld layers)", h.n_layers,
                 (long long)nl * repeat);
        h.n_done = h.n_live;
        return check_flags(ctx, h, where);
    }
    ctx->err.clear();
    return ORQA_OK;
}

}  // namespace

extern "C" {

orqa_status orqa_run_program(orqa_ctx* ctx, const orqa_layer_desc* layers, int32_t n_layers, int32_t repeat,
                             double delta, double* expect_out, int64_t n_expect_out) {
    if (!ctx) return ORQA_EINVAL;
    return ORQA_DISPATCH(ctx, run_program_impl, ctx, layers, n_layers, repeat, delta, expect_out, n_expect_out,
                         nullptr);
}

orqa_status orqa_get_tuning(orqa_ctx* ctx, orqa_tuning* out) {
    if (!ctx || !out) return ORQA_EINVAL;
    out->range_target = ctx->range_target;
    out->sub_max = ctx->sub_max;
    out->bucket_density = ctx->bucket_density;
    out->grid_per_sm = ctx->grid_per_sm;
    return ORQA_OK;
}

orqa_status orqa_set_tuning(orqa_ctx* ctx, const orqa_tuning* in) {
    if (!ctx || !in) return ORQA_EINVAL;
    if (in->range_target < MIN_RANGE_TARGET || in->range_target > 4096 || in->sub_max < 128 || in->sub_max > LB_MAX ||
        in->bucket_density < 8 || in->bucket_density > 128 ||
        in->grid_per_sm < 1 ||
        in->grid_per_sm > 32)
        return fail(ctx, ORQA_EINVAL, "set_tuning: value out of range");
    // a fine bucket holds at most bucket_density strings on average at full
    // capacity and must fit one shared-memory sub-range; units arrive in
    // clumps of up to 32 strings, so the bucket-size tail is wider than a
    // Poisson one: keep a factor 3 of margin
    if (in->sub_max < 3 * in->bucket_density)
        return fail(ctx, ORQA_EINVAL, "set_tuning: sub_max must be at least 3 x bucket_density");
    const long long nf = fine_buckets(ctx->cap, in->bucket_density);
    if (nf > ctx->n_fine_max) return fail(ctx, ORQA_EINVAL, "set_tuning: bucket arrays too small");
    ctx->range_target = in->range_target;
    ctx->sub_max = in->sub_max;
    ctx->bucket_density = in->bucket_density;
    ctx->grid_per_sm = in->grid_per_sm;
    ctx->n_fine = (int)nf;
    ctx->fshift = 64 - __builtin_ctzll((unsigned long long)nf);
    return ORQA_OK;
}

orqa_status orqa_autotune(orqa_ctx* ctx, const orqa_layer_desc* layers, int32_t n_layers, int32_t repeat,
                          double delta, int32_t trials, orqa_tuning* best, double* best_ms) {
    if (!ctx) return ORQA_EINVAL;
    if (trials < 1 || trials > 100) return fail(ctx, ORQA_EINVAL, "autotune: trials must be 1..100");
    // snapshot of the operator, restored before every run
    const long long n0 = ctx->n;
    const size_t W = (size_t)ctx->W;
    std::vector<uint64_t> x((size_t)std::max(1ll, n0) * W), z((size_t)std::max(1ll, n0) * W);
    std::vector<double> c((size_t)std::max(1ll, n0));
    std::vector<int32_t> pid((size_t)std::max(1ll, n0));
    int64_t got = 0;
    orqa_status st = orqa_export_batch(ctx, n0, x.data(), z.data(), c.data(), pid.data(), &got);
    if (st != ORQA_OK) return st;
    const double clean0 = ctx->clean_delta;
    auto restore = [&]() -> orqa_status {
        orqa_status s2 = set_from(ctx, got, x.data(), z.data(), c.data(), ctx->P > 1 ? pid.data() : nullptr,
                                  cudaMemcpyHostToDevice);
        if (s2 == ORQA_OK) ctx->clean_delta = clean0;
        return s2;
    };
    long long per_rep = 0;
    for (int l = 0; l < n_layers && layers; ++l) per_rep += layers[l].expect_after ? 1 : 0;
    std::vector<double> results((size_t)std::max(1ll, per_rep * repeat * ctx->P));
    auto measure = [&](const orqa_tuning& t, double* ms) -> orqa_status {
        orqa_status s2 = orqa_set_tuning(ctx, &t);
        if (s2 != ORQA_OK) return s2;
        double bestv = 1e300;
        for (int k = 0; k <= trials; ++k) {  // run 0 captures the graph and is not timed
            if ((s2 = restore()) != ORQA_OK) return s2;
            float g = 0.f;
            s2 = ORQA_DISPATCH(ctx, run_program_impl, ctx, layers, n_layers, repeat, delta, results.data(),
                               (int64_t)results.size(), &g);
            if (s2 != ORQA_OK) return s2;
            if (k > 0) bestv = std::min(bestv, (double)g);
        }
        *ms = bestv;
        return ORQA_OK;
    };
    orqa_tuning cur_t;
    orqa_get_tuning(ctx, &cur_t);
    const orqa_tuning start_t = cur_t;
    // a failed run leaves the starting tuning and operator in place, and the
    // message of the failure
    auto give_up = [&](orqa_status s) -> orqa_status {
        const std::string msg = ctx->err;
        orqa_set_tuning(ctx, &start_t);
        restore();
        ctx->err = msg;
        return s;
    };
    double cur_ms = 0.0;
    if ((st = measure(cur_t, &cur_ms)) != ORQA_OK) return give_up(st);
    const int targets[] = {192, 256, 320, 448, 640};
    const int subs[] = {LB_MAX / 2, LB_MAX};
    const int densities[] = {16, 32, 64, 80};
    const int grids[] = {8, 16, 32};
    for (int param = 0; param < 4; ++param) {
        const int* vals = param == 0 ? targets : param == 1 ? subs : param == 2 ? densities : grids;
        const int nv = param == 0 ? 5 : param == 1 ? 2 : param == 2 ? 4 : 3;
        for (int i = 0; i < nv; ++i) {
            orqa_tuning t = cur_t;
            int& field = param == 0 ? t.range_target : param == 1 ? t.sub_max : param == 2 ? t.bucket_density
                                                                                        : t.grid_per_sm;
            if (field == vals[i]) continue;
            field = vals[i];
            if (fine_buckets(ctx->cap, t.bucket_density) > ctx->n_fine_max) continue;
            if (t.sub_max < 3 * t.bucket_density) continue;
            double ms = 0.0;
            if ((st = measure(t, &ms)) != ORQA_OK) return give_up(st);
            if (ms < cur_ms) {
                cur_ms = ms;
                cur_t = t;
            }
        }
    }
    if ((st = orqa_set_tuning(ctx, &cur_t)) != ORQA_OK) return st;
    if ((st = restore()) != ORQA_OK) return st;
    if (best) *best = cur_t;
    if (best_ms) *best_ms = cur_ms;
    ctx->err.clear();
    return ORQA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Sharding by a hash of the z plane (orqa_shard.cuh): placement, the split
// of the strings another rank owns after a ZZ layer, and their merge-free
// arrival.
// ---------------------------------------------------------------------------
namespace {

template <int W, typename T>
orqa_status shard_split_impl(orqa_ctx* ctx, int R, int rank, long long send_cap, uint64_t* send, int64_t* counts_out) {
    const long long n = ctx->n;
    for (int r = 0; r < R; ++r) counts_out[r] = 0;
    if (n == 0) return ORQA_OK;
    unsigned long long* d_cnt = reinterpret_cast<unsigned long long*>(ctx->partials);
    unsigned long long* d_cur = d_cnt + SHARD_MAX_RANKS;
    CUDA_TRY(ctx, cudaMemsetAsync(d_cnt, 0, (size_t)R * 8, ctx->stream));
    const StrList src = ctx->buf[ctx->cur];
    k_shard_count<W><<<grid_for(ctx, n), 256, (size_t)R * 4, ctx->stream>>>(src, n, R, d_cnt);
    LAUNCH_CHECK(ctx);
    std::vector<unsigned long long> cnt((size_t)R);
    CUDA_TRY(ctx, cudaMemcpyAsync(cnt.data(), d_cnt, (size_t)R * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    const long long out = n - (long long)cnt[(size_t)rank];
    if (out > send_cap) {
        char b[160];
        snprintf(b, sizeof b, "shard_split: %lld strings leave, send buffer holds %lld", out, send_cap);
        return fail(ctx, ORQA_ECAPACITY, b);
    }
    if (out > 0 && !send) return fail(ctx, ORQA_EINVAL, "shard_split: null send buffer");
    std::vector<unsigned long long> cur((size_t)R, 0ull);
    unsigned long long run = 0;
    for (int r = 0; r < R; ++r) {
        if (r == rank) continue;
        cur[(size_t)r] = run;
        run += cnt[(size_t)r];
    }
    CUDA_TRY(ctx, cudaMemcpyAsync(d_cur, cur.data(), (size_t)R * 8, cudaMemcpyHostToDevice, ctx->stream));
    if (reset_counters(ctx) != ORQA_OK) return ORQA_ECUDA;
    const int keep = (ctx->cur + 1) % 3;
    k_shard_scatter<W, T><<<grid_for(ctx, n), 256, 0, ctx->stream>>>(src, n, R, rank, ctx->buf[keep], d_cur, send,
                                                                    send_cap, ctx->ctr);
    LAUNCH_CHECK(ctx);
    Counters h{};
    orqa_status st = sync_counters(ctx, &h);
    if (st != ORQA_OK) return st;
    if ((st = check_flags(ctx, h, "shard_split")) != ORQA_OK) return st;
    if ((long long)h.n_done != (long long)cnt[(size_t)rank]) return fail(ctx, ORQA_ECUDA, "shard_split: count mismatch");
    for (int r = 0; r < R; ++r) counts_out[r] = r == rank ? 0 : (int64_t)cnt[(size_t)r];
    return host_commit(ctx, keep, (long long)h.n_done);
}

template <int W, typename T>
orqa_status shard_append_impl(orqa_ctx* ctx, long long m, const uint64_t* recv) {
    if (m == 0) return ORQA_OK;
    k_shard_append<W, T><<<grid_for(ctx, m), 256, 0, ctx->stream>>>(recv, m, ctx->buf[ctx->cur], ctx->n);
    LAUNCH_CHECK(ctx);
    return host_commit(ctx, ctx->cur, ctx->n + m);
}

}  // namespace

extern "C" {

orqa_status orqa_shard_owner(int32_t n_qubits, int64_t n, const uint64_t* z, int32_t n_ranks, int32_t* out) {
    if (n_qubits < 1 || n_qubits > 128 || n < 0 || n_ranks < 1 || n_ranks > SHARD_MAX_RANKS ||
        (n > 0 && (!z || !out)))
        return ORQA_EINVAL;
    const int W = n_qubits <= 64 ? 1 : 2;
    for (int64_t i = 0; i < n; ++i) out[i] = shard_owner(z + i * W, W, n_ranks);
    return ORQA_OK;
}

orqa_status orqa_shard_split(orqa_ctx* ctx, int32_t n_ranks, int32_t rank, int64_t send_cap, uint64_t* send,
                             int64_t* send_counts) {
    if (!ctx) return ORQA_EINVAL;
    if (n_ranks < 1 || n_ranks > SHARD_MAX_RANKS || rank < 0 || rank >= n_ranks || send_cap < 0 || !send_counts)
        return fail(ctx, ORQA_EINVAL, "shard_split: bad arguments");
    if (ctx->P > 1) return fail(ctx, ORQA_ESTATE, "shard_split: not for batched contexts");
    orqa_status st = settle_zz(ctx);
    if (st != ORQA_OK) return st;
    st = ORQA_DISPATCH(ctx, shard_split_impl, ctx, n_ranks, rank, send_cap, send, send_counts);
    if (st == ORQA_OK) ctx->err.clear();
    return st;
}

orqa_status orqa_shard_append(orqa_ctx* ctx, int64_t n, const uint64_t* recv) {
    if (!ctx) return ORQA_EINVAL;
    if (n < 0 || (n > 0 && !recv)) return fail(ctx, ORQA_EINVAL, "shard_append: bad arguments");
    if (ctx->P > 1) return fail(ctx, ORQA_ESTATE, "shard_append: not for batched contexts");
    if (ctx->n + n > ctx->cap) return fail(ctx, ORQA_ECAPACITY, "shard_append: result exceeds capacity");
    orqa_status st = settle_zz(ctx);
    if (st != ORQA_OK) return st;
    st = ORQA_DISPATCH(ctx, shard_append_impl, ctx, n, recv);
    if (st == ORQA_OK) ctx->err.clear();
    return st;
}

}  // extern "C"
