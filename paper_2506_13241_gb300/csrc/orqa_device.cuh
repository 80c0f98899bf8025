// Device-side building blocks of liborqa: string planes, bit helpers,
// hashing and warp-aggregated appends.  Pauli strings are (x, z) bit planes
// of W uint64 words (see include/orqa.h); coefficients are FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace orqa {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int MAX_QUBITS = 128;
constexpr int CHUNK_BITS = 5;     // rotation qubits per unit pass: 2^5 = one warp
constexpr int32_t SLOT_EMPTY = -1;
constexpr int32_t SLOT_BUSY = -2;
constexpr long long SPIN_LIMIT = 1LL << 22;   // default bound of every spin-wait

// String list in structure-of-arrays form.  x and z are string-major
// (word w of string i at x[i*W + w]) so that W = 2 loads as one 16-byte
// vector per plane.
struct StrList {
    uint64_t* x;
    uint64_t* z;
    double* c;
    uint64_t* h;     // per-string unit-key hash for the next chunk pass (active list only)
    int32_t* rank;   // per-string rank inside its fine bucket (active list only)
    uint16_t* pid;   // problem index per string (batched contexts), else null
};

// Error bits of Counters::err.
constexpr unsigned ERR_OVERFLOW = 1u;         // an append would have exceeded capacity
constexpr unsigned ERR_TIMEOUT = 2u;          // a bounded spin-wait gave up
constexpr unsigned ERR_TABLE_FULL = 4u;       // the merge hash table had no free slot
constexpr unsigned ERR_BUCKET_OVERFLOW = 8u;  // a CTA range exceeded its shared-memory capacity
constexpr unsigned ERR_PASS_LIMIT = 16u;      // an X layer needed more chunk passes than qubits allow
// A run of at most 128 X gates needs at most ceil(128 / CHUNK_BITS) = 26
// chunk passes; the pass loops stop (with ERR_PASS_LIMIT) beyond this.
constexpr int MAX_PASSES = 32;

// Device counters.  The fields before `err` describe the layer (or merge)
// in progress and are cleared when it starts.  `err` is sticky within a
// captured program: once set, every later layer kernel returns at once, so
// the operator of the last completed layer stays intact.  `n_live` is the
// size of the committed operator; only commit kernels and the host write it.
struct Counters {
    unsigned long long n_done;       // strings appended to the output list
    unsigned long long n_next;       // strings appended to the next active list
    unsigned long long n_units;      // units created in the hash table
    unsigned long long unit_cursor;  // next free element slot for unit offsets
    unsigned long long branch_events;
    unsigned long long dropped;
    unsigned long long pairs_one;    // pair updates with one member present (2 DMUL)
    unsigned long long pairs_two;    // pair updates with both present (4 DMUL + 2 DADD)
    unsigned long long n_active;     // strings in the active list of the current pass
    unsigned long long split_dropped;  // strings the entry split dropped
    unsigned long long peak;         // largest output + active count seen in the layer
    unsigned long long n_in;         // |O| entering the layer (captured programs)
    double dropped_sq;               // sum of c^2 over the strings truncation removed
    // The layer's string-gate updates are the sum over its gates (ascending
    // qubits) of |O| before the gate: ng n_in - split_dropped (ng - 1) +
    // upd_w, where upd_w sums, over every unit and gate, the unit's
    // population change at that gate times the number of the layer's gates
    // above it (two's complement: the sum may be negative).
    unsigned long long upd_w;
    unsigned int range_cursor;       // next CTA range of the unit kernel
    int pass;                        // chunk pass in progress
    unsigned int err;                // ERR_* bits
    unsigned int n_layers;           // layers committed since the last host reset
    unsigned long long n_live;       // |O| of the committed operator
    int cur;                         // buffer holding the committed operator
    int pad;
};

// True in every thread of the block iff an error bit is set.  The test is
// block-uniform (one read, broadcast by the barrier), so a kernel can return
// on it without leaving a warp or a barrier partly populated.  Every thread
// of the block must call it.
__device__ __forceinline__ bool block_aborted(const Counters* ctr) {
    return __syncthreads_or(threadIdx.x == 0 && *(const volatile unsigned*)&ctr->err != 0u) != 0;
}

// Totals of a captured program, accumulated on the device layer by layer.
struct ProgramStats {
    unsigned long long updates;      // sum over gates of |O| before the gate
    unsigned long long peak;         // largest intermediate set
    unsigned long long branch_events;
    unsigned long long dropped;
    unsigned long long pairs_one;
    unsigned long long pairs_two;
    unsigned long long passes;       // chunk passes of all X layers
    unsigned long long x_layers;     // X layers completed
    double dropped_sq;               // sum of c^2 of the truncated strings (with norm tracking)
};

// Per-problem rotation table of a batched X layer: entry p * MAX_QUBITS + q
// holds (cos, sin) of problem p's angle on qubit q; the FP32 table holds
// them as float pairs (cos_hi, sin_hi, cos_lo, sin_lo) with hi + lo the
// FP64 value to about 2^-48.
struct RotTable {
    const double2* f64;
    const float4* f32;
};

// Per-layer parameters of a run of X rotations (strictly ascending qubits).
struct RxRun {
    uint64_t mask[2];        // qubits of the run
    int32_t q_first;         // first (lowest) qubit of the run
    uint32_t dbits32;        // threshold as FP32 magnitude bits: smallest float >= delta
    uint64_t dbits64;        // threshold as FP64 magnitude bits
    double delta;            // absolute truncation threshold
    int32_t track_norm;      // 1: add c^2 of every string truncation removes to Counters::dropped_sq
    int32_t uniform;         // 1: every gate of the run has the same angle (and no per-problem table)
    RotTable tab;            // batched contexts: per-problem angles (else null)
    double cs[MAX_QUBITS];   // cos(theta_q), exact at Clifford angles
    double sn[MAX_QUBITS];   // sin(theta_q)
    float csf[MAX_QUBITS];   // the same as float pairs hi + lo (FP32 form)
    float snf[MAX_QUBITS];
    float cslf[MAX_QUBITS];
    float snlf[MAX_QUBITS];
};

// cos and sin of one gate in the coefficient type's arithmetic: FP64
// values, or (FP32 form) float pairs hi + lo that carry the FP64 value, so
// the rounding of cos and sin to float does not bias every product.
template <typename T>
struct Rot;

template <>
struct Rot<double> {
    double c, s;
};

template <>
struct Rot<float> {
    float c, s, cl, sl;
};

// ZZ layer parameters.  Edges of one Clifford mode form a set; a set is
// stored as offset groups: the edges (i, i + d) of the set, as the mask of
// their left endpoints i.  Sets are applied in order.
//   mode 1: (cos, sin) = (-1, 0)  anticommuting strings change sign
//   mode 2: (cos, sin) = ( 0,-1)  z_i, z_j flip; sign flips iff the
//                                  anticommuting site was Y
//   mode 3: (cos, sin) = ( 0,+1)  z_i, z_j flip; sign flips iff it was X
constexpr int MAX_ZZ_GROUPS = 256;
constexpr int MAX_ZZ_SETS = 32;

struct ZZGroups {
    int32_t n_sets;
    int32_t n_groups;
    int32_t set_mode[MAX_ZZ_SETS];
    int32_t set_end[MAX_ZZ_SETS];    // one past the set's last group
    int32_t d[MAX_ZZ_GROUPS];
    uint64_t mask[MAX_ZZ_GROUPS][2];
};

template <int W>
__device__ __forceinline__ void load_plane(const uint64_t* __restrict__ p, long long i,
                                           uint64_t (&v)[W]) {
    if constexpr (W == 2) {
        ulonglong2 t = reinterpret_cast<const ulonglong2*>(p)[i];
        v[0] = t.x;
        v[1] = t.y;
    } else {
        v[0] = p[i];
    }
}

template <int W>
__device__ __forceinline__ void load_plane_cg(const uint64_t* p, long long i, uint64_t (&v)[W]) {
    if constexpr (W == 2) {
        ulonglong2 t = __ldcg(reinterpret_cast<const ulonglong2*>(p) + i);
        v[0] = t.x;
        v[1] = t.y;
    } else {
        v[0] = __ldcg(p + i);
    }
}

template <int W>
__device__ __forceinline__ void store_plane(uint64_t* p, long long i, const uint64_t (&v)[W]) {
    if constexpr (W == 2) {
        reinterpret_cast<ulonglong2*>(p)[i] = make_ulonglong2(v[0], v[1]);
    } else {
        p[i] = v[0];
    }
}

// Register-only bit access for W-word planes (no dynamic array indexing, so
// the planes stay in registers).
// v >> d and v << d on W-word planes, 0 < d < 64 W.
template <int W>
__device__ __forceinline__ void shr_planes(const uint64_t (&v)[W], int d, uint64_t (&r)[W]) {
    if constexpr (W == 1) {
        r[0] = v[0] >> d;
    } else {
        if (d >= 64) {
            r[0] = v[1] >> (d - 64);
            r[1] = 0;
        } else {
            r[0] = (v[0] >> d) | (v[1] << (64 - d));
            r[1] = v[1] >> d;
        }
    }
}

template <int W>
__device__ __forceinline__ void shl_planes(const uint64_t (&v)[W], int d, uint64_t (&r)[W]) {
    if constexpr (W == 1) {
        r[0] = v[0] << d;
    } else {
        if (d >= 64) {
            r[1] = v[0] << (d - 64);
            r[0] = 0;
        } else {
            r[1] = (v[1] << d) | (v[0] >> (64 - d));
            r[0] = v[0] << d;
        }
    }
}

// Number of the run's gates (set bits of its 128-bit qubit mask) above q.
__device__ __forceinline__ int gates_above(const uint64_t (&m)[2], int q) {
    const uint64_t lo = q >= 64 ? 0ull : (q == 63 ? 0ull : m[0] >> (q + 1));
    const uint64_t hi = q >= 64 ? (q == 127 ? 0ull : m[1] >> (q - 63)) : m[1];
    return __popcll(lo) + __popcll(hi);
}

// One ZZ layer of Clifford angles on one string, in closed form (the rule
// is derived above k_rzz_layer): z becomes z xor C0 per set, and the return
// value is 1 iff the coefficient changes sign.
template <int W>
__device__ __forceinline__ unsigned zz_conjugate(const ZZGroups& G, const uint64_t (&x)[W], uint64_t (&z)[W]) {
    unsigned neg = 0;
    int g = 0;
    for (int k = 0; k < G.n_sets; ++k) {
        uint64_t c0[W], c1[W];
#pragma unroll
        for (int w = 0; w < W; ++w) c0[w] = c1[w] = 0;
        for (; g < G.set_end[k]; ++g) {
            const int d = G.d[g];
            uint64_t sh[W], a[W], b[W];
            shr_planes<W>(x, d, sh);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                a[w] = (x[w] ^ sh[w]) & G.mask[g][w];
                c1[w] ^= c0[w] & a[w];
                c0[w] ^= a[w];
            }
            shl_planes<W>(a, d, b);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                c1[w] ^= c0[w] & b[w];
                c0[w] ^= b[w];
            }
        }
        const int mode = G.set_mode[k];
        unsigned par = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t t;
            if (mode == 1)
                t = x[w] & c0[w];
            else if (mode == 2)
                t = x[w] & ((z[w] & c0[w]) ^ c1[w]);
            else
                t = x[w] & ((z[w] & c0[w]) ^ c1[w] ^ c0[w]);
            par ^= (unsigned)__popcll(t);
        }
        neg ^= par & 1u;
        if (mode != 1) {
#pragma unroll
            for (int w = 0; w < W; ++w) z[w] ^= c0[w];
        }
    }
    return neg;
}

template <int W>
__device__ __forceinline__ int bit_of(const uint64_t (&v)[W], int q) {
    if constexpr (W == 1) {
        return (int)((v[0] >> q) & 1ull);
    } else {
        const uint64_t w = (q < 64) ? v[0] : v[1];
        return (int)((w >> (q & 63)) & 1ull);
    }
}

template <int W>
__device__ __forceinline__ void set_bit(uint64_t (&v)[W], int q) {
    if constexpr (W == 1) {
        v[0] |= 1ull << q;
    } else {
        const uint64_t b = 1ull << (q & 63);
        if (q < 64)
            v[0] |= b;
        else
            v[1] |= b;
    }
}

template <int W>
__device__ __forceinline__ bool all_zero(const uint64_t (&v)[W]) {
    uint64_t acc = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) acc |= v[w];
    return acc == 0;
}

__device__ __forceinline__ uint64_t mix64(uint64_t h) {
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h;
}

// Hash of a (z, x) key: one odd-constant multiply per word, then the mix64
// finaliser, whose top bits pick fine buckets and low bits pick shared-memory
// slots.  Equality is always decided on the full key.
// `salt` is the problem index in batched contexts (0 otherwise), so equal
// strings of different problems land in different buckets and slots.
template <int W>
__device__ __forceinline__ uint64_t hash_key(const uint64_t (&z)[W], const uint64_t (&xb)[W],
                                             unsigned salt = 0) {
    uint64_t h = z[0] * 0x9e3779b97f4a7c15ull ^ (xb[0] * 0xc2b2ae3d27d4eb4full + 0x165667b19e3779f9ull);
    if constexpr (W == 2) {
        h ^= (z[1] * 0xd6e8feb86659fd93ull) ^ ((xb[1] * 0x94d049bb133111ebull) >> 1);
        h += 0x27d4eb2f165667c5ull;
    }
    h ^= (uint64_t)salt * 0x9fb21c651e98df25ull;
    return mix64(h);
}

// A unit-key hash carries the string's problem index in bits 16..31; fine
// buckets use the top bits and shared-memory slots the low 10 bits, so the
// embedded index changes neither.
constexpr int PID_SHIFT = 16;

__device__ __forceinline__ uint64_t with_pid(uint64_t h, unsigned pid) {
    return (h & ~(0xffffull << PID_SHIFT)) | ((uint64_t)(pid & 0xffffu) << PID_SHIFT);
}

__device__ __forceinline__ unsigned pid_of(uint64_t h) { return (unsigned)(h >> PID_SHIFT) & 0xffffu; }

// Position of the k-th set bit (0-based, k < popcount(v)) of v.
__device__ __forceinline__ int nth_set_bit(uint64_t v, int k) {
    int pos = 0;
    int c = __popc((unsigned)v);
    if (k >= c) {
        k -= c;
        v >>= 32;
        pos = 32;
    }
    unsigned w = (unsigned)v;
    c = __popc(w & 0xffffu);
    if (k >= c) {
        k -= c;
        w >>= 16;
        pos += 16;
    }
    c = __popc(w & 0xffu);
    if (k >= c) {
        k -= c;
        w >>= 8;
        pos += 8;
    }
    c = __popc(w & 0xfu);
    if (k >= c) {
        k -= c;
        w >>= 4;
        pos += 4;
    }
    c = __popc(w & 0x3u);
    if (k >= c) {
        k -= c;
        w >>= 2;
        pos += 2;
    }
    if (k >= (int)(w & 1u)) pos += 1;
    return pos;
}

// Positions (ascending) of the set bits of f whose rank is in
// [skip, skip + CHUNK_BITS) (pos, the count is returned) and in
// [skip + CHUNK_BITS, skip + 2 CHUNK_BITS) (pos2, np2), in one sweep.
template <int W>
__device__ __forceinline__ int chunk_positions2(const uint64_t (&f)[W], int skip, int (&pos)[CHUNK_BITS],
                                                int (&pos2)[CHUNK_BITS], int& np2) {
    int r = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t v = f[w];
        if (r == 2 * CHUNK_BITS) break;
        const int cnt = __popcll(v);
        if (skip >= cnt) {
            skip -= cnt;
            continue;
        }
        if (skip > 0) {
            v &= ~((1ull << nth_set_bit(v, skip)) - 1ull);
            skip = 0;
        }
        while (v != 0 && r < 2 * CHUNK_BITS) {
            const int p = 64 * w + (__ffsll((long long)v) - 1);
            if (r < CHUNK_BITS)
                pos[r] = p;
            else
                pos2[r - CHUNK_BITS] = p;
            ++r;
            v &= v - 1;
        }
    }
    np2 = r > CHUNK_BITS ? r - CHUNK_BITS : 0;
    return r < CHUNK_BITS ? r : CHUNK_BITS;
}

// chunk_positions2 with the first chunk's positions packed 7 bits each
// (position j at bits 7j .. 7j + 6; returns their count) and the second
// chunk as a bit mask m2 with np2 bits: registers only, no indexed arrays.
template <int W>
__device__ __forceinline__ int chunk_positions2_packed(const uint64_t (&f)[W], int skip, uint64_t& packed,
                                                       uint64_t (&m2)[W], int& np2) {
    int r = 0;
    packed = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) m2[w] = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t v = f[w];
        if (r == 2 * CHUNK_BITS) break;
        const int cnt = __popcll(v);
        if (skip >= cnt) {
            skip -= cnt;
            continue;
        }
        if (skip > 0) {
            v &= ~((1ull << nth_set_bit(v, skip)) - 1ull);
            skip = 0;
        }
        while (v != 0 && r < 2 * CHUNK_BITS) {
            const int b = __ffsll((long long)v) - 1;
            if (r < CHUNK_BITS)
                packed |= (uint64_t)(64 * w + b) << (7 * r);
            else
                m2[w] |= 1ull << b;
            ++r;
            v &= v - 1;
        }
    }
    np2 = r > CHUNK_BITS ? r - CHUNK_BITS : 0;
    return r < CHUNK_BITS ? r : CHUNK_BITS;
}

__device__ __forceinline__ int packed_pos(uint64_t packed, int j) { return (int)((packed >> (7 * j)) & 127u); }

// Mask m of the set bits of f whose rank among the set bits is in
// [skip, skip + CHUNK_BITS) (the chunk of one pass); returns their count.
template <int W>
__device__ __forceinline__ int chunk_mask(const uint64_t (&f)[W], int skip, uint64_t (&m)[W]) {
    int r = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        m[w] = 0;
        uint64_t v = f[w];
        const int cnt = __popcll(v);
        if (r == CHUNK_BITS || skip >= cnt) {
            skip = r == CHUNK_BITS ? skip : skip - cnt;
            continue;
        }
        if (skip > 0) {
            v &= ~((1ull << nth_set_bit(v, skip)) - 1ull);
            skip = 0;
        }
        // the lowest CHUNK_BITS - r set bits of v
        const int take = min(__popcll(v), CHUNK_BITS - r);
        const uint64_t above = take < __popcll(v) ? ~((1ull << nth_set_bit(v, take)) - 1ull) : 0ull;
        m[w] = v & ~above;
        r += take;
    }
    return r;
}

// The bits of x at the positions of mask m, in ascending order (a unit slot).
template <int W>
__device__ __forceinline__ int gather_bits(const uint64_t (&x)[W], const uint64_t (&m)[W]) {
    int idx = 0, j = 0;
#pragma unroll
    for (int w = 0; w < W; ++w)
        for (uint64_t v = m[w]; v; v &= v - 1, ++j) idx |= (int)((x[w] >> (__ffsll((long long)v) - 1)) & 1ull) << j;
    return idx;
}

// Hash of a string's unit key for chunk pass `pass`: z, and x with the
// chunk's bits cleared (the unit definition of the layer kernels).
template <int W>
__device__ __forceinline__ uint64_t unit_hash(const uint64_t (&x)[W], const uint64_t (&z)[W], const uint64_t* mask,
                                              int pass, unsigned pid) {
    uint64_t f[W], m[W], xb[W];
#pragma unroll
    for (int w = 0; w < W; ++w) f[w] = z[w] & mask[w];
    chunk_mask<W>(f, CHUNK_BITS * pass, m);
#pragma unroll
    for (int w = 0; w < W; ++w) xb[w] = x[w] & ~m[w];
    return with_pid(hash_key<W>(z, xb, pid), pid);
}

// Warp-aggregated append: every lane of a full warp calls it; lanes with
// pred get consecutive slots.  Returns the slot (or -1 if !pred).
__device__ __forceinline__ long long warp_append(bool pred, unsigned long long* cursor) {
    unsigned m = __ballot_sync(FULL_MASK, pred);
    if (m == 0) return -1;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(cursor, (unsigned long long)__popc(m));
    base = __shfl_sync(FULL_MASK, base, leader);
    if (!pred) return -1;
    return (long long)(base + __popc(m & ((1u << lane) - 1u)));
}

// Sum of a 64-bit value over a full warp (every lane calls it; all lanes
// receive the total), exact for per-lane values below 2^59: the low 16,
// middle 16 and high 32 bits are summed separately in 32 bits (at most
// 32 * (2^16 - 1) and 32 * 2^27), so a warp's total may exceed 2^32.
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
    const unsigned lo = __reduce_add_sync(FULL_MASK, (unsigned)(v & 0xffffu));
    const unsigned mid = __reduce_add_sync(FULL_MASK, (unsigned)((v >> 16) & 0xffffu));
    const unsigned hi = __reduce_add_sync(FULL_MASK, (unsigned)(v >> 32));
    return (unsigned long long)lo + ((unsigned long long)mid << 16) + ((unsigned long long)hi << 32);
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL_MASK, v, d);
    return v;
}

// Coefficient types: FP64 (the default) and FP32 (ORQA_FLAG_FP32).  Zero and
// threshold tests are integer tests on the magnitude bits of the stored
// type; thresholds arrive as magnitude bits of that type.
template <typename T>
struct Coef;

template <>
struct Coef<double> {
    __device__ static unsigned long long mag(double v) {
        return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    }
    __device__ static double negate(double v) {
        return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
    }
    __device__ static unsigned long long to_slot(double v) { return (unsigned long long)__double_as_longlong(v); }
    __device__ static double from_slot(unsigned long long b) { return __longlong_as_double((long long)b); }
    __device__ static unsigned long long threshold(const RxRun& r) { return r.dbits64; }
    // (cos, sin) of problem p's angle on qubit q
    __device__ static Rot<double> rot(const RxRun& r, unsigned p, int q) {
        if (r.tab.f64) {
            const double2 v = r.tab.f64[p * MAX_QUBITS + q];
            return {v.x, v.y};
        }
        return {r.cs[q], r.sn[q]};
    }
};

template <>
struct Coef<float> {
    __device__ static unsigned long long mag(float v) { return (unsigned long long)(__float_as_uint(v) & 0x7fffffffu); }
    __device__ static float negate(float v) { return __uint_as_float(__float_as_uint(v) ^ 0x80000000u); }
    __device__ static unsigned long long to_slot(float v) { return (unsigned long long)__float_as_uint(v); }
    __device__ static float from_slot(unsigned long long b) { return __uint_as_float((unsigned)b); }
    __device__ static unsigned long long threshold(const RxRun& r) { return r.dbits32; }
    __device__ static Rot<float> rot(const RxRun& r, unsigned p, int q) {
        if (r.tab.f32) {
            const float4 v = r.tab.f32[p * MAX_QUBITS + q];
            return {v.x, v.y, v.z, v.w};
        }
        return {r.csf[q], r.snf[q], r.cslf[q], r.snlf[q]};
    }
};

// Truncation test of Algorithm 1 (keep iff c != 0 and |c| >= delta) on the
// IEEE bit patterns: for non-negative values the magnitude order is the
// unsigned order of the magnitude bits, so the test is exact and uses no
// floating-point instruction (FP64 issue is the scarce resource on GB300).
// tbits: the threshold as magnitude bits of T.
template <typename T>
__device__ __forceinline__ bool keep_t(T v, unsigned long long tbits) {
    const unsigned long long m = Coef<T>::mag(v);
    return m != 0ull && m >= tbits;
}

// a*b + c*d (+ a small correction `extra`) in FP32 with the compensated
// scheme Dot2 (Ogita, Rump, Oishi 2005): exact products by FMA
// (TwoProduct), exact sum by TwoSum, and the error terms added before the
// final rounding.
__device__ __forceinline__ float dot2f(float a, float b, float c, float d, float extra) {
    const float p = __fmul_rn(a, b), ep = __fmaf_rn(a, b, -p);
    const float q = __fmul_rn(c, d), eq = __fmaf_rn(c, d, -q);
    const float s = __fadd_rn(p, q);
    const float t = __fsub_rn(s, p);
    const float es = __fadd_rn(__fsub_rn(p, __fsub_rn(s, t)), __fsub_rn(q, t));
    return __fadd_rn(s, __fadd_rn(es, __fadd_rn(__fadd_rn(ep, eq), extra)));
}

// (hi + lo) * v rounded once to float: TwoProduct of hi * v plus lo * v.
__device__ __forceinline__ float mul_pair(float hi, float lo, float v) {
    const float p = __fmul_rn(hi, v);
    const float e = __fmaf_rn(hi, v, -p);
    return __fadd_rn(p, __fmaf_rn(lo, v, e));
}

// One-member pair (Eq. update_rule with the partner absent): (cos v, sin v).
__device__ __forceinline__ void one_member(const Rot<float>& r, float v, float& pc, float& ps) {
    pc = mul_pair(r.c, r.cl, v);
    ps = mul_pair(r.s, r.sl, v);
}

// Pair update of Eq. (update_rule) with both members present:
// (c_Z, c_Y) -> (cos c_Z - sin c_Y, cos c_Y + sin c_Z).
__device__ __forceinline__ void pair_update(const Rot<float>& r, float a, float b, float& na, float& nb) {
    na = dot2f(r.c, a, -r.s, b, __fmaf_rn(r.cl, a, -__fmul_rn(r.sl, b)));
    nb = dot2f(r.c, b, r.s, a, __fmaf_rn(r.cl, b, __fmul_rn(r.sl, a)));
}

// One entry of a level's pair list, either case: u1 is the coefficient of
// the present member (c_Z of a two-member pair), u2 that of the other
// member (c_Y), or u1 again when the pair has one member; y_side says that
// member is the sigma_y string.  Two members: (cos c_Z - sin c_Y,
// cos c_Y + sin c_Z), every product and sum rounded once in that order.
// One member: (cos c, sin c) at sigma_z, (-sin c, cos c) at sigma_y.  In
// FP64, cos u1 and sin u2 serve both cases (a one-member pair needs exactly
// those two products), so entries of both kinds share one pass of a list.
__device__ __forceinline__ void pair_entry(const Rot<double>& r, double u1, double u2, bool two, bool y_side,
                                           double& na, double& nb) {
    const double p = __dmul_rn(r.c, u1), q = __dmul_rn(r.s, u2);
    if (two) {
        na = __dsub_rn(p, q);
        nb = __dadd_rn(__dmul_rn(r.c, u2), __dmul_rn(r.s, u1));
    } else {
        // sigma_z present: (cos c, sin c); sigma_y present: (-sin c, cos c)
        na = y_side ? Coef<double>::negate(q) : p;
        nb = y_side ? p : q;
    }
}

// A pair with one member present, u its coefficient: exactly the one-member
// case of pair_entry (cos u, sin u at sigma_z; -sin u, cos u at sigma_y).
__device__ __forceinline__ void lone_entry(const Rot<double>& r, double u, bool y_side, double& na, double& nb) {
    const double p = __dmul_rn(r.c, u), q = __dmul_rn(r.s, u);
    na = y_side ? Coef<double>::negate(q) : p;
    nb = y_side ? p : q;
}

__device__ __forceinline__ void lone_entry(const Rot<float>& r, float u, bool y_side, float& na, float& nb) {
    float p, q;
    one_member(r, u, p, q);
    na = y_side ? Coef<float>::negate(q) : p;
    nb = y_side ? p : q;
}

__device__ __forceinline__ void pair_entry(const Rot<float>& r, float u1, float u2, bool two, bool y_side,
                                           float& na, float& nb) {
    if (two) {
        pair_update(r, u1, u2, na, nb);
    } else {
        float p, q;
        one_member(r, u1, p, q);
        na = y_side ? Coef<float>::negate(q) : p;
        nb = y_side ? p : q;
    }
}

}  // namespace orqa
