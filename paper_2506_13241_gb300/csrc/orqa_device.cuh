// Device-side building blocks of liborqa: string planes, bit helpers,
// hashing and warp-aggregated appends.  Pauli strings are (x, z) bit planes
// of W uint64 words (see include/orqa.h); coefficients are FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace orqa {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int MAX_QUBITS = 128;
constexpr int MAX_EDGES = 1024;   // ZZ gates per kernel launch
constexpr int CHUNK_BITS = 5;     // rotation qubits per unit pass: 2^5 = one warp
constexpr int32_t SLOT_EMPTY = -1;
constexpr int32_t SLOT_BUSY = -2;
constexpr long long SPIN_LIMIT = 1LL << 22;

// String list in structure-of-arrays form.  x and z are string-major
// (word w of string i at x[i*W + w]) so that W = 2 loads as one 16-byte
// vector per plane.
struct StrList {
    uint64_t* x;
    uint64_t* z;
    double* c;
};

// Device counters shared by the kernels of one call.
struct Counters {
    unsigned long long n_done;       // strings appended to the output list
    unsigned long long n_next;       // strings appended to the next active list
    unsigned long long n_units;      // units created in the hash table
    unsigned long long unit_cursor;  // next free element slot for unit offsets
    unsigned long long branch_events;
    unsigned long long dropped;
    unsigned int overflow;           // an append would have exceeded capacity
    unsigned int timeout;            // a bounded spin-wait gave up
    unsigned int table_full;         // the hash table had no free slot
    unsigned int pad;
    double expect_partial[1];        // unused placeholder (keeps 8-byte alignment)
};

// Per-layer parameters of a run of X rotations (strictly ascending qubits).
struct RxRun {
    uint64_t mask[2];        // qubits of the run
    int32_t q_first;         // first (lowest) qubit of the run
    int32_t pad;
    double delta;            // absolute truncation threshold
    double cs[MAX_QUBITS];   // cos(theta_q), exact at Clifford angles
    double sn[MAX_QUBITS];   // sin(theta_q)
};

// ZZ layer parameters: one mode per edge.
//   mode 1: (cos, sin) = (-1, 0)  anticommuting strings change sign
//   mode 2: (cos, sin) = ( 0,-1)  z_i, z_j flip; sign flips iff the
//                                  anticommuting site was Y
//   mode 3: (cos, sin) = ( 0,+1)  z_i, z_j flip; sign flips iff it was X
struct ZZLayer {
    int32_t n_edges;
    int32_t pad;
    uint8_t qi[MAX_EDGES];
    uint8_t qj[MAX_EDGES];
    uint8_t mode[MAX_EDGES];
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

__device__ __forceinline__ int get_bit(const uint64_t* v, int q) {
    return (int)((v[q >> 6] >> (q & 63)) & 1ull);
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

template <int W>
__device__ __forceinline__ uint64_t hash_key(const uint64_t (&z)[W], const uint64_t (&xb)[W]) {
    uint64_t h = 0x9e3779b97f4a7c15ull;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        h = mix64(h ^ z[w]) + 0x632be59bd9b4e019ull;
        h = mix64(h ^ xb[w]) + 0x2545f4914f6cdd1dull;
    }
    return h;
}

// Positions (ascending) of the set bits of f whose rank among the set bits
// is in [skip, skip + CHUNK_BITS); returns how many were found and whether
// set bits of rank >= skip + CHUNK_BITS remain.
template <int W>
__device__ __forceinline__ int chunk_positions(const uint64_t (&f)[W], int skip, int (&pos)[CHUNK_BITS],
                                               bool& more) {
    int r = 0;
    more = false;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t v = f[w];
        int cnt = __popcll(v);
        if (r == CHUNK_BITS) {
            more = more || (v != 0);
            continue;
        }
        if (skip >= cnt) {
            skip -= cnt;
            continue;
        }
        while (skip > 0) {
            v &= v - 1;
            --skip;
        }
        while (v != 0 && r < CHUNK_BITS) {
            pos[r++] = 64 * w + (__ffsll((long long)v) - 1);
            v &= v - 1;
        }
        if (v != 0) more = true;
    }
    return r;
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

// Truncation test of Algorithm 1 (keep iff c != 0 and |c| >= delta) done on
// the IEEE bit patterns: for non-negative doubles the magnitude order is the
// unsigned integer order of (bits & 0x7fff...), so this is exact and costs
// no FP64 instruction (FP64 issue rate is the scarce resource on GB300).
// delta_bits is the bit pattern of delta >= 0.
__device__ __forceinline__ bool keep_bits(double v, unsigned long long delta_bits) {
    const unsigned long long m = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    return m != 0ull && m >= delta_bits;
}

__device__ __forceinline__ bool keep_coef(double v, double delta) {
    return keep_bits(v, (unsigned long long)__double_as_longlong(delta));
}

__device__ __forceinline__ bool nonzero_bits(double v) {
    return ((unsigned long long)__double_as_longlong(v) << 1) != 0ull;
}

}  // namespace orqa
