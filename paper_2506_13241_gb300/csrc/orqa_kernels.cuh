// Kernels of liborqa.  Each kernel cites the passage of arXiv 2506.13241
// whose operation it performs.  Coefficient products and sums use explicit
// round-to-nearest intrinsics (no FMA contraction), so a coefficient is
// fl(fl(cos*a) +- fl(sin*b)) exactly as the per-gate update of Eq.
// (update_rule) evaluates it on a CPU.
#pragma once

#include "orqa_device.cuh"

namespace orqa {

// ---------------------------------------------------------------------------
// ZZ layer (Clifford).  Conjugation by exp(-i theta/2 Z_i Z_j) at theta a
// multiple of pi/2 (Eq. eq:u with theta_zz = -pi/2; Eq. update_rule with
// cos in {0, +-1}).  A string anticommutes with Z_i Z_j iff x_i xor x_j = 1;
// for cos = 0 its image is the single string with z_i, z_j flipped and
// coefficient (-1)^((B+1)/2) sin(theta) c, which for sin = -1 flips the sign
// iff the anticommuting site (the endpoint with x = 1) is Y before the gate.
//
// All gates of a set commute, so the set is applied in closed form.  Let
// n_s be the number of anticommuting edges at site s (neighbours t with
// x_t != x_s) and C0, C1 the planes of its bits 0 and 1.  Every such edge
// flips z_s, so z' = z xor C0.  Taking the edges in any order, the sign
// flips once per edge whose x = 1 endpoint s has odd z_s at that moment:
// z_s(original) summed over the n_s edges at s, plus one flip per pair of
// edges at s (the earlier one flips z_s for the later one), i.e.
//   sign(sin = -1) = parity(x & ((z & C0) ^ C1)),
//   sign(sin = +1) = parity(x & ((z & C0) ^ C1 ^ C0))   (flip iff X),
//   sign(cos = -1) = parity(x & C0)                      (one per edge).
// C0, C1 come from offset groups: the anticommuting edges (i, i + d) of a
// group are a = (x ^ (x >> d)) & mask, counted at i (a) and at i + d
// (a << d) by a 2-bit carry-save counter.  In place: one read of x, z, c and
// one write of z, c per string.
// ---------------------------------------------------------------------------
// The operator is the committed one (n = n_live strings, read on the device).
template <int W, typename T>
__global__ void __launch_bounds__(256) k_rzz_layer(StrList s, long long cap, Counters* ctr,
                                                   const __grid_constant__ ZZGroups G) {
    if (block_aborted(ctr)) return;
    const long long n = min((long long)ctr->n_live, cap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t x[W], z[W];
        load_plane<W>(s.x, i, x);
        load_plane<W>(s.z, i, z);
        const unsigned neg = zz_conjugate<W>(G, x, z);
        store_plane<W>(s.z, i, z);
        if (neg) {
            T* c = reinterpret_cast<T*>(s.c) + i;
            *c = Coef<T>::negate(*c);
        }
    }
}

// ---------------------------------------------------------------------------
// Stand-alone truncation (the truncate loop of Algorithm 1): copies the
// strings that are kept to dst, order-preserving within a warp,
// warp-aggregated appends.  Absolute form: keep iff c != 0 and |c| >= delta.
// Relative form (Eq. truncation1, STRICT): keep iff c != 0 and |c| > thr,
// thr = eps0 * max|c|.  Both are integer tests on the magnitude bits of the
// stored type (tbits: the threshold in that type, rounded so that the test
// on the stored value equals the test against the FP64 threshold).
// ---------------------------------------------------------------------------
template <int W, typename T, bool STRICT>
__global__ void __launch_bounds__(256) k_truncate(StrList src, long long n, StrList dst,
                                                  long long cap, unsigned long long tbits, Counters* ctr) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n + 31) & ~31ll;
    const T* __restrict__ sc = reinterpret_cast<const T*>(src.c);
    double drop_sq = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        T c = 0;
        if (i < n) c = sc[i];
        const unsigned long long m = Coef<T>::mag(c);
        const bool keep = (i < n) && (STRICT ? (m > tbits) : keep_t<T>(c, tbits));
        if (i < n && !keep) drop_sq = fma((double)c, (double)c, drop_sq);
        const long long slot = warp_append(keep, &ctr->n_done);
        if (keep) {
            if (slot < cap) {
                uint64_t x[W], z[W];
                load_plane<W>(src.x, i, x);
                load_plane<W>(src.z, i, z);
                store_plane<W>(dst.x, slot, x);
                store_plane<W>(dst.z, slot, z);
                reinterpret_cast<T*>(dst.c)[slot] = c;
                if (dst.pid) dst.pid[slot] = src.pid[i];
            } else {
                atomicOr(&ctr->err, ERR_OVERFLOW);
            }
        }
    }
    drop_sq = warp_sum_f64(drop_sq);  // the loop is warp-uniform (n_round and stride are multiples of 32)
    if ((threadIdx.x & 31) == 0 && drop_sq != 0.0) atomicAdd(&ctr->dropped_sq, drop_sq);
}

// max |c| as the largest magnitude bit pattern (exact: for non-negative
// doubles the order of the bit patterns is the order of the values).
template <typename T>
__global__ void __launch_bounds__(256) k_absmax(const T* c, long long n, unsigned long long* out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long m = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        m = max(m, Coef<T>::mag(c[i]));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_down_sync(FULL_MASK, m, d));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// ---------------------------------------------------------------------------
// Duplicate merge, step 1 (the insert-or-add of Algorithm 1 for an arbitrary
// input): each string finds or creates its entry in an open-addressing hash
// table keyed by the whole string and takes a rank among its duplicates.
// Entries ("units") are numbered in creation order with warp-aggregated
// counters; a waiting lane spins on a slot another thread is publishing, with
// an iteration limit that sets the timeout flag.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256) k_merge_assign(StrList src, long long n, int32_t* table,
                                                      long long table_mask, uint64_t* unit_z, uint64_t* unit_x,
                                                      uint16_t* unit_pid, int32_t* unit_count, int32_t* uid_out,
                                                      int32_t* rank_out, Counters* ctr, long long spin_limit) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n + 31) & ~31ll;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        uint64_t x[W], z[W];
        bool done = i >= n;
        long long slot = 0;
        unsigned pid = 0;
        if (!done) {
            load_plane<W>(src.x, i, x);
            load_plane<W>(src.z, i, z);
            if (src.pid) pid = src.pid[i];
            slot = (long long)(hash_key<W>(z, x, pid) & (uint64_t)table_mask);
        }
        int my_uid = -1;
        long long probes = 0;
        while (__any_sync(FULL_MASK, !done)) {
            int v = SLOT_EMPTY;
            bool claimed = false;
            if (!done) {
                v = atomicCAS(&table[slot], SLOT_EMPTY, SLOT_BUSY);
                claimed = (v == SLOT_EMPTY);
            }
            const long long u = warp_append(claimed, &ctr->n_units);
            if (claimed) {
                store_plane<W>(unit_z, u, z);
                store_plane<W>(unit_x, u, x);
                if (unit_pid) unit_pid[u] = (uint16_t)pid;
                unit_count[u] = 0;
                __threadfence();
                atomicExch(&table[slot], (int32_t)u);
                my_uid = (int)u;
                done = true;
            }
            __syncwarp();
            if (!done) {
                long long spins = 0;
                while (v == SLOT_BUSY && spins < spin_limit) {
                    v = *((volatile int32_t*)&table[slot]);
                    ++spins;
                }
                if (v == SLOT_BUSY) {
                    atomicOr(&ctr->err, ERR_TIMEOUT);
                    done = true;
                } else {
                    __threadfence();
                    uint64_t kz[W], kx[W];
                    load_plane_cg<W>(unit_z, v, kz);
                    load_plane_cg<W>(unit_x, v, kx);
                    bool eq = !unit_pid || __ldcg(unit_pid + v) == (uint16_t)pid;
#pragma unroll
                    for (int w = 0; w < W; ++w) eq = eq && (kz[w] == z[w]) && (kx[w] == x[w]);
                    if (eq) {
                        my_uid = v;
                        done = true;
                    } else {
                        slot = (slot + 1) & table_mask;
                        if (++probes > table_mask) {
                            atomicOr(&ctr->err, ERR_TABLE_FULL);
                            done = true;
                        }
                    }
                }
            }
        }
        if (i < n) {
            uid_out[i] = my_uid;
            if (my_uid >= 0) rank_out[i] = atomicAdd(&unit_count[my_uid], 1);
        }
    }
}

// Marks every slot of the merge hash table as being published (a test hook
// of the bounded wait above: every insertion then waits until its limit).
__global__ void k_fill_busy(int32_t* table, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        table[i] = SLOT_BUSY;
}

// Gives every unit a contiguous element range (in arbitrary unit order):
// a warp scan of the counts plus one atomic per warp.
__global__ void __launch_bounds__(256) k_merge_offsets(const int32_t* unit_count,
                                                      long long* unit_off, Counters* ctr) {
    const long long nu = (long long)*((volatile unsigned long long*)&ctr->n_units);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (nu + 31) & ~31ll;
    const int lane = threadIdx.x & 31;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n_round; u += stride) {
        const int cnt = (u < nu) ? unit_count[u] : 0;
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(FULL_MASK, incl, d);
            if (lane >= d) incl += t;
        }
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(&ctr->unit_cursor, (unsigned long long)incl);
        base = __shfl_sync(FULL_MASK, base, 31);
        if (u < nu) unit_off[u] = (long long)base + incl - cnt;
    }
}

// Moves each string's coefficient into its entry's range (as FP64: the
// duplicates of an entry are summed in an FP64 accumulator).
template <typename Tin>
__global__ void __launch_bounds__(256) k_merge_scatter(const Tin* c, long long n, const int32_t* uid,
                                                       const int32_t* rank, const long long* unit_off,
                                                       double* sorted_c) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int u = uid[i];
        if (u < 0) continue;
        sorted_c[unit_off[u] + rank[i]] = (double)c[i];
    }
}

// ---------------------------------------------------------------------------
// Duplicate merge, step 4: one thread per entry sums the coefficients of its
// equal strings and keeps the sum if it is non-zero and not below delta.
// ---------------------------------------------------------------------------
template <int W, typename Tout>
__global__ void __launch_bounds__(256) k_merge_reduce(const uint64_t* unit_z,
                                                      const uint64_t* unit_xb,
                                                      const uint16_t* unit_pid,
                                                      const int32_t* unit_count,
                                                      const long long* unit_off,
                                                      const double* sorted_c, unsigned long long tbits,
                                                      StrList dst, long long cap, Counters* ctr) {
    const long long nu = (long long)*((volatile unsigned long long*)&ctr->n_units);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (nu + 31) & ~31ll;
    double drop_sq = 0.0;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n_round; u += stride) {
        double acc = 0.0;
        if (u < nu) {
            const int m = unit_count[u];
            const long long off = unit_off[u];
            acc = sorted_c[off];
            for (int e = 1; e < m; ++e) acc = __dadd_rn(acc, sorted_c[off + e]);
        }
        const Tout v = (Tout)acc;
        const bool keep = (u < nu) && keep_t<Tout>(v, tbits);
        const long long slot = warp_append(keep, &ctr->n_done);
        if (keep) {
            if (slot < cap) {
                uint64_t z[W], x[W];
                load_plane<W>(unit_z, u, z);
                load_plane<W>(unit_xb, u, x);
                store_plane<W>(dst.x, slot, x);
                store_plane<W>(dst.z, slot, z);
                reinterpret_cast<Tout*>(dst.c)[slot] = v;
                if (dst.pid) dst.pid[slot] = unit_pid[u];
            } else {
                atomicOr(&ctr->err, ERR_OVERFLOW);
            }
        } else if (u < nu) {
            atomicAdd(&ctr->dropped, 1ull);
            const double v64 = (double)v;
            drop_sq = fma(v64, v64, drop_sq);
        }
    }
    drop_sq = warp_sum_f64(drop_sq);  // the loop is warp-uniform
    if ((threadIdx.x & 31) == 0 && drop_sq != 0.0) atomicAdd(&ctr->dropped_sq, drop_sq);
}

// ---------------------------------------------------------------------------
// <0|O|0> (Eq. magnetization): sum of c over strings with x = 0.  Per-block
// partial sums in a fixed grid, then one thread adds them in block order.
// ---------------------------------------------------------------------------
constexpr int EXPECT_BLOCKS = 1024;

// n = n_live strings of the committed operator, read on the device.
template <int W, typename T>
__global__ void __launch_bounds__(256) k_expect_partial(StrList s, long long cap, const Counters* ctr,
                                                        double* partials) {
    __shared__ double red[8];
    const long long n = min((long long)ctr->n_live, cap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    double acc = 0.0;
    const T* __restrict__ c = reinterpret_cast<const T*>(s.c);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t x[W];
        load_plane<W>(s.x, i, x);
        if (all_zero<W>(x)) acc = __dadd_rn(acc, (double)c[i]);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(FULL_MASK, acc, d));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b = __dadd_rn(b, red[k]);
        partials[blockIdx.x] = b;
    }
}

// One warp adds the block partials in a fixed order: lane l sums partials
// l, l+32, ... in sequence, then a fixed shuffle tree combines the lanes.
__global__ void k_expect_final(const double* partials, int nblocks, double* out, const Counters* ctr) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32 || blockIdx.x != 0) return;
    double acc = 0.0;
    for (int k = lane; k < nblocks; k += 32) acc = __dadd_rn(acc, partials[k]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(FULL_MASK, acc, d));
    if (lane == 0) *out = ctr->err ? __longlong_as_double(0x7ff8000000000000ll) : acc;  // NaN after an error
}

// ---------------------------------------------------------------------------
// Norms of the committed operator: sum of c^2 (FP64, per-block partials in
// a fixed grid, then added in block order, so the result does not depend on
// timing) and max |c| (exact, as the largest magnitude bit pattern).  They
// carry the unitarity invariant of Eq. (update_rule): a rotation keeps sum
// c^2, so between two layers it falls exactly by the sum of c^2 that the
// truncation of Eq. (truncation1) removes (up to rounding).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_norms_partial(const T* c, long long cap, const Counters* ctr,
                                                       double* partials, unsigned long long* max_bits) {
    __shared__ double red[8];
    const long long n = min((long long)ctr->n_live, cap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    double acc = 0.0;
    unsigned long long m = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T v = c[i];
        const double d = (double)v;
        acc = __dadd_rn(acc, __dmul_rn(d, d));
        m = max(m, Coef<T>::mag(v));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        acc = __dadd_rn(acc, __shfl_down_sync(FULL_MASK, acc, d));
        m = max(m, __shfl_down_sync(FULL_MASK, m, d));
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = acc;
        if (m) atomicMax(max_bits, m);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b = __dadd_rn(b, red[k]);
        partials[blockIdx.x] = b;
    }
}

// ---------------------------------------------------------------------------
// <0|O_p|0> of every problem p of a batched context.  Each block adds the
// diagonal strings it meets into per-problem shared-memory accumulators;
// the block partials of problem p are then added in block order.
// ---------------------------------------------------------------------------
constexpr int EXPECT_BATCH_BLOCKS = 256;

template <int W, typename T>
__global__ void __launch_bounds__(256) k_expect_batch_partial(StrList s, long long cap, const Counters* ctr,
                                                              int n_problems, double* partials) {
    extern __shared__ double acc_p[];
    for (int p = threadIdx.x; p < n_problems; p += blockDim.x) acc_p[p] = 0.0;
    __syncthreads();
    const long long n = min((long long)ctr->n_live, cap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const T* __restrict__ c = reinterpret_cast<const T*>(s.c);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t x[W];
        load_plane<W>(s.x, i, x);
        if (all_zero<W>(x)) atomicAdd(&acc_p[s.pid[i]], (double)c[i]);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n_problems; p += blockDim.x)
        partials[(long long)blockIdx.x * n_problems + p] = acc_p[p];
}

__global__ void __launch_bounds__(256) k_expect_batch_final(const double* partials, int nblocks, int n_problems,
                                                            double* out, const Counters* ctr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_problems) return;
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc = __dadd_rn(acc, partials[(long long)b * n_problems + p]);
    out[p] = ctr->err ? __longlong_as_double(0x7ff8000000000000ll) : acc;  // NaN after an error
}

// Live strings per problem.
__global__ void __launch_bounds__(256) k_problem_sizes(const uint16_t* pid, long long cap, const Counters* ctr,
                                                       int n_problems, unsigned long long* out) {
    extern __shared__ unsigned cnt_p[];
    for (int p = threadIdx.x; p < n_problems; p += blockDim.x) cnt_p[p] = 0u;
    __syncthreads();
    const long long n = min((long long)ctr->n_live, cap);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt_p[pid[i]], 1u);
    __syncthreads();
    for (int p = threadIdx.x; p < n_problems; p += blockDim.x)
        if (cnt_p[p]) atomicAdd(&out[p], (unsigned long long)cnt_p[p]);
}

// Commit of a layer computed into buffer `cur`: its output list becomes the
// operator.  Skipped after an error, so the last completed layer's operator
// stays committed.
__global__ void k_commit(Counters* ctr, int cur) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || ctr->err) return;
    ctr->n_live = ctr->n_done;
    ctr->cur = cur;
    ctr->n_layers += 1;
}

// ---------------------------------------------------------------------------
// Rotation about a general Pauli string J (Eq. update_rule for any sigma_J).
// U^dagger P U for U = exp(-i theta J / 2) is P when P commutes with J and
// cos(theta) P + i sin(theta) J P otherwise, with J P = i^B(J,P) sigma_{J xor P}
// and B odd, so the child's factor is i^(1 + B): -1 for B = 1, +1 for B = 3.
// B(J, P) mod 4 is counted per qubit from the single-qubit products (XY, YZ,
// ZX give +1; XZ, YX, ZY give -1).  Each string writes itself (cos c) and,
// if it anticommutes, its child (+-sin c) to a staging list; the duplicate
// merge then sums the at most two terms of every string and truncates.
// ---------------------------------------------------------------------------
struct PauliGen {
    uint64_t x[2], z[2];     // J as planes
    double c, s;             // cos(theta), sin(theta), exact at Clifford angles
    float ch, sh, cl, sl;    // the same as float pairs hi + lo (FP32 form)
};

template <int W>
__device__ __forceinline__ int phase_exponent_jp(const PauliGen& J, const uint64_t (&x)[W], const uint64_t (&z)[W]) {
    int plus = 0, minus = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint64_t jx = J.x[w] & ~J.z[w], jy = J.x[w] & J.z[w], jz = ~J.x[w] & J.z[w];
        const uint64_t px = x[w] & ~z[w], py = x[w] & z[w], pz = ~x[w] & z[w];
        plus += __popcll((jx & py) | (jy & pz) | (jz & px));
        minus += __popcll((jx & pz) | (jy & px) | (jz & py));
    }
    return (plus - minus) & 3;
}

template <typename T>
__device__ __forceinline__ void pauli_products(const PauliGen& J, T v, T& pc, T& ps);

template <>
__device__ __forceinline__ void pauli_products<double>(const PauliGen& J, double v, double& pc, double& ps) {
    pc = __dmul_rn(J.c, v);
    ps = __dmul_rn(J.s, v);
}

template <>
__device__ __forceinline__ void pauli_products<float>(const PauliGen& J, float v, float& pc, float& ps) {
    pc = mul_pair(J.ch, J.cl, v);
    ps = mul_pair(J.sh, J.sl, v);
}

template <int W, typename T>
__global__ void __launch_bounds__(256) k_pauli_expand(StrList src, long long n, StrList dst, long long cap,
                                                      const __grid_constant__ PauliGen J, Counters* ctr) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n + 31) & ~31ll;
    const int lane = threadIdx.x & 31;
    const T* __restrict__ sc = reinterpret_cast<const T*>(src.c);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        uint64_t x[W], z[W];
        T c = 0;
        unsigned anti = 0, pid = 0;
        const bool live = i < n;
        if (live) {
            load_plane<W>(src.x, i, x);
            load_plane<W>(src.z, i, z);
            c = sc[i];
            if (src.pid) pid = src.pid[i];
#pragma unroll
            for (int w = 0; w < W; ++w) anti ^= (unsigned)__popcll((x[w] & J.z[w]) ^ (z[w] & J.x[w]));
            anti &= 1u;
        }
        const unsigned cnt = live ? 1u + anti : 0u;
        unsigned incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned t = __shfl_up_sync(FULL_MASK, incl, d);
            if (lane >= d) incl += t;
        }
        const unsigned total = __shfl_sync(FULL_MASK, incl, 31);
        unsigned long long base = 0;
        if (lane == 31 && total) base = atomicAdd(&ctr->n_done, (unsigned long long)total);
        base = __shfl_sync(FULL_MASK, base, 31);
        const unsigned nb = __popc(__ballot_sync(FULL_MASK, anti != 0));
        if (lane == 0 && nb) atomicAdd(&ctr->branch_events, (unsigned long long)nb);
        if (!live) continue;
        long long slot = (long long)(base + incl - cnt);
        T keep = c, child = 0;
        if (anti) {
            T ps;
            pauli_products<T>(J, c, keep, ps);
            child = (phase_exponent_jp<W>(J, x, z) == 1) ? Coef<T>::negate(ps) : ps;
        }
        if (slot + (long long)cnt > cap) {
            atomicOr(&ctr->err, ERR_OVERFLOW);
            continue;
        }
        store_plane<W>(dst.x, slot, x);
        store_plane<W>(dst.z, slot, z);
        reinterpret_cast<T*>(dst.c)[slot] = keep;
        if (dst.pid) dst.pid[slot] = (uint16_t)pid;
        if (anti) {
            ++slot;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                x[w] ^= J.x[w];
                z[w] ^= J.z[w];
            }
            store_plane<W>(dst.x, slot, x);
            store_plane<W>(dst.z, slot, z);
            reinterpret_cast<T*>(dst.c)[slot] = child;
            if (dst.pid) dst.pid[slot] = (uint16_t)pid;
        }
    }
}

// ---------------------------------------------------------------------------
// Pauli-string density D_t(x) (App. D): counts of the live strings by sign
// and by bin of |x| = |c| / max|c|.  tbits[k] (k = 0..n_bins) are the
// magnitude bits, in the stored type, of the bin edges t_k = max * e_k
// (ascending, t_n_bins = max); bin k holds t_k <= |c| < t_{k+1} (the last
// bin also |c| = max), and bin n_bins counts |c| < t_0.  counts[s * (n_bins
// + 1) + k] with s = 0 for c > 0 and s = 1 for c < 0.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_histogram(const T* c, long long cap, const Counters* ctr,
                                                   const unsigned long long* tbits, int n_bins,
                                                   unsigned long long* counts) {
    extern __shared__ unsigned hist_s[];
    const int nb2 = 2 * (n_bins + 1);
    for (int k = threadIdx.x; k < nb2; k += blockDim.x) hist_s[k] = 0u;
    __syncthreads();
    const long long n = min((long long)ctr->n_live, cap);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T v = c[i];
        const unsigned long long m = Coef<T>::mag(v);
        int bin;
        if (m < tbits[0]) {
            bin = n_bins;
        } else {  // largest k <= n_bins - 1 with tbits[k] <= m
            int lo = 0, hi = n_bins - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tbits[mid] <= m)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            bin = lo;
        }
        const int sgn = (Coef<T>::to_slot(v) >> (sizeof(T) * 8 - 1)) & 1;
        atomicAdd(&hist_s[sgn * (n_bins + 1) + bin], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nb2; k += blockDim.x)
        if (hist_s[k]) atomicAdd(&counts[k], (unsigned long long)hist_s[k]);
}

// Start of an X layer inside a captured program: clears the layer counters
// (not the error bits or the committed operator) and the per-qubit
// population deltas, and records |O| entering the layer.
__global__ void k_layer_begin(Counters* ctr) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ctr->n_done = ctr->n_next = ctr->n_units = ctr->unit_cursor = 0;
    ctr->branch_events = ctr->dropped = ctr->pairs_one = ctr->pairs_two = 0;
    ctr->n_active = ctr->split_dropped = ctr->peak = ctr->upd_w = 0;
    ctr->dropped_sq = 0.0;
    ctr->n_in = ctr->n_live;
    ctr->range_cursor = 0;
    ctr->pass = 0;
}

// End of an X layer of ng gates inside a captured program: commits its
// output list (buffer `cur`) and adds the layer to the program totals (the
// updates as Counters::upd_w states).
__global__ void k_layer_end_x(Counters* ctr, int cur, int ng, ProgramStats* ps) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || ctr->err) return;
    const unsigned long long upd = (unsigned long long)ng * ctr->n_in -
                                   ctr->split_dropped * (unsigned long long)(ng - 1) + ctr->upd_w;
    ctr->n_live = ctr->n_done;
    ctr->cur = cur;
    ctr->n_layers += 1;
    ps->updates += upd;
    if (ctr->peak > ps->peak) ps->peak = ctr->peak;
    ps->branch_events += ctr->branch_events;
    ps->dropped += ctr->dropped;
    ps->pairs_one += ctr->pairs_one;
    ps->pairs_two += ctr->pairs_two;
    ps->dropped_sq += ctr->dropped_sq;
    ps->passes += (unsigned long long)ctr->pass;
    ps->x_layers += 1;
}

// End of a ZZ layer inside a captured program (applied in place, or held
// back for the next X layer's entry split: |O| and the buffer are
// unchanged).
__global__ void k_layer_end_zz(Counters* ctr, int n_gates, ProgramStats* ps) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || ctr->err) return;
    ctr->n_layers += 1;
    ps->updates += ctr->n_live * (unsigned long long)n_gates;
    if (ctr->n_live > ps->peak) ps->peak = ctr->n_live;
}

// Sets the committed operator from the host (after a host-side commit).
__global__ void k_set_live(Counters* ctr, long long n, int cur) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ctr->n_live = (unsigned long long)n;
    ctr->cur = cur;
}

}  // namespace orqa
