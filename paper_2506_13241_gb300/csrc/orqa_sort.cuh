// Canonical order of the operator O = sum_I O_I sigma_I (Eq. define_O): the
// strings sorted by their 256-bit key, x words from the highest to the
// lowest, then z words likewise (big-endian over the planes), after the
// problem index in batched contexts.
//
// LSD radix sort with 8-bit digits.  A digit that is the same for every
// string (found by one OR / AND reduction per key word) cannot change the
// order and is skipped, so an operator confined to a few qubits takes few
// passes.  Each pass moves whole strings (x, z, c, problem index) from one
// string buffer to another; the passes alternate between the two buffers
// that do not hold the committed operator, which is only read.  A pass is
// stable: every block owns a contiguous chunk of the input and walks it in
// order, tile by tile, ranking equal digits by warp match masks and warp
// order, so equal digits keep their input order.
#pragma once

#include "orqa_device.cuh"

namespace orqa {

constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_DIGITS = 256;

// Key word k of string i, least significant first: z[0..W-1], x[0..W-1],
// then the problem index (batched contexts).
template <int W>
__device__ __forceinline__ uint64_t sort_word(const StrList& s, long long i, int k) {
    if (k < W) return s.z[i * W + k];
    if (k < 2 * W) return s.x[i * W + (k - W)];
    return s.pid ? (uint64_t)s.pid[i] : 0ull;
}

// or_and[2k] |= OR and or_and[2k + 1] &= AND of key word k over the n
// strings (the host sets them to 0 and ~0 first).
template <int W>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_bits(StrList s, long long n, int K,
                                                            unsigned long long* or_and) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int k = 0; k < K; ++k) {
        unsigned long long o = 0ull, a = ~0ull;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const uint64_t v = sort_word<W>(s, i, k);
            o |= v;
            a &= v;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            o |= __shfl_xor_sync(FULL_MASK, o, d);
            a &= __shfl_xor_sync(FULL_MASK, a, d);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicOr(&or_and[2 * k], o);
            atomicAnd(&or_and[2 * k + 1], a);
        }
    }
}

// Digit counts of block b's chunk [b * chunk, min(n, (b + 1) * chunk)),
// stored digit-major: hist[d * G + b].
template <int W>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist(StrList s, long long n, long long chunk, int k,
                                                            int shift, unsigned* hist, int G) {
    __shared__ unsigned h[SORT_DIGITS];
    for (int d = threadIdx.x; d < SORT_DIGITS; d += blockDim.x) h[d] = 0u;
    __syncthreads();
    const long long lo = (long long)blockIdx.x * chunk, hi = min(n, lo + chunk);
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
        atomicAdd(&h[(sort_word<W>(s, i, k) >> shift) & 255u], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < SORT_DIGITS; d += blockDim.x) hist[(long long)d * G + blockIdx.x] = h[d];
}

// Exclusive scan, in place, of the `total` digit-major counts (one block of
// 1024 threads; every thread scans a contiguous segment).
__global__ void __launch_bounds__(1024) k_sort_scan(unsigned* hist, int total) {
    __shared__ unsigned warp_tot[32];
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int per = (total + 1023) / 1024;
    const int lo = min(total, t * per), hi = min(total, lo + per);
    unsigned s = 0;
    for (int i = lo; i < hi; ++i) s += hist[i];
    unsigned incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned v = __shfl_up_sync(FULL_MASK, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) warp_tot[wp] = incl;
    __syncthreads();
    if (wp == 0) {
        const unsigned v = warp_tot[lane];
        unsigned w = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned u = __shfl_up_sync(FULL_MASK, w, d);
            if (lane >= d) w += u;
        }
        warp_tot[lane] = w - v;
    }
    __syncthreads();
    unsigned run = warp_tot[wp] + incl - s;
    for (int i = lo; i < hi; ++i) {
        const unsigned c = hist[i];
        hist[i] = run;
        run += c;
    }
}

// Stable scatter of block b's chunk by digit (shift) of key word k: string
// i goes to offs[d * G + b] + (strings of digit d before it in the chunk).
template <int W, typename T>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter(StrList src, StrList dst, long long n, long long chunk,
                                                               int k, int shift, const unsigned* offs, int G) {
    __shared__ unsigned base[SORT_DIGITS];
    __shared__ unsigned whist[SORT_WARPS][SORT_DIGITS];
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    for (int d = tid; d < SORT_DIGITS; d += blockDim.x) base[d] = offs[(long long)d * G + blockIdx.x];
    const long long lo = (long long)blockIdx.x * chunk, hi = min(n, lo + chunk);
    for (long long t0 = lo; t0 < hi; t0 += SORT_THREADS) {  // block-uniform
        for (int j = tid; j < SORT_WARPS * SORT_DIGITS; j += SORT_THREADS) (&whist[0][0])[j] = 0u;
        __syncthreads();
        const long long i = t0 + tid;
        const bool valid = i < hi;
        // invalid lanes take a digit no valid lane has, so they match only themselves
        const unsigned d = valid ? (unsigned)((sort_word<W>(src, i, k) >> shift) & 255u) : 256u + lane;
        const unsigned peers = __match_any_sync(FULL_MASK, d);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == 31 - __clz(peers)) whist[wp][d] = __popc(peers);
        __syncthreads();
        unsigned tile_cnt = 0;
        if (tid < SORT_DIGITS) {  // exclusive prefix over the warps, per digit
            for (int w = 0; w < SORT_WARPS; ++w) {
                const unsigned c = whist[w][tid];
                whist[w][tid] = tile_cnt;
                tile_cnt += c;
            }
        }
        __syncthreads();
        if (valid) {
            const long long pos = (long long)base[d] + whist[wp][d] + rank;
            uint64_t x[W], z[W];
            load_plane<W>(src.x, i, x);
            load_plane<W>(src.z, i, z);
            store_plane<W>(dst.x, pos, x);
            store_plane<W>(dst.z, pos, z);
            reinterpret_cast<T*>(dst.c)[pos] = reinterpret_cast<const T*>(src.c)[i];
            if (dst.pid) dst.pid[pos] = src.pid[i];
        }
        __syncthreads();
        if (tid < SORT_DIGITS) base[tid] += tile_cnt;
    }
}

}  // namespace orqa
