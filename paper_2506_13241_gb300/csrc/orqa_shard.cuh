// Sharding of one operator over R ranks by a hash of the z plane (the
// multi-device form of the ORQA partition, Eq. eq:Om, with the owner map
// f of Eq. distributor replaced by a hash of z alone).
//
// An X rotation flips x bits only, so every string that an X layer can
// merge with a given string (its partners P xor X_q) has the same z plane:
// with strings placed by owner(z), an X layer -- branching, merging and
// truncation -- needs no data from another rank.  A ZZ layer maps each
// string to exactly one string, z' = z xor (L x) with the sign rule of
// Eq. update_rule: afterwards the strings whose new owner is another rank
// move there in one exchange, and since the layer is a bijection they are
// distinct from every string already held there, so no merge follows.
#pragma once

#include "orqa_device.cuh"

namespace orqa {

constexpr int SHARD_MAX_RANKS = 512;  // ORQA_SHARD_MAX_RANKS

// Owner rank of a z plane: a 64-bit mix of its words, reduced mod R.  The
// same code runs on the host (placement) and on the device (exchange).
__host__ __device__ __forceinline__ uint64_t shard_mix(uint64_t h) {
    h ^= h >> 31;
    h *= 0x7fb5d329728ea185ull;
    h ^= h >> 27;
    h *= 0x81dadef4bc2dd44dull;
    h ^= h >> 33;
    return h;
}

__host__ __device__ __forceinline__ int shard_owner(const uint64_t* z, int W, int n_ranks) {
    uint64_t h = shard_mix(z[0] + 0x9e3779b97f4a7c15ull);
    if (W == 2) h = shard_mix(h ^ z[1]);
    return (int)(h % (uint64_t)n_ranks);
}

// Strings per owner rank (counts[r], zeroed by the host).
template <int W>
__global__ void __launch_bounds__(256) k_shard_count(StrList s, long long n, int n_ranks, unsigned long long* counts) {
    extern __shared__ unsigned cnt_r[];
    for (int r = threadIdx.x; r < n_ranks; r += blockDim.x) cnt_r[r] = 0u;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        uint64_t z[W];
        load_plane<W>(s.z, i, z);
        atomicAdd(&cnt_r[shard_owner(z, W, n_ranks)], 1u);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n_ranks; r += blockDim.x)
        if (cnt_r[r]) atomicAdd(&counts[r], (unsigned long long)cnt_r[r]);
}

// Exchange records: 2W + 1 words per string, x words, z words, then the
// coefficient's bit pattern (a float in the low 32 bits in the FP32 form).
// Strings owned by `rank` are appended to `keep` (ctr->n_done); the others
// go to send[cursor[owner]++] (cursor: the start of each destination's run).
template <int W, typename T>
__global__ void __launch_bounds__(256) k_shard_scatter(StrList s, long long n, int n_ranks, int rank, StrList keep,
                                                       unsigned long long* cursor, uint64_t* send, long long send_cap,
                                                       Counters* ctr) {
    const long long n_round = (n + 31) & ~31ll;
    const int lane = threadIdx.x & 31;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_round;
         i += (long long)gridDim.x * blockDim.x) {  // warp-uniform
        const bool live = i < n;
        uint64_t x[W], z[W];
        T c = 0;
        int o = -1;
        if (live) {
            load_plane<W>(s.x, i, x);
            load_plane<W>(s.z, i, z);
            c = reinterpret_cast<const T*>(s.c)[i];
            o = shard_owner(z, W, n_ranks);
        }
        const long long k = warp_append(live && o == rank, &ctr->n_done);
        if (live && o == rank && k < n) {
            store_plane<W>(keep.x, k, x);
            store_plane<W>(keep.z, k, z);
            reinterpret_cast<T*>(keep.c)[k] = c;
        }
        // one atomic per destination present in the warp
        const bool out = live && o != rank;
        const unsigned peers = __match_any_sync(FULL_MASK, out ? o : -1);
        const int leader = __ffs(peers) - 1;
        unsigned long long b = 0;
        if (out && lane == leader) b = atomicAdd(&cursor[o], (unsigned long long)__popc(peers));
        b = __shfl_sync(FULL_MASK, b, leader);  // every lane takes its group leader's base
        if (out) {
            const long long slot = (long long)b + __popc(peers & ((1u << lane) - 1u));
            if (slot >= send_cap) {  // only after a count mismatch; never write past the buffer
                atomicOr(&ctr->err, ERR_OVERFLOW);
                continue;
            }
            uint64_t* r = send + slot * (2 * W + 1);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                r[w] = x[w];
                r[W + w] = z[w];
            }
            r[2 * W] = Coef<T>::to_slot(c);
        }
    }
}

// Appends n exchange records to the committed buffer at position base.
template <int W, typename T>
__global__ void __launch_bounds__(256) k_shard_append(const uint64_t* recv, long long n, StrList s, long long base) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint64_t* r = recv + i * (2 * W + 1);
        uint64_t x[W], z[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            x[w] = r[w];
            z[w] = r[W + w];
        }
        store_plane<W>(s.x, base + i, x);
        store_plane<W>(s.z, base + i, z);
        reinterpret_cast<T*>(s.c)[base + i] = Coef<T>::from_slot(r[2 * W]);
    }
}

}  // namespace orqa
