// X-rotation layer pipeline (Eq. update_rule applied gate by gate with the
// truncation of Algorithm 1), organised for GB300.
//
// A run of X rotations on ascending qubits (mask M) never changes z, so it
// acts independently on every group of strings with equal z and equal x
// outside F = z & M.  Inside a group a string anticommutes exactly with the
// gates of F.  The run is applied in chunk passes: pass p applies the gates
// of the F bits of rank [5p, 5p + 5) to "units" -- strings with equal z and
// equal x outside those <= 5 chunk bits -- so a unit is a dense vector over
// at most 32 x-patterns and never exchanges coefficients with another unit.
// Processing the gates of one unit in order with truncation after each is
// exactly Algorithm 1 restricted to that unit, because the gates outside
// the unit's chunk act trivially on it and truncation is per string.
//
// Each pass:
//   1. fine-bucket counts of the active strings (filled by the kernel that
//      wrote them): bucket = top bits of the hash of the unit key;
//   2. exclusive scan of the counts;
//   3. one streaming scatter of the active strings into bucket order (which
//      also clears the counts for the next pass);
//   4. persistent CTAs claim contiguous ranges of ~range_target strings
//      (whole buckets, so whole units), build the units in shared memory and
//      update them there.
// Survivors are appended to the output list (no chunk left) or to the next
// active list, whose bucket counts are accumulated on the fly.
#pragma once

#include "orqa_device.cuh"

namespace orqa {

// Four warps per CTA and seven CTAs per SM (shared memory: 32,000 B per
// CTA at W = 2 in FP64; 7 x 128 threads leave 73 registers a thread): with
// the sub-range barriers of small CTAs the warps wait less for the slowest
// one than with 8-warp CTAs (measured at the 1e9-string heavy-hex workload:
// 4-warp CTAs x 6 were 3-4% faster than 8 warps x 3 and faster than 32
// units per warp; 7 per SM are 5% faster than 6).  FP32 coefficients need
// 22,776 B and 64 registers, so 8 CTAs fit (3% faster than 7).
constexpr int LB_THREADS = 128;
constexpr int LB_CTAS_PER_SM = 7;  // resident unit-kernel CTAs per SM (launch bound), FP64
// FP32 coefficients: smaller shared-memory rows leave room for one more CTA
template <typename T>
constexpr int lb_ctas() { return sizeof(T) == 4 ? 8 : LB_CTAS_PER_SM; }
constexpr int LB_WARPS = LB_THREADS / 32;
constexpr int LB_MAX = 256;         // most strings one CTA sub-range may hold
constexpr int LB_TARGET = 448;      // strings per CTA range, on average (default tuning)
constexpr int LB_TABLE = 512;       // shared-memory hash slots (load <= 1/2)
constexpr int LB_UPW = 16;          // units a warp owns per round (lanes 0..15)
constexpr int LB_UPW_LOG = 4;
constexpr int LB_RU = LB_WARPS * LB_UPW;  // dense unit rows (LB_UPW per warp)
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int fine_bucket(uint64_t h, int fshift) { return (int)(h >> fshift); }

// A string that a chunk pass sends on to the next carries its slot in its
// next unit (the bits of x at the next chunk's positions) in bits 10..14 of
// its unit-key hash, and its x with those bits cleared (the next unit key's
// x): the unit kernel knows both once per unit, so the next pass's load
// needs no chunk search.  (The entry split writes full x; pass 0 searches.)
// Fine buckets use the top bits of the hash, shared-memory slots the low 9
// bits and the problem index bits 16..31.
constexpr int IDX_SHIFT = 10;

__device__ __forceinline__ uint64_t with_idx(uint64_t h, unsigned idx) {
    return (h & ~(0x1full << IDX_SHIFT)) | ((uint64_t)(idx & 31u) << IDX_SHIFT);
}

__device__ __forceinline__ int idx_of(uint64_t h) { return (int)(h >> IDX_SHIFT) & 31; }

// Fine-bucket counts are 16-bit, two per 32-bit word (half the footprint of
// the randomly addressed count array).  A string takes its rank in its
// bucket in two steps, so that several increments can be in flight before
// their results are used: bucket_add returns the word before the increment,
// bucket_old the string's rank from it.  A bucket holds at most sub_max <=
// 512 strings in a valid pass; the caller raises ERR_BUCKET_OVERFLOW for a
// rank of 2^15 or more, so no count ever carries into its neighbour unseen
// (every later kernel returns once the error is set).
__device__ __forceinline__ unsigned bucket_add(uint32_t* counts, int b) {
    return atomicAdd(&counts[b >> 1], 1u << (16 * (b & 1)));
}

__device__ __forceinline__ int bucket_old(unsigned word, int b) { return (int)((word >> (16 * (b & 1))) & 0xffffu); }

__device__ __forceinline__ int bucket_count(const uint32_t* counts, long long b) {
    return (int)((counts[b >> 1] >> (16 * (b & 1))) & 0xffffu);
}

// ---------------------------------------------------------------------------
// Entry split of a run (see the header comment): strings with F = 0 only
// meet the truncation and go to the output list; the others go to the active
// list.  A string already below delta is removed by the truncation after the
// run's first gate unless that gate acts on it first.  Active strings are
// counted into their pass-0 fine bucket.
// ---------------------------------------------------------------------------
// Exclusive block-wide scan of one int per thread (all threads call it);
// total receives the sum.
__device__ __forceinline__ int block_scan_exclusive(int v, int* warp_tot, int& total) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(FULL_MASK, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) warp_tot[wp] = incl;
    __syncthreads();
    if (wp == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? warp_tot[lane] : 0;
        int ti = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(FULL_MASK, ti, d);
            if (lane >= d) ti += u;
        }
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == nw - 1) warp_tot[32] = ti;
    }
    __syncthreads();
    const int r = warp_tot[wp] + incl - v;
    total = warp_tot[32];
    __syncthreads();
    return r;
}

// Each block takes tiles of SPLIT_ITEMS strings per thread: all loads of a
// tile are issued before any decision, and the tile's outputs are reserved
// with one atomic per list (a block scan gives every string its slot).
// ZZ: a ZZ layer of Clifford angles (G) that precedes the X layer is applied
// here first, string by string (zz_conjugate), instead of by a pass of its
// own over the operator: it maps each string to one string with |c|
// unchanged, so the routing below sees exactly the strings that the layer
// on its own would have left.
constexpr int SPLIT_ITEMS = 2;

template <int W, typename T, bool ZZ>
__global__ void __launch_bounds__(256) k_rx_split(StrList src, StrList done, StrList active, long long cap,
                                                  const __grid_constant__ RxRun run, Counters* ctr,
                                                  uint32_t* fcount, int fshift, const __grid_constant__ ZZGroups G) {
    __shared__ int warp_tot[33];
    __shared__ unsigned long long s_base[2];
    if (block_aborted(ctr)) return;
    const long long n = min((long long)ctr->n_live, cap);
    const long long tile = (long long)blockDim.x * SPLIT_ITEMS;
    const unsigned long long dbits = Coef<T>::threshold(run);
    const T* __restrict__ sc = reinterpret_cast<const T*>(src.c);
    unsigned long long my_drop = 0;
    double my_drop_sq = 0.0;
    for (long long t0 = (long long)blockIdx.x * tile; t0 < n; t0 += (long long)gridDim.x * tile) {  // block-uniform
        uint64_t z[SPLIT_ITEMS][W];
        uint64_t xz[ZZ ? SPLIT_ITEMS : 1][W];  // x, loaded up front only for the ZZ stage
        T c[SPLIT_ITEMS];
        int kind[SPLIT_ITEMS];  // 0: not live or dropped, 1: output list, 2: active list
#pragma unroll
        for (int k = 0; k < SPLIT_ITEMS; ++k) {
            const long long i = t0 + (long long)k * blockDim.x + threadIdx.x;
            kind[k] = 0;
            c[k] = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) z[k][w] = 0;
            if (i < n) {
                load_plane<W>(src.z, i, z[k]);
                c[k] = sc[i];
                if constexpr (ZZ) load_plane<W>(src.x, i, xz[k]);
            }
        }
        int nd = 0, na = 0;
#pragma unroll
        for (int k = 0; k < SPLIT_ITEMS; ++k) {
            const long long i = t0 + (long long)k * blockDim.x + threadIdx.x;
            if (i >= n) continue;
            if constexpr (ZZ) {
                if (zz_conjugate<W>(G, xz[k], z[k])) c[k] = Coef<T>::negate(c[k]);
            }
            uint64_t f[W], acc = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                f[w] = z[k][w] & run.mask[w];
                acc |= f[w];
            }
            const bool keep = keep_t<T>(c[k], dbits);
            bool act = acc != 0;
            if (act && !keep && !bit_of<W>(f, run.q_first)) act = false;  // dropped before its gates
            kind[k] = act ? 2 : (keep ? 1 : 0);
            nd += kind[k] == 1;
            na += kind[k] == 2;
            if (kind[k] == 0) {
                my_drop += 1;
                const double cd = (double)c[k];
                my_drop_sq = fma(cd, cd, my_drop_sq);
            }
        }
        int total;
        const int pre = block_scan_exclusive(nd | (na << 16), warp_tot, total);
        if (threadIdx.x == 0) {
            const unsigned td = (unsigned)total & 0xffffu, ta = (unsigned)total >> 16;
            s_base[0] = td ? atomicAdd(&ctr->n_done, (unsigned long long)td) : 0ull;
            s_base[1] = ta ? atomicAdd(&ctr->n_next, (unsigned long long)ta) : 0ull;
        }
        __syncthreads();
        long long sd = (long long)(s_base[0] + (unsigned)(pre & 0xffff));
        long long sa = (long long)(s_base[1] + (unsigned)(pre >> 16));
        // the tile's routed strings: stores and hashes first, then the
        // bucket counts of the active ones back to back, so that a thread's
        // returning atomics overlap
        long long slot[SPLIT_ITEMS];
        uint64_t hh[SPLIT_ITEMS];
#pragma unroll
        for (int k = 0; k < SPLIT_ITEMS; ++k) {
            const long long i = t0 + (long long)k * blockDim.x + threadIdx.x;
            const bool act = kind[k] == 2;
            slot[k] = act ? sa++ : (kind[k] == 1 ? sd++ : -1);
            hh[k] = 0;
            if (!kind[k]) continue;
            StrList dst = act ? active : done;
            const unsigned pid = src.pid ? src.pid[i] : 0u;
            uint64_t x[W];
            if constexpr (ZZ) {
#pragma unroll
                for (int w = 0; w < W; ++w) x[w] = xz[k][w];
            } else {
                load_plane<W>(src.x, i, x);
            }
            if (slot[k] < cap) {
                store_plane<W>(dst.x, slot[k], x);
                store_plane<W>(dst.z, slot[k], z[k]);
                reinterpret_cast<T*>(dst.c)[slot[k]] = c[k];
                if (dst.pid) dst.pid[slot[k]] = (uint16_t)pid;
            } else {
                atomicOr(&ctr->err, ERR_OVERFLOW);
            }
            if (act) hh[k] = unit_hash<W>(x, z[k], run.mask, 0, pid);
        }
        unsigned word[SPLIT_ITEMS];
#pragma unroll
        for (int k = 0; k < SPLIT_ITEMS; ++k)
            word[k] = kind[k] == 2 ? bucket_add(fcount, fine_bucket(hh[k], fshift)) : 0u;
        bool over = false;
#pragma unroll
        for (int k = 0; k < SPLIT_ITEMS; ++k)
            if (kind[k] == 2) {
                const int rk = bucket_old(word[k], fine_bucket(hh[k], fshift));
                over = over || rk >= 0x8000;
                if (slot[k] < cap) {
                    active.h[slot[k]] = hh[k];
                    active.rank[slot[k]] = rk;
                }
            }
        if (over) atomicOr(&ctr->err, ERR_BUCKET_OVERFLOW);
        __syncthreads();  // s_base is rewritten by the next tile
    }
    const unsigned long long wd = warp_sum64(my_drop);
    const double wsq = warp_sum_f64(my_drop_sq);
    if ((threadIdx.x & 31) == 0 && wd) {
        atomicAdd(&ctr->dropped, wd);
        atomicAdd(&ctr->split_dropped, wd);
        atomicAdd(&ctr->dropped_sq, wsq);
    }
}

// Pass bookkeeping between the kernels of an X layer (one thread): the list
// just written becomes the active list of the next pass.  With use_cond it
// also sets the condition of the enclosing graph loop (another pass is
// needed iff strings are active and no error was raised).
// pass_limit (at most MAX_PASSES) bounds the loop.
__global__ void k_pass_advance(Counters* ctr, int first, cudaGraphConditionalHandle cond, int use_cond,
                               int pass_limit) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long na = ctr->n_next;
    ctr->n_active = na;
    ctr->n_next = 0;
    ctr->range_cursor = 0;
    ctr->pass = first ? 0 : ctr->pass + 1;
    if (na > 0 && ctr->pass >= pass_limit) atomicOr(&ctr->err, ERR_PASS_LIMIT);
    const unsigned long long pk = ctr->n_done + na;
    if (pk > ctr->peak) ctr->peak = pk;
    if (use_cond) cudaGraphSetConditional(cond, (na > 0 && ctr->err == 0) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Exclusive scan of the fine-bucket counts (n = number of buckets, a
// multiple of SCAN_TILE): tile sums, a one-block scan of the tile sums,
// then offsets[b]; offsets[n] = total.  Offsets are 32-bit (every total is
// at most the capacity, < 2^31), which halves the table the scatter gathers
// from at random.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const uint32_t* counts, uint32_t* offsets,
                                                             long long* tile_sums, const Counters* ctr) {
    if (block_aborted(ctr)) return;
    __shared__ int warp_tot[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = bucket_count(counts, base + k);
        s += v[k];
    }
    int total;
    int run = block_scan_exclusive(s, warp_tot, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        offsets[base + k] = (uint32_t)run;
        run += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block; n_tiles <= SCAN_TILE.  All counts fit in int (they sum to at
// most the capacity, < 2^31).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_top(long long* tile_sums, int n_tiles,
                                                           const Counters* ctr) {
    if (block_aborted(ctr)) return;
    __shared__ int warp_tot[33];
    const int t = threadIdx.x;
    int v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int i = t * SCAN_ITEMS + k;
        v[k] = i < n_tiles ? (int)tile_sums[i] : 0;
        s += v[k];
    }
    int total;
    int run = block_scan_exclusive(s, warp_tot, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int i = t * SCAN_ITEMS + k;
        if (i < n_tiles) tile_sums[i] = run;
        run += v[k];
    }
    if (t == 0) tile_sums[SCAN_TILE] = total;
}

// Final scan step.  Also derives the CTA ranges of the unit kernel: range j
// is the buckets whose start offset lies in [j*T, (j+1)*T), so its first
// bucket is range_start[j] = min{b : offsets[b] >= j*T}.  Bucket b is that
// first bucket exactly for the j with offsets[b-1] < j*T <= offsets[b]; the
// end offsets[n] = total closes the last ranges, and range_start[J] = n for
// J = ceil(total / T).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_add(uint32_t* offsets, const long long* tile_sums,
                                                           const uint32_t* counts, long long n,
                                                           int32_t* range_start, long long T,
                                                           const Counters* ctr) {
    if (block_aborted(ctr)) return;
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    const long long add = tile_sums[blockIdx.x];
    const long long total = tile_sums[SCAN_TILE];
    const long long J = (total + T - 1) / T;
    long long prev = (base == 0) ? -1 : (long long)offsets[base] + add - bucket_count(counts, base - 1);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const long long o = (long long)offsets[base + k] + add;
        offsets[base + k] = (uint32_t)o;
        const long long jlo = (prev < 0) ? 0 : prev / T + 1;
        const long long jhi = min(o / T, J - 1);
        for (long long j = jlo; j <= jhi; ++j) range_start[j] = (int32_t)(base + k);
        prev = o;
    }
    if (base + SCAN_ITEMS == n) {  // the end bucket boundary
        offsets[n] = (uint32_t)total;
        for (long long j = prev / T + 1; j <= J - 1; ++j) range_start[j] = (int32_t)n;
        range_start[J] = (int32_t)n;
    }
}

// ---------------------------------------------------------------------------
// Scatter of the active strings into fine-bucket order, using the unit-key
// hash and the rank inside its bucket that the producing kernel stored with
// each string (the value its bucket-count atomic returned), so the position
// is offsets[bucket] + rank and no atomic is needed here.  The bucket-ordered
// copy is an array of
// records of whole 32-byte sectors -- (x, z, c, h) padded to 64 bytes for
// W = 2, exactly 32 bytes for W = 1 -- so the scattered writes never leave a
// partly written sector.
// ---------------------------------------------------------------------------
constexpr int SCATTER_ILP = 4;

template <int W, typename T>
__device__ __forceinline__ void store_record(void* base, long long i, const uint64_t (&x)[W],
                                             const uint64_t (&z)[W], T c, uint64_t h) {
    if constexpr (W == 2) {
        ulonglong2* r = reinterpret_cast<ulonglong2*>(base) + 4 * i;
        r[0] = make_ulonglong2(x[0], x[1]);
        r[1] = make_ulonglong2(z[0], z[1]);
        r[2] = make_ulonglong2(Coef<T>::to_slot(c), h);
        r[3] = make_ulonglong2(0ull, 0ull);  // completes the second sector
    } else {
        ulonglong2* r = reinterpret_cast<ulonglong2*>(base) + 2 * i;
        r[0] = make_ulonglong2(x[0], z[0]);
        r[1] = make_ulonglong2(Coef<T>::to_slot(c), h);
    }
}

template <int W, typename T>
__device__ __forceinline__ void load_record(const void* base, long long i, uint64_t (&x)[W], uint64_t (&z)[W],
                                            T& c, uint64_t& h) {
    if constexpr (W == 2) {
        const ulonglong2* r = reinterpret_cast<const ulonglong2*>(base) + 4 * i;
        const ulonglong2 a = r[0], b = r[1], d = r[2];
        x[0] = a.x;
        x[1] = a.y;
        z[0] = b.x;
        z[1] = b.y;
        c = Coef<T>::from_slot(d.x);
        h = d.y;
    } else {
        const ulonglong2* r = reinterpret_cast<const ulonglong2*>(base) + 2 * i;
        const ulonglong2 a = r[0], d = r[1];
        x[0] = a.x;
        z[0] = a.y;
        c = Coef<T>::from_slot(d.x);
        h = d.y;
    }
}

__host__ __device__ constexpr int record_bytes(int W) { return W == 2 ? 64 : 32; }

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    const unsigned lo = __shfl_sync(FULL_MASK, (unsigned)v, src);
    const unsigned hi = __shfl_sync(FULL_MASK, (unsigned)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}

// The records of 32 strings are staged in shared memory and written back
// cooperatively: RQ = record_bytes / 16 consecutive lanes store the 16-byte
// quarters of one record, so every store instruction writes 32 / RQ whole
// records instead of 32 scattered 16-byte pieces.
template <int W, typename T>
__global__ void __launch_bounds__(256) k_bucket_scatter(StrList src, long long cap, int fshift,
                                                        const uint32_t* __restrict__ offsets, void* dst,
                                                        uint32_t* fcount, long long n_fine, Counters* ctr) {
    constexpr int RQ = record_bytes(W) / 16;  // 16-byte quarters per record
    __shared__ uint4 stage[256 / 32][32][RQ];
    if (block_aborted(ctr)) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long long n = min((long long)ctr->n_active, cap);
    // the counts were consumed by the scan; clear them for the next pass
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < n_fine / 2;
         b += (long long)gridDim.x * blockDim.x)
        fcount[b] = 0u;
    const long long stride = (long long)gridDim.x * blockDim.x * SCATTER_ILP;
    for (long long base = (long long)blockIdx.x * blockDim.x * SCATTER_ILP + threadIdx.x;
         base - threadIdx.x < n; base += stride) {  // warp-uniform: all lanes iterate together
        long long slot[SCATTER_ILP];
        uint64_t h[SCATTER_ILP];
#pragma unroll
        for (int k = 0; k < SCATTER_ILP; ++k) {
            const long long i = base + (long long)k * blockDim.x;
            h[k] = 0;
            slot[k] = -1;
            if (i < n) {
                h[k] = src.h[i];
                slot[k] = src.rank[i];
            }
        }
#pragma unroll
        for (int k = 0; k < SCATTER_ILP; ++k)
            if (slot[k] >= 0) slot[k] += (long long)offsets[fine_bucket(h[k], fshift)];
#pragma unroll
        for (int k = 0; k < SCATTER_ILP; ++k) {
            const long long i = base + (long long)k * blockDim.x;
            long long sl = slot[k];
            if (sl >= cap) {  // only reachable after an undetected count error; never write past the records
                atomicOr(&ctr->err, ERR_OVERFLOW);
                sl = -1;
            }
            if (sl >= 0) {
                uint64_t x[W], z[W];
                load_plane<W>(src.x, i, x);
                load_plane<W>(src.z, i, z);
                const T c = reinterpret_cast<const T*>(src.c)[i];
                if constexpr (W == 2) {
                    stage[wp][lane][0] = make_uint4((unsigned)x[0], (unsigned)(x[0] >> 32), (unsigned)x[1],
                                                    (unsigned)(x[1] >> 32));
                    stage[wp][lane][1] = make_uint4((unsigned)z[0], (unsigned)(z[0] >> 32), (unsigned)z[1],
                                                    (unsigned)(z[1] >> 32));
                } else {
                    stage[wp][lane][0] = make_uint4((unsigned)x[0], (unsigned)(x[0] >> 32), (unsigned)z[0],
                                                    (unsigned)(z[0] >> 32));
                }
                const unsigned long long cs = Coef<T>::to_slot(c);
                stage[wp][lane][RQ == 4 ? 2 : 1] =
                    make_uint4((unsigned)cs, (unsigned)(cs >> 32), (unsigned)h[k], (unsigned)(h[k] >> 32));
                if constexpr (RQ == 4) stage[wp][lane][3] = make_uint4(0u, 0u, 0u, 0u);  // completes the sector
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < RQ; ++r) {
                const int rec = r * (32 / RQ) + lane / RQ, qi = lane % RQ;
                const long long s_rec = (long long)shfl64((uint64_t)sl, rec);
                if (s_rec >= 0)
                    reinterpret_cast<uint4*>(dst)[s_rec * RQ + qi] = stage[wp][rec][qi];
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// CTA-local unit processing.
//
// A CTA loads its range (whole fine buckets, so whole units) into shared
// memory, groups the strings into units with a shared-memory hash table on
// the exact key (z, x outside the chunk) and lists the strings of every unit
// contiguously.  A unit is a 32-slot row (slot = the string's chunk bits)
// with a 32-bit occupancy mask.  Each warp claims groups of LB_UPW units
// from a shared cursor and processes them with warp-level synchronisation
// only.  For chunk level j the pair {slot l, slot l | 2^j} (bit j of l
// clear) holds the strings P (sigma_z at the level's qubit q) and
// P xor X_q (sigma_y); by Eq. (update_rule) with B(Z,X) = 1, B(Y,X) = -1,
//     new c_Z = cos c_Z - sin c_Y,   new c_Y = cos c_Y + sin c_Z,
// an absent member counting as 0 (Algorithm 1 inserts it), then the
// truncation c == 0 or |c| < delta.  The pairs of a level (found with two
// mask operations per unit) go to one warp list -- the one-member pairs
// (2 DMUL) first, then the two-member pairs (2 more DMUL + 2 DADD) --
// processed by all lanes in one pass, and the outputs of a group are
// enumerated one per lane.  FP64 instructions thus run on full warps
// (GB300 issues FP64 at 2 lanes per clock per SM whatever the active mask)
// and no lane loops over one unit's members.
// ---------------------------------------------------------------------------
// One work item of the unit kernel: buckets [b_lo, b_next) of range rj
// (whose buckets end at b_end), holding strings [s0, s1) of the bucket order.
struct SubRange {
    long long s0, s1;
    int rj, b_lo, b_next, b_end;
};

template <int W, typename T>
struct LocalSmem {
    uint64_t sx[W][LB_MAX];     // x with the chunk bits cleared
    uint64_t sz[W][LB_MAX];
    T sc[LB_MAX];
    T dense[LB_RU][32];         // unit rows: slot l of row r at column dcol(r, l)
    alignas(4) uint16_t table[LB_TABLE];  // hash table of string indices (0xffff: empty), then unit masks
    unsigned occ[LB_RU];
    int16_t s_unit[LB_MAX];     // home slot, then representative, then unit id
    int16_t u_rep[LB_MAX];
    int16_t s_order[LB_MAX];    // the strings in unit order
    int16_t ustart[LB_MAX + 1]; // first position of each unit in that order
    union {
        struct {
            int16_t rep_uid[LB_MAX];      // unit id of a representative
            int32_t rep_cnt[LB_MAX / 2];  // strings per representative, two 16-bit counts per word
        } g;                              // grouping phases
        Rot<T> hrot[LB_RU];               // unit phase: cos and sin of each unit's current gate
    } ph;
    uint16_t spid[LB_MAX];      // problem index of each string
    uint8_t s_idx[LB_MAX];
    int warp_tot[33];
    double drop_sq[LB_WARPS];   // per warp: sum of c^2 dropped (norm tracking only)
    int group_cursor;           // next unit group a warp claims
    SubRange cur, nx;           // the sub-range in work and the next one
    int n_units;
};

// Column of slot l in dense row r: the slot XOR the row's low bits, so that
// the same slot of different rows (the common case in a level's pair list)
// falls in different shared-memory banks.
__device__ __forceinline__ int dcol(int r, int l) { return l ^ (r & 15); }

__device__ __forceinline__ unsigned level_mask(int j) {
    // slots whose bit j is clear
    return j == 0 ? 0x55555555u : j == 1 ? 0x33333333u : j == 2 ? 0x0f0f0f0fu : j == 3 ? 0x00ff00ffu : 0x0000ffffu;
}

// Position of the k-th set bit (0-based) of a 32-bit mask.
__device__ __forceinline__ int nth_set_bit32(unsigned w, int k) {
    int pos = 0;
    int c = __popc(w & 0xffffu);
    if (k >= c) { k -= c; w >>= 16; pos += 16; }
    c = __popc(w & 0xffu);
    if (k >= c) { k -= c; w >>= 8; pos += 8; }
    c = __popc(w & 0xfu);
    if (k >= c) { k -= c; w >>= 4; pos += 4; }
    c = __popc(w & 0x3u);
    if (k >= c) { k -= c; w >>= 2; pos += 2; }
    if (k >= (int)(w & 1u)) pos += 1;
    return pos;
}

__device__ __forceinline__ unsigned warp_exclusive_scan(unsigned v, unsigned& total) {
    const int lane = threadIdx.x & 31;
    unsigned incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned t = __shfl_up_sync(FULL_MASK, incl, d);
        if (lane >= d) incl += t;
    }
    total = __shfl_sync(FULL_MASK, incl, 31);
    return incl - v;
}


// Prepares the next work item (one warp, all lanes): the rest of the
// current range, or else the next non-empty range claimed from the device
// cursor.  Its end is the last bucket boundary b <= b_end with
// offsets[b] - offsets[b_lo] <= sub_max, found by a 32-way search: the
// offsets are nondecreasing, so of 32 boundaries spread over [lo, hi] the
// qualifying ones form a prefix, and each step shrinks the interval 32-fold
// (a range can span many empty buckets when few strings are active).
// Its records (contiguous in bucket order, rec_bytes each) are then
// prefetched into L2 with one bulk copy-engine request, so that the load
// phase of the next sub-range reads L2 instead of DRAM.
template <typename Smem>
__device__ __forceinline__ void next_subrange(Smem& S, Counters* ctr, const int32_t* __restrict__ range_start,
                                              const uint32_t* __restrict__ offsets, long long J, int sub_max,
                                              bool first, const void* bk, int rec_bytes) {
    const int lane = threadIdx.x & 31;
    int rj, b_lo, b_end;
    if (!first && S.cur.b_next < S.cur.b_end) {
        rj = S.cur.rj;
        b_lo = S.cur.b_next;
        b_end = S.cur.b_end;
    } else {
        for (;;) {  // warp-uniform; skips empty ranges
            int r = 0;
            if (lane == 0) r = (int)atomicAdd(&ctr->range_cursor, 1u);
            r = __shfl_sync(FULL_MASK, r, 0);
            rj = r;
            if (r >= J) break;
            b_lo = range_start[r];
            b_end = range_start[r + 1];
            if (b_lo < b_end) break;
        }
    }
    if (rj >= J) {
        if (lane == 0) S.nx.rj = rj;
        return;
    }
    const long long base = (long long)offsets[b_lo];
    int lo = b_lo, hi = b_end;  // lo qualifies; the answer lies in [lo, hi]
    while (lo < hi) {           // warp-uniform
        const long long span = hi - lo;
        const int cand = lo + (int)((span * (lane + 1) + 31) >> 5);  // nondecreasing, last = hi
        const unsigned bal = __ballot_sync(FULL_MASK, (long long)offsets[cand] - base <= sub_max);
        const int K = __popc(bal);
        if (K == 32) {
            lo = hi;
            break;
        }
        const int first_bad = __shfl_sync(FULL_MASK, cand, K);
        const int last_good = __shfl_sync(FULL_MASK, cand, K > 0 ? K - 1 : 0);
        if (K > 0) lo = last_good;
        hi = first_bad - 1;
    }
    const long long end = (long long)offsets[lo];
    if (lane == 0 && end > base) {  // whole records: 16-byte aligned, a multiple of 16 bytes
        const char* p = static_cast<const char*>(bk) + base * rec_bytes;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((unsigned)((end - base) * rec_bytes))
                     : "memory");
    }
    if (lane == 0) {
        S.nx.rj = rj;
        S.nx.b_lo = b_lo;
        S.nx.b_next = lo;
        S.nx.b_end = b_end;
        S.nx.s0 = base;
        S.nx.s1 = end;
    }
}

// Persistent: each CTA claims ranges from a device cursor until none is
// left, so the grid can be fixed (as in a captured graph) and uneven ranges
// balance across CTAs.  The number of ranges J = ceil(total / range_target)
// and the pass index are read from the device.  A sub-range holds at most
// sub_max <= LB_MAX strings (the load of the shared-memory hash table is at
// most sub_max / LB_TABLE).  TRACK adds up the c^2 of the dropped strings
// (the norm bookkeeping); the timed path is compiled without it.
template <int W, typename T, bool TRACK>
__global__ void __launch_bounds__(LB_THREADS, lb_ctas<T>()) k_bucket_local(
    const void* bk, const uint32_t* __restrict__ offsets, const int32_t* __restrict__ range_start,
    long long n_fine, int range_target, int sub_max, const __grid_constant__ RxRun run, StrList done,
    StrList next, long long cap, Counters* ctr, uint32_t* fcount_next, int fshift) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LocalSmem<W, T>& S = *reinterpret_cast<LocalSmem<W, T>*>(smem_raw);
    if (block_aborted(ctr)) return;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const unsigned long long dbits = Coef<T>::threshold(run);
    const int pass = ctr->pass;
    const long long J = ((long long)offsets[n_fine] + range_target - 1) / range_target;

    // per-lane event counts stay far below 2^32 (a launch handles at most
    // 5 entries per string of the capacity, < 2^31, spread over every lane of
    // the grid); the warp totals are summed in 64 bits
    unsigned my_branch = 0, my_drop = 0;
    unsigned long long my_one = 0, my_two = 0, my_upd = 0;  // my_upd: see Counters::upd_w
    if (TRACK && tid < LB_WARPS) S.drop_sq[tid] = 0.0;
    // The work items are sub-ranges; the next one (claiming a new range when
    // the current range is done) is prepared by warp LB_WARPS - 1 while the
    // other warps work on the current one's units, so the latency of the
    // claim and the bound search overlaps useful work.
    if (wp == LB_WARPS - 1) next_subrange(S, ctr, range_start, offsets, J, sub_max, true, bk, record_bytes(W));
    for (;;) {  // block-uniform
    __syncthreads();  // the prepared item is visible; the previous one is finished
    // every thread reads the prepared item (warp LB_WARPS - 1 rewrites it
    // only in the unit phase, after the barriers below), so the table
    // clearing and the load share one phase
    const SubRange cur = S.nx;
    if (tid == 0) {
        S.cur = cur;
        S.n_units = 0;
    }
    if (cur.rj >= J) break;
    if (cur.b_next == cur.b_lo) {  // one bucket alone exceeds sub_max
        if (tid == 0) atomicOr(&ctr->err, ERR_BUCKET_OVERFLOW);
        break;
    }
    for (int t = tid; t < LB_TABLE; t += LB_THREADS) S.table[t] = 0xffffu;
    for (int t = tid; t < LB_MAX / 2; t += LB_THREADS) S.ph.g.rep_cnt[t] = 0;
    const long long s0 = cur.s0;
    const int m = (int)(cur.s1 - cur.s0);

    // ---- load the range; key of a string = (z, x with the chunk bits cleared)
    for (int i = tid; i < m; i += LB_THREADS) {
        uint64_t x[W], z[W], h;
        T c;
        load_record<W, T>(bk, s0 + i, x, z, c, h);
        int idx;
        if (pass == 0) {  // from the entry split: full x
            uint64_t f[W], m[W];
#pragma unroll
            for (int w = 0; w < W; ++w) f[w] = z[w] & run.mask[w];
            chunk_mask<W>(f, 0, m);
            idx = gather_bits<W>(x, m);
#pragma unroll
            for (int w = 0; w < W; ++w) x[w] &= ~m[w];
        } else {  // from the previous pass: the unit key's x and the slot
            idx = idx_of(h);
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            S.sx[w][i] = x[w];
            S.sz[w][i] = z[w];
        }
        S.sc[i] = c;
        S.spid[i] = (uint16_t)pid_of(h);
        S.s_idx[i] = (uint8_t)idx;
        S.s_unit[i] = (int16_t)(h & (uint64_t)(LB_TABLE - 1));  // home slot, replaced below
    }
    __syncthreads();
    // ---- units: shared-memory hash table on the exact key
    for (int i = tid; i < m; i += LB_THREADS) {
        uint64_t xb[W], z[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            xb[w] = S.sx[w][i];
            z[w] = S.sz[w][i];
        }
        const uint16_t pi = S.spid[i];
        int slot = S.s_unit[i];
        int rep = i;
        for (int probe = 0; probe < LB_TABLE; ++probe) {  // 2*LB_MAX slots: never full
            const unsigned short old = atomicCAS(&S.table[slot], (unsigned short)0xffffu, (unsigned short)i);
            if (old == 0xffffu) break;
            const int v = old;
            bool eq = S.spid[v] == pi;
#pragma unroll
            for (int w = 0; w < W; ++w) eq = eq && (S.sz[w][v] == z[w]) && (S.sx[w][v] == xb[w]);
            if (eq) {
                rep = v;
                break;
            }
            slot = (slot + 1) & (LB_TABLE - 1);
        }
        S.s_unit[i] = (int16_t)rep;
        if (rep == i) {  // a new unit: its id, in arbitrary order
            const int u = atomicAdd(&S.n_units, 1);
            S.ph.g.rep_uid[i] = (int16_t)u;
            S.u_rep[u] = (int16_t)i;
        }
        atomicAdd(&S.ph.g.rep_cnt[rep >> 1], 1 << (16 * (rep & 1)));
    }
    __syncthreads();
    const int n_units = S.n_units;
    // ---- the strings of each unit as a contiguous list
    constexpr int PER_T = LB_MAX / LB_THREADS;
    {
        int v[PER_T], cnt = 0;
#pragma unroll
        for (int k = 0; k < PER_T; ++k) {
            const int u = tid * PER_T + k;
            v[k] = 0;
            if (u < n_units) {
                const int r = S.u_rep[u];
                v[k] = (S.ph.g.rep_cnt[r >> 1] >> (16 * (r & 1))) & 0xffff;
            }
            cnt += v[k];
        }
        int total;
        int run = block_scan_exclusive(cnt, S.warp_tot, total);
#pragma unroll
        for (int k = 0; k < PER_T; ++k) {
            const int u = tid * PER_T + k;
            if (u < n_units) S.ustart[u] = (int16_t)run;
            run += v[k];
        }
        if (tid == 0) {
            S.ustart[n_units] = (int16_t)total;
            S.group_cursor = 0;
        }
    }
    // occupancy masks of the units, in the hash table's storage (free now)
    uint32_t* uocc = reinterpret_cast<uint32_t*>(S.table);
    for (int u = tid; u < n_units; u += LB_THREADS) uocc[u] = 0u;
    __syncthreads();
    for (int i = tid; i < m; i += LB_THREADS) {
        const int r = S.s_unit[i];
        const int u = S.ph.g.rep_uid[r];
        const int k = ((atomicSub(&S.ph.g.rep_cnt[r >> 1], 1 << (16 * (r & 1))) >> (16 * (r & 1))) & 0xffff) - 1;
        S.s_order[S.ustart[u] + k] = (int16_t)i;
        S.s_unit[i] = (int16_t)u;
        atomicOr(&uocc[u], 1u << S.s_idx[i]);
    }
    __syncthreads();

    // ---- unit groups: a warp claims LB_UPW consecutive units at a time
    // (lane L < LB_UPW owns unit g + L, in dense row ub + L) and works on
    // them with warp-level synchronisation only
    const int ub = wp * LB_UPW;  // first dense row of this warp
    if (wp == LB_WARPS - 1) next_subrange(S, ctr, range_start, offsets, J, sub_max, false, bk, record_bytes(W));
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(&S.group_cursor, LB_UPW);
        g = __shfl_sync(FULL_MASK, g, 0);
        if (g >= n_units) break;  // warp-uniform
        const int u = g + lane;
        const bool own = lane < LB_UPW && u < n_units;
        uint64_t z[W], xb[W], xn[W];
        uint64_t ppos = 0;  // this pass's chunk positions, 7 bits each (packed_pos)
        int np = 0;
        bool more = false;
        unsigned upid = 0, nidx = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) z[w] = xb[w] = xn[w] = 0;
        if (own) {
            const int rep = S.u_rep[u];
            upid = S.spid[rep];
            uint64_t f[W], m2[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                z[w] = S.sz[w][rep];
                xb[w] = S.sx[w][rep];
                f[w] = z[w] & run.mask[w];
            }
            int np2 = 0;
            np = chunk_positions2_packed<W>(f, CHUNK_BITS * pass, ppos, m2, np2);
            more = np2 > 0;
            // the next pass's key: x outside the next chunk (this chunk's bits
            // are set per output string below; the two chunks are disjoint),
            // and the slot in the next unit, the same for all the unit's outputs
            nidx = (unsigned)gather_bits<W>(xb, m2);
            // a unit's strings all go on or all end: its outputs' x is the
            // next pass's key x (next chunk cleared) or the unit key's x
#pragma unroll
            for (int w = 0; w < W; ++w) xn[w] = more ? xb[w] & ~m2[w] : xb[w];
        }
        if (lane < LB_UPW) S.occ[ub + lane] = own ? uocc[u] : 0u;
        // strings of this warp's units into their slots (a contiguous run of
        // the unit-ordered list)
        {
            const int k_lo = S.ustart[g], k_hi = S.ustart[min(g + LB_UPW, n_units)];
            for (int k = k_lo + lane; k < k_hi; k += 32) {
                const int i = S.s_order[k];
                const int r = ub + S.s_unit[i] - g;
                S.dense[r][dcol(r, S.s_idx[i])] = S.sc[i];
            }
        }
        __syncwarp();
        const int wnp = __reduce_max_sync(FULL_MASK, np);
        for (int j = 0; j < wnp; ++j) {
            const int bit = 1 << j;
            const unsigned mj = level_mask(j);
            const bool act = own && np > j;
            unsigned sgl = 0, dbl = 0, hi = 0;
            int pop_before = 0, qj = 0;
            if (act) {
                const unsigned o = S.occ[ub + lane];
                const unsigned lo = o & mj;
                hi = (o >> bit) & mj;
                sgl = lo ^ hi;
                dbl = lo & hi;
                pop_before = __popc(o);
                qj = packed_pos(ppos, j);
                // one gate angle for the whole run: a uniform parameter read
                S.ph.hrot[ub + lane] = run.uniform ? Coef<T>::rot(run, 0u, run.q_first) : Coef<T>::rot(run, upid, qj);
            }
            unsigned tot;
            const unsigned o12 = warp_exclusive_scan((unsigned)__popc(sgl) | ((unsigned)__popc(dbl) << 16), tot);
            const unsigned n1 = tot & 0xffffu, n2 = tot >> 16;
            my_one += n1;
            my_two += n2;
            __syncwarp();  // the owners' hrot entries are visible
            // entry t of the level: the one-member pairs at [0, n1), the
            // two-member pairs at [n1, n1 + n2), each kind in owner-lane
            // order; a lane finds its entry's owner by a binary search of
            // the owners' exclusive counts and its slot as the r-th set bit
            for (unsigned t0 = 0; t0 < n1 + n2; t0 += 32) {  // warp-uniform
                const unsigned t = t0 + lane;
                const bool two = t >= n1;
                const unsigned rk = two ? t - n1 : t;
                const int sh = two ? 16 : 0;
                int lo = 0, hi2 = LB_UPW - 1;
                unsigned base = 0;  // exclusive count of owner lo (lane 0: 0)
#pragma unroll
                for (int step = 0; step < LB_UPW_LOG; ++step) {
                    const int mid = (lo + hi2 + 1) >> 1;
                    const unsigned fm = (__shfl_sync(FULL_MASK, o12, mid) >> sh) & 0xffffu;
                    if (fm <= rk) {
                        lo = mid;
                        base = fm;
                    } else {
                        hi2 = mid - 1;
                    }
                }
                const unsigned ms = __shfl_sync(FULL_MASK, sgl, lo);
                const unsigned md = __shfl_sync(FULL_MASK, dbl, lo);
                const unsigned mh = __shfl_sync(FULL_MASK, hi, lo);
                if (t >= n1 + n2) continue;
                const int la = nth_set_bit32(two ? md : ms, (int)(rk - base));
                const int ur = ub + lo;
                const bool y_side = !two && ((mh >> la) & 1u);
                const int lb = la | bit;
                const T u1 = S.dense[ur][dcol(ur, y_side ? lb : la)];
                T na, nb;
                if (t0 + 32 <= n1) {  // warp-uniform: one-member entries only (2 products)
                    lone_entry(S.ph.hrot[ur], u1, y_side, na, nb);
                } else {
                    const T u2 = two ? S.dense[ur][dcol(ur, lb)] : u1;
                    pair_entry(S.ph.hrot[ur], u1, u2, two, y_side, na, nb);
                }
                const bool ka = keep_t<T>(na, dbits), kb = keep_t<T>(nb, dbits);
                my_drop += (unsigned)(!ka) + (unsigned)(!kb);
                if constexpr (TRACK) {
                    if (!(ka && kb)) {
                        const double da = ka ? 0.0 : (double)na, db = kb ? 0.0 : (double)nb;
                        atomicAdd(&S.drop_sq[wp], fma(da, da, db * db));
                    }
                }
                S.dense[ur][dcol(ur, la)] = na;
                S.dense[ur][dcol(ur, lb)] = nb;
                // occupancy of the pair before (both, or the present member) and after
                const unsigned was = two ? ((1u << la) | (1u << lb)) : (1u << (y_side ? lb : la));
                const unsigned now = (ka ? (1u << la) : 0u) | (kb ? (1u << lb) : 0u);
                if (was & ~now) atomicAnd(&S.occ[ur], ~(was & ~now));
                if (now & ~was) atomicOr(&S.occ[ur], now & ~was);
            }
            __syncwarp();
            if (act) {
                const int d = __popc(S.occ[ub + lane]) - pop_before;
                my_branch += (unsigned)pop_before;
                my_upd += (unsigned long long)((long long)d * gates_above(run.mask, qj));
            }
        }
        // ---- outputs: flattened over the warp, one reservation per warp and list
        const unsigned occ = own ? S.occ[ub + lane] : 0u;
        const unsigned nout = __popc(occ);
        unsigned wtot;
        const unsigned flat = warp_exclusive_scan(nout, wtot);
        unsigned ntot;
        const unsigned noff = warp_exclusive_scan(more ? nout : 0u, ntot);
        unsigned long long bd = 0, bn = 0;
        if (lane == 0) {
            if (wtot > ntot) bd = atomicAdd(&ctr->n_done, (unsigned long long)(wtot - ntot));
            if (ntot) bn = atomicAdd(&ctr->n_next, (unsigned long long)ntot);
        }
        const unsigned long long base_done = shfl64(bd, 0), base_next = shfl64(bn, 0);
        const unsigned doff = flat - noff;  // done-list offset of this lane's unit
        // done and next offsets of a lane's unit (each at most LB_UPW * 32 < 2^10)
        const unsigned dn_off = doff | (noff << 10);
        for (unsigned kb = 0; kb < wtot; kb += 32) {
            const unsigned k = kb + lane;
            // owner lane: last L < LB_UPW with flat(L) <= k
            int lo = 0, hi2 = LB_UPW - 1;
            unsigned fl = 0;  // flat offset of owner lo (lane 0: 0)
#pragma unroll
            for (int step = 0; step < LB_UPW_LOG; ++step) {
                const int mid = (lo + hi2 + 1) >> 1;
                const unsigned fm = __shfl_sync(FULL_MASK, flat, mid);
                if (fm <= k) {
                    lo = mid;
                    fl = fm;
                } else {
                    hi2 = mid - 1;
                }
            }
            const int L = lo;
            const unsigned oc = __shfl_sync(FULL_MASK, occ, L);
            // problem index, chunk size, next-pass flag and next slot, packed
            const unsigned pk =
                __shfl_sync(FULL_MASK, upid | ((unsigned)np << 16) | ((unsigned)more << 19) | (nidx << 20), L);
            const unsigned ppl = pk & 0xffffu;
            const int npl = (int)((pk >> 16) & 7u);
            const bool mr = ((pk >> 19) & 1u) != 0;
            const unsigned nxi = pk >> 20;
            const unsigned dno = __shfl_sync(FULL_MASK, dn_off, L);
            const unsigned dof = dno & 1023u, nof = dno >> 10;
            const uint64_t pp = shfl64(ppos, L);
            uint64_t x[W], zz[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                x[w] = shfl64(xn[w], L);
                zz[w] = shfl64(z[w], L);
            }
            if (k >= wtot) continue;
            const int r = (int)(k - fl);
            const int l = nth_set_bit32(oc, r);
#pragma unroll
            for (int j = 0; j < CHUNK_BITS; ++j)
                if (j < npl && ((l >> j) & 1)) {
                    set_bit<W>(x, packed_pos(pp, j));
                }
            const long long slot = (long long)(mr ? base_next + nof + r : base_done + dof + r);
            StrList dst = mr ? next : done;
            uint64_t h = 0;
            unsigned word = 0;
            int b = 0;
            if (mr) {  // the bucket count is in flight during the stores
                h = with_idx(with_pid(hash_key<W>(zz, x, ppl), ppl), nxi);  // x: outside the next chunk
                b = fine_bucket(h, fshift);
                word = bucket_add(fcount_next, b);
            }
            if (slot < cap) {
                store_plane<W>(dst.x, slot, x);
                store_plane<W>(dst.z, slot, zz);
                reinterpret_cast<T*>(dst.c)[slot] = S.dense[ub + L][dcol(ub + L, l)];
                if (dst.pid) dst.pid[slot] = (uint16_t)ppl;
                if (mr) dst.h[slot] = h;
            } else {
                atomicOr(&ctr->err, ERR_OVERFLOW);
            }
            if (mr) {
                const int rk = bucket_old(word, b);
                if (rk >= 0x8000) atomicOr(&ctr->err, ERR_BUCKET_OVERFLOW);
                if (slot < cap) dst.rank[slot] = rk;
            }
        }
        __syncwarp();
    }
    }
    const unsigned long long nb = warp_sum64(my_branch);
    const unsigned long long nd = warp_sum64(my_drop);
    if (lane == 0 && (nb | nd)) {
        atomicAdd(&ctr->branch_events, nb);
        atomicAdd(&ctr->dropped, nd);
        atomicAdd(&ctr->pairs_one, my_one);
        atomicAdd(&ctr->pairs_two, my_two);
        if (TRACK) atomicAdd(&ctr->dropped_sq, S.drop_sq[wp]);
    }
    const unsigned long long nu = warp_sum64(my_upd);
    if (lane == 0 && nu) atomicAdd(&ctr->upd_w, nu);
}

}  // namespace orqa
