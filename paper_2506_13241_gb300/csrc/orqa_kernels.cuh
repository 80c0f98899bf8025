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
// cos in {0, +-1}).  A string anticommutes with Z_i Z_j iff x_i xor x_j = 1.
// For cos = 0 its image is the single string with z_i, z_j flipped and
// coefficient (-1)^((B+1)/2) sin(theta) c; working out B(I, Z_i Z_j) for the
// anticommuting site gives: for sin = -1 the sign flips iff that site was Y
// (x = z = 1) before the gate, for sin = +1 iff it was X.  Edges are applied
// in array order, each seeing the planes left by the previous ones.  In
// place: one read and one write of z and c per string.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256) k_rzz_layer(StrList s, long long n,
                                                   const __grid_constant__ ZZLayer L) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t x[W], z[W];
        load_plane<W>(s.x, i, x);
        load_plane<W>(s.z, i, z);
        unsigned neg = 0;
        for (int e = 0; e < L.n_edges; ++e) {
            const int qi = L.qi[e], qj = L.qj[e], mode = L.mode[e];
            const int xi = get_bit(x, qi), xj = get_bit(x, qj);
            if ((xi ^ xj) == 0) continue;
            if (mode == 1) {
                neg ^= 1u;
                continue;
            }
            const int zsrc = xi ? get_bit(z, qi) : get_bit(z, qj);
            neg ^= (mode == 2) ? (unsigned)zsrc : (unsigned)(zsrc ^ 1);
            z[qi >> 6] ^= 1ull << (qi & 63);
            z[qj >> 6] ^= 1ull << (qj & 63);
        }
        store_plane<W>(s.z, i, z);
        if (neg) s.c[i] = -s.c[i];
    }
}

// ---------------------------------------------------------------------------
// Stand-alone truncation (the truncate loop of Algorithm 1): copies the
// strings with c != 0 and |c| >= delta to dst, order-preserving within a
// warp, warp-aggregated appends.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256) k_truncate(StrList src, long long n, StrList dst,
                                                  long long cap, double delta, Counters* ctr) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n + 31) & ~31ll;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        double c = 0.0;
        if (i < n) c = src.c[i];
        const bool keep = (i < n) && keep_coef(c, delta);
        const long long slot = warp_append(keep, &ctr->n_done);
        if (keep) {
            if (slot < cap) {
                uint64_t x[W], z[W];
                load_plane<W>(src.x, i, x);
                load_plane<W>(src.z, i, z);
                store_plane<W>(dst.x, slot, x);
                store_plane<W>(dst.z, slot, z);
                dst.c[slot] = c;
            } else {
                ctr->overflow = 1u;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// X-rotation layer, entry split.  The run's gates are X_q for q in mask, in
// ascending q, each followed by truncation (Algorithm 1).  A string with
// F = z & mask = 0 commutes with every gate of the run and only meets the
// truncation; a string with F != 0 anticommutes with exactly the gates of F
// and goes to the active list.  A string already below delta is removed by
// the truncation after the run's first gate unless that gate acts on it
// first, so it is kept only when F holds q_first.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256) k_rx_split(StrList src, long long n, StrList done,
                                                  StrList active, long long cap,
                                                  const __grid_constant__ RxRun run, Counters* ctr) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n + 31) & ~31ll;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        uint64_t x[W], z[W], f[W];
        double c = 0.0;
        bool live = i < n;
        bool act = false, keep = false;
        if (live) {
            load_plane<W>(src.z, i, z);
            c = src.c[i];
#pragma unroll
            for (int w = 0; w < W; ++w) f[w] = z[w] & run.mask[w];
            act = !all_zero<W>(f);
            keep = keep_coef(c, run.delta);
            if (act && !keep && !get_bit(f, run.q_first)) act = false;  // dropped before its gates
        }
        const bool to_done = live && !act && keep;
        const long long sd = warp_append(to_done, &ctr->n_done);
        const long long sa = warp_append(act, &ctr->n_next);
        if (to_done || act) {
            const long long slot = to_done ? sd : sa;
            StrList dst = to_done ? done : active;
            if (slot < cap) {
                load_plane<W>(src.x, i, x);
                store_plane<W>(dst.x, slot, x);
                store_plane<W>(dst.z, slot, z);
                dst.c[slot] = c;
            } else {
                ctr->overflow = 1u;
            }
        }
        const unsigned nd = __popc(__ballot_sync(FULL_MASK, live && !act && !keep));
        if ((threadIdx.x & 31) == 0 && nd) atomicAdd(&ctr->dropped, (unsigned long long)nd);
    }
}

// ---------------------------------------------------------------------------
// Unit assignment.  A unit is the set of strings that one chunk pass can
// couple: same z, and same x outside the chunk C (the set bits of
// F = z & mask whose rank lies in [CHUNK_BITS*pass, CHUNK_BITS*(pass+1))).
// The rotations of the chunk only flip x bits inside C, so a unit never
// exchanges coefficients with another one.  Each string finds (or creates)
// its unit in an open-addressing hash table keyed by (z, x & ~C), takes a
// rank inside it, and records its chunk index (its x bits at C, packed).
// In full-key mode (merge of duplicates) the key is the whole string.
// ---------------------------------------------------------------------------
template <int W, bool FULL_KEY>
__global__ void __launch_bounds__(256) k_unit_assign(
    StrList src, long long n, const __grid_constant__ RxRun run, int pass, int32_t* table,
    long long table_mask, uint64_t* unit_z, uint64_t* unit_xb, int32_t* unit_count,
    int32_t* uid_out, int32_t* rank_out, uint8_t* idx_out, Counters* ctr) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n + 31) & ~31ll;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        uint64_t x[W], z[W], xb[W];
        bool done = i >= n;
        int idx = 0;
        long long slot = 0;
        if (!done) {
            load_plane<W>(src.x, i, x);
            load_plane<W>(src.z, i, z);
#pragma unroll
            for (int w = 0; w < W; ++w) xb[w] = x[w];
            if (!FULL_KEY) {
                uint64_t f[W];
#pragma unroll
                for (int w = 0; w < W; ++w) f[w] = z[w] & run.mask[w];
                int pos[CHUNK_BITS];
                bool more;
                const int np = chunk_positions<W>(f, CHUNK_BITS * pass, pos, more);
                for (int j = 0; j < np; ++j) {
                    idx |= get_bit(x, pos[j]) << j;
                    xb[pos[j] >> 6] &= ~(1ull << (pos[j] & 63));
                }
            }
            slot = (long long)(hash_key<W>(z, xb) & (uint64_t)table_mask);
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
                store_plane<W>(unit_xb, u, xb);
                unit_count[u] = 0;
                __threadfence();
                atomicExch(&table[slot], (int32_t)u);
                my_uid = (int)u;
                done = true;
            }
            __syncwarp();
            if (!done) {
                long long spins = 0;
                while (v == SLOT_BUSY && spins < SPIN_LIMIT) {
                    v = *((volatile int32_t*)&table[slot]);
                    ++spins;
                }
                if (v == SLOT_BUSY) {
                    atomicExch(&ctr->timeout, 1u);
                    done = true;
                } else {
                    __threadfence();
                    uint64_t kz[W], kx[W];
                    load_plane_cg<W>(unit_z, v, kz);
                    load_plane_cg<W>(unit_xb, v, kx);
                    bool eq = true;
#pragma unroll
                    for (int w = 0; w < W; ++w) eq = eq && (kz[w] == z[w]) && (kx[w] == xb[w]);
                    if (eq) {
                        my_uid = v;
                        done = true;
                    } else {
                        slot = (slot + 1) & table_mask;
                        if (++probes > table_mask) {
                            atomicExch(&ctr->table_full, 1u);
                            done = true;
                        }
                    }
                }
            }
        }
        if (i < n) {
            uid_out[i] = my_uid;
            if (my_uid >= 0) rank_out[i] = atomicAdd(&unit_count[my_uid], 1);
            if (!FULL_KEY) idx_out[i] = (uint8_t)idx;
        }
    }
}

// Gives every unit a contiguous element range (in arbitrary unit order):
// a warp scan of the counts plus one atomic per warp.
__global__ void __launch_bounds__(256) k_unit_offsets(const int32_t* unit_count,
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

// Moves each string's coefficient (and chunk index) into its unit's range.
template <bool WITH_IDX>
__global__ void __launch_bounds__(256) k_unit_scatter(const double* c, long long n,
                                                      const int32_t* uid, const int32_t* rank,
                                                      const uint8_t* idx, const long long* unit_off,
                                                      double* sorted_c, uint8_t* sorted_idx) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int u = uid[i];
        if (u < 0) continue;
        const long long pos = unit_off[u] + rank[i];
        sorted_c[pos] = c[i];
        if (WITH_IDX) sorted_idx[pos] = idx[i];
    }
}

// ---------------------------------------------------------------------------
// Unit processing.  A unit is a dense vector over the 2^k x-patterns of its
// k <= 5 chunk qubits (slot l holds the coefficient of the string whose
// chunk bits spell l, 0 if absent).  For each chunk qubit q (ascending, the
// gate order) the slots l and l | (1 << j) (bit j clear) hold the pair
// {P, P xor X_q} with P at sigma_z and its partner at sigma_y on q; both
// anticommute with X_q.  By Eq. (update_rule) with B(Z,X) = 1, B(Y,X) = -1:
//   new c_Z = cos c_Z - sin c_Y,   new c_Y = cos c_Y + sin c_Z,
// where an absent partner counts as 0 (Algorithm 1's insert-or-add creates
// it), followed by truncation (c == 0 or |c| < delta).
//
// A warp holds UNITS_PER_WARP units in shared memory.  Per chunk level it
// first lists the pairs with a non-zero member (integer tests only), then
// updates just those pairs, 32 pairs per instruction: the FP64 work is
// proportional to the live strings, not to the 32 slots of every unit.
// Survivors go to the output list if no chunk of F remains, else to the
// next active list, with one output reservation per block and round.
// ---------------------------------------------------------------------------
constexpr int PROCESS_WARPS = 8;
constexpr int UNITS_PER_WARP = 8;

template <int W>
__global__ void __launch_bounds__(PROCESS_WARPS * 32) k_unit_process(
    const uint64_t* unit_z, const uint64_t* unit_xb, const int32_t* unit_count,
    const long long* unit_off, const double* sorted_c, const uint8_t* sorted_idx,
    const __grid_constant__ RxRun run, int pass, StrList done, StrList next, long long cap,
    Counters* ctr, unsigned long long* pop_delta) {
    constexpr int K = UNITS_PER_WARP;
    __shared__ double dense[PROCESS_WARPS][K][32];
    __shared__ uint16_t work[PROCESS_WARPS][K * 16];
    __shared__ uint64_t uz[PROCESS_WARPS][K][W], uxb[PROCESS_WARPS][K][W];
    __shared__ uint8_t upos[PROCESS_WARPS][K][CHUNK_BITS];
    __shared__ int8_t unp[PROCESS_WARPS][K];
    __shared__ uint8_t umore[PROCESS_WARPS][K];
    __shared__ int um[PROCESS_WARPS][K];
    __shared__ long long uoff[PROCESS_WARPS][K];
    __shared__ int blk_delta[MAX_QUBITS];
    __shared__ unsigned warp_cnt[2][PROCESS_WARPS];
    __shared__ unsigned long long warp_base[2][PROCESS_WARPS];
    __shared__ unsigned long long blk_branch, blk_drop;
    for (int t = threadIdx.x; t < MAX_QUBITS; t += blockDim.x) blk_delta[t] = 0;
    if (threadIdx.x == 0) {
        blk_branch = 0;
        blk_drop = 0;
    }
    __syncthreads();
    const long long nu = (long long)*((volatile unsigned long long*)&ctr->n_units);
    const int lane = threadIdx.x & 31;
    const int wp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(run.delta);
    const long long per_block = (long long)PROCESS_WARPS * K;
    unsigned long long my_branch = 0, my_drop = 0;
    double (*dn)[32] = dense[wp];
    for (long long base = (long long)blockIdx.x * per_block; base < nu; base += (long long)gridDim.x * per_block) {
        // unit headers: lane r < K loads unit r of this warp
        if (lane < K) {
            const long long u = base + (long long)wp * K + lane;
            int np = 0, m = 0;
            long long off = 0;
            bool more = false;
            uint64_t z[W], xb[W], f[W];
#pragma unroll
            for (int w = 0; w < W; ++w) z[w] = xb[w] = 0;
            int pos[CHUNK_BITS] = {0, 0, 0, 0, 0};
            if (u < nu) {
                m = unit_count[u];
                off = unit_off[u];
                load_plane<W>(unit_z, u, z);
                load_plane<W>(unit_xb, u, xb);
#pragma unroll
                for (int w = 0; w < W; ++w) f[w] = z[w] & run.mask[w];
                np = chunk_positions<W>(f, CHUNK_BITS * pass, pos, more);
            }
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uz[wp][lane][w] = z[w];
                uxb[wp][lane][w] = xb[w];
            }
#pragma unroll
            for (int j = 0; j < CHUNK_BITS; ++j) upos[wp][lane][j] = (uint8_t)pos[j];
            unp[wp][lane] = (int8_t)np;
            umore[wp][lane] = more ? 1 : 0;
            um[wp][lane] = m;
            uoff[wp][lane] = off;
        }
#pragma unroll
        for (int r = 0; r < K; ++r) dn[r][lane] = 0.0;
        __syncwarp();
        for (int r = 0; r < K; ++r) {
            const int m = um[wp][r];
            const long long off = uoff[wp][r];
            for (int e = lane; e < m; e += 32) dn[r][sorted_idx[off + e]] = sorted_c[off + e];
        }
        __syncwarp();
        for (int j = 0; j < CHUNK_BITS; ++j) {
            const int bit = 1 << j;
            // list the live pairs (Z-side slot index) of every unit with a level-j gate
            int npairs = 0;
            int pop_before[K];
#pragma unroll
            for (int r = 0; r < K; ++r) {
                pop_before[r] = 0;
                if (unp[wp][r] <= j) continue;  // warp-uniform
                const bool nz = nonzero_bits(dn[r][lane]);
                pop_before[r] = __popc(__ballot_sync(FULL_MASK, nz));
                const bool nzp = __shfl_xor_sync(FULL_MASK, nz, bit);
                const bool live = ((lane & bit) == 0) && (nz || nzp);
                const unsigned b = __ballot_sync(FULL_MASK, live);
                if (live) work[wp][npairs + __popc(b & lt_mask)] = (uint16_t)(r * 32 + lane);
                npairs += __popc(b);
            }
            __syncwarp();
            for (int w = lane; w < npairs; w += 32) {
                const int slot = work[wp][w];
                const int r = slot >> 5, la = slot & 31, lb = la | bit;
                const int q = upos[wp][r][j];
                const double co = run.cs[q], sn = run.sn[q];
                const double a = dn[r][la], b = dn[r][lb];
                double na = __dsub_rn(__dmul_rn(co, a), __dmul_rn(sn, b));
                double nb = __dadd_rn(__dmul_rn(co, b), __dmul_rn(sn, a));
                const bool ka = keep_bits(na, dbits), kb = keep_bits(nb, dbits);
                my_drop += (unsigned long long)(!ka) + (unsigned long long)(!kb);
                dn[r][la] = ka ? na : 0.0;
                dn[r][lb] = kb ? nb : 0.0;
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < K; ++r) {
                if (unp[wp][r] <= j) continue;
                const int pop_after = __popc(__ballot_sync(FULL_MASK, nonzero_bits(dn[r][lane])));
                if (lane == 0) {
                    my_branch += (unsigned long long)pop_before[r];
                    if (pop_after != pop_before[r]) atomicAdd(&blk_delta[upos[wp][r][j]], pop_after - pop_before[r]);
                }
            }
        }
        // one reservation per block and destination for the whole round
        unsigned cnt_done = 0, cnt_next = 0;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const unsigned k = __popc(__ballot_sync(FULL_MASK, nonzero_bits(dn[r][lane])));
            if (umore[wp][r])
                cnt_next += k;
            else
                cnt_done += k;
        }
        if (lane == 0) {
            warp_cnt[0][wp] = cnt_done;
            warp_cnt[1][wp] = cnt_next;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            const int d = threadIdx.x;
            unsigned long long tot = 0;
            for (int k = 0; k < PROCESS_WARPS; ++k) {
                warp_base[d][k] = tot;
                tot += warp_cnt[d][k];
            }
            unsigned long long b = 0;
            if (tot) b = atomicAdd(d == 0 ? &ctr->n_done : &ctr->n_next, tot);
            for (int k = 0; k < PROCESS_WARPS; ++k) warp_base[d][k] += b;
        }
        __syncthreads();
        unsigned long long ob_done = warp_base[0][wp], ob_next = warp_base[1][wp];
        for (int r = 0; r < K; ++r) {
            const double v = dn[r][lane];
            const bool keep = nonzero_bits(v);
            const unsigned bal = __ballot_sync(FULL_MASK, keep);
            const bool more = umore[wp][r] != 0;
            unsigned long long& ob = more ? ob_next : ob_done;
            if (keep) {
                const long long slot = (long long)(ob + __popc(bal & lt_mask));
                if (slot < cap) {
                    uint64_t x[W], z[W];
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        x[w] = uxb[wp][r][w];
                        z[w] = uz[wp][r][w];
                    }
                    const int np = unp[wp][r];
                    for (int j = 0; j < np; ++j)
                        if ((lane >> j) & 1) {
                            const int p = upos[wp][r][j];
                            x[p >> 6] |= 1ull << (p & 63);
                        }
                    StrList dst = more ? next : done;
                    store_plane<W>(dst.x, slot, x);
                    store_plane<W>(dst.z, slot, z);
                    dst.c[slot] = v;
                } else {
                    ctr->overflow = 1u;
                }
            }
            ob += __popc(bal);
        }
        __syncthreads();
    }
    // lanes 1..31 also carry drop counts from the pair loop
    my_drop = __reduce_add_sync(FULL_MASK, (unsigned)my_drop);
    if (lane == 0) {
        atomicAdd(&blk_branch, my_branch);
        atomicAdd(&blk_drop, my_drop);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < MAX_QUBITS; t += blockDim.x)
        if (blk_delta[t]) atomicAdd(&pop_delta[t], (unsigned long long)(long long)blk_delta[t]);
    if (threadIdx.x == 0) {
        if (blk_branch) atomicAdd(&ctr->branch_events, blk_branch);
        if (blk_drop) atomicAdd(&ctr->dropped, blk_drop);
    }
}

// ---------------------------------------------------------------------------
// Duplicate merge (insert-or-add of Algorithm 1): one thread per unit of
// equal strings sums their coefficients and keeps the sum if it is non-zero
// and not below delta.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256) k_merge_reduce(const uint64_t* unit_z,
                                                      const uint64_t* unit_xb,
                                                      const int32_t* unit_count,
                                                      const long long* unit_off,
                                                      const double* sorted_c, double delta,
                                                      StrList dst, long long cap, Counters* ctr) {
    const long long nu = (long long)*((volatile unsigned long long*)&ctr->n_units);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (nu + 31) & ~31ll;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n_round; u += stride) {
        double acc = 0.0;
        if (u < nu) {
            const int m = unit_count[u];
            const long long off = unit_off[u];
            acc = sorted_c[off];
            for (int e = 1; e < m; ++e) acc = __dadd_rn(acc, sorted_c[off + e]);
        }
        const bool keep = (u < nu) && keep_coef(acc, delta);
        const long long slot = warp_append(keep, &ctr->n_done);
        if (keep) {
            if (slot < cap) {
                uint64_t z[W], x[W];
                load_plane<W>(unit_z, u, z);
                load_plane<W>(unit_xb, u, x);
                store_plane<W>(dst.x, slot, x);
                store_plane<W>(dst.z, slot, z);
                dst.c[slot] = acc;
            } else {
                ctr->overflow = 1u;
            }
        } else if (u < nu) {
            atomicAdd(&ctr->dropped, 1ull);
        }
    }
}

// ---------------------------------------------------------------------------
// <0|O|0> (Eq. magnetization): sum of c over strings with x = 0.  Per-block
// partial sums in a fixed grid, then one thread adds them in block order.
// ---------------------------------------------------------------------------
constexpr int EXPECT_BLOCKS = 1024;

template <int W>
__global__ void __launch_bounds__(256) k_expect_partial(StrList s, long long n, double* partials) {
    __shared__ double red[8];
    const long long stride = (long long)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t x[W];
        load_plane<W>(s.x, i, x);
        if (all_zero<W>(x)) acc = __dadd_rn(acc, s.c[i]);
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
__global__ void k_expect_final(const double* partials, int nblocks, double* out) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32 || blockIdx.x != 0) return;
    double acc = 0.0;
    for (int k = lane; k < nblocks; k += 32) acc = __dadd_rn(acc, partials[k]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(FULL_MASK, acc, d));
    if (lane == 0) *out = acc;
}

}  // namespace orqa
