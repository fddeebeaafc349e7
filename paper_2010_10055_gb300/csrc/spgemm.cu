// spgemm.cu -- C = A At over the overlap semiring (Sec. IV-D), row-wise on the GPU.
//
// Semiring: multiplying A_ij by At_jk takes the positions of k-mer j in reads i and k; adding
// counts one more shared k-mer and keeps the positions of up to max_seeds of them. Which seeds
// are kept is fixed order-free: the max_seeds shared k-mers with the smallest column index.
// Every update below is commutative (a count increment and an insertion into a "smallest S"
// list), so any parallel order gives the same C bit for bit.
//
// Passes (one thread block per row of C, rows binned by table size):
//  1. row_work   w_i = sum over j in row i of (nnz(At_j) - 1): products of row i, diagonal excluded.
//  2. symbolic   a hash table keyed by the partner read k, with a count per key, sized from a
//                guess (w_i / 2 slots: partners are far fewer than products because every true
//                overlap shares many k-mers). A row whose table fills past 3/4 is marked and
//                redone with 2 * min(w_i, n - 1) slots in a per-block global slice.
//                Records nnz_i = #{k : count >= min_shared} and distinct_i = #{k}.
//  3. scan nnz_i -> C.row_ptr; numeric classes from distinct_i (exact table sizes).
//  4. numeric    hash table (key, count, S seed words). A seed word is
//                (index of j within row i) << 32 | At value, so its numeric order is the order
//                of j; inserting into the S-slot list is a chain of atomicMin's that pushes the
//                loser down. Entries with count >= min_shared are compacted, bitonic-sorted by
//                k and written to C; seed positions are resolved from A's row.
// Fused path (default): no symbolic pass; tables sized from a guess, overflowing rows redone in
// global memory. A row with many products first walks them once to mark, in two bit filters in
// shared memory, the partners seen once and seen twice; the table then takes only partners whose
// seen-twice bit is set -- every partner with count >= 2, all its products, plus the few count-1
// partners that share a filter bit with another -- so it is sized for the kept partners rather
// than every partner (reads sharing one chance k-mer outnumber true overlaps many times over in
// large genomes). Entries below min_shared are dropped when the row is written, as before, so C is
// unchanged.
// Products of a row are enumerated warp by warp: a warp takes 32 consecutive entries of A's row,
// scans their At row lengths in registers, and walks the flattened product list 32 at a time,
// each lane finding its entry with a 5-step shuffle search.
#include <mutex>
#include <optional>

#include "check.cuh"
#include "ops.cuh"

namespace sg {

constexpr int SP_MAX_SEEDS = 8;

constexpr int SP_NCLS = 9;        // shared-memory classes per pass (one per table size)
constexpr int SP_MINLOG = 6;      // smallest table: 64 slots

__device__ __forceinline__ uint32_t hash_slot(int32_t k, int log2T) {
    return ((uint32_t)k * 2654435761u) >> (32 - log2T);
}

__host__ __device__ __forceinline__ int64_t pow2_at_least(int64_t x) {
    int64_t t = 1;
    while (t < x) t <<= 1;
    return t;
}

struct SpArgs {
    const int64_t *a_rp;
    const int32_t *a_col;
    const uint32_t *a_val;
    const int64_t *t_rp;
    const int32_t *t_col;
    const uint32_t *t_val;
    const int64_t *a_beg;     // per A entry (i, j): start of At row j
    const uint32_t *a_len;    // per A entry: length of At row j
    const uint64_t *t_pair;   // At entries as (val << 32 | col): one sector per product
    int64_t n;
    uint32_t min_shared;
    int S;
    uint32_t *err;  // DEV_OVERFLOW if the numeric pass ever disagrees with the symbolic sizes
};

// One warp per row: w_i, and for every entry (i, j) the start and length of At row j, so that
// the two passes stream these instead of gathering At's row pointers at random.
__global__ void row_work_kernel(const int64_t *__restrict__ a_rp, const int32_t *__restrict__ a_col,
                                const int64_t *__restrict__ t_rp, int64_t n, int64_t *__restrict__ work,
                                int64_t *__restrict__ a_beg, uint32_t *__restrict__ a_len) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    int64_t w = 0;
    for (int64_t a = a_rp[row] + lane; a < a_rp[row + 1]; a += 32) {
        const int32_t j = a_col[a];
        const int64_t b = t_rp[j], e = t_rp[j + 1];
        a_beg[a] = b;
        a_len[a] = (uint32_t)(e - b);
        w += e - b - 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) work[row] = w;
}

// Row classes: a row whose table needs at most 2^log2T[c] slots goes to class c; larger rows go
// to the global class (index ncls). lists[c * n + x] = rows of class c; counts[c] = its size.
struct Classes {
    int log2T[SP_NCLS];
    int ncls;
};

__global__ void classify_kernel(const int64_t *__restrict__ need, int64_t n, Classes cl,
                                unsigned long long *__restrict__ counts, int32_t *__restrict__ lists) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t u = need[i];
    if (u <= 0) return;
    int c = cl.ncls;
    for (int q = 0; q < cl.ncls; q++)
        if (u <= ((int64_t)1 << cl.log2T[q])) { c = q; break; }
    unsigned long long p = atomicAdd(counts + c, 1ull);
    if (SG_IN_BOUNDS((int64_t)p < n, 302, p)) lists[(int64_t)c * n + (int64_t)p] = (int32_t)i;
}

// symbolic table request: nextpow2(max(64, w >> shift)), capped at the exact bound 2 * min(w, n - 1)
__global__ void sym_need_kernel(const int64_t *__restrict__ work, int64_t n, int shift, int64_t *__restrict__ need) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t w = work[i];
    if (w <= 0) { need[i] = 0; return; }
    int64_t exact = pow2_at_least(2 * (w < n - 1 ? w : n - 1));
    int64_t guess = pow2_at_least((w >> shift) > 64 ? (w >> shift) : 64);
    need[i] = guess < exact ? guess : exact;
}

// numeric table request: nextpow2(2 * distinct), at least 64
__global__ void num_need_kernel(const int64_t *__restrict__ dist, int64_t n, int64_t *__restrict__ need) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t d = dist[i];
    need[i] = d > 0 ? pow2_at_least(2 * d > 64 ? 2 * d : 64) : 0;
}

// ------------------------------------------------------------------- product enumeration
// Calls f(k, vk, idx) for every product of row i: k = partner read (k != i), vk = the At value
// (PAIR only), idx = index of the A entry within row i. Stops (per warp) once *stop is nonzero.
// Each lane takes SP_U products per step, so a warp has SP_U gathers of At in flight at once.
constexpr int SP_U = 2;

template <bool PAIR, class F>
__device__ __forceinline__ void for_each_product(const SpArgs &g, int32_t i, int64_t r0, int64_t r1,
                                                 const volatile int *stop, F &&f) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t a0 = r0 + (int64_t)warp * 32; a0 < r1; a0 += (int64_t)nwarps * 32) {
        // one decision for the whole warp: the lanes may not have reconverged after the divergent
        // table updates, and a lane that left here would strand the others in the shuffles below
        if (stop && __any_sync(0xffffffffu, *stop != 0)) return;
        const int64_t a = a0 + lane;
        int64_t beg = 0, len = 0;
        if (a < r1) {
            beg = g.a_beg[a];
            len = g.a_len[a];
        }
        int64_t inc = len;  // inclusive scan of the lengths across the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int64_t excl = inc - len;
        const int64_t total = __shfl_sync(0xffffffffu, inc, 31);
        for (int64_t base = 0; base < total; base += 32 * SP_U) {
            int owner[SP_U];
            int64_t b[SP_U];
            uint64_t pr[SP_U];
#pragma unroll
            for (int u = 0; u < SP_U; u++) {
                const int64_t p = base + u * 32 + lane;
                int ow = 0;  // largest lane whose exclusive prefix is <= p
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    const int64_t v = __shfl_sync(0xffffffffu, excl, (ow + s) & 31);
                    if (ow + s < 32 && v <= p) ow += s;
                }
                const int64_t ob = __shfl_sync(0xffffffffu, beg, ow);
                const int64_t oe = __shfl_sync(0xffffffffu, excl, ow);
                owner[u] = ow;
                b[u] = p < total ? ob + (p - oe) : -1;
            }
#pragma unroll
            for (int u = 0; u < SP_U; u++)  // all gathers first, then the table updates
                if (b[u] >= 0) pr[u] = PAIR ? g.t_pair[b[u]] : (uint64_t)(uint32_t)g.t_col[b[u]];
#pragma unroll
            for (int u = 0; u < SP_U; u++) {
                if (b[u] < 0) continue;
                const int32_t k = (int32_t)(uint32_t)pr[u];
                if (k != i) f(k, (uint32_t)(pr[u] >> 32), a0 - r0 + owner[u]);
            }
        }
    }
}

// ---------------------------------------------------------------------------- symbolic
// Table in shared memory (GSLICE == false, 2^log2T slots, may overflow) or in this block's slice
// of a global pool (GSLICE == true, 2 * min(w_i, n - 1) slots rounded up: never overflows).
template <bool GSLICE>
__global__ void __launch_bounds__(512) symbolic_kernel(SpArgs g, const int32_t *__restrict__ rows,
                                                      const unsigned long long *__restrict__ nrows_p, int log2T,
                                                      const int64_t *__restrict__ work, int32_t *__restrict__ gpool,
                                                      int64_t slice, int32_t *__restrict__ ovf_list,
                                                      unsigned long long *__restrict__ ovf_count,
                                                      int64_t *__restrict__ nnz_row, int64_t *__restrict__ distinct_row) {
    extern __shared__ __align__(16) int32_t sym_tab[];
    __shared__ int s_ins, s_ovf;
    __shared__ int32_t s_red[2 * 16];
    const int64_t nrows = (int64_t)*nrows_p;
    for (int64_t rb = blockIdx.x; rb < nrows; rb += gridDim.x) {
        const int32_t i = rows[rb];
        int lT = log2T;
        int32_t *keys = sym_tab;
        if (GSLICE) {
            const int64_t w = work[i];
            const int64_t T = pow2_at_least(2 * (w < g.n - 1 ? w : g.n - 1));
            lT = 0;
            while (((int64_t)1 << lT) < T) lT++;
            keys = gpool + (int64_t)blockIdx.x * slice;
        }
        const int32_t T = 1 << lT;
        uint32_t *cnt = (uint32_t *)(keys + T);
        const int cap = GSLICE ? T : (T >> 1) + (T >> 2);
        for (int x = threadIdx.x; x < T; x += blockDim.x) {
            keys[x] = -1;
            cnt[x] = 0;
        }
        if (threadIdx.x == 0) {
            s_ins = 0;
            s_ovf = 0;
        }
        __syncthreads();
        const uint32_t msk = (uint32_t)T - 1u;
        for_each_product<false>(g, i, g.a_rp[i], g.a_rp[i + 1], GSLICE ? nullptr : &s_ovf,
                                [&](int32_t k, uint32_t, int64_t) {
            uint32_t h = hash_slot(k, lT);
            for (int probe = 0; probe < T; probe++) {
                int32_t cur = ((volatile int32_t *)keys)[h];
                if (cur == -1) {
                    const int32_t old = atomicCAS(keys + h, -1, k);
                    if (old == -1) {
                        if (atomicAdd(&s_ins, 1) >= cap) s_ovf = 1;
                        atomicAdd(cnt + h, 1u);
                        return;
                    }
                    cur = old;
                }
                if (cur == k) {
                    atomicAdd(cnt + h, 1u);
                    return;
                }
                h = (h + 1) & msk;
            }
            s_ovf = 1;  // went round the whole table
        });
        __syncthreads();
        if (s_ovf) {  // table too small for this row: the global-slice pass redoes it
            if (threadIdx.x == 0) {
                const unsigned long long q = atomicAdd(ovf_count, 1ull);
                if (SG_IN_BOUNDS((int64_t)q < g.n, 301, q)) ovf_list[q] = i;
            }
            __syncthreads();
            continue;
        }
        int32_t nz = 0, dist = 0;
        for (int x = threadIdx.x; x < T; x += blockDim.x) {
            if (keys[x] != -1) {
                dist++;
                if (cnt[x] >= g.min_shared) nz++;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            nz += __shfl_xor_sync(0xffffffffu, nz, o);
            dist += __shfl_xor_sync(0xffffffffu, dist, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_red[2 * (threadIdx.x >> 5)] = nz;
            s_red[2 * (threadIdx.x >> 5) + 1] = dist;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t a = 0, b = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
                a += s_red[2 * w];
                b += s_red[2 * w + 1];
            }
            nnz_row[i] = a;
            distinct_row[i] = b;
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- numeric
// One table of T slots: sort buffer [T/2] u64 | keys [T] i32 | counts [T] u32 | seeds [T][S] u32,
// in shared memory (GSLICE == false) or in this block's global slice. A seed is the index of the
// A entry (i, j) within row i; its order is the order of j, so the S smallest indices are the
// S shared k-mers with the smallest columns (reading r4). The positions are looked up when the
// row is written: pos_i from A's entry, pos_k from At's row j (sorted by read).
constexpr uint32_t SEED_NONE = 0xFFFFFFFFu;

// guessed: a table sized from a guess may hold up to 3/4 T partners, so its sort buffer has T
// entries; an exact-size table (T >= 2 x distinct) needs T/2.
__host__ __device__ inline size_t num_table_bytes(int64_t T, int S, bool guessed = false) {
    return (size_t)(guessed ? T : T / 2) * 8 + (size_t)T * (8 + 4 * (size_t)S);
}

// At value of partner k in At row [b, b + len) (t_pair = val << 32 | col, ascending col).
__device__ __forceinline__ uint32_t at_value(const uint64_t *__restrict__ t_pair, int64_t b, int64_t len, int32_t k) {
    int64_t lo = b, hi = b + len;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int32_t)(uint32_t)t_pair[mid] <= k) lo = mid; else hi = mid;
    }
    return (uint32_t)(t_pair[lo] >> 32);
}

// FUSED == false: the table size comes from the symbolic pass's exact distinct count (need[i]) and
// row i is written to C at c_rp[i]. FUSED == true (no symbolic pass): shared-memory tables are
// sized from a guess; a row whose table fills past 3/4 stops and is appended to ovf_list, to be
// redone in a global-memory table of the exact bound 2 min(w_i, n - 1) (GSLICE, never overflows);
// a finished row is written to the temporary arrays at c_rp[i] (room for min(w_i / t, n - 1)
// entries) and its length to nnz_row[i].
// FILT (fused shared-memory tables only, min_shared >= 2): the seen-once / seen-twice filters of
// 2^log2F bits each sit before the table; partner k maps to bit k when n <= 2^log2F, else to a
// multiplicative hash of k.
template <bool GSLICE, bool FUSED, bool FILT = false>
__global__ void __launch_bounds__(1024) numeric_kernel(SpArgs g, const int32_t *__restrict__ rows,
                                                     const unsigned long long *__restrict__ nrows_p, int log2T,
                                                     int log2F,
                                                     const int64_t *__restrict__ need, unsigned char *__restrict__ gpool,
                                                     int64_t slice_bytes, const int64_t *__restrict__ c_rp,
                                                     int32_t *__restrict__ c_col, uint32_t *__restrict__ c_cnt,
                                                     uint32_t *__restrict__ c_si, uint32_t *__restrict__ c_sk,
                                                     int64_t c_nnz, const int64_t *__restrict__ work,
                                                     int32_t *__restrict__ ovf_list,
                                                     unsigned long long *__restrict__ ovf_count,
                                                     int64_t *__restrict__ nnz_row) {
    extern __shared__ __align__(16) unsigned char num_raw[];
    __shared__ int s_ctr, s_ins, s_ovf;
    const int S = g.S;
    const int64_t nrows = (int64_t)*nrows_p;
    for (int64_t rb = blockIdx.x; rb < nrows; rb += gridDim.x) {
        const int32_t i = rows[rb];
        if (!SG_IN_BOUNDS(i >= 0 && i < g.n, 307, i)) continue;
        int lT = log2T;
        unsigned char *tb = FILT ? num_raw + ((size_t)2 << log2F) / 8 : num_raw;
        uint32_t *F1 = (uint32_t *)num_raw, *F2 = F1 + ((1 << log2F) >> 5);
        if (GSLICE) {
            int64_t T;
            if (FUSED) {
                const int64_t w = work[i];
                T = pow2_at_least(2 * (w < g.n - 1 ? w : g.n - 1));
            } else {
                T = need[i];
            }
            lT = 0;
            while (lT < 31 && ((int64_t)1 << lT) < T) lT++;
            if (!SG_IN_BOUNDS(num_table_bytes((int64_t)1 << lT, S) <= (size_t)slice_bytes, 306, T)) continue;
            tb = gpool + (int64_t)blockIdx.x * slice_bytes;
        }
        const int32_t T = 1 << lT;
        const bool guessed = FUSED && !GSLICE;
        const int ob_cap = guessed ? T : (T >> 1);  // sort buffer entries
        uint64_t *obuf = (uint64_t *)tb;
        int32_t *keys = (int32_t *)(obuf + ob_cap);
        uint32_t *cnt = (uint32_t *)(keys + T);
        uint32_t *seeds = cnt + T;
        for (int x = threadIdx.x; x < T; x += blockDim.x) {
            keys[x] = -1;
            cnt[x] = 0;
        }
        for (int x = threadIdx.x; x < T * S; x += blockDim.x) seeds[x] = SEED_NONE;
        if (FILT)
            for (int x = threadIdx.x; x < (2 << log2F) >> 5; x += blockDim.x) F1[x] = 0u;  // F1 and F2
        if (threadIdx.x == 0) {
            s_ctr = 0;
            s_ins = 0;
            s_ovf = 0;
        }
        __syncthreads();
        const int64_t r0 = g.a_rp[i], r1 = g.a_rp[i + 1];
        const uint32_t msk = (uint32_t)T - 1u;
        const bool fid = g.n <= ((int64_t)1 << log2F);
        auto fbit = [&](int32_t k) -> uint32_t {
            return fid ? (uint32_t)k & ((1u << log2F) - 1u) : ((uint32_t)k * 2654435761u) >> (32 - log2F);
        };
        if (FILT) {  // seen once -> F1, seen again -> F2 (bits are only ever set)
            for_each_product<false>(g, i, r0, r1, nullptr, [&](int32_t k, uint32_t, int64_t) {
                const uint32_t b = fbit(k), m = 1u << (b & 31u);
                if (((volatile uint32_t *)F2)[b >> 5] & m) return;
                if (atomicOr(F1 + (b >> 5), m) & m) atomicOr(F2 + (b >> 5), m);
            });
            __syncthreads();
        }
        const int cap = (T >> 1) + (T >> 2);  // guessed tables: at most 3/4 T partners
        for_each_product<false>(g, i, r0, r1, guessed ? &s_ovf : nullptr, [&](int32_t k, uint32_t, int64_t idx) {
            if (guessed && *(volatile int *)&s_ovf) return;  // the row is abandoned
            if (FILT) {  // seen once only: count 1 < min_shared
                const uint32_t b = fbit(k);
                if (!((F2[b >> 5] >> (b & 31u)) & 1u)) return;
            }
            uint32_t h = hash_slot(k, lT);
            bool found = false;
            // exact sizes (T >= 2 * distinct_i) always find a free slot or k; a guessed table may
            // fill up, which ends the row (s_ovf)
            for (int probe = 0; probe < T; probe++) {
                int32_t cur = ((volatile int32_t *)keys)[h];
                if (cur == -1) {
                    const int32_t old = atomicCAS(keys + h, -1, k);
                    if (old == -1) {
                        if (guessed && atomicAdd(&s_ins, 1) >= cap) s_ovf = 1;
                        found = true;
                        break;
                    }
                    cur = old;
                }
                if (cur == k) {
                    found = true;
                    break;
                }
                h = (h + 1) & msk;
            }
            if (!found) {
                s_ovf = 1;
                return;
            }
            atomicAdd(cnt + h, 1u);
            if (S > 0) {
                uint32_t v = (uint32_t)idx;
                uint32_t *sl = seeds + (int64_t)h * S;
                for (int q = 0; q < S; q++) {
                    const uint32_t old = atomicMin(sl + q, v);
                    if (old > v) v = old;  // the larger one moves on to the next slot
                    if (v == SEED_NONE) break;
                }
            }
        });
        __syncthreads();
        if (guessed && s_ovf) {  // table too small for this row: the global-memory pass redoes it
            if (threadIdx.x == 0) {
                const unsigned long long q = atomicAdd(ovf_count, 1ull);
                if (SG_IN_BOUNDS((int64_t)q < g.n, 304, q)) ovf_list[q] = i;
            }
            __syncthreads();
            continue;
        }
        for (int x = threadIdx.x; x < T; x += blockDim.x) {
            if (keys[x] != -1 && cnt[x] >= g.min_shared) {
                const int p = atomicAdd(&s_ctr, 1);
                if (SG_IN_BOUNDS(p < ob_cap, 303, p)) obuf[p] = ((uint64_t)(uint32_t)keys[x] << 32) | (uint32_t)x;
            }
        }
        __syncthreads();
        const int nv = s_ctr < ob_cap ? s_ctr : ob_cap;  // s_ctr <= ob_cap by the table sizes
        if (!SG_IN_BOUNDS(s_ctr <= ob_cap, 305, s_ctr)) {}
        int P2 = 1;
        while (P2 < nv) P2 <<= 1;
        for (int x = nv + threadIdx.x; x < P2; x += blockDim.x) obuf[x] = ~0ull;
        __syncthreads();
        for (int kk = 2; kk <= P2; kk <<= 1) {
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int x = threadIdx.x; x < P2; x += blockDim.x) {
                    const int y = x ^ jj;
                    if (y > x) {
                        const uint64_t a = obuf[x], b = obuf[y];
                        const bool up = (x & kk) == 0;
                        if ((a > b) == up) {
                            obuf[x] = b;
                            obuf[y] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        const int64_t e0 = c_rp[i];
        const int64_t room = c_rp[i + 1] - e0;
        if ((FUSED ? nv > room : nv != room) && threadIdx.x == 0) atomicOr(g.err, (uint32_t)DEV_OVERFLOW);
        const int nw = nv < room ? nv : (int)room;
        if (FUSED && threadIdx.x == 0) nnz_row[i] = nw;
        for (int q = threadIdx.x; q < nw; q += blockDim.x) {
            const uint64_t w = obuf[q];
            const uint32_t slot = (uint32_t)w;
            const int32_t k = (int32_t)(w >> 32);
            const int64_t e = e0 + q;
            c_col[e] = k;
            c_cnt[e] = cnt[slot];
            for (int s = 0; s < S; s++) {
                const uint32_t sd = seeds[(int64_t)slot * S + s];
                uint32_t si = 0xFFFFFFFFu, sk = 0xFFFFFFFFu;
                if (sd != SEED_NONE) {
                    const int64_t a = r0 + sd;
                    const uint32_t vi = g.a_val[a];
                    const uint32_t vk = at_value(g.t_pair, g.a_beg[a], g.a_len[a], k);
                    si = vi & 0x7FFFFFFFu;
                    sk = (vk & 0x7FFFFFFFu) | ((vi ^ vk) & 0x80000000u);
                }
                c_si[(int64_t)s * c_nnz + e] = si;
                c_sk[(int64_t)s * c_nnz + e] = sk;
            }
        }
        __syncthreads();
    }
}

static inline int64_t blocks_for(int64_t n, int nt) { return (n + nt - 1) / nt; }

// Sampled rows (every stride-th row, one block each): the products w, and the bits set in the
// seen-once and seen-twice filters after the row's products -- about its distinct partners and
// its partners seen at least twice. sums = {sum w, sum F1 bits, sum F2 bits}.
__global__ void __launch_bounds__(512) sample_kernel(SpArgs g, const int64_t *__restrict__ work, int64_t stride,
                                                    int log2F, unsigned long long *__restrict__ sums) {
    extern __shared__ __align__(16) uint32_t smp_f[];
    __shared__ unsigned long long s_c[2];
    const int64_t i = (int64_t)blockIdx.x * stride;
    if (i >= g.n) return;
    const int nw = (1 << log2F) >> 5;
    uint32_t *F1 = smp_f, *F2 = smp_f + nw;
    for (int x = threadIdx.x; x < 2 * nw; x += blockDim.x) smp_f[x] = 0u;
    if (threadIdx.x < 2) s_c[threadIdx.x] = 0ull;
    __syncthreads();
    const bool fid = g.n <= ((int64_t)1 << log2F);
    for_each_product<false>(g, (int32_t)i, g.a_rp[i], g.a_rp[i + 1], nullptr, [&](int32_t k, uint32_t, int64_t) {
        const uint32_t b = fid ? (uint32_t)k & ((1u << log2F) - 1u) : ((uint32_t)k * 2654435761u) >> (32 - log2F);
        const uint32_t m = 1u << (b & 31u);
        if (((volatile uint32_t *)F2)[b >> 5] & m) return;
        if (atomicOr(F1 + (b >> 5), m) & m) atomicOr(F2 + (b >> 5), m);
    });
    __syncthreads();
    unsigned long long c1 = 0, c2 = 0;
    for (int x = threadIdx.x; x < nw; x += blockDim.x) {
        c1 += __popc(F1[x]);
        c2 += __popc(F2[x]);
    }
    atomicAdd(&s_c[0], c1);
    atomicAdd(&s_c[1], c2);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(sums, (unsigned long long)(work[i] > 0 ? work[i] : 0));
        atomicAdd(sums + 1, s_c[0]);
        atomicAdd(sums + 2, s_c[1]);
    }
}

// Fused path: guessed table size and the row's output room min(w / t, n - 1). The guess is
// (w * fu) >> 16 for a sampled partner ratio fu (fixed point), or w >> shift without a sample.
// Rows with w >= fwork (fwork > 0) take the filtered pass: their guess ((w * ff) >> 16, or
// w >> fshift, at most fcap = the largest filtered shared-memory table) goes to need_f and need is
// 0, else need_f is 0.
__global__ void fused_need_kernel(const int64_t *__restrict__ work, int64_t n, int shift, uint64_t fu, uint32_t t,
                                  int64_t fwork, int fshift, uint64_t ff, int64_t fcap, int64_t *__restrict__ need,
                                  int64_t *__restrict__ need_f, int64_t *__restrict__ room) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t w = work[i];
    need_f[i] = 0;
    if (w <= 0) {
        need[i] = 0;
        room[i] = 0;
        return;
    }
    const bool filt = fwork > 0 && w >= fwork;
    const uint64_t mul = filt ? ff : fu;
    const int64_t g0 = mul ? (int64_t)(((unsigned __int128)w * mul) >> 16) : (w >> (filt ? fshift : shift));
    const int64_t exact = pow2_at_least(2 * (w < n - 1 ? w : n - 1));
    int64_t guess = pow2_at_least(g0 > 64 ? g0 : 64);
    if (filt && guess > fcap) guess = fcap;  // kept partners are few: try the largest table first
    (filt ? need_f : need)[i] = guess < exact ? guess : exact;
    if (filt) need[i] = 0;
    const int64_t r = w / t;
    room[i] = r < n - 1 ? r : n - 1;
}

// Fused path: copies each row's entries from the temporary arrays (row i at tmp_off[i], seeds
// slot-major with stride tmp_n) to C (row i at c_rp[i], stride nnz). One warp per row.
__global__ void compact_c_kernel(const int64_t *__restrict__ tmp_off, int64_t tmp_n, const int32_t *__restrict__ t_col,
                                 const uint32_t *__restrict__ t_cnt, const uint32_t *__restrict__ t_si,
                                 const uint32_t *__restrict__ t_sk, int S, const int64_t *__restrict__ c_rp, int64_t n,
                                 int64_t nnz, int32_t *__restrict__ c_col, uint32_t *__restrict__ c_cnt,
                                 uint32_t *__restrict__ c_si, uint32_t *__restrict__ c_sk) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int64_t src = tmp_off[row], dst = c_rp[row], len = c_rp[row + 1] - dst;
    for (int64_t e = lane; e < len; e += 32) {
        c_col[dst + e] = t_col[src + e];
        c_cnt[dst + e] = t_cnt[src + e];
        for (int q = 0; q < S; q++) {
            c_si[(int64_t)q * nnz + dst + e] = t_si[(int64_t)q * tmp_n + src + e];
            c_sk[(int64_t)q * nnz + dst + e] = t_sk[(int64_t)q * tmp_n + src + e];
        }
    }
}

__global__ void pair_kernel(const int32_t *__restrict__ col, const uint32_t *__restrict__ val, int64_t nnz,
                            uint64_t *__restrict__ pair) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) pair[e] = ((uint64_t)val[e] << 32) | (uint32_t)col[e];
}

// threads per block for a table of 2^log2T slots: tables of 4 k slots and more leave one or two
// blocks per SM, so those blocks bring more warps to hide the gathers' latency
static int pick_threads(int log2T) { return log2T <= 7 ? 64 : (log2T <= 10 ? 128 : (log2T <= 11 ? 256 : 512)); }

// numeric launches of 4 K slots and more run one block per SM: spgemm_big_threads (512 or 1024)
static int pick_numeric_threads(int log2T, bool filtered) {
    const int big = (int)tune("spgemm_big_threads");
    if (log2T >= 12) return big;
    return filtered ? (log2T <= 11 ? 256 : 512) : pick_threads(log2T);
}

// Launch names by table size, so that per-kernel timing separates the classes.
static const char *const SYM_NAMES[] = {"spgemm_symbolic_t64", "spgemm_symbolic_t128", "spgemm_symbolic_t256",
                                        "spgemm_symbolic_t512", "spgemm_symbolic_t1k", "spgemm_symbolic_t2k",
                                        "spgemm_symbolic_t4k", "spgemm_symbolic_t8k", "spgemm_symbolic_t16k"};
static const char *const NUM_NAMES[] = {"spgemm_numeric_t64", "spgemm_numeric_t128", "spgemm_numeric_t256",
                                        "spgemm_numeric_t512", "spgemm_numeric_t1k", "spgemm_numeric_t2k",
                                        "spgemm_numeric_t4k", "spgemm_numeric_t8k", "spgemm_numeric_t16k"};
static const char *const FIL_NAMES[] = {"spgemm_numeric_f64", "spgemm_numeric_f128", "spgemm_numeric_f256",
                                        "spgemm_numeric_f512", "spgemm_numeric_f1k", "spgemm_numeric_f2k",
                                        "spgemm_numeric_f4k", "spgemm_numeric_f8k", "spgemm_numeric_f16k"};

sg_status overlap_impl(const sg_csr_u32 *A, const sg_csr_u32 *At, uint32_t min_shared, int S,
                       sg_overlap_csr *C, cudaStream_t s, Scratch &sc) {
    const int64_t n = A->n_rows;
    const int NT = 256;
    constexpr int NCNT = SP_NCLS + 2;  // classes + global class + overflow counter
    uint32_t *err = sc.get<uint32_t>(1);
    int64_t *work = sc.get<int64_t>(n + 1);
    int64_t *need = sc.get<int64_t>(n + 1);
    int64_t *nnz_row = sc.get<int64_t>(n + 1);
    int64_t *dist = sc.get<int64_t>(n + 1);
    unsigned long long *counts = sc.get<unsigned long long>(4 * NCNT + 4);
    int32_t *lists = sc.get<int32_t>((size_t)(SP_NCLS + 1) * (n + 1));
    int32_t *ovf = sc.get<int32_t>(2 * (n + 1));  // overflow list | unused list of the re-run
    if (!err || !work || !need || !nnz_row || !dist || !counts || !lists || !ovf) return SG_ERR_OOM;
    unsigned long long *sym_counts = counts, *num_counts = counts + NCNT, *unused = counts + 2 * NCNT;
    unsigned long long *ovf_count = counts + SP_NCLS + 1;
    unsigned long long *fz_counts = counts + 2 * NCNT + 1, *fz_ovf = fz_counts + SP_NCLS + 1;
    unsigned long long *ff_counts = counts + 3 * NCNT + 1;  // filtered rows' classes + global class
    SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    SG_CUDA_TRY(cudaMemsetAsync(counts, 0, (4 * NCNT + 4) * sizeof(unsigned long long), s));
    SG_CUDA_TRY(cudaMemsetAsync(nnz_row, 0, (n + 1) * sizeof(int64_t), s));
    SG_CUDA_TRY(cudaMemsetAsync(dist, 0, (n + 1) * sizeof(int64_t), s));
    int64_t *a_beg = sc.get<int64_t>(A->nnz + 1);
    uint32_t *a_len = sc.get<uint32_t>(A->nnz + 1);
    uint64_t *t_pair = sc.get<uint64_t>(At->nnz + 1);
    if (!a_beg || !a_len || !t_pair) return SG_ERR_OOM;
    SpArgs g{A->row_ptr, A->col, A->val, At->row_ptr, At->col, At->val, a_beg, a_len, t_pair,
             n, min_shared, S, err};
    std::optional<StageScope> stage;
    stage.emplace("SpGEMMSymbolic", s);
    SG_LAUNCH("row_work", row_work_kernel, blocks_for(n * 32, 256), 256, 0, s, A->row_ptr, A->col, At->row_ptr, n,
              work, a_beg, a_len);
    SG_LAUNCH("at_pairs", pair_kernel, blocks_for(At->nnz, 256), 256, 0, s, At->col, At->val, At->nnz, t_pair);
    const int nsm = sm_count();
    const int grid = (int)(nsm * tune("spgemm_blocks_per_sm"));
    // numeric: one class per table size from 2^6 while the table and its sort buffer fit in 160 KB
    Classes num{};
    num.ncls = 0;
    while (num.ncls < SP_NCLS && num_table_bytes((int64_t)1 << (SP_MINLOG + num.ncls), S) <= (160u << 10)) {
        num.log2T[num.ncls] = SP_MINLOG + num.ncls;
        num.ncls++;
    }
    Classes fz{};  // the fused pass's guessed tables (larger sort buffer; up to 220 KB: one block per SM)
    fz.ncls = 0;
    while (fz.ncls < SP_NCLS && num_table_bytes((int64_t)1 << (SP_MINLOG + fz.ncls), S, true) <= (220u << 10)) {
        fz.log2T[fz.ncls] = SP_MINLOG + fz.ncls;
        fz.ncls++;
    }
    // filtered rows (fused path): two filters of 2^log2F bits, one bit per read while n fits
    int log2F = 10;
    while (log2F < (int)tune("spgemm_filter_log2") && ((int64_t)1 << log2F) < n) log2F++;
    const size_t fbytes = ((size_t)2 << log2F) / 8;
    Classes ff{};
    ff.ncls = 0;
    while (ff.ncls < SP_NCLS &&
           num_table_bytes((int64_t)1 << (SP_MINLOG + ff.ncls), S, true) + fbytes <= (220u << 10)) {
        ff.log2T[ff.ncls] = SP_MINLOG + ff.ncls;
        ff.ncls++;
    }
    // global-memory tables of the exact bound 2 min(w, n - 1) (rows beyond shared memory)
    const int64_t Tmax = pow2_at_least(2 * (n > 1 ? n - 1 : 1));
    const int64_t gslice_bytes = (int64_t)((num_table_bytes(Tmax, S) + 255) & ~(size_t)255);

    // ---- fused path (no symbolic pass): guessed tables, rows written to a temporary region
    if (tune("spgemm_fused")) {
        stage.emplace("SpGEMMNumeric", s);
        int64_t *room = sc.get<int64_t>(n + 1), *tmp_off = sc.get<int64_t>(n + 1), *need_f = sc.get<int64_t>(n + 1);
        int32_t *lists_f = sc.get<int32_t>((size_t)(SP_NCLS + 1) * (n + 1));
        if (!room || !tmp_off || !need_f || !lists_f) return SG_ERR_OOM;
        // filtered rows: mode 2 always, mode 1 when the sample finds under half the partners recur
        const int64_t fmode = tune("spgemm_filter_mode");
        int64_t fwork = min_shared >= 2 && ff.ncls > 0 && fmode > 0 ? tune("spgemm_filter_work") : 0;
        // table guesses from a sample of rows (large inputs only): partners per product, r1 distinct
        // and r2 seen at least twice
        uint64_t fu = 0, ffq = 0;
        const int64_t nsamp = A->nnz >= tune("spgemm_sample_min_nnz") ? tune("spgemm_sample_rows") : 0;
        bool recur = true;  // without a sample, mode 1 does not filter
        if (nsamp > 0 && n > 0) {
            const int64_t stride = n > nsamp ? n / nsamp : 1;
            const int64_t nb = (n + stride - 1) / stride;
            unsigned long long *sums = counts + 4 * NCNT + 1;  // zeroed with the counters
            SG_CUDA_TRY(ensure_smem(sample_kernel, fbytes));
            SG_LAUNCH("spgemm_sample", sample_kernel, nb, 256, fbytes, s, g, (const int64_t *)work, stride, log2F,
                      sums);
            unsigned long long h[3] = {0, 0, 0};
            SG_CUDA_TRY(read_back(h, sums, sizeof(h), s));
            if (h[0] > 0) {
                const double pct = (double)tune("spgemm_guess_pct") / 100.0;
                const double r1 = (double)h[1] / (double)h[0], r2 = (double)h[2] / (double)h[0];
                fu = (uint64_t)(pct * r1 * 65536.0) + 1;
                ffq = (uint64_t)(pct * r2 * 65536.0) + 1;
                recur = r1 < 2.0 * r2;  // most partners recur: the filter would keep nearly all
            }
        }
        if (fmode == 1 && recur) fwork = 0;
        SG_LAUNCH("fused_need", fused_need_kernel, blocks_for(n, NT), NT, 0, s, (const int64_t *)work, n,
                  (int)tune("num_guess_shift"), fu, min_shared, fwork, (int)tune("spgemm_filter_shift"), ffq,
                  ff.ncls > 0 ? (int64_t)1 << ff.log2T[ff.ncls - 1] : (int64_t)64, need, need_f, room);
        SG_TRY(exclusive_scan<int64_t>(room, tmp_off, n, s, err));
        SG_LAUNCH("classify", classify_kernel, blocks_for(n, NT), NT, 0, s, need, n, fz, fz_counts, lists);
        if (fwork)
            SG_LAUNCH("classify", classify_kernel, blocks_for(n, NT), NT, 0, s, need_f, n, ff, ff_counts, lists_f);
        unsigned long long h_fz[NCNT], h_ff[NCNT];
        int64_t tmp_n = 0;
        uint32_t herr = 0;
        SG_CUDA_TRY(cudaMemcpyAsync(h_ff, ff_counts, sizeof(h_ff), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaMemcpyAsync(h_fz, fz_counts, sizeof(h_fz), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(read_back(&tmp_n, tmp_off + n, sizeof(int64_t), s));
        if (herr & DEV_TIMEOUT) return timeout_error("overlap_spgemm");
        const double tmp_bytes = (double)tmp_n * (8.0 + 8.0 * S);
        // the region is reserved, mostly untouched: at most half of what the device can still give
        const double avail = (double)device_bytes_available();
        if (tmp_bytes <= (double)tune("spgemm_fused_max_mb") * 1048576.0 && tmp_bytes <= 0.5 * avail) {
            int32_t *t_col = sc.get<int32_t>(tmp_n + 1);
            uint32_t *t_cnt = sc.get<uint32_t>(tmp_n + 1);
            uint32_t *t_si = sc.get<uint32_t>((size_t)S * tmp_n + 1), *t_sk = sc.get<uint32_t>((size_t)S * tmp_n + 1);
            if (!t_col || !t_cnt || !t_si || !t_sk) return SG_ERR_OOM;
            for (int c = 0; c < fz.ncls; c++) {
                if (!h_fz[c]) continue;
                const size_t sm = num_table_bytes((int64_t)1 << fz.log2T[c], S, true);
                SG_CUDA_TRY(ensure_smem(numeric_kernel<false, true>, sm));
                SG_LAUNCH(NUM_NAMES[fz.log2T[c] - SP_MINLOG], (numeric_kernel<false, true>), grid,
                          pick_numeric_threads(fz.log2T[c], false), sm, s, g, lists + (int64_t)c * n, fz_counts + c,
                          fz.log2T[c], 0,
                          (const int64_t *)need, (unsigned char *)nullptr, (int64_t)0, (const int64_t *)tmp_off,
                          t_col, t_cnt, t_si, t_sk, tmp_n, (const int64_t *)work, ovf, fz_ovf, nnz_row);
            }
            for (int c = 0; fwork && c < ff.ncls; c++) {  // rows with many products: filtered first
                if (!h_ff[c]) continue;
                const size_t sm = num_table_bytes((int64_t)1 << ff.log2T[c], S, true) + fbytes;
                SG_CUDA_TRY(ensure_smem(numeric_kernel<false, true, true>, sm));
                SG_LAUNCH(FIL_NAMES[ff.log2T[c] - SP_MINLOG], (numeric_kernel<false, true, true>), grid,
                          pick_numeric_threads(ff.log2T[c], true), sm, s, g, lists_f + (int64_t)c * n, ff_counts + c,
                          ff.log2T[c], log2F, (const int64_t *)need_f, (unsigned char *)nullptr, (int64_t)0,
                          (const int64_t *)tmp_off, t_col, t_cnt, t_si, t_sk, tmp_n, (const int64_t *)work, ovf,
                          fz_ovf, nnz_row);
            }
            unsigned long long n_ovf = 0;
            SG_CUDA_TRY(read_back(&n_ovf, fz_ovf, sizeof(n_ovf), s));
            const unsigned long long n_big = h_fz[fz.ncls], n_big_f = fwork ? h_ff[ff.ncls] : 0;
            if (n_big + n_big_f + n_ovf > 0) {
                unsigned long long rows_g = n_big > n_ovf ? n_big : n_ovf;
                rows_g = rows_g > n_big_f ? rows_g : n_big_f;
                const int ggrid = (int)(rows_g < (unsigned long long)nsm * 2 ? rows_g : (unsigned long long)nsm * 2);
                unsigned char *pool = sc.get<unsigned char>((size_t)gslice_bytes * ggrid);
                if (!pool) return SG_ERR_OOM;
                if (n_big)
                    SG_LAUNCH("spgemm_numeric_gmem", (numeric_kernel<true, true>), ggrid, 512, 0, s, g,
                              lists + (int64_t)fz.ncls * n, fz_counts + fz.ncls, 0, 0, (const int64_t *)need, pool,
                              gslice_bytes, (const int64_t *)tmp_off, t_col, t_cnt, t_si, t_sk, tmp_n,
                              (const int64_t *)work, ovf + n + 1, unused, nnz_row);
                if (n_big_f)
                    SG_LAUNCH("spgemm_numeric_gmem", (numeric_kernel<true, true>), ggrid, 512, 0, s, g,
                              lists_f + (int64_t)ff.ncls * n, ff_counts + ff.ncls, 0, 0, (const int64_t *)need_f,
                              pool, gslice_bytes, (const int64_t *)tmp_off, t_col, t_cnt, t_si, t_sk, tmp_n,
                              (const int64_t *)work, ovf + n + 1, unused, nnz_row);
                if (n_ovf)
                    SG_LAUNCH("spgemm_numeric_gmem", (numeric_kernel<true, true>), ggrid, 512, 0, s, g,
                              (const int32_t *)ovf, fz_ovf, 0, 0, (const int64_t *)need, pool, gslice_bytes,
                              (const int64_t *)tmp_off, t_col, t_cnt, t_si, t_sk, tmp_n, (const int64_t *)work,
                              ovf + n + 1, unused, nnz_row);
            }
            SG_ALLOC(C->row_ptr, int64_t, n + 1, s);
            SG_TRY(exclusive_scan<int64_t>(nnz_row, C->row_ptr, n, s, err));
            int64_t nnz = 0;
            SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            SG_CUDA_TRY(read_back(&nnz, C->row_ptr + n, sizeof(int64_t), s));
            if (herr & DEV_TIMEOUT) return timeout_error("overlap_spgemm");
            if (herr) {
                set_error("overlap_spgemm: a row exceeded its output bound (internal error)");
                return SG_ERR_OVERFLOW;
            }
            C->n = n;
            C->nnz = nnz;
            C->max_seeds = S;
            SG_ALLOC(C->col, int32_t, nnz, s);
            SG_ALLOC(C->count, uint32_t, nnz, s);
            SG_ALLOC(C->seed_i, uint32_t, (int64_t)S * nnz, s);
            SG_ALLOC(C->seed_k, uint32_t, (int64_t)S * nnz, s);
            SG_LAUNCH("compact_c", compact_c_kernel, blocks_for(n * 32, 256), 256, 0, s, (const int64_t *)tmp_off,
                      tmp_n, (const int32_t *)t_col, (const uint32_t *)t_cnt, (const uint32_t *)t_si,
                      (const uint32_t *)t_sk, S, (const int64_t *)C->row_ptr, n, nnz, C->col, C->count, C->seed_i,
                      C->seed_k);
            return SG_OK;
        }
        // the temporary region would exceed its budget: the two-pass path below
    }

    // ---- symbolic: guessed shared-memory tables of 2^6 .. 2^14 slots, one class per size
    Classes sym{};
    sym.ncls = SP_NCLS;
    for (int c = 0; c < SP_NCLS; c++) sym.log2T[c] = SP_MINLOG + c;
    SG_LAUNCH("sym_need", sym_need_kernel, blocks_for(n, NT), NT, 0, s, work, n, (int)tune("sym_guess_shift"),
              need);
    SG_LAUNCH("classify", classify_kernel, blocks_for(n, NT), NT, 0, s, need, n, sym, sym_counts, lists);
    for (int c = 0; c < sym.ncls; c++) {
        const size_t sm = (size_t)(2 << sym.log2T[c]) * sizeof(int32_t);
        SG_CUDA_TRY(ensure_smem(symbolic_kernel<false>, sm));
        SG_LAUNCH(SYM_NAMES[sym.log2T[c] - SP_MINLOG], symbolic_kernel<false>, grid, pick_threads(sym.log2T[c]), sm,
                  s, g,
                  lists + (int64_t)c * n, sym_counts + c, sym.log2T[c], (const int64_t *)work, (int32_t *)nullptr,
                  (int64_t)0, ovf, ovf_count, nnz_row, dist);
    }
    // rows too large for any shared-memory table, and rows whose guessed table overflowed
    unsigned long long h_sym[NCNT];
    SG_CUDA_TRY(read_back(h_sym, sym_counts, sizeof(h_sym), s));
    const unsigned long long n_big = h_sym[sym.ncls], n_ovf = h_sym[SP_NCLS + 1];
    if (n_big + n_ovf > 0) {
        const int64_t slice = 2 * pow2_at_least(2 * (n > 1 ? n - 1 : 1));  // keys + counts of the largest row
        const unsigned long long rows_g = n_big > n_ovf ? n_big : n_ovf;
        const int grid = (int)(rows_g < (unsigned long long)nsm * 2 ? rows_g : (unsigned long long)nsm * 2);
        int32_t *pool = sc.get<int32_t>((size_t)slice * grid);
        if (!pool) return SG_ERR_OOM;
        if (n_big)
            SG_LAUNCH("spgemm_symbolic_gmem", symbolic_kernel<true>, grid, 512, 0, s, g,
                      lists + (int64_t)sym.ncls * n, sym_counts + sym.ncls, 0, (const int64_t *)work, pool, slice,
                      ovf, ovf_count, nnz_row, dist);
        if (n_ovf)  // global-slice tables never overflow, so this pass never appends to the list
            SG_LAUNCH("spgemm_symbolic_gmem", symbolic_kernel<true>, grid, 512, 0, s, g, (const int32_t *)ovf,
                      ovf_count, 0, (const int64_t *)work, pool, slice, ovf + n + 1, unused, nnz_row, dist);
    }

    // ---- C row pointers; numeric classes from the exact distinct counts
    stage.emplace("SpGEMMNumeric", s);
    SG_ALLOC(C->row_ptr, int64_t, n + 1, s);
    SG_TRY(exclusive_scan<int64_t>(nnz_row, C->row_ptr, n, s, err));
    SG_LAUNCH("num_need", num_need_kernel, blocks_for(n, NT), NT, 0, s, dist, n, need);
    SG_LAUNCH("classify", classify_kernel, blocks_for(n, NT), NT, 0, s, need, n, num, num_counts, lists);
    int64_t nnz = 0;
    unsigned long long h_num[NCNT];
    uint32_t herr = 0;
    SG_CUDA_TRY(cudaMemcpyAsync(h_num, num_counts, sizeof(h_num), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(read_back(&nnz, C->row_ptr + n, sizeof(int64_t), s));
    if (herr & DEV_TIMEOUT) return timeout_error("overlap_spgemm");  // before anything uses row_ptr
    C->n = n;
    C->nnz = nnz;
    C->max_seeds = S;
    SG_ALLOC(C->col, int32_t, nnz, s);
    SG_ALLOC(C->count, uint32_t, nnz, s);
    SG_ALLOC(C->seed_i, uint32_t, (int64_t)S * nnz, s);
    SG_ALLOC(C->seed_k, uint32_t, (int64_t)S * nnz, s);
    for (int c = 0; c < num.ncls; c++) {
        if (!h_num[c]) continue;
        const size_t sm = num_table_bytes((int64_t)1 << num.log2T[c], S);
        SG_CUDA_TRY(ensure_smem(numeric_kernel<false, false>, sm));
        SG_LAUNCH(NUM_NAMES[num.log2T[c] - SP_MINLOG], (numeric_kernel<false, false>), grid,
                  pick_numeric_threads(num.log2T[c], false), sm, s, g, lists + (int64_t)c * n, num_counts + c,
                  num.log2T[c], 0,
                  (const int64_t *)need, (unsigned char *)nullptr, (int64_t)0, (const int64_t *)C->row_ptr, C->col,
                  C->count, C->seed_i, C->seed_k, nnz, (const int64_t *)nullptr, (int32_t *)nullptr,
                  (unsigned long long *)nullptr, (int64_t *)nullptr);
    }
    if (h_num[num.ncls]) {
        const int ggrid =
            (int)(h_num[num.ncls] < (unsigned long long)nsm * 2 ? h_num[num.ncls] : (unsigned long long)nsm * 2);
        unsigned char *pool = sc.get<unsigned char>((size_t)gslice_bytes * ggrid);
        if (!pool) return SG_ERR_OOM;
        SG_LAUNCH("spgemm_numeric_gmem", (numeric_kernel<true, false>), ggrid, 512, 0, s, g,
                  lists + (int64_t)num.ncls * n, num_counts + num.ncls, 0, 0, (const int64_t *)need, pool,
                  gslice_bytes,
                  (const int64_t *)C->row_ptr, C->col, C->count, C->seed_i, C->seed_k, nnz, (const int64_t *)nullptr,
                  (int32_t *)nullptr, (unsigned long long *)nullptr, (int64_t *)nullptr);
    }
    SG_CUDA_TRY(read_back(&herr, err, sizeof(uint32_t), s));
    if (herr & DEV_TIMEOUT) return timeout_error("overlap_spgemm");
    if (herr) {
        set_error("overlap_spgemm: numeric and symbolic passes disagree on a row size (internal error)");
        return SG_ERR_OVERFLOW;
    }
    return SG_OK;
}

}  // namespace sg

extern "C" sg_status sg_overlap_spgemm(const sg_csr_u32 *A, const sg_csr_u32 *At, uint32_t min_shared,
                                       int32_t max_seeds, sg_overlap_csr *C, sg_stream_t stream) {
    if (!C) {
        sg::set_error("overlap_spgemm: NULL output struct");
        return SG_ERR_INVALID;
    }
    *C = sg_overlap_csr{};
    if (!A || !At || max_seeds < 0 || max_seeds > sg::SP_MAX_SEEDS || min_shared < 1 || A->n_rows != At->n_cols ||
        A->n_cols != At->n_rows || A->nnz != At->nnz || A->n_rows < 0 || A->n_rows >= ((int64_t)1 << 31) ||
        !A->row_ptr || !At->row_ptr) {
        sg::set_error("overlap_spgemm: invalid arguments");
        return SG_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    sg_status st;
    {
        sg::Scratch sc(s);
        st = sg::overlap_impl(A, At, min_shared, max_seeds, C, s, sc);
    }
    if (st != SG_OK) sg_free_overlap(C, stream);
    return st;
}

extern "C" void sg_free_overlap(sg_overlap_csr *c, sg_stream_t stream) {
    if (!c) return;
    cudaStream_t s = (cudaStream_t)stream;
    sg::dfree(c->row_ptr, s);
    sg::dfree(c->col, s);
    sg::dfree(c->count, s);
    sg::dfree(c->seed_i, s);
    sg::dfree(c->seed_k, s);
    *c = sg_overlap_csr{};
}
