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
#include <algorithm>
#include <mutex>
#include <optional>
#include <vector>

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
    int64_t n;      // rows of A handled by this call
    uint32_t min_shared;
    int S;
    uint32_t *err;  // DEV_OVERFLOW if the numeric pass ever disagrees with the symbolic sizes
    int64_t np;     // partners: columns of At (all reads); n = np unless A is a row range of a larger A
    int64_t row0;   // read id of row 0 of A (nonzero only for a row range), for the diagonal
    const struct AtRec *t_rec;  // At rows as 32-byte records (fused pass), or nullptr
};

// One At row as a 32-byte record: its start in At, its length and, when it has at most AT_INL
// entries, their reads. An A entry's products then cost one aligned 32-byte load -- one DRAM
// sector -- instead of a row-pointer gather plus a gather of the row.
constexpr int AT_INL = 5;
struct __align__(32) AtRec {
    int64_t b;
    uint32_t len;
    int32_t r[AT_INL];
};
static_assert(sizeof(AtRec) == 32, "one sector per record");

__device__ __forceinline__ AtRec load_rec(const AtRec *p) {
    const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint4 y = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
    AtRec r;
    r.b = (int64_t)(((uint64_t)x.y << 32) | x.x);
    r.len = x.z;
    r.r[0] = (int32_t)x.w;
    r.r[1] = (int32_t)y.x;
    r.r[2] = (int32_t)y.y;
    r.r[3] = (int32_t)y.z;
    r.r[4] = (int32_t)y.w;
    return r;
}

// One thread per row j of At: its record.
__global__ void at_rec_kernel(const int64_t *__restrict__ t_rp, const int32_t *__restrict__ t_col, int64_t m,
                              AtRec *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int64_t b = t_rp[j], len = t_rp[j + 1] - b;
    uint4 x, y;
    x.x = (uint32_t)b;
    x.y = (uint32_t)((uint64_t)b >> 32);
    x.z = len > 0xFFFFFFFFll ? 0xFFFFFFFFu : (uint32_t)len;
    int32_t r[AT_INL];
#pragma unroll
    for (int t = 0; t < AT_INL; t++) r[t] = (len <= AT_INL && t < len) ? t_col[b + t] : -1;
    x.w = (uint32_t)r[0];
    y.x = (uint32_t)r[1];
    y.y = (uint32_t)r[2];
    y.z = (uint32_t)r[3];
    y.w = (uint32_t)r[4];
    reinterpret_cast<uint4 *>(out + j)[0] = x;
    reinterpret_cast<uint4 *>(out + j)[1] = y;
}

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
__global__ void sym_need_kernel(const int64_t *__restrict__ work, int64_t n, int64_t np, int shift,
                                int64_t *__restrict__ need) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t w = work[i];
    if (w <= 0) { need[i] = 0; return; }
    int64_t exact = pow2_at_least(2 * (w < np - 1 ? w : np - 1));
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
            const int64_t T = pow2_at_least(2 * (w < g.np - 1 ? w : g.np - 1));
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
        for_each_product<false>(g, (int32_t)(g.row0 + i), g.a_rp[i], g.a_rp[i + 1], GSLICE ? nullptr : &s_ovf,
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
// S shared k-mers with the smallest columns, the seeds kept (a choice that does not depend on the
// order of the updates). The positions are looked up when the row is written: pos_i from A's
// entry, pos_k from At's row j (sorted by read).
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
                T = pow2_at_least(2 * (w < g.np - 1 ? w : g.np - 1));
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
        const bool fid = g.np <= ((int64_t)1 << log2F);
        auto fbit = [&](int32_t k) -> uint32_t {
            return fid ? (uint32_t)k & ((1u << log2F) - 1u) : ((uint32_t)k * 2654435761u) >> (32 - log2F);
        };
        if (FILT) {  // seen once -> F1, seen again -> F2 (bits are only ever set)
            for_each_product<false>(g, (int32_t)(g.row0 + i), r0, r1, nullptr, [&](int32_t k, uint32_t, int64_t) {
                const uint32_t b = fbit(k), m = 1u << (b & 31u);
                if (((volatile uint32_t *)F2)[b >> 5] & m) return;
                if (atomicOr(F1 + (b >> 5), m) & m) atomicOr(F2 + (b >> 5), m);
            });
            __syncthreads();
        }
        const int cap = (T >> 1) + (T >> 2);  // guessed tables: at most 3/4 T partners
        for_each_product<false>(g, (int32_t)(g.row0 + i), r0, r1, guessed ? &s_ovf : nullptr, [&](int32_t k, uint32_t, int64_t idx) {
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

// ------------------------------------------------------------------------ fused numeric pass
// The default numeric pass. Each block takes a row i of C and walks A's row: for an entry (i, j)
// it reads the extent of At row j and, in the upper-triangle form, finds read i in it (At rows
// are sorted by read); the products are the At entries after i (upper) or all but i (whole
// rows). No per-entry table of At extents is stored beforehand: the extent is read where it is
// used, so each A entry costs one gather of At's row pointers and one of its (short) row.
//
// Upper-triangle form: C is symmetric (the shared set of (i, k) is that of (k, i); C_ki's seeds
// are C_ik's with the two positions swapped and the same rc bit), so only partners k > i are
// tabulated, which halves the table work. C is then assembled from the upper triangle U by
// writing each U row in place and its mirror into the lower part of the partner's row
// (mirror_c_kernel, packed records), whose entries are put in column order by a sort per row
// (sort_lower_kernel).
//
// Table slot (64 bits): partner << 32 | count; empty = ~0. A product whose partner is present
// costs one 64-bit atomicAdd on the slot; a new partner claims an empty slot and counts itself
// with one atomicCAS. Seeds, by max_seeds: 1 -> one u32 slot kept by atomicMin; 2 -> one u64 word
// (smallest << 32 | second smallest) replaced by atomicCAS only while the new index is smaller
// than the second (later indices, the common case, cost one load); more -> the atomicMin chain.
//
// Finished rows reserve their entries in a temporary region by one atomicAdd on a cursor (row i
// at tmp_off[i]); a row that finds the region full is listed for a retry in a grown region.

// Extent [beg, beg + len) of the products of A entry a of row gi (read id): the tail of At row
// j = a_col[a] after read gi (UPPER), or the whole row (gi itself is skipped by the caller). With
// records, a row of at most AT_INL entries is read from its record: *rec receives it and *t0 the
// index of the first product within it; *t0 = -1 otherwise (the products are read from t_col).
template <bool UPPER>
__device__ __forceinline__ void at_extent(const SpArgs &g, int64_t a, int32_t gi, int64_t &beg, uint32_t &len,
                                          AtRec *rec = nullptr, int *t0 = nullptr) {
    const int32_t j = g.a_col[a];
    int64_t b, e;
    if (g.t_rec) {
        const AtRec r = load_rec(g.t_rec + j);
        b = r.b;
        if (r.len <= AT_INL) {
            int t = 0;
            if (UPPER) {
#pragma unroll
                for (int q = 0; q < AT_INL; q++)
                    if (q < (int)r.len && r.r[q] <= gi) t = q + 1;
            }
            beg = b + t;
            len = r.len - (uint32_t)t;
            if (rec) *rec = r;
            if (t0) *t0 = t;
            return;
        }
        e = b + (int64_t)r.len;
    } else {
        b = g.t_rp[j];
        e = g.t_rp[j + 1];
    }
    if (t0) *t0 = -1;
    int64_t lo = b;
    if (UPPER) {
        int64_t hi = e;
        while (lo < hi) {  // first entry of At row j with read > gi
            const int64_t mid = (lo + hi) >> 1;
            if (g.t_col[mid] <= gi) lo = mid + 1; else hi = mid;
        }
    }
    beg = lo;
    len = (uint32_t)(e - lo);
}

// Products of row i (read id gi) with their partner counts: f(k, idx) for every product, k = the
// partner, idx = index of the A entry within the row; k == gi is skipped. Warp-cooperative: a warp
// takes 32 consecutive entries of A's row, finds their extents, scans their lengths (32-bit) and
// walks the flattened products TU_U x 32 at a time, each lane finding its entry by a 5-step
// shuffle search; the gathers of the next step are issued before the current step's table
// updates. Stops (per warp, at a chunk boundary) once *stop is nonzero.
constexpr int TU_U = 2;

// With records (g.t_rec), wb is this block's buffer of AT_INL x 32 ints per warp: each lane puts
// its record's reads there, and a product of a short row is read from it instead of from t_col.
constexpr int WB_PER_WARP = 32 * AT_INL;

template <bool UPPER, class F>
__device__ __forceinline__ void enum_fused(const SpArgs &g, int32_t gi, int64_t r0, int64_t r1,
                                           const volatile int *stop, int32_t *wb, F &&f) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int32_t *wbw = wb ? wb + warp * WB_PER_WARP : nullptr;
    for (int64_t a0 = r0 + (int64_t)warp * 32; a0 < r1; a0 += (int64_t)nwarps * 32) {
        if (stop && __any_sync(0xffffffffu, *stop != 0)) return;
        const int64_t a = a0 + lane;
        int64_t beg = 0;
        uint32_t len = 0;
        int wsrc = -1;  // index in wbw of this lane's first product, or -1: products in t_col
        AtRec rec;
        int t0 = -1;
        if (a < r1) {
            if (wbw) at_extent<UPPER>(g, a, gi, beg, len, &rec, &t0);
            else at_extent<UPPER>(g, a, gi, beg, len);
        }
        if (wbw) {
            __syncwarp();  // the previous chunk's reads of wbw are done
            if (t0 >= 0) {
#pragma unroll
                for (int q = 0; q < AT_INL; q++) wbw[lane * AT_INL + q] = rec.r[q];
                wsrc = lane * AT_INL + t0;
            }
            __syncwarp();  // every lane's reads are in wbw
        }
        uint32_t inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t excl = inc - len;
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        if (total == 0) continue;
        int32_t kk[TU_U];
        uint32_t ix[TU_U];
        auto gather = [&](uint32_t base) {
#pragma unroll
            for (int u = 0; u < TU_U; u++) {
                const uint32_t p = base + u * 32 + lane;
                int ow = 0;  // largest lane whose exclusive prefix is <= p
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    const uint32_t v = __shfl_sync(0xffffffffu, excl, (ow + s) & 31);
                    if (ow + s < 32 && v <= p) ow += s;
                }
                const int64_t ob = __shfl_sync(0xffffffffu, beg, ow);
                const uint32_t oe = __shfl_sync(0xffffffffu, excl, ow);
                const int os = __shfl_sync(0xffffffffu, wsrc, ow);
                ix[u] = (uint32_t)(a0 - r0) + (uint32_t)ow;
                kk[u] = p >= total ? gi : (os >= 0 ? wbw[os + (int)(p - oe)] : g.t_col[ob + (p - oe)]);
            }
        };
        gather(0);
        for (uint32_t base = 0; base < total; base += 32 * TU_U) {
            int32_t k_cur[TU_U];
            uint32_t i_cur[TU_U];
#pragma unroll
            for (int u = 0; u < TU_U; u++) {
                k_cur[u] = kk[u];
                i_cur[u] = ix[u];
            }
            if (base + 32 * TU_U < total) gather(base + 32 * TU_U);
#pragma unroll
            for (int u = 0; u < TU_U; u++)
                if (k_cur[u] != gi) f(k_cur[u], i_cur[u]);
        }
    }
}

constexpr uint64_t SLOT_EMPTY = ~0ull;

// At value of partner k in At row [b, b + len) (ascending reads), from the col and val arrays.
__device__ __forceinline__ uint32_t at_value_cv(const int32_t *__restrict__ t_col, const uint32_t *__restrict__ t_val,
                                                int64_t b, int64_t len, int32_t k) {
    int64_t lo = b, hi = b + len;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (t_col[mid] <= k) lo = mid; else hi = mid;
    }
    return t_val[lo];
}

// Bytes of one table of T slots with S seeds: slots u64[T] | seeds | sort buffer u64[T / 2].
__host__ __device__ inline size_t tab_seed_bytes(int64_t T, int S) {
    return S == 0 ? 0 : (S == 2 ? (size_t)T * 8 : (size_t)T * 4 * (size_t)S);
}
__host__ __device__ inline size_t tab_bytes(int64_t T, int S) {
    return (size_t)T * 8 + tab_seed_bytes(T, S) + (size_t)(T / 2) * 8;
}

// Where finished rows go: the temporary region (capacity cap entries, seeds slot-major with stride
// cap), its cursor, each row's offset and length, the rows to retry, and (upper form) the number of
// mirrored entries each row of C will receive.
struct TmpOut {
    int32_t *col;
    uint32_t *cnt, *si, *sk;
    int64_t cap;
    unsigned long long *cursor;
    int64_t *off, *len;
    int32_t *retry;
    unsigned long long *n_retry;
    uint32_t *colcnt;
};

// The numeric pass. GSLICE == false: a guessed table in shared memory; a table filling past 3/4,
// or keeping more than T / 2 partners, ends the row, which is appended to ovf_list. GSLICE ==
// true: a table of the exact bound 2 min(w, np - 1) slots in this block's slice of global memory,
// where w = wl[rb] is the row's product count (never overflows). SK: 0, 1, 2 seeds as above; 3 =
// the chain. FILT: the seen-once / seen-twice filters (2^log2F bits each) mark the partners of
// the row first, and only partners seen twice reach the table (min_shared >= 2).
// Registers of the numeric pass: at most 40 per thread, so that 48 warps fit an SM (64 registers
// would allow 32); the compiler spills a few bytes to stay under it.
#ifndef SG_TAB_BOUNDS
#define SG_TAB_BOUNDS __maxnreg__(40)
#endif

template <bool GSLICE, int SK, bool FILT, bool UPPER>
__global__ void SG_TAB_BOUNDS tab_numeric_kernel(SpArgs g, const int32_t *__restrict__ rows,
                                                         const unsigned long long *__restrict__ nrows_p, int log2T,
                                                         int log2F, unsigned char *__restrict__ gpool,
                                                         int64_t slice_bytes, const int64_t *__restrict__ wl,
                                                         TmpOut o, int32_t *__restrict__ ovf_list,
                                                         unsigned long long *__restrict__ ovf_count, int64_t wb_off,
                                                         int8_t *__restrict__ ovf_lt) {
    extern __shared__ __align__(16) unsigned char tab_raw[];
    int32_t *wb = g.t_rec ? (int32_t *)(tab_raw + wb_off) : nullptr;  // record reads, per warp
    __shared__ int s_ctr, s_ins, s_ovf, s_full, s_fail;
    __shared__ unsigned long long s_e0;
    const int S = g.S;
    const int64_t nrows = (int64_t)*nrows_p;
    for (int64_t rb = blockIdx.x; rb < nrows; rb += gridDim.x) {
        const int32_t i = rows[rb];
        if (!SG_IN_BOUNDS(i >= 0 && i < g.n, 308, i)) continue;
        const int32_t gi = (int32_t)(g.row0 + i);
        int lT = log2T;
        unsigned char *tb = FILT ? tab_raw + ((size_t)2 << log2F) / 8 : tab_raw;
        uint32_t *F1 = (uint32_t *)tab_raw, *F2 = F1 + ((1 << log2F) >> 5);
        if (GSLICE) {
            const int64_t w = wl[rb];
            const int64_t T = pow2_at_least(2 * (w < g.np - 1 ? w : g.np - 1));
            lT = 0;
            while (lT < 31 && ((int64_t)1 << lT) < T) lT++;
            if (!SG_IN_BOUNDS(tab_bytes((int64_t)1 << lT, S) <= (size_t)slice_bytes, 309, T)) continue;
            tb = gpool + (int64_t)blockIdx.x * slice_bytes;
        }
        const int32_t T = 1 << lT;
        const int ob_cap = T >> 1;
        uint64_t *slot = (uint64_t *)tb;
        unsigned char *sd = tb + (size_t)T * 8;
        uint64_t *seed2 = (uint64_t *)sd;
        uint32_t *seed1 = (uint32_t *)sd;
        uint64_t *obuf = (uint64_t *)(sd + tab_seed_bytes(T, S));
        for (int x = threadIdx.x; x < T; x += blockDim.x) slot[x] = SLOT_EMPTY;
        if (SK == 2)
            for (int x = threadIdx.x; x < T; x += blockDim.x) seed2[x] = ~0ull;
        else if (SK != 0)
            for (int x = threadIdx.x; x < T * S; x += blockDim.x) seed1[x] = SEED_NONE;
        if (FILT)
            for (int x = threadIdx.x; x < (2 << log2F) >> 5; x += blockDim.x) F1[x] = 0u;
        if (threadIdx.x == 0) {
            s_ctr = 0;
            s_ins = 0;
            s_ovf = 0;
            s_full = 0;
        }
        __syncthreads();
        const int64_t r0 = g.a_rp[i], r1 = g.a_rp[i + 1];
        const uint32_t msk = (uint32_t)T - 1u;
        const bool fid = g.np <= ((int64_t)1 << log2F);
        auto fbit = [&](int32_t k) -> uint32_t {
            return fid ? (uint32_t)k & ((1u << log2F) - 1u) : ((uint32_t)k * 2654435761u) >> (32 - log2F);
        };
        if (FILT) {  // seen once -> F1, seen again -> F2 (bits are only ever set)
            enum_fused<UPPER>(g, gi, r0, r1, nullptr, wb, [&](int32_t k, uint32_t) {
                const uint32_t b = fbit(k), m = 1u << (b & 31u);
                if (((volatile uint32_t *)F2)[b >> 5] & m) return;
                if (atomicOr(F1 + (b >> 5), m) & m) atomicOr(F2 + (b >> 5), m);
            });
            __syncthreads();
        }
        const int cap = (T >> 1) + (T >> 2);
        enum_fused<UPPER>(g, gi, r0, r1, GSLICE ? nullptr : &s_ovf, wb, [&](int32_t k, uint32_t idx) {
            if (!GSLICE && *(volatile int *)&s_ovf) return;
            if (FILT) {
                const uint32_t b = fbit(k);
                if (!((F2[b >> 5] >> (b & 31u)) & 1u)) return;
            }
            uint32_t h = hash_slot(k, lT);
            int probe = 0;
            uint64_t w2 = 0;
            for (;;) {
                uint64_t v = ((volatile uint64_t *)slot)[h];
                if (v == SLOT_EMPTY) {
                    v = atomicCAS((unsigned long long *)(slot + h), SLOT_EMPTY, ((uint64_t)(uint32_t)k << 32) | 1ull);
                    if (v == SLOT_EMPTY) {
                        if (!GSLICE && atomicAdd(&s_ins, 1) >= cap) s_ovf = 1;
                        w2 = ~0ull;  // a new partner's seeds are still empty, or being filled
                        break;
                    }
                }
                if ((int32_t)(v >> 32) == k) {
                    if (SK == 2) w2 = seed2[h];  // issued before the count update; the CAS below checks it
                    atomicAdd((unsigned long long *)(slot + h), 1ull);
                    break;
                }
                h = (h + 1) & msk;
                if (++probe == T) {  // went round the whole table
                    s_ovf = 1;
                    return;
                }
            }
            if (SK == 1) {
                atomicMin(seed1 + h, idx);
            } else if (SK == 2) {
                uint64_t w = w2;
                for (;;) {
                    const uint32_t m1 = (uint32_t)(w >> 32), m2 = (uint32_t)w;
                    if (idx >= m2 && w != ~0ull) break;  // indices of one partner are distinct
                    const uint64_t nw = idx < m1 ? (((uint64_t)idx << 32) | m1) : (((uint64_t)m1 << 32) | idx);
                    const uint64_t old = atomicCAS((unsigned long long *)(seed2 + h), w, nw);
                    if (old == w) break;
                    w = old;
                }
            } else if (SK == 3) {
                uint32_t v = idx;
                uint32_t *sl = seed1 + (int64_t)h * S;
                for (int q = 0; q < S; q++) {
                    const uint32_t old = atomicMin(sl + q, v);
                    if (old > v) v = old;
                    if (v == SEED_NONE) break;
                }
            }
        });
        __syncthreads();
        // kept partners -> sort buffer; a guessed table may keep more than it holds (s_full), an
        // exact one (T >= 2 x partners) never does. s_ovf is not written past the barrier above.
        if (GSLICE || !s_ovf) {
            for (int x = threadIdx.x; x < T; x += blockDim.x) {
                const uint64_t v = slot[x];
                if (v != SLOT_EMPTY && (uint32_t)v >= g.min_shared) {
                    const int p = atomicAdd(&s_ctr, 1);
                    if (SG_IN_BOUNDS(!GSLICE || p < ob_cap, 310, p) && p < ob_cap)
                        obuf[p] = (v & 0xFFFFFFFF00000000ull) | (uint32_t)x;
                    else
                        s_full = 1;
                }
            }
        }
        __syncthreads();
        if (!GSLICE && (s_ovf || s_full)) {  // the global-memory pass redoes the row
            if (threadIdx.x == 0) {
                const unsigned long long q = atomicAdd(ovf_count, 1ull);
                if (SG_IN_BOUNDS((int64_t)q < g.n, 311, q)) {
                    ovf_list[q] = i;
                    if (ovf_lt) ovf_lt[q] = (int8_t)lT;  // the table that was too small
                }
            }
            __syncthreads();
            continue;
        }
        const int nv = s_ctr < ob_cap ? s_ctr : ob_cap;
        if (threadIdx.x == 0) {  // reserve the row's entries in the temporary region
            const unsigned long long e0 = atomicAdd(o.cursor, (unsigned long long)nv);
            s_e0 = e0;
            s_fail = e0 + (unsigned long long)nv > (unsigned long long)o.cap;
            if (s_fail) {
                const unsigned long long q = atomicAdd(o.n_retry, 1ull);
                if (SG_IN_BOUNDS((int64_t)q < g.n, 316, q)) o.retry[q] = i;
            } else {
                o.off[i] = (int64_t)e0;
                o.len[i] = nv;
            }
        }
        int P2 = 1;
        while (P2 < nv) P2 <<= 1;
        for (int x = nv + threadIdx.x; x < P2; x += blockDim.x) obuf[x] = ~0ull;
        __syncthreads();
        if (s_fail) continue;  // the region is full: the row is redone in a grown one
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
        const int64_t e0 = (int64_t)s_e0;
        for (int q = threadIdx.x; q < nv; q += blockDim.x) {
            const uint64_t wq = obuf[q];
            const uint32_t x = (uint32_t)wq;
            const int32_t k = (int32_t)(wq >> 32);
            const int64_t e = e0 + q;
            o.col[e] = k;
            o.cnt[e] = (uint32_t)slot[x];
            if (o.colcnt) atomicAdd(o.colcnt + k, 1u);
            for (int s = 0; s < S; s++) {
                uint32_t sdx;
                if (SK == 2) sdx = s == 0 ? (uint32_t)(seed2[x] >> 32) : (uint32_t)seed2[x];
                else sdx = seed1[(int64_t)x * S + s];
                uint32_t si = SEED_NONE, sk = SEED_NONE;
                if (sdx != SEED_NONE) {
                    const int64_t a = r0 + sdx;
                    const uint32_t vi = g.a_val[a];
                    const int32_t j = g.a_col[a];
                    uint32_t vk;
                    if (g.t_rec) {
                        const AtRec rr = load_rec(g.t_rec + j);
                        if (rr.len <= AT_INL) {
                            int q = 0;
#pragma unroll
                            for (int t = 1; t < AT_INL; t++)
                                if (t < (int)rr.len && rr.r[t] <= k) q = t;
                            vk = g.t_val[rr.b + q];
                        } else {
                            vk = at_value_cv(g.t_col, g.t_val, rr.b, rr.len, k);
                        }
                    } else {
                        const int64_t tb0 = g.t_rp[j];
                        vk = at_value_cv(g.t_col, g.t_val, tb0, g.t_rp[j + 1] - tb0, k);
                    }
                    si = vi & 0x7FFFFFFFu;
                    sk = (vk & 0x7FFFFFFFu) | ((vi ^ vk) & 0x80000000u);
                }
                o.si[(int64_t)s * o.cap + e] = si;
                o.sk[(int64_t)s * o.cap + e] = sk;
            }
        }
        __syncthreads();
    }
}

// Products of listed rows (one warp each), for the exact global-memory tables and the retry
// region's size: wl[q] = w of row rows[q], *wmax = the largest, *room = sum of min(w / t, np - 1).
template <bool UPPER>
__global__ void rows_work_kernel(SpArgs g, const int32_t *__restrict__ rows, const unsigned long long *__restrict__ cnt_p,
                                 int64_t *__restrict__ wl, unsigned long long *__restrict__ wmax,
                                 unsigned long long *__restrict__ room) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= (int64_t)*cnt_p) return;
    const int32_t i = rows[q];
    if (!SG_IN_BOUNDS(i >= 0 && i < g.n, 317, i)) return;
    const int32_t gi = (int32_t)(g.row0 + i);
    int64_t w = 0;
    for (int64_t a = g.a_rp[i] + lane; a < g.a_rp[i + 1]; a += 32) {
        int64_t beg;
        uint32_t len;
        at_extent<UPPER>(g, a, gi, beg, len);
        w += len;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (!UPPER) w -= g.a_rp[i + 1] - g.a_rp[i];  // the diagonal: one product per entry
    if (lane == 0) {
        wl[q] = w;
        atomicMax(wmax, (unsigned long long)w);
        const int64_t r = std::min<int64_t>(w / g.min_shared, UPPER ? g.np - 1 - gi : g.np - 1);
        atomicAdd(room, (unsigned long long)(r > 0 ? r : 0));
    }
}

// Sampled rows (every stride-th row, one block each): the row's A entries, and the bits set in the
// seen-once and seen-twice filters after its products -- about its distinct partners and its
// partners seen at least twice. sums = {sum of A entries, sum F1 bits, sum F2 bits}.
template <bool UPPER>
__global__ void __launch_bounds__(512) sample_fx_kernel(SpArgs g, int64_t stride, int log2F,
                                                       unsigned long long *__restrict__ sums) {
    extern __shared__ __align__(16) uint32_t smp_f[];
    __shared__ unsigned long long s_c[2];
    const int64_t i = (int64_t)blockIdx.x * stride;
    if (i >= g.n) return;
    const int nw = (1 << log2F) >> 5;
    uint32_t *F1 = smp_f, *F2 = smp_f + nw;
    for (int x = threadIdx.x; x < 2 * nw; x += blockDim.x) smp_f[x] = 0u;
    if (threadIdx.x < 2) s_c[threadIdx.x] = 0ull;
    __syncthreads();
    const bool fid = g.np <= ((int64_t)1 << log2F);
    int32_t *wb = g.t_rec ? (int32_t *)(smp_f + 2 * nw) : nullptr;
    enum_fused<UPPER>(g, (int32_t)(g.row0 + i), g.a_rp[i], g.a_rp[i + 1], nullptr, wb, [&](int32_t k, uint32_t) {
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
        atomicAdd(sums, (unsigned long long)(g.a_rp[i + 1] - g.a_rp[i]));
        atomicAdd(sums + 1, s_c[0]);
        atomicAdd(sums + 2, s_c[1]);
    }
}

// Table requests of the fused pass, from each row's number of A entries L: a guess of
// (L * fu) >> 16 partners (fu = sampled partners per A entry, fixed point), at least 64 slots.
// Rows with L >= fwork (fwork > 0) take the filtered pass: their guess ((L * ff) >> 16, at most
// fcap = the largest filtered shared-memory table) goes to need_f and need is 0, else need_f is 0.
__global__ void fx_need_kernel(const int64_t *__restrict__ a_rp, int64_t n, uint64_t fu, int64_t fwork, uint64_t ff,
                               int64_t fcap, int64_t tcap, int64_t *__restrict__ need, int64_t *__restrict__ need_f) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t L = a_rp[i + 1] - a_rp[i];
    need_f[i] = 0;
    if (L <= 0) {
        need[i] = 0;
        return;
    }
    const bool filt = fwork > 0 && L >= fwork;
    const int64_t g0 = (int64_t)(((unsigned __int128)L * (filt ? ff : fu)) >> 16);
    int64_t guess = pow2_at_least(g0 > 64 ? g0 : 64);
    if (guess > tcap) guess = tcap;  // no row has more partners than the table bound for all reads
    if (filt && guess > fcap) guess = fcap;
    (filt ? need_f : need)[i] = guess;
    if (filt) need[i] = 0;
}

// C from the upper triangle U (rows at tmp_off, lengths nnz_row, seeds slot-major with stride
// tmp_n). One warp per row i of U: its entries go to C row i after the lower part (colcnt[i]
// entries), in order; each entry (i, k) also goes, mirrored (seed positions swapped, same rc bit),
// as one packed record (col, count, then si, sk per seed slot: 2 + 2S words) to a free place
// (cursor[k], zeroed) of row k's part of the lower record array (from lrp[k]); sort_lower_kernel
// moves those into C in column order.
__global__ void mirror_c_kernel(const int64_t *__restrict__ tmp_off, const int64_t *__restrict__ nnz_row,
                                int64_t tmp_n, const int32_t *__restrict__ t_col, const uint32_t *__restrict__ t_cnt,
                                const uint32_t *__restrict__ t_si, const uint32_t *__restrict__ t_sk, int S,
                                const uint32_t *__restrict__ colcnt, const int64_t *__restrict__ c_rp,
                                const int64_t *__restrict__ lrp, int64_t n, int64_t nnz, int64_t nnz_l,
                                uint32_t *__restrict__ cursor, int32_t *__restrict__ c_col,
                                uint32_t *__restrict__ c_cnt, uint32_t *__restrict__ c_si,
                                uint32_t *__restrict__ c_sk, uint32_t *__restrict__ lrec) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int64_t len = nnz_row[row];
    if (len == 0) return;
    const int64_t src = tmp_off[row], dst = c_rp[row] + colcnt[row];
    const int RS = 2 + 2 * S;
    for (int64_t e = lane; e < len; e += 32) {
        const int32_t k = t_col[src + e];
        const uint32_t cnt = t_cnt[src + e];
        c_col[dst + e] = k;
        c_cnt[dst + e] = cnt;
        if (!SG_IN_BOUNDS(k > row && k < n, 312, k)) continue;
        const uint32_t p = atomicAdd(cursor + k, 1u);
        const int64_t m = lrp[k] + p;
        if (!SG_IN_BOUNDS(p < colcnt[k] && m < nnz_l, 313, p)) continue;
        uint32_t *r = lrec + m * RS;
        r[0] = (uint32_t)row;
        r[1] = cnt;
        for (int q = 0; q < S; q++) {
            const uint32_t si = t_si[(int64_t)q * tmp_n + src + e], sk = t_sk[(int64_t)q * tmp_n + src + e];
            c_si[(int64_t)q * nnz + dst + e] = si;
            c_sk[(int64_t)q * nnz + dst + e] = sk;
            const bool none = si == SEED_NONE;
            r[2 + 2 * q] = none ? SEED_NONE : (sk & 0x7FFFFFFFu);
            r[3 + 2 * q] = none ? SEED_NONE : (si | (sk & 0x80000000u));
        }
    }
}

// Moves each row's lower part (colcnt[i] packed records from lrp[i], distinct columns < i, in
// arbitrary order) into C at c_rp[i] in column order. One block per row of up to lmax (<=
// LOWER_SMEM) entries: keys (column << 32 | offset) bitonic-sorted in shared memory, then each
// record copied from its offset. Longer parts are listed for lower_big_kernel.
constexpr int LOWER_SMEM = 4096;
constexpr int LOWER_NT = 256;

__device__ __forceinline__ void lower_copy(const uint32_t *__restrict__ r, int64_t to, int S, int64_t nnz,
                                           int32_t *__restrict__ c_col, uint32_t *__restrict__ c_cnt,
                                           uint32_t *__restrict__ c_si, uint32_t *__restrict__ c_sk) {
    c_col[to] = (int32_t)r[0];
    c_cnt[to] = r[1];
    for (int q = 0; q < S; q++) {
        c_si[(int64_t)q * nnz + to] = r[2 + 2 * q];
        c_sk[(int64_t)q * nnz + to] = r[3 + 2 * q];
    }
}

template <class K>
__device__ __forceinline__ void block_bitonic(K *key, int64_t P2) {
    for (int64_t kk = 2; kk <= P2; kk <<= 1) {
        for (int64_t jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int64_t x = threadIdx.x; x < P2; x += blockDim.x) {
                const int64_t y = x ^ jj;
                if (y > x) {
                    const K a = key[x], c = key[y];
                    if ((a > c) == ((x & kk) == 0)) {
                        key[x] = c;
                        key[y] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(LOWER_NT) sort_lower_kernel(const uint32_t *__restrict__ colcnt,
                                                           const int64_t *__restrict__ lrp,
                                                           const int64_t *__restrict__ c_rp, int64_t n, int64_t nnz,
                                                           int S, const uint32_t *__restrict__ lrec,
                                                           int32_t *__restrict__ c_col, uint32_t *__restrict__ c_cnt,
                                                           uint32_t *__restrict__ c_si, uint32_t *__restrict__ c_sk,
                                                           unsigned long long *__restrict__ big_count,
                                                           int32_t *__restrict__ big_rows, int lmax) {
    __shared__ uint64_t key[LOWER_SMEM];
    const int RS = 2 + 2 * S;
    for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
        const int64_t L = colcnt[row];
        if (L == 0) continue;
        const int64_t lb = lrp[row], b = c_rp[row];
        if (L > lmax) {
            if (threadIdx.x == 0) {
                const unsigned long long q = atomicAdd(big_count, 1ull);
                if (SG_IN_BOUNDS((int64_t)q < n, 314, q)) big_rows[q] = (int32_t)row;
            }
            continue;
        }
        if (L == 1) {
            if (threadIdx.x == 0) lower_copy(lrec + lb * RS, b, S, nnz, c_col, c_cnt, c_si, c_sk);
            continue;
        }
        int64_t P2 = 1;
        while (P2 < L) P2 <<= 1;
        for (int64_t x = threadIdx.x; x < P2; x += blockDim.x)
            key[x] = x < L ? (((uint64_t)lrec[(lb + x) * RS] << 32) | (uint32_t)x) : ~0ull;
        __syncthreads();
        block_bitonic(key, P2);
        for (int64_t x = threadIdx.x; x < L; x += blockDim.x)
            lower_copy(lrec + (lb + (uint32_t)key[x]) * RS, b + x, S, nnz, c_col, c_cnt, c_si, c_sk);
        __syncthreads();
    }
}

// Lower parts longer than LOWER_SMEM: one block per listed row, its keys sorted in this block's
// slice of global scratch (P2 = the next power of two of the length, 8 bytes each).
__global__ void __launch_bounds__(1024) lower_big_kernel(const uint32_t *__restrict__ colcnt,
                                                       const int64_t *__restrict__ lrp,
                                                       const int64_t *__restrict__ c_rp, int64_t nnz, int S,
                                                       const int32_t *__restrict__ rows,
                                                       const unsigned long long *__restrict__ nrows_p,
                                                       uint64_t *__restrict__ gpool, int64_t slice,
                                                       const uint32_t *__restrict__ lrec, int32_t *__restrict__ c_col,
                                                       uint32_t *__restrict__ c_cnt, uint32_t *__restrict__ c_si,
                                                       uint32_t *__restrict__ c_sk) {
    const int64_t nrows = (int64_t)*nrows_p;
    const int RS = 2 + 2 * S;
    uint64_t *key = gpool + (int64_t)blockIdx.x * slice;
    for (int64_t rb = blockIdx.x; rb < nrows; rb += gridDim.x) {
        const int32_t row = rows[rb];
        const int64_t L = colcnt[row], lb = lrp[row], b = c_rp[row];
        int64_t P2 = 1;
        while (P2 < L) P2 <<= 1;
        if (!SG_IN_BOUNDS(P2 <= slice, 315, L)) continue;
        for (int64_t x = threadIdx.x; x < P2; x += blockDim.x)
            key[x] = x < L ? (((uint64_t)lrec[(lb + x) * RS] << 32) | (uint32_t)x) : ~0ull;
        __syncthreads();
        block_bitonic(key, P2);
        for (int64_t x = threadIdx.x; x < L; x += blockDim.x)
            lower_copy(lrec + (lb + (uint32_t)key[x]) * RS, b + x, S, nnz, c_col, c_cnt, c_si, c_sk);
        __syncthreads();
    }
}

// C from the upper triangle U (rows at tmp_off, lengths nnz_row, seeds slot-major with stride
// tmp_n). One warp per row i of U: its entries go to C row i after the lower part (colcnt[i]
// entries), in order; every entry (i, k) also writes, at its row-major rank rpu[i] + e, a sort key
// (the partner k) and a value (i << 33 | its position in C). A stable sort by key then lists each
// column's entries by ascending row, which is the order of the mirrored entries in the lower part
// of row k (lower_fill_kernel).
constexpr int MIRROR_POS_BITS = 33;
// An entry of U as one 32-byte record (count, then si, sk per seed slot) for max_seeds <= 3, so
// that its mirror gathers one sector instead of 1 + 2 max_seeds words of C's arrays.
constexpr int MIRROR_REC_SEEDS = 3;
struct __align__(32) MirrorRec {
    uint32_t w[8];
};

__global__ void mirror_keys_kernel(const int64_t *__restrict__ tmp_off, const int64_t *__restrict__ nnz_row,
                                   int64_t tmp_n, const int32_t *__restrict__ t_col,
                                   const uint32_t *__restrict__ t_cnt, const uint32_t *__restrict__ t_si,
                                   const uint32_t *__restrict__ t_sk, int S, const uint32_t *__restrict__ colcnt,
                                   const int64_t *__restrict__ c_rp, const int64_t *__restrict__ rpu, int64_t n,
                                   int64_t nnz, int32_t *__restrict__ c_col, uint32_t *__restrict__ c_cnt,
                                   uint32_t *__restrict__ c_si, uint32_t *__restrict__ c_sk,
                                   uint32_t *__restrict__ mkey, uint64_t *__restrict__ mval,
                                   MirrorRec *__restrict__ mrec) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int64_t len = nnz_row[row];
    if (len == 0) return;
    const int64_t src = tmp_off[row], dst = c_rp[row] + colcnt[row], u0 = rpu[row];
    for (int64_t e = lane; e < len; e += 32) {
        const int32_t k = t_col[src + e];
        const uint32_t cnt = t_cnt[src + e];
        c_col[dst + e] = k;
        c_cnt[dst + e] = cnt;
        MirrorRec r = {};
        r.w[0] = cnt;
        for (int q = 0; q < S; q++) {
            const uint32_t si = t_si[(int64_t)q * tmp_n + src + e], sk = t_sk[(int64_t)q * tmp_n + src + e];
            c_si[(int64_t)q * nnz + dst + e] = si;
            c_sk[(int64_t)q * nnz + dst + e] = sk;
            if (q < MIRROR_REC_SEEDS) {
                r.w[1 + 2 * q] = si;
                r.w[2 + 2 * q] = sk;
            }
        }
        mkey[u0 + e] = (uint32_t)k;
        if (mrec) {  // the mirror reads this record by its index in U instead of C's arrays at dst + e
            mrec[u0 + e] = r;
            mval[u0 + e] = ((uint64_t)row << MIRROR_POS_BITS) | (uint64_t)(u0 + e);
        } else {
            mval[u0 + e] = ((uint64_t)row << MIRROR_POS_BITS) | (uint64_t)(dst + e);
        }
    }
}

// Sorted mirror list -> lower parts: entry q of the list (partner k, row i, position p of C_ik)
// is the (q - lrp[k])-th entry of row k's lower part: C_ki with the count of C_ik and its seeds'
// positions swapped (same rc bit).
__global__ void lower_fill_kernel(const uint32_t *__restrict__ mkey, const uint64_t *__restrict__ mval, int64_t nu,
                                  const int64_t *__restrict__ lrp, const int64_t *__restrict__ c_rp, int64_t n,
                                  int64_t nnz, int S, int32_t *__restrict__ c_col, uint32_t *__restrict__ c_cnt,
                                  uint32_t *__restrict__ c_si, uint32_t *__restrict__ c_sk,
                                  const MirrorRec *__restrict__ mrec) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nu) return;
    const uint32_t k = mkey[q];
    const uint64_t v = mval[q];
    // p: the U entry's position in C, or (records) its index in U
    const int64_t i = (int64_t)(v >> MIRROR_POS_BITS), p = (int64_t)(v & ((1ull << MIRROR_POS_BITS) - 1));
    if (!SG_IN_BOUNDS(k < n && p < (mrec ? nu : nnz), 312, q)) return;
    const int64_t d = c_rp[k] + (q - lrp[k]);
    if (!SG_IN_BOUNDS(d >= c_rp[k] && d < c_rp[k + 1], 313, d)) return;
    c_col[d] = (int32_t)i;
    MirrorRec r = {};
    if (mrec) {
        const uint4 *pr = reinterpret_cast<const uint4 *>(mrec + p);
        const uint4 a = __ldg(pr), b = __ldg(pr + 1);
        r.w[0] = a.x; r.w[1] = a.y; r.w[2] = a.z; r.w[3] = a.w;
        r.w[4] = b.x; r.w[5] = b.y; r.w[6] = b.z; r.w[7] = b.w;
    }
    c_cnt[d] = mrec ? r.w[0] : c_cnt[p];
    for (int s = 0; s < S; s++) {
        const uint32_t si = mrec ? r.w[1 + 2 * s] : c_si[(int64_t)s * nnz + p];
        const uint32_t sk = mrec ? r.w[2 + 2 * s] : c_sk[(int64_t)s * nnz + p];
        const bool none = si == SEED_NONE;
        c_si[(int64_t)s * nnz + d] = none ? SEED_NONE : (sk & 0x7FFFFFFFu);
        c_sk[(int64_t)s * nnz + d] = none ? SEED_NONE : (si | (sk & 0x80000000u));
    }
}

// nnz of C's rows in the upper-triangle form: U row i plus its mirrored entries.
__global__ void c_rowlen_kernel(const int64_t *__restrict__ nnz_row, const uint32_t *__restrict__ colcnt, int64_t n,
                                int64_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = nnz_row[i] + colcnt[i];
}

static inline int64_t blocks_for(int64_t n, int nt) { return (n + nt - 1) / nt; }

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

// Rows whose guessed table overflowed (ovf[0 .. *cnt_p), with the log2 size that was too small
// in lt) go to the smallest class at least 2^shift times larger, or to the global class.
__global__ void escalate_kernel(const int32_t *__restrict__ ovf, const int8_t *__restrict__ lt,
                                const unsigned long long *__restrict__ cnt_p, int shift, Classes cl, int64_t n,
                                unsigned long long *__restrict__ counts, int32_t *__restrict__ lists) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)*cnt_p) return;
    const int want = lt[q] + shift;
    int c = cl.ncls;
    for (int x = 0; x < cl.ncls; x++)
        if (cl.log2T[x] >= want) { c = x; break; }
    const unsigned long long p = atomicAdd(counts + c, 1ull);
    if (SG_IN_BOUNDS((int64_t)p < n, 318, p)) lists[(int64_t)c * n + (int64_t)p] = ovf[q];
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

// threads per block of the fused pass: enough warps that the blocks shared memory lets reside on
// one SM bring about spgemm_tab_warps warps (64 = the SM's limit) between them; for tables of 4 K
// slots and more, spgemm_tab_warps_big
// tsm = the table's (and filters') shared memory, warp_bytes = each warp's record buffer; code =
// log2T, negated for unfiltered tables (for the fixed choice when spgemm_tab_warps is 0)
static int pick_tab_threads(size_t tsm, size_t warp_bytes, int code) {
    const int log2T = code < 0 ? -code : code;
    int64_t want = tune("spgemm_tab_warps");
    if (want <= 0) return pick_numeric_threads(log2T, code > 0);
    if (log2T >= 12) want = tune("spgemm_tab_warps_big");
    int64_t threads = 64;
    for (;;) {
        const size_t bytes = tsm + warp_bytes * (size_t)(threads / 32);
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(32, (int64_t)((227u << 10) / bytes)));
        if (threads >= 1024 || blocks * (threads / 32) >= want) break;
        threads <<= 1;
    }
    return (int)threads;
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
                       sg_overlap_csr *C, cudaStream_t s, Scratch &sc, const OverlapOpts &opt) {
    const int64_t n = A->n_rows, np = At->n_cols;
    const int NT = 256;
    constexpr int NCNT = SP_NCLS + 2;  // classes + global class + overflow counter
    uint32_t *err = sc.get<uint32_t>(1);
    int64_t *work = sc.get<int64_t>(n + 1);
    int64_t *need = sc.get<int64_t>(n + 1);
    int64_t *nnz_row = sc.get<int64_t>(n + 1);
    int64_t *dist = sc.get<int64_t>(n + 1);
    unsigned long long *counts = sc.get<unsigned long long>(4 * NCNT + 10);
    int32_t *lists = sc.get<int32_t>((size_t)(SP_NCLS + 1) * (n + 1));
    int32_t *ovf = sc.get<int32_t>(2 * (n + 1));  // overflow list | unused list of the re-run
    if (!err || !work || !need || !nnz_row || !dist || !counts || !lists || !ovf) return SG_ERR_OOM;
    unsigned long long *sym_counts = counts, *num_counts = counts + NCNT, *unused = counts + 2 * NCNT;
    unsigned long long *ovf_count = counts + SP_NCLS + 1;
    unsigned long long *fz_counts = counts + 2 * NCNT + 1, *fz_ovf = fz_counts + SP_NCLS + 1;
    unsigned long long *ff_counts = counts + 3 * NCNT + 1;  // filtered rows' classes + global class
    SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    SG_CUDA_TRY(cudaMemsetAsync(counts, 0, (4 * NCNT + 10) * sizeof(unsigned long long), s));
    SG_CUDA_TRY(cudaMemsetAsync(nnz_row, 0, (n + 1) * sizeof(int64_t), s));
    SG_CUDA_TRY(cudaMemsetAsync(dist, 0, (n + 1) * sizeof(int64_t), s));
    uint64_t *t_pair = nullptr;  // only the two-pass kernels read At as (val << 32 | col) pairs
    SpArgs g{A->row_ptr, A->col, A->val, At->row_ptr, At->col, At->val, nullptr, nullptr, t_pair,
             n, min_shared, S, err, np, opt.row0, nullptr};
    const bool fused = opt.whole_rows || tune("spgemm_fused") != 0;
    const bool upper = fused && !opt.whole_rows && tune("spgemm_upper") != 0;
    std::optional<StageScope> stage;
    const int nsm = sm_count();
    const int grid = (int)(nsm * tune("spgemm_blocks_per_sm"));
    // the fused pass reads At through 32-byte row records when they fit beside everything else
    // (not for row ranges: every range would build them again, outside its budget)
    const int64_t m = At->n_rows;
    AtRec *recs = nullptr;
    if (fused && !opt.whole_rows && tune("spgemm_at_records") && m > 0 &&
        (double)m * sizeof(AtRec) <= 0.25 * (double)device_bytes_available()) {
        recs = sc.get<AtRec>(m);
        if (!recs) return SG_ERR_OOM;
        stage.emplace("SpGEMMSymbolic", s);
        SG_LAUNCH("at_records", at_rec_kernel, blocks_for(m, 256), 256, 0, s, At->row_ptr, At->col, m, recs);
        g.t_rec = recs;
    }
    // shared memory of the per-warp record buffers, for a block of `threads`
    auto wbb = [&](int threads) -> size_t { return recs ? (size_t)(threads / 32) * WB_PER_WARP * 4 : 0; };
    // numeric (two-pass form): one class per table size from 2^6 while table and sort buffer fit in 160 KB
    Classes num{};
    num.ncls = 0;
    while (num.ncls < SP_NCLS && num_table_bytes((int64_t)1 << (SP_MINLOG + num.ncls), S) <= (160u << 10)) {
        num.log2T[num.ncls] = SP_MINLOG + num.ncls;
        num.ncls++;
    }
    // the fused pass's guessed tables (up to 220 KB with the record buffers of 1024 threads: one
    // block per SM)
    const size_t tab_limit = (220u << 10) - wbb(1024);
    Classes fz{};
    fz.ncls = 0;
    while (fz.ncls < SP_NCLS && tab_bytes((int64_t)1 << (SP_MINLOG + fz.ncls), S) <= tab_limit) {
        fz.log2T[fz.ncls] = SP_MINLOG + fz.ncls;
        fz.ncls++;
    }
    // filtered rows (fused path): two filters of 2^log2F bits, one bit per read while np fits
    int log2F = 10;
    while (log2F < (int)tune("spgemm_filter_log2") && ((int64_t)1 << log2F) < np) log2F++;
    const size_t fbytes = ((size_t)2 << log2F) / 8;
    Classes ff{};
    ff.ncls = 0;
    while (ff.ncls < SP_NCLS && tab_bytes((int64_t)1 << (SP_MINLOG + ff.ncls), S) + fbytes <= tab_limit) {
        ff.log2T[ff.ncls] = SP_MINLOG + ff.ncls;
        ff.ncls++;
    }
    // global-memory tables of the exact bound 2 min(w, np - 1) for the two-pass form's largest row
    const int64_t Tmax = pow2_at_least(2 * (np > 1 ? np - 1 : 1));
    const int64_t gslice_bytes = (int64_t)((num_table_bytes(Tmax, S) + 255) & ~(size_t)255);
    const int SK = S <= 2 ? S : 3;

    // ---- fused path (no symbolic pass): guessed tables, rows written to a temporary region
    if (fused) {
        stage.emplace("SpGEMMNumeric", s);
        int64_t *tmp_off = sc.get<int64_t>(n + 1), *need_f = sc.get<int64_t>(n + 1), *lrp = sc.get<int64_t>(n + 1);
        int32_t *lists_f = sc.get<int32_t>((size_t)(SP_NCLS + 1) * (n + 1));
        int32_t *retry = sc.get<int32_t>(n + 1);
        uint32_t *colcnt = upper ? sc.get<uint32_t>(n + 1) : nullptr;
        if (!tmp_off || !need_f || !lrp || !lists_f || !retry || (upper && !colcnt)) return SG_ERR_OOM;
        if (upper) SG_CUDA_TRY(cudaMemsetAsync(colcnt, 0, (n + 1) * sizeof(uint32_t), s));
        // counters after the class counts (4 NCNT + 1 of them), all zeroed above
        unsigned long long *tcur = counts + 4 * NCNT + 1;     // temporary region cursor
        unsigned long long *n_retry = counts + 4 * NCNT + 2;  // rows that found the region full
        unsigned long long *gw = counts + 4 * NCNT + 3;       // {largest w, room} of listed rows (2)
        unsigned long long *big_count = counts + 4 * NCNT + 5;  // long mirrored parts
        unsigned long long *sums = counts + 4 * NCNT + 6;     // sample sums (3)
        // sampled rows: distinct partners (r1) and partners seen at least twice (r2) per A entry
        const int64_t fmode = tune("spgemm_filter_mode");
        int64_t fwork = min_shared >= 2 && ff.ncls > 0 && fmode > 0 ? tune("spgemm_filter_work") : 0;
        double r1 = 0.0, r2 = 0.0;
        const int64_t nsamp = tune("spgemm_sample_rows");
        if (nsamp > 0 && n > 0 && A->nnz > 0) {
            const int64_t stride = n > nsamp ? n / nsamp : 1;
            const int64_t nb = (n + stride - 1) / stride;
            const size_t ssm = fbytes + wbb(256);
            if (upper) {
                SG_CUDA_TRY(ensure_smem(sample_fx_kernel<true>, ssm));
                SG_LAUNCH("spgemm_sample", sample_fx_kernel<true>, nb, 256, ssm, s, g, stride, log2F, sums);
            } else {
                SG_CUDA_TRY(ensure_smem(sample_fx_kernel<false>, ssm));
                SG_LAUNCH("spgemm_sample", sample_fx_kernel<false>, nb, 256, ssm, s, g, stride, log2F, sums);
            }
            unsigned long long h[3] = {0, 0, 0};
            SG_CUDA_TRY(read_back(h, sums, sizeof(h), s));
            if (h[0] > 0) {
                r1 = (double)h[1] / (double)h[0];
                r2 = (double)h[2] / (double)h[0];
            }
        }
        if (r1 == 0.0) r1 = r2 = 1.0;  // no sample: a partner per A entry
        const bool recur = r1 < 2.0 * r2;  // most partners recur: the filter would keep nearly all
        if (fmode == 1 && recur) fwork = 0;
        const double pct = (double)tune("spgemm_guess_pct") / 100.0;
        const uint64_t fu = (uint64_t)(pct * r1 * 65536.0) + 1, ffq = (uint64_t)(pct * r2 * 65536.0) + 1;
        SG_LAUNCH("fused_need", fx_need_kernel, blocks_for(n, NT), NT, 0, s, A->row_ptr, n, fu, fwork, ffq,
                  ff.ncls > 0 ? (int64_t)1 << ff.log2T[ff.ncls - 1] : (int64_t)64, Tmax, need, need_f);
        SG_LAUNCH("classify", classify_kernel, blocks_for(n, NT), NT, 0, s, need, n, fz, fz_counts, lists);
        if (fwork)
            SG_LAUNCH("classify", classify_kernel, blocks_for(n, NT), NT, 0, s, need_f, n, ff, ff_counts, lists_f);
        unsigned long long h_fz[NCNT], h_ff[NCNT];
        uint32_t herr = 0;
        SG_CUDA_TRY(cudaMemcpyAsync(h_ff, ff_counts, sizeof(h_ff), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaMemcpyAsync(h_fz, fz_counts, sizeof(h_fz), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(read_back(&herr, err, sizeof(uint32_t), s));
        if (herr & DEV_TIMEOUT) return timeout_error("overlap_spgemm");
        // the temporary region: the sampled kept partners per A entry (r2 for min_shared >= 2, r1
        // for 1) times nnz(A), with room to spare; rows that find it full are redone in a grown one
        int64_t cap = opt.tmp_cap;
        if (cap <= 0) {
            const double kept = (min_shared >= 2 ? r2 : r1) * (double)A->nnz + 4.0 * (double)n;
            cap = (int64_t)((double)tune("spgemm_tmp_pct") / 100.0 * kept) + 64;
        }
        const double tmp_bytes = (double)cap * (8.0 + 8.0 * S);
        // at most half of what the device can still give (a row range was sized for its budget)
        const double avail = (double)device_bytes_available();
        if (opt.whole_rows ||
            (tmp_bytes <= (double)tune("spgemm_fused_max_mb") * 1048576.0 && tmp_bytes <= 0.5 * avail)) {
            TmpOut o{};
            o.col = sc.get<int32_t>(cap + 1);
            o.cnt = sc.get<uint32_t>(cap + 1);
            o.si = sc.get<uint32_t>((size_t)S * cap + 1);
            o.sk = sc.get<uint32_t>((size_t)S * cap + 1);
            if (!o.col || !o.cnt || !o.si || !o.sk) return SG_ERR_OOM;
            o.cap = cap;
            o.cursor = tcur;
            o.off = tmp_off;
            o.len = nnz_row;
            o.retry = retry;
            o.n_retry = n_retry;
            o.colcnt = colcnt;
            // one launch per table class; the seed form (SK), the filter and the form pick the kernel
            const int carve = (int)tune("spgemm_smem_carveout");
            auto launch_tab = [&](bool filt, int log2T, const int32_t *rl, const unsigned long long *cnt,
                                  const char *name, int32_t *ol, unsigned long long *oc, int8_t *olt) -> sg_status {
                const size_t tsm = tab_bytes((int64_t)1 << log2T, S) + (filt ? fbytes : 0);
                const int nt = pick_tab_threads(tsm, wbb(32), filt ? log2T : -log2T);
                const size_t sm = tsm + wbb(nt);
                const int64_t wb_off = (int64_t)tsm;
#define SG_TAB_LAUNCH(SKV, FV, UV)                                                                          \
    do {                                                                                                    \
        SG_CUDA_TRY(ensure_smem(tab_numeric_kernel<false, SKV, FV, UV>, sm));                               \
        if (carve >= 0)                                                                                     \
            SG_CUDA_TRY(cudaFuncSetAttribute(tab_numeric_kernel<false, SKV, FV, UV>,                        \
                                             cudaFuncAttributePreferredSharedMemoryCarveout, carve));       \
        SG_LAUNCH(name, (tab_numeric_kernel<false, SKV, FV, UV>), grid, nt, sm, s, g, rl, cnt, log2T, log2F, \
                  (unsigned char *)nullptr, (int64_t)0, (const int64_t *)nullptr, o, ol, oc, wb_off, olt);  \
    } while (0)
#define SG_TAB_SK(FV, UV)                      \
    do {                                       \
        if (SK == 0) SG_TAB_LAUNCH(0, FV, UV); \
        else if (SK == 1) SG_TAB_LAUNCH(1, FV, UV); \
        else if (SK == 2) SG_TAB_LAUNCH(2, FV, UV); \
        else SG_TAB_LAUNCH(3, FV, UV);         \
    } while (0)
                if (filt && upper) SG_TAB_SK(true, true);
                else if (filt) SG_TAB_SK(true, false);
                else if (upper) SG_TAB_SK(false, true);
                else SG_TAB_SK(false, false);
#undef SG_TAB_SK
#undef SG_TAB_LAUNCH
                return SG_OK;
            };
            // rows in exact global-memory tables: their products first (table sizes), then the pass
            int64_t *wl = sc.get<int64_t>(n + 1);
            if (!wl) return SG_ERR_OOM;
            auto launch_gtab = [&](const int32_t *rl, const unsigned long long *cnt, unsigned long long nrows)
                -> sg_status {
                SG_CUDA_TRY(cudaMemsetAsync(gw, 0, 2 * sizeof(unsigned long long), s));
                if (upper)
                    SG_LAUNCH("spgemm_rows_work", rows_work_kernel<true>, blocks_for((int64_t)nrows * 32, 256), 256, 0,
                              s, g, rl, cnt, wl, gw, gw + 1);
                else
                    SG_LAUNCH("spgemm_rows_work", rows_work_kernel<false>, blocks_for((int64_t)nrows * 32, 256), 256,
                              0, s, g, rl, cnt, wl, gw, gw + 1);
                unsigned long long wmax = 0;
                SG_CUDA_TRY(read_back(&wmax, gw, sizeof(wmax), s));
                const int64_t T = pow2_at_least(2 * std::min<int64_t>(std::max<int64_t>((int64_t)wmax, 1),
                                                                      np > 1 ? np - 1 : 1));
                const int64_t slice = (int64_t)((tab_bytes(T, S) + 255) & ~(size_t)255);
                int ggrid = (int)std::min<unsigned long long>(nrows, (unsigned long long)nsm * 2);
                if (opt.gmem_bytes) ggrid = (int)std::max<int64_t>(1, std::min<int64_t>(ggrid, (int64_t)opt.gmem_bytes / slice));
                unsigned char *pool = sc.get<unsigned char>((size_t)slice * ggrid);
                if (!pool) return SG_ERR_OOM;
                const size_t gsm = wbb(512);
#define SG_GTAB_LAUNCH(SKV, UV)                                                                                  \
    SG_LAUNCH("spgemm_numeric_gmem", (tab_numeric_kernel<true, SKV, false, UV>), ggrid, 512, gsm, s, g, rl, cnt, \
              0, 0, pool, slice, (const int64_t *)wl, o, ovf + n + 1, unused, (int64_t)0, (int8_t *)nullptr)
#define SG_GTAB_SK(UV)                     \
    do {                                   \
        if (SK == 0) SG_GTAB_LAUNCH(0, UV); \
        else if (SK == 1) SG_GTAB_LAUNCH(1, UV); \
        else if (SK == 2) SG_GTAB_LAUNCH(2, UV); \
        else SG_GTAB_LAUNCH(3, UV);        \
    } while (0)
                if (upper) SG_GTAB_SK(true);
                else SG_GTAB_SK(false);
#undef SG_GTAB_SK
#undef SG_GTAB_LAUNCH
                sc.release(pool);
                return SG_OK;
            };
            // rows whose guessed table overflows are tried once more in a table 4 x larger while
            // one fits in shared memory (esc: second-round class lists and counts, their overflow
            // list), else redone in global memory
            const int esc_shift = (int)tune("spgemm_escalate");
            int8_t *ovf_lt = esc_shift > 0 ? sc.get<int8_t>(n + 1) : nullptr;
            unsigned long long *esc_counts = esc_shift > 0 ? sc.get<unsigned long long>(NCNT + 1) : nullptr;
            int32_t *esc_lists = esc_shift > 0 ? sc.get<int32_t>((size_t)(SP_NCLS + 1) * (n + 1)) : nullptr;
            int32_t *esc_ovf = esc_shift > 0 ? sc.get<int32_t>(n + 1) : nullptr;
            if (esc_shift > 0 && (!ovf_lt || !esc_counts || !esc_lists || !esc_ovf)) return SG_ERR_OOM;
            if (esc_shift > 0) SG_CUDA_TRY(cudaMemsetAsync(esc_counts, 0, (NCNT + 1) * sizeof(unsigned long long), s));
            for (int c = 0; c < fz.ncls; c++) {
                if (!h_fz[c]) continue;
                SG_TRY(launch_tab(false, fz.log2T[c], lists + (int64_t)c * n, fz_counts + c,
                                  NUM_NAMES[fz.log2T[c] - SP_MINLOG], ovf, fz_ovf, ovf_lt));
            }
            for (int c = 0; fwork && c < ff.ncls; c++) {  // rows with many entries: filtered first
                if (!h_ff[c]) continue;
                SG_TRY(launch_tab(true, ff.log2T[c], lists_f + (int64_t)c * n, ff_counts + c,
                                  FIL_NAMES[ff.log2T[c] - SP_MINLOG], ovf, fz_ovf, nullptr));
            }
            unsigned long long n_ovf = 0, h_esc[NCNT + 1] = {};
            SG_CUDA_TRY(read_back(&n_ovf, fz_ovf, sizeof(n_ovf), s));
            // filtered rows' overflows (no size recorded) are escalated past every class
            const bool escalate = esc_shift > 0 && n_ovf > 0 && !fwork;
            if (escalate) {
                SG_LAUNCH("escalate", escalate_kernel, blocks_for((int64_t)n_ovf, NT), NT, 0, s, (const int32_t *)ovf,
                          (const int8_t *)ovf_lt, (const unsigned long long *)fz_ovf, esc_shift, fz, n, esc_counts,
                          esc_lists);
                SG_CUDA_TRY(read_back(h_esc, esc_counts, sizeof(h_esc), s));
                for (int c = 0; c < fz.ncls; c++) {
                    if (!h_esc[c]) continue;
                    SG_TRY(launch_tab(false, fz.log2T[c], esc_lists + (int64_t)c * n, esc_counts + c,
                                      NUM_NAMES[fz.log2T[c] - SP_MINLOG], esc_ovf, esc_counts + NCNT, nullptr));
                }
            }
            const unsigned long long n_big = h_fz[fz.ncls], n_big_f = fwork ? h_ff[ff.ncls] : 0;
            if (n_big) SG_TRY(launch_gtab(lists + (int64_t)fz.ncls * n, fz_counts + fz.ncls, n_big));
            if (n_big_f) SG_TRY(launch_gtab(lists_f + (int64_t)ff.ncls * n, ff_counts + ff.ncls, n_big_f));
            if (escalate) {
                unsigned long long n_ovf2 = 0;
                SG_CUDA_TRY(read_back(&n_ovf2, esc_counts + NCNT, sizeof(n_ovf2), s));
                if (h_esc[fz.ncls])
                    SG_TRY(launch_gtab(esc_lists + (int64_t)fz.ncls * n, esc_counts + fz.ncls, h_esc[fz.ncls]));
                if (n_ovf2) SG_TRY(launch_gtab((const int32_t *)esc_ovf, esc_counts + NCNT, n_ovf2));
            } else if (n_ovf) {
                SG_TRY(launch_gtab((const int32_t *)ovf, fz_ovf, n_ovf));
            }
            // rows that found the region full: grow it by their exact room and redo them
            unsigned long long n_rt = 0;
            SG_CUDA_TRY(read_back(&n_rt, n_retry, sizeof(n_rt), s));
            if (n_rt) {
                int32_t *rl = sc.get<int32_t>(n_rt + 1);
                unsigned long long *rc = sc.get<unsigned long long>(1);
                if (!rl || !rc) return SG_ERR_OOM;
                SG_CUDA_TRY(cudaMemcpyAsync(rl, retry, n_rt * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                SG_CUDA_TRY(cudaMemcpyAsync(rc, n_retry, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
                SG_CUDA_TRY(cudaMemsetAsync(gw, 0, 2 * sizeof(unsigned long long), s));
                if (upper)
                    SG_LAUNCH("spgemm_rows_work", rows_work_kernel<true>, blocks_for((int64_t)n_rt * 32, 256), 256, 0,
                              s, g, (const int32_t *)rl, (const unsigned long long *)rc, wl, gw, gw + 1);
                else
                    SG_LAUNCH("spgemm_rows_work", rows_work_kernel<false>, blocks_for((int64_t)n_rt * 32, 256), 256,
                              0, s, g, (const int32_t *)rl, (const unsigned long long *)rc, wl, gw, gw + 1);
                unsigned long long hroom = 0;
                SG_CUDA_TRY(read_back(&hroom, gw + 1, sizeof(hroom), s));
                TmpOut o2 = o;
                o2.cap = cap + (int64_t)hroom;
                o2.col = sc.get<int32_t>(o2.cap + 1);
                o2.cnt = sc.get<uint32_t>(o2.cap + 1);
                o2.si = sc.get<uint32_t>((size_t)S * o2.cap + 1);
                o2.sk = sc.get<uint32_t>((size_t)S * o2.cap + 1);
                if (!o2.col || !o2.cnt || !o2.si || !o2.sk) return SG_ERR_OOM;
                SG_CUDA_TRY(cudaMemcpyAsync(o2.col, o.col, cap * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                SG_CUDA_TRY(cudaMemcpyAsync(o2.cnt, o.cnt, cap * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
                for (int q = 0; q < S; q++) {
                    SG_CUDA_TRY(cudaMemcpyAsync(o2.si + (int64_t)q * o2.cap, o.si + (int64_t)q * cap,
                                                cap * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
                    SG_CUDA_TRY(cudaMemcpyAsync(o2.sk + (int64_t)q * o2.cap, o.sk + (int64_t)q * cap,
                                                cap * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
                }
                for (const void *p : {(const void *)o.col, (const void *)o.cnt, (const void *)o.si, (const void *)o.sk})
                    sc.release(p);
                const unsigned long long c0 = (unsigned long long)cap;  // successful rows lie below cap
                SG_CUDA_TRY(cudaMemcpyAsync(tcur, &c0, sizeof(c0), cudaMemcpyHostToDevice, s));
                SG_CUDA_TRY(cudaMemsetAsync(n_retry, 0, sizeof(unsigned long long), s));
                o = o2;
                cap = o2.cap;
                SG_TRY(launch_gtab((const int32_t *)rl, (const unsigned long long *)rc, n_rt));
                unsigned long long n_rt2 = 0;
                SG_CUDA_TRY(read_back(&n_rt2, n_retry, sizeof(n_rt2), s));
                if (n_rt2) {
                    set_error("overlap_spgemm: %llu rows did not fit the grown region (internal error)", n_rt2);
                    return SG_ERR_OVERFLOW;
                }
            }
            if (debug_record_classes()) {  // test hook: which launch handled each row
                std::vector<int32_t> &rec = debug_classes();
                rec.assign(n, -1);
                std::vector<int32_t> h;
                auto mark = [&](const int32_t *dl, unsigned long long cnt, int code, bool add) -> sg_status {
                    h.resize(cnt);
                    if (cnt) SG_CUDA_TRY(read_back(h.data(), dl, cnt * sizeof(int32_t), s));
                    for (int32_t r : h)
                        if (r >= 0 && r < n) rec[r] = add ? rec[r] + code : code;
                    return SG_OK;
                };
                for (int c = 0; c <= fz.ncls; c++)
                    SG_TRY(mark(lists + (int64_t)c * n, h_fz[c], c < fz.ncls ? fz.log2T[c] : 32, false));
                for (int c = 0; fwork && c <= ff.ncls; c++)
                    SG_TRY(mark(lists_f + (int64_t)c * n, h_ff[c], c < ff.ncls ? 16 + ff.log2T[c] : 33, false));
                SG_TRY(mark(ovf, n_ovf, 64, true));
                if (escalate) {  // second round: 96 + log2 of the larger table, 32 + 96 global
                    for (int c = 0; c <= fz.ncls; c++)
                        SG_TRY(mark(esc_lists + (int64_t)c * n, h_esc[c], c < fz.ncls ? 96 + fz.log2T[c] : 128, false));
                    unsigned long long n_ovf2 = 0;
                    SG_CUDA_TRY(read_back(&n_ovf2, esc_counts + NCNT, sizeof(n_ovf2), s));
                    SG_TRY(mark(esc_ovf, n_ovf2, 64, true));
                }
            }
            int64_t *clen = upper ? need_f : nnz_row;  // need_f is free once the classes have run
            if (upper)
                SG_LAUNCH("c_rowlen", c_rowlen_kernel, blocks_for(n, NT), NT, 0, s, (const int64_t *)nnz_row,
                          (const uint32_t *)colcnt, n, need_f);
            SG_ALLOC(C->row_ptr, int64_t, n + 1, s);
            SG_TRY(exclusive_scan<int64_t>(clen, C->row_ptr, n, s, err));
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
            if (!upper) {
                SG_LAUNCH("compact_c", compact_c_kernel, blocks_for(n * 32, 256), 256, 0, s, (const int64_t *)tmp_off,
                          cap, (const int32_t *)o.col, (const uint32_t *)o.cnt, (const uint32_t *)o.si,
                          (const uint32_t *)o.sk, S, (const int64_t *)C->row_ptr, n, nnz, C->col, C->count,
                          C->seed_i, C->seed_k);
                return SG_OK;
            }
            // C = U + U^T: U rows in place; the mirrored entries of each column, in row order
            SG_TRY(exclusive_scan<uint32_t>(colcnt, lrp, n, s, err));
            int64_t nnz_l = 0;
            SG_CUDA_TRY(read_back(&nnz_l, lrp + n, sizeof(int64_t), s));
            if (tune("spgemm_mirror_sort") && nnz < ((int64_t)1 << MIRROR_POS_BITS)) {
                int64_t *rpu = need;  // free once the classes have run
                SG_TRY(exclusive_scan<int64_t>(nnz_row, rpu, n, s, err));
                uint32_t *mk0 = sc.get<uint32_t>(nnz_l + 1), *mk1 = sc.get<uint32_t>(nnz_l + 1);
                uint64_t *mv0 = sc.get<uint64_t>(nnz_l + 1), *mv1 = sc.get<uint64_t>(nnz_l + 1);
                if (!mk0 || !mk1 || !mv0 || !mv1) return SG_ERR_OOM;
                // U's entries as records, where the seeds fit one (nnz_l = nnz(U): every U entry is mirrored)
                MirrorRec *mrec = nullptr;
                if (tune("spgemm_mirror_rec") && S <= MIRROR_REC_SEEDS) {
                    mrec = sc.get<MirrorRec>(nnz_l + 1);
                    if (!mrec) return SG_ERR_OOM;
                }
                SG_LAUNCH("mirror_c", mirror_keys_kernel, blocks_for(n * 32, 256), 256, 0, s,
                          (const int64_t *)tmp_off, (const int64_t *)nnz_row, cap, (const int32_t *)o.col,
                          (const uint32_t *)o.cnt, (const uint32_t *)o.si, (const uint32_t *)o.sk, S,
                          (const uint32_t *)colcnt, (const int64_t *)C->row_ptr, (const int64_t *)rpu, n, nnz, C->col,
                          C->count, C->seed_i, C->seed_k, mk0, mv0, mrec);
                for (const void *p : {(const void *)o.col, (const void *)o.cnt, (const void *)o.si, (const void *)o.sk})
                    sc.release(p);
                int kbits = 1;
                while (kbits < 32 && ((int64_t)1 << kbits) < n) kbits++;
                bool alt = false;
                SG_TRY((radix_sort_pairs<uint32_t, uint64_t>(mk0, mv0, mk1, mv1, nnz_l, kbits, &alt, s, err)));
                SG_LAUNCH("lower_fill", lower_fill_kernel, blocks_for(nnz_l, 256), 256, 0, s,
                          (const uint32_t *)(alt ? mk1 : mk0), (const uint64_t *)(alt ? mv1 : mv0), nnz_l,
                          (const int64_t *)lrp, (const int64_t *)C->row_ptr, n, nnz, S, C->col, C->count, C->seed_i,
                          C->seed_k, (const MirrorRec *)mrec);
                SG_CUDA_TRY(read_back(&herr, err, sizeof(uint32_t), s));  // the sort waits between tiles
                if (herr & DEV_TIMEOUT) return timeout_error("overlap_spgemm");
                return SG_OK;
            }
            uint32_t *cursor = sc.get<uint32_t>(n + 1);
            uint32_t *lrec = sc.get<uint32_t>((size_t)(2 + 2 * S) * nnz_l + 1);
            if (!cursor || !lrec) return SG_ERR_OOM;
            SG_CUDA_TRY(cudaMemsetAsync(cursor, 0, (n + 1) * sizeof(uint32_t), s));
            SG_LAUNCH("mirror_c", mirror_c_kernel, blocks_for(n * 32, 256), 256, 0, s, (const int64_t *)tmp_off,
                      (const int64_t *)nnz_row, cap, (const int32_t *)o.col, (const uint32_t *)o.cnt,
                      (const uint32_t *)o.si, (const uint32_t *)o.sk, S, (const uint32_t *)colcnt,
                      (const int64_t *)C->row_ptr, (const int64_t *)lrp, n, nnz, nnz_l, cursor, C->col, C->count,
                      C->seed_i, C->seed_k, lrec);
            for (const void *p : {(const void *)o.col, (const void *)o.cnt, (const void *)o.si, (const void *)o.sk})
                sc.release(p);
            int32_t *big_rows = ovf;  // free once the redo passes have run
            SG_LAUNCH("sort_lower", sort_lower_kernel, (int64_t)nsm * 8, LOWER_NT, 0, s, (const uint32_t *)colcnt,
                      (const int64_t *)lrp, (const int64_t *)C->row_ptr, n, nnz, S, (const uint32_t *)lrec, C->col,
                      C->count, C->seed_i, C->seed_k, big_count, big_rows,
                      (int)std::min<int64_t>(tune("spgemm_lower_smem"), LOWER_SMEM));
            unsigned long long n_lbig = 0;
            SG_CUDA_TRY(read_back(&n_lbig, big_count, sizeof(n_lbig), s));
            if (n_lbig) {
                int64_t slice = 1;
                while (slice < n) slice <<= 1;  // a lower part holds fewer than n entries
                const int lgrid = (int)(n_lbig < (unsigned long long)nsm ? n_lbig : (unsigned long long)nsm);
                uint64_t *kpool = sc.get<uint64_t>((size_t)slice * lgrid);
                if (!kpool) return SG_ERR_OOM;
                SG_LAUNCH("sort_lower_big", lower_big_kernel, lgrid, 1024, 0, s, (const uint32_t *)colcnt,
                          (const int64_t *)lrp, (const int64_t *)C->row_ptr, nnz, S, (const int32_t *)big_rows,
                          (const unsigned long long *)big_count, kpool, slice, (const uint32_t *)lrec, C->col,
                          C->count, C->seed_i, C->seed_k);
            }
            return SG_OK;
        }
        // the temporary region would exceed its budget: the two-pass path below
    }
    // ---- two-pass form: row work and At extents per A entry, symbolic sizes, exact tables
    int64_t *a_beg = sc.get<int64_t>(A->nnz + 1);
    uint32_t *a_len = sc.get<uint32_t>(A->nnz + 1);
    if (!a_beg || !a_len) return SG_ERR_OOM;
    g.a_beg = a_beg;
    g.a_len = a_len;
    stage.emplace("SpGEMMSymbolic", s);
    SG_LAUNCH("row_work", row_work_kernel, blocks_for(n * 32, 256), 256, 0, s, A->row_ptr, A->col, At->row_ptr, n,
              work, a_beg, a_len);
    g.t_pair = t_pair = sc.get<uint64_t>(At->nnz + 1);
    if (!t_pair) return SG_ERR_OOM;
    SG_LAUNCH("at_pairs", pair_kernel, blocks_for(At->nnz, 256), 256, 0, s, At->col, At->val, At->nnz, t_pair);

    // ---- symbolic: guessed shared-memory tables of 2^6 .. 2^14 slots, one class per size
    Classes sym{};
    sym.ncls = SP_NCLS;
    for (int c = 0; c < SP_NCLS; c++) sym.log2T[c] = SP_MINLOG + c;
    SG_LAUNCH("sym_need", sym_need_kernel, blocks_for(n, NT), NT, 0, s, work, n, np, (int)tune("sym_guess_shift"),
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
        const int64_t slice = 2 * pow2_at_least(2 * (np > 1 ? np - 1 : 1));  // keys + counts of the largest row
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

// ------------------------------------------------------------------------------------------
// Memory-bounded formation of C in row tiles (the paper's closing remark, Sec. VIII: form C in
// parts under a memory bound instead of all at once). Rows of C are independent, so C is formed
// for a range of A's rows at a time -- A's row pointers of the range rebased to 0, partners still
// every read of At, whole rows (the mirrored form needs every earlier row) -- and each finished
// tile is handed to the caller and freed before the next one starts.
namespace sg {

constexpr int64_t TILE_ROW_BYTES = 256;           // per-row arrays of one tile (row pointers, classes...)
constexpr int64_t TILE_FIXED_BYTES = 4ll << 20;   // counters and allocation rounding of one tile

// Per row: the bytes the row adds to a tile (the temporary and the final room for its entries of
// C, min(w / t, np - 1) each, twice; and the per-row arrays) and its products w (whole row,
// diagonal excluded). One warp per row.
__global__ void tile_est_kernel(const int64_t *__restrict__ a_rp, const int32_t *__restrict__ a_col,
                                const int64_t *__restrict__ t_rp, int64_t n, int64_t np, uint32_t t, int S,
                                int64_t *__restrict__ bytes, int64_t *__restrict__ work) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    int64_t w = 0;
    for (int64_t a = a_rp[row] + lane; a < a_rp[row + 1]; a += 32) {
        const int32_t j = a_col[a];
        w += t_rp[j + 1] - t_rp[j] - 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) {
        const int64_t room = std::min<int64_t>(w / t, np - 1);
        bytes[row] = 2 * (8 + 8 * (int64_t)S) * room + TILE_ROW_BYTES;
        work[row] = w;
    }
}

__global__ void rebase_rows_kernel(const int64_t *__restrict__ rp, int64_t r0, int64_t nr, int64_t *__restrict__ out) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x <= nr) out[x] = rp[r0 + x] - rp[r0];
}

}  // namespace sg

extern "C" sg_status sg_overlap_spgemm_tiled(const sg_csr_u32 *A, const sg_csr_u32 *At, uint32_t min_shared,
                                             int32_t max_seeds, size_t budget_bytes, sg_overlap_tile_fn fn,
                                             void *user, int64_t *n_tiles, sg_stream_t stream) {
    using namespace sg;
    if (n_tiles) *n_tiles = 0;
    if (!A || !At || !fn || max_seeds < 0 || max_seeds > SP_MAX_SEEDS || min_shared < 1 || A->n_rows != At->n_cols ||
        A->n_cols != At->n_rows || A->nnz != At->nnz || A->n_rows < 0 || A->n_rows >= ((int64_t)1 << 31) ||
        !A->row_ptr || !At->row_ptr || budget_bytes == 0) {
        set_error("overlap_spgemm_tiled: invalid arguments");
        return SG_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->n_rows, np = At->n_cols;
    const int S = max_seeds;
    if (n == 0) return SG_OK;
    // per-row bytes and products, and A's row pointers, on the host
    std::vector<int64_t> hb(n), hw(n), hrp(n + 1);
    {
        Scratch sc(s);
        int64_t *db = sc.get<int64_t>(n), *dw = sc.get<int64_t>(n);
        if (!db || !dw) return SG_ERR_OOM;
        SG_LAUNCH("tile_est", tile_est_kernel, (n * 32 + 255) / 256, 256, 0, s, A->row_ptr, A->col, At->row_ptr, n,
                  np, min_shared, S, db, dw);
        SG_CUDA_TRY(cudaMemcpyAsync(hb.data(), db, n * 8, cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaMemcpyAsync(hw.data(), dw, n * 8, cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaMemcpyAsync(hrp.data(), A->row_ptr, (n + 1) * 8, cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // the redo pass's global table for a tile whose largest row has w products
    auto gslice = [&](int64_t w) -> int64_t {
        const int64_t T = pow2_at_least(2 * std::min<int64_t>(std::max<int64_t>(w, 1), np > 1 ? np - 1 : 1));
        return (int64_t)((tab_bytes(T, S) + 255) & ~(size_t)255);
    };
    int64_t tiles = 0;
    for (int64_t r0 = 0; r0 < n;) {
        // the longest range from r0 whose rows, one global table for its largest row and the fixed
        // part fit the budget
        int64_t acc = TILE_FIXED_BYTES, wmax = 0, r1 = r0, room = 0;
        while (r1 < n) {
            const int64_t wm = std::max(wmax, hw[r1]);
            if (acc + hb[r1] + gslice(wm) > (int64_t)budget_bytes) break;
            acc += hb[r1];
            room += std::min<int64_t>(hw[r1] / min_shared, np - 1);
            wmax = wm;
            r1++;
        }
        if (r1 == r0) {
            set_error("overlap_spgemm_tiled: row %lld alone needs about %lld bytes, more than the budget of %zu",
                      (long long)r0, (long long)(TILE_FIXED_BYTES + hb[r0] + gslice(hw[r0])), budget_bytes);
            return SG_ERR_BUDGET;
        }
        const int64_t nr = r1 - r0, base = hrp[r0];
        sg_overlap_csr Ct{};
        sg_status st;
        {
            Scratch sc(s);
            int64_t *rp = sc.get<int64_t>(nr + 1);
            if (!rp) return SG_ERR_OOM;
            SG_LAUNCH("rebase_rows", rebase_rows_kernel, (nr + 256) / 256, 256, 0, s, A->row_ptr, r0, nr, rp);
            sg_csr_u32 At_{*At};
            sg_csr_u32 Ar{nr, A->n_cols, hrp[r1] - base, rp, A->col + base, A->val + base};
            OverlapOpts opt;
            opt.row0 = r0;
            opt.whole_rows = true;
            opt.gmem_bytes = (size_t)((int64_t)budget_bytes - acc);  // >= one table for the largest row
            opt.tmp_cap = room + 1;  // exact bound: no row of the tile finds the region full
            st = overlap_impl(&Ar, &At_, min_shared, S, &Ct, s, sc, opt);
        }
        if (st == SG_OK && cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("overlap_spgemm_tiled: tile of rows %lld..%lld failed", (long long)r0, (long long)r1);
            st = SG_ERR_CUDA;
        }
        if (st == SG_OK) st = fn(&Ct, r0, user);
        sg_free_overlap(&Ct, stream);
        if (st != SG_OK) return st;
        tiles++;
        if (n_tiles) *n_tiles = tiles;
        r0 = r1;
    }
    return SG_OK;
}
