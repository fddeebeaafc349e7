// spgemm.cu -- C = A At over the overlap semiring (Sec. IV-D), row-wise on the GPU.
//
// Semiring: multiplying A_ij by At_jk takes the positions of k-mer j in reads i and k; adding
// counts one more shared k-mer and keeps the positions of up to max_seeds of them. Which seeds
// are kept is fixed order-free: the max_seeds shared k-mers with the smallest column index.
// Every update below is commutative (a count increment and an insertion into a "smallest S"
// list), so any parallel order gives the same C bit for bit.
//
// Passes:
//  1. row_work    w_i = sum over j in row i of (nnz(At_j) - 1): products of row i, diagonal excluded.
//  2. bin rows by hash-table size (power of two >= 2 * min(w_i, n - 1)).
//  3. symbolic    per row, a hash table keyed by the partner read k with a count per key; records
//                 nnz_i = #{k : count >= min_shared} and distinct_i = #{k}.
//  4. scan nnz_i -> C.row_ptr; re-bin rows by 2 * distinct_i.
//  5. numeric     per row, a hash table (key, count, S seed words). A seed word is
//                 (index of j within row i) << 32 | At value, so its numeric order is the order
//                 of j; inserting into the S-slot list is a chain of atomicMin's that pushes the
//                 loser down. Entries with count >= min_shared are compacted, bitonic-sorted by k
//                 and written to C; seed positions are resolved from A's row.
// Tables live in shared memory (one block per row) up to a size limit, else in a global pool.
#include "prim.cuh"

namespace sg {

constexpr int SP_NT = 256;
constexpr int SP_NT_BIG = 512;
constexpr int SP_CH = 1024;  // A entries staged per chunk
constexpr int SP_MAX_SEEDS = 8;
constexpr uint64_t SEED_NONE = ~0ull;

__device__ __forceinline__ uint32_t hash_slot(int32_t k, int log2T) {
    return ((uint32_t)k * 2654435761u) >> (32 - log2T);
}

// Find or insert key k; returns its slot. T = 1 << log2T, never full (load <= 1/2).
__device__ __forceinline__ uint32_t table_slot(int32_t *keys, int32_t k, int log2T) {
    const uint32_t msk = (1u << log2T) - 1u;
    uint32_t h = hash_slot(k, log2T);
    for (;;) {
        int32_t cur = ((volatile int32_t *)keys)[h];
        if (cur == k) return h;
        if (cur == -1) {
            int32_t old = atomicCAS(keys + h, -1, k);
            if (old == -1 || old == k) return h;
        }
        h = (h + 1) & msk;
    }
}

__global__ void row_work_kernel(const int64_t *__restrict__ a_rp, const int32_t *__restrict__ a_col,
                                const int64_t *__restrict__ t_rp, int64_t n, int64_t *__restrict__ work) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    int64_t w = 0;
    for (int64_t a = a_rp[row] + lane; a < a_rp[row + 1]; a += 32) {
        int32_t j = a_col[a];
        w += t_rp[j + 1] - t_rp[j] - 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) work[row] = w;
}

// Bin classes: log2 of the table size. Classes 0..NB-1 are shared-memory bins with table sizes
// 2^min_log2[c]..; the last class is the global-memory bin.
struct Bins {
    static constexpr int NB = 5;  // 4 smem classes + 1 global
    int log2T[NB - 1];            // table size of each smem class
    int nsmem;                    // smem classes in use (the rest go global)
};

// bin[i] = class of row i (or -1 when the row has no products); counts[c]++; for the global
// class, gsize[i] = table slots needed.
__global__ void bin_kernel(const int64_t *__restrict__ ub, int64_t n, int64_t cap, Bins bins,
                           int32_t *__restrict__ bin, unsigned long long *__restrict__ counts,
                           int64_t *__restrict__ gsize) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t u = ub[i] < cap ? ub[i] : cap;
    int b = -1;
    int64_t g = 0;
    if (u > 0) {
        int l = 0;
        while (((int64_t)1 << l) < 2 * u) l++;
        b = bins.nsmem;
        for (int c = 0; c < bins.nsmem; c++)
            if (l <= bins.log2T[c]) { b = c; break; }
        if (b == bins.nsmem) g = (int64_t)1 << l;
        atomicAdd(counts + b, 1ull);
    }
    bin[i] = b;
    gsize[i] = g;
}

__global__ void bin_fill_kernel(const int32_t *__restrict__ bin, int64_t n, const int64_t *__restrict__ base,
                                unsigned long long *__restrict__ cursor, int32_t *__restrict__ rows) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = bin[i];
    if (b < 0) return;
    unsigned long long p = atomicAdd(cursor + b, 1ull);
    rows[base[b] + (int64_t)p] = (int32_t)i;
}

// Staging of one chunk of row i of A: the columns, At row starts, and the exclusive prefix of
// At row lengths. Returns the number of products of the chunk.
template <int NT>
__device__ __forceinline__ int64_t stage_chunk(const int64_t *__restrict__ t_rp, const int32_t *__restrict__ a_col,
                                               int64_t a0, int cnt, int32_t *s_j, int64_t *s_beg,
                                               int64_t *s_pre, int64_t *s_tmp) {
    int64_t len = 0;
    int64_t beg = 0;
    int32_t j = 0;
    // each thread owns SP_CH / NT consecutive entries
    constexpr int PER = SP_CH / NT;
    int64_t loc[PER];
    int64_t sum = 0;
#pragma unroll
    for (int q = 0; q < PER; q++) {
        int c = threadIdx.x * PER + q;
        len = 0;
        if (c < cnt) {
            j = a_col[a0 + c];
            beg = t_rp[j];
            len = t_rp[j + 1] - beg;
            s_j[c] = j;
            s_beg[c] = beg;
        }
        loc[q] = sum;
        sum += len;
    }
    int64_t total;
    int64_t pre = block_exclusive_scan<NT>(sum, s_tmp, &total);
#pragma unroll
    for (int q = 0; q < PER; q++) {
        int c = threadIdx.x * PER + q;
        if (c < cnt) s_pre[c] = pre + loc[q];
    }
    if (threadIdx.x == 0) s_pre[cnt] = total;
    __syncthreads();
    return total;
}

// index c in [0, cnt) with s_pre[c] <= p < s_pre[c + 1]
__device__ __forceinline__ int find_chunk_entry(const int64_t *s_pre, int cnt, int64_t p) {
    int lo = 0, hi = cnt;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (s_pre[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

struct SpArgs {
    const int64_t *a_rp;
    const int32_t *a_col;
    const uint32_t *a_val;
    const int64_t *t_rp;
    const int32_t *t_col;
    const uint32_t *t_val;
    int64_t n;
    uint32_t min_shared;
    int S;
    uint32_t *err;  // DEV_OVERFLOW if the numeric pass ever disagrees with the symbolic sizes
};

// ---------------------------------------------------------------------------- symbolic
template <int NT, bool GMEM>
__global__ void __launch_bounds__(NT) symbolic_kernel(SpArgs g, const int32_t *__restrict__ rows, int64_t nrows,
                                                     int log2T, int32_t *__restrict__ gpool,
                                                     const int64_t *__restrict__ goff, int64_t *__restrict__ nnz_row,
                                                     int64_t *__restrict__ distinct_row) {
    extern __shared__ __align__(16) unsigned char sp_raw[];
    int32_t *s_j = (int32_t *)sp_raw;
    int64_t *s_beg = (int64_t *)(s_j + SP_CH);
    int64_t *s_pre = s_beg + SP_CH;
    int64_t *s_tmp = s_pre + SP_CH + 2;
    int32_t *tab = (int32_t *)(s_tmp + 32);  // keys [T] then counts [T]
    __shared__ int32_t s_red[2 * (NT / 32)];
    for (int64_t rb = blockIdx.x; rb < nrows; rb += gridDim.x) {
        const int32_t i = rows[rb];
        int lT = log2T;
        int32_t *keys;
        if (GMEM) {
            const int64_t T = goff[i + 1] - goff[i];  // a power of two
            keys = gpool + 2 * goff[i];
            lT = 0;
            while (((int64_t)1 << lT) < T) lT++;
        } else {
            keys = tab;
        }
        const int32_t T = 1 << lT;
        uint32_t *cnt = (uint32_t *)(keys + T);
        for (int x = threadIdx.x; x < T; x += NT) {
            keys[x] = -1;
            cnt[x] = 0;
        }
        __syncthreads();
        const int64_t r0 = g.a_rp[i], r1 = g.a_rp[i + 1];
        for (int64_t a0 = r0; a0 < r1; a0 += SP_CH) {
            int cntc = (int)((r1 - a0) < SP_CH ? (r1 - a0) : SP_CH);
            int64_t P = stage_chunk<NT>(g.t_rp, g.a_col, a0, cntc, s_j, s_beg, s_pre, s_tmp);
            for (int64_t p = threadIdx.x; p < P; p += NT) {
                int c = find_chunk_entry(s_pre, cntc, p);
                int32_t k = g.t_col[s_beg[c] + (p - s_pre[c])];
                if (k == i) continue;
                uint32_t h = table_slot(keys, k, lT);
                atomicAdd(cnt + h, 1u);
            }
            __syncthreads();
        }
        int32_t nz = 0, dist = 0;
        for (int x = threadIdx.x; x < T; x += NT) {
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
            for (int w = 0; w < NT / 32; w++) {
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
template <int NT, bool GMEM>
__global__ void __launch_bounds__(NT) numeric_kernel(SpArgs g, const int32_t *__restrict__ rows, int64_t nrows,
                                                    int log2T, int tab_off, unsigned char *__restrict__ gpool,
                                                    const int64_t *__restrict__ goff,
                                                    const int64_t *__restrict__ c_rp, int32_t *__restrict__ c_col,
                                                    uint32_t *__restrict__ c_cnt, uint32_t *__restrict__ c_si,
                                                    uint32_t *__restrict__ c_sk, int64_t c_nnz) {
    extern __shared__ __align__(16) unsigned char sp_raw[];
    // chunk staging region (reused as the output sort buffer once accumulation is done)
    int32_t *s_j = (int32_t *)sp_raw;
    int64_t *s_beg = (int64_t *)(s_j + SP_CH);
    int64_t *s_pre = s_beg + SP_CH;
    int64_t *s_tmp = s_pre + SP_CH + 2;
    unsigned char *tab_smem = sp_raw + tab_off;  // tab_off >= staging bytes and >= T/2 * 8
    __shared__ int s_ctr[1];
    const int S = g.S;
    for (int64_t rb = blockIdx.x; rb < nrows; rb += gridDim.x) {
        const int32_t i = rows[rb];
        int lT = log2T;
        unsigned char *tb;
        uint64_t *obuf;
        if (GMEM) {
            int64_t T = goff[i + 1] - goff[i];
            lT = 0;
            while (((int64_t)1 << lT) < T) lT++;
            // per slot: 8 (key, count) + 8 S (seeds) + 8 (sort buffer of T/2 u64, padded to keep
            // every row 8-byte aligned)
            tb = gpool + goff[i] * (int64_t)(16 + 8 * S);
            obuf = (uint64_t *)(tb + ((int64_t)1 << lT) * (8 + 8 * S));
        } else {
            tb = tab_smem;
            obuf = (uint64_t *)sp_raw;
        }
        const int32_t T = 1 << lT;
        uint64_t *seeds = (uint64_t *)tb;                 // [T][S]
        int32_t *keys = (int32_t *)(seeds + (int64_t)T * S);
        uint32_t *cnt = (uint32_t *)(keys + T);
        for (int x = threadIdx.x; x < T; x += NT) {
            keys[x] = -1;
            cnt[x] = 0;
        }
        for (int x = threadIdx.x; x < T * S; x += NT) seeds[x] = SEED_NONE;
        if (threadIdx.x == 0) s_ctr[0] = 0;
        __syncthreads();
        const int64_t r0 = g.a_rp[i], r1 = g.a_rp[i + 1];
        for (int64_t a0 = r0; a0 < r1; a0 += SP_CH) {
            int cntc = (int)((r1 - a0) < SP_CH ? (r1 - a0) : SP_CH);
            int64_t P = stage_chunk<NT>(g.t_rp, g.a_col, a0, cntc, s_j, s_beg, s_pre, s_tmp);
            for (int64_t p = threadIdx.x; p < P; p += NT) {
                int c = find_chunk_entry(s_pre, cntc, p);
                int64_t b = s_beg[c] + (p - s_pre[c]);
                int32_t k = g.t_col[b];
                if (k == i) continue;
                uint32_t h = table_slot(keys, k, lT);
                atomicAdd(cnt + h, 1u);
                if (S > 0) {
                    // seed word: (index of j within row i) << 32 | value of At_jk
                    unsigned long long v = ((unsigned long long)(a0 - r0 + c) << 32) | g.t_val[b];
                    unsigned long long *sl = (unsigned long long *)(seeds + (int64_t)h * S);
                    for (int q = 0; q < S; q++) {
                        unsigned long long old = atomicMin(sl + q, v);
                        if (old > v) v = old;  // the larger one moves on to the next slot
                        if (v == SEED_NONE) break;
                    }
                }
            }
            __syncthreads();
        }
        // compact entries with count >= min_shared as (k << 32 | slot)
        for (int x = threadIdx.x; x < T; x += NT) {
            if (keys[x] != -1 && cnt[x] >= g.min_shared) {
                int p = atomicAdd(s_ctr, 1);
                obuf[p] = ((uint64_t)(uint32_t)keys[x] << 32) | (uint32_t)x;
            }
        }
        __syncthreads();
        const int nv = s_ctr[0];
        int P2 = 1;
        while (P2 < nv) P2 <<= 1;
        for (int x = nv + threadIdx.x; x < P2; x += NT) obuf[x] = ~0ull;
        __syncthreads();
        for (int kk = 2; kk <= P2; kk <<= 1) {
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int x = threadIdx.x; x < P2; x += NT) {
                    int y = x ^ jj;
                    if (y > x) {
                        uint64_t a = obuf[x], b = obuf[y];
                        bool up = (x & kk) == 0;
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
        if (nv != room && threadIdx.x == 0) atomicOr(g.err, (uint32_t)DEV_OVERFLOW);
        const int nw = nv < room ? nv : (int)room;
        for (int q = threadIdx.x; q < nw; q += NT) {
            uint64_t w = obuf[q];
            uint32_t slot = (uint32_t)w;
            int64_t e = e0 + q;
            c_col[e] = (int32_t)(w >> 32);
            c_cnt[e] = cnt[slot];
            for (int s = 0; s < S; s++) {
                uint64_t sd = seeds[(int64_t)slot * S + s];
                uint32_t si = 0xFFFFFFFFu, sk = 0xFFFFFFFFu;
                if (sd != SEED_NONE) {
                    uint32_t vi = g.a_val[r0 + (int64_t)(sd >> 32)];
                    uint32_t vk = (uint32_t)sd;
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

static size_t chunk_bytes() { return SP_CH * 4 + SP_CH * 8 + (SP_CH + 2) * 8 + 32 * 8; }
static size_t symbolic_smem(int log2T) { return chunk_bytes() + (size_t)(2 << log2T) * 4; }
// the output sort buffer (T/2 u64) overlaps the staging region; the table follows both
static size_t numeric_tab_off(int log2T) {
    size_t T = (size_t)1 << log2T;
    size_t stage = chunk_bytes();
    if (stage < T / 2 * 8) stage = T / 2 * 8;
    return (stage + 15) & ~(size_t)15;
}
static size_t numeric_smem(int log2T, int S) {
    return numeric_tab_off(log2T) + ((size_t)1 << log2T) * (8 + 8 * (size_t)S);
}

// Bins rows by table size and returns per-class row lists. ub[i] = upper bound of keys of row i.
struct BinResult {
    int64_t count[Bins::NB];
    int64_t base[Bins::NB + 1];
    int32_t *rows;   // rows of class c at rows[base[c] .. base[c+1])
    int64_t *goff;   // [n+1] exclusive scan of global table sizes (slots)
    int64_t gtotal;  // global pool slots
};

static sg_status bin_rows(const int64_t *ub, int64_t n, const Bins &bins, Scratch &sc, cudaStream_t s,
                          BinResult *out) {
    const int NT = 256;
    int32_t *bin = sc.get<int32_t>(n + 1);
    unsigned long long *counts = sc.get<unsigned long long>(2 * Bins::NB);
    int64_t *gsize = sc.get<int64_t>(n + 1);
    out->goff = sc.get<int64_t>(n + 1);
    int64_t *dbase = sc.get<int64_t>(Bins::NB + 1);
    out->rows = sc.get<int32_t>(n + 1);
    if (!bin || !counts || !gsize || !out->goff || !dbase || !out->rows) return SG_ERR_OOM;
    SG_CUDA_TRY(cudaMemsetAsync(counts, 0, 2 * Bins::NB * sizeof(unsigned long long), s));
    SG_LAUNCH("bin_rows", bin_kernel, blocks_for(n, NT), NT, 0, s, ub, n, (int64_t)(n > 0 ? n - 1 : 0), bins, bin,
              counts, gsize);
    SG_TRY(exclusive_scan<int64_t>(gsize, out->goff, n, s));
    unsigned long long hc[Bins::NB];
    SG_CUDA_TRY(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaMemcpyAsync(&out->gtotal, out->goff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    out->base[0] = 0;
    for (int c = 0; c < Bins::NB; c++) {
        out->count[c] = (int64_t)hc[c];
        out->base[c + 1] = out->base[c] + out->count[c];
    }
    SG_CUDA_TRY(cudaMemcpyAsync(dbase, out->base, sizeof(int64_t) * (Bins::NB + 1), cudaMemcpyHostToDevice, s));
    SG_LAUNCH("bin_fill", bin_fill_kernel, blocks_for(n, NT), NT, 0, s, bin, n, dbase, counts + Bins::NB,
              out->rows);
    return SG_OK;
}

static int grid_for(int64_t rows) {
    int64_t g = rows < 152 * 16 ? rows : 152 * 16;
    return (int)(g > 0 ? g : 0);
}

static sg_status overlap_impl(const sg_csr_u32 *A, const sg_csr_u32 *At, uint32_t min_shared, int S,
                              sg_overlap_csr *C, cudaStream_t s, Scratch &sc) {
    const int64_t n = A->n_rows;
    uint32_t *err = sc.get<uint32_t>(1);
    if (!err) return SG_ERR_OOM;
    SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    SpArgs g{A->row_ptr, A->col, A->val, At->row_ptr, At->col, At->val, n, min_shared, S, err};
    int64_t *work = sc.get<int64_t>(n + 1);
    int64_t *nnz_row = sc.get<int64_t>(n + 1);
    int64_t *dist = sc.get<int64_t>(n + 1);
    if (!work || !nnz_row || !dist) return SG_ERR_OOM;
    SG_CUDA_TRY(cudaMemsetAsync(nnz_row, 0, (n + 1) * sizeof(int64_t), s));
    SG_CUDA_TRY(cudaMemsetAsync(dist, 0, (n + 1) * sizeof(int64_t), s));
    SG_LAUNCH("row_work", row_work_kernel, blocks_for(n * 32, 256), 256, 0, s, A->row_ptr, A->col, At->row_ptr, n,
              work);

    // symbolic: smem classes up to 2^14 slots (128 KB of keys + counts)
    Bins sb{};
    sb.nsmem = 4;
    sb.log2T[0] = 8; sb.log2T[1] = 10; sb.log2T[2] = 12; sb.log2T[3] = 14;
    BinResult br{};
    SG_TRY(bin_rows(work, n, sb, sc, s, &br));
    int32_t *gpool_sym = nullptr;
    const int sg_glob = sb.nsmem;  // index of the global-memory class
    if (br.count[sg_glob] > 0) {
        gpool_sym = sc.get<int32_t>(2 * br.gtotal);
        if (!gpool_sym) return SG_ERR_OOM;
    }
    for (int c = 0; c < sb.nsmem; c++) {
        if (!br.count[c]) continue;
        size_t sm = symbolic_smem(sb.log2T[c]);
        SG_CUDA_TRY(cudaFuncSetAttribute(symbolic_kernel<SP_NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm));
        SG_LAUNCH("spgemm_symbolic", (symbolic_kernel<SP_NT, false>), grid_for(br.count[c]), SP_NT, sm, s, g,
                  br.rows + br.base[c], br.count[c], sb.log2T[c], (int32_t *)nullptr, (const int64_t *)nullptr,
                  nnz_row, dist);
    }
    if (br.count[sg_glob]) {
        size_t sm = chunk_bytes();
        SG_LAUNCH("spgemm_symbolic_gmem", (symbolic_kernel<SP_NT_BIG, true>), grid_for(br.count[sg_glob]),
                  SP_NT_BIG, sm, s, g, br.rows + br.base[sg_glob], br.count[sg_glob], 0, gpool_sym,
                  (const int64_t *)br.goff, nnz_row, dist);
    }

    // C row pointers
    SG_ALLOC(C->row_ptr, int64_t, n + 1, s);
    SG_TRY(exclusive_scan<int64_t>(nnz_row, C->row_ptr, n, s));

    // numeric bins from the exact distinct-key counts
    Bins nb{};
    nb.nsmem = 0;
    const int lmax = S <= 2 ? 12 : (S <= 4 ? 11 : 10);  // keep the table + staging under ~120 KB
    for (int l = 8; l <= lmax && nb.nsmem < Bins::NB - 1; l += 2) nb.log2T[nb.nsmem++] = l;
    if (nb.log2T[nb.nsmem - 1] != lmax) nb.log2T[nb.nsmem - 1] = lmax;
    BinResult nr{};
    SG_TRY(bin_rows(dist, n, nb, sc, s, &nr));  // synchronises: C.row_ptr is complete too
    int64_t nnz = 0;
    SG_CUDA_TRY(read_back(&nnz, C->row_ptr + n, sizeof(int64_t), s));
    C->n = n;
    C->nnz = nnz;
    C->max_seeds = S;
    SG_ALLOC(C->col, int32_t, nnz, s);
    SG_ALLOC(C->count, uint32_t, nnz, s);
    SG_ALLOC(C->seed_i, uint32_t, (int64_t)S * nnz, s);
    SG_ALLOC(C->seed_k, uint32_t, (int64_t)S * nnz, s);
    unsigned char *gpool_num = nullptr;
    const int ng_glob = nb.nsmem;
    if (nr.count[ng_glob] > 0) {
        gpool_num = sc.get<unsigned char>((size_t)nr.gtotal * (16 + 8 * (size_t)S));
        if (!gpool_num) return SG_ERR_OOM;
    }
    for (int c = 0; c < nb.nsmem; c++) {
        if (!nr.count[c]) continue;
        size_t sm = numeric_smem(nb.log2T[c], S);
        SG_CUDA_TRY(cudaFuncSetAttribute(numeric_kernel<SP_NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm));
        SG_LAUNCH("spgemm_numeric", (numeric_kernel<SP_NT, false>), grid_for(nr.count[c]), SP_NT, sm, s, g,
                  nr.rows + nr.base[c], nr.count[c], nb.log2T[c], (int)numeric_tab_off(nb.log2T[c]),
                  (unsigned char *)nullptr,
                  (const int64_t *)nullptr, (const int64_t *)C->row_ptr, C->col, C->count, C->seed_i, C->seed_k,
                  nnz);
    }
    if (nr.count[ng_glob]) {
        size_t sm = chunk_bytes();
        SG_LAUNCH("spgemm_numeric_gmem", (numeric_kernel<SP_NT_BIG, true>), grid_for(nr.count[ng_glob]),
                  SP_NT_BIG, sm, s, g, nr.rows + nr.base[ng_glob], nr.count[ng_glob], 0, 0, gpool_num,
                  (const int64_t *)nr.goff, (const int64_t *)C->row_ptr, C->col, C->count, C->seed_i, C->seed_k,
                  nnz);
    }
    uint32_t herr = 0;
    SG_CUDA_TRY(read_back(&herr, err, sizeof(uint32_t), s));
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
