// kmer.cu -- reads -> A (reads x reliable k-mers) and At, on the GPU.
//
// Sec. II: a k-mer's canonical form is the smaller of its code and its reverse complement's.
// Sec. IV-C: k-mers are counted in two phases -- a Bloom filter sees every k-mer, and only
// k-mers it has already seen go on to be counted exactly -- and a k-mer is kept when its
// frequency lies in the reliable range [lo, hi].
// Sec. IV-D: A_ij holds the position of k-mer j in read i (here: pos | strand << 31 at the
// lowest such position).
//
// Pipeline (all on `stream`):
//  0. window_codes   one walk over the reads writes every window's canonical code and strand.
//  1. bloom_insert   every code is OR-ed into the blocked Bloom filter B1 (all probe bits in one
//                    32-bit word, so "already present" is decided by one atomic); a code found
//                    present is OR-ed into B2 ("seen at least twice"). Skipped when lo == 1.
//  2. cand_count     per thread, the windows whose code tests positive in B2. Every occurrence
//                    of a k-mer with frequency >= 2 passes (false positives only add singletons,
//                    which the exact count below drops).
//  3. cand_emit      writes (code, position | strand) at scanned offsets, so the candidates stay
//                    in position order, i.e. (read, pos) order.
//  4. radix sort by code (stable): equal codes form segments in (read, pos) order; positions are
//     then resolved to (read, pos).
//  5. segments -> exact frequency (segment length) -> reliable flag -> column = rank of the
//     reliable code; within a reliable segment the first entry of each read is its lowest
//     position: those entries are At's row, already sorted by read.
//  6. A = At transposed by a stable radix sort on the read id (columns stay ascending).
#include <type_traits>

#include "check.cuh"
#include "ops.cuh"

namespace sg {

constexpr int KM_NT = 256;
constexpr int KM_W = 32;                  // windows per thread
constexpr int KM_CHUNK = KM_NT * KM_W;    // windows per block

// 32-bit mix of a 64-bit k-mer code (multiply-xorshift finaliser).
__device__ __forceinline__ uint32_t hash32(uint64_t code, uint32_t seed) {
    uint32_t h = (uint32_t)code * 0x9E3779B1u + seed;
    h ^= (uint32_t)(code >> 32) * 0x85EBCA77u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}

// Blocked Bloom filter: a key sets 4 bits of one 32-bit word, so whether all of them were
// already set is decided by the single atomicOr that sets them.
struct Bloom {
    uint32_t *words;
    uint32_t nwords;
    uint32_t seed;
    __device__ __forceinline__ void probe(uint64_t code, uint32_t *idx, uint32_t *mask) const {
        const uint32_t h = hash32(code, seed);
        *idx = __umulhi(h, nwords);
        const uint32_t g = h * 0x85EBCA6Bu;  // bit positions from a second mix
        *mask = (1u << (g >> 27)) | (1u << ((g >> 22) & 31u)) | (1u << ((g >> 17) & 31u)) |
                (1u << ((g >> 12) & 31u));
    }
};

// Per-thread cursor over the job map (reads are visited in increasing order).
struct JobCursor {
    JobMap m;
    int64_t jb = 0, jlo = 0, jhi = -1;
    __device__ __forceinline__ uint64_t key(uint64_t code, int64_t r) {
        if (!m.ro) return code;
        if (r < jlo || r >= jhi) {  // last job b with ro[b] <= r
            int64_t lo = 0, hi = m.njobs;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (m.ro[mid] <= r) lo = mid; else hi = mid;
            }
            jb = lo;
            jlo = m.ro[lo];
            jhi = m.ro[lo + 1];
        }
        return ((uint64_t)jb << m.kbits) | code;
    }
};

// Visits the windows [c0 + t*KM_W, c0 + (t+1)*KM_W) of thread t in position order, calling
// f(code, strand, read, pos, local start) for each window of k A/C/G/T bases inside one read, where
// the local start (in [t*KM_W, (t+1)*KM_W)) indexes the block's chunk. K > 0 makes k a
// compile-time constant (K == 0: k taken from k_rt). Indices inside the block are 32-bit.
template <int K, class F>
__device__ __forceinline__ void for_each_window(const uint8_t *__restrict__ sm, int64_t c0, int64_t total,
                                                const int64_t *__restrict__ off, int64_t n, int k_rt,
                                                F &&f) {
    const int k = K > 0 ? K : k_rt;
    const int ls = threadIdx.x * KM_W;
    const int64_t qs = c0 + ls;
    if (qs >= total || n <= 0) return;
    int le = ls + KM_W + k - 1;  // exclusive, local to the block
    if (c0 + le > total) le = (int)(total - c0);
    // read containing qs: last r with off[r] <= qs
    int64_t lo = 0, hi = n;  // invariant: off[lo] <= qs < off[hi] (off[n] = total > qs)
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= qs) lo = mid; else hi = mid;
    }
    int64_t r = lo;
    int64_t rbase = off[r] - c0;  // start of read r relative to the block
    int64_t nx = off[r + 1] - c0;
    int next = nx > (int64_t)0x7fffffff ? 0x7fffffff : (int)nx;
    const uint64_t mask = (1ull << (2 * k)) - 1;
    const int rs = 2 * (k - 1);
    uint64_t fw = 0, rc = 0;
    int run = 0;
    for (int q = ls; q < le; q++) {
        // crossed into the next read (skips empty reads); r + 1 < n keeps every access in
        // bounds even when the offsets turn out to be invalid (reported after this pass)
        while (q >= next && r + 1 < n) {
            r++;
            rbase = off[r] - c0;
            nx = off[r + 1] - c0;
            next = nx > (int64_t)0x7fffffff ? 0x7fffffff : (int)nx;
            run = 0;
        }
        const uint32_t c = sm[q];
        const bool ok = (c == 'A') | (c == 'C') | (c == 'G') | (c == 'T');
        const uint32_t t = (c >> 1) & 3u;
        const uint32_t b = t ^ (t >> 1);  // A=0 C=1 G=2 T=3
        fw = ((fw << 2) | b) & mask;
        rc = (rc >> 2) | ((uint64_t)(3u - b) << rs);
        run = ok ? run + 1 : 0;
        if (run >= k && q - k + 1 >= ls) {
            const uint64_t code = fw < rc ? fw : rc;
            const uint32_t strand = rc < fw ? 1u : 0u;
            f(code, strand, r, (uint32_t)(q - k + 1 - rbase), q - k + 1);
        }
    }
}

// Stages the block's bases in shared memory. The reads stream through once per pass, so they
// are loaded evict-first (ld.global.cs) to keep the filters resident in L2; 16-byte loads when
// the chunk start is 16-byte aligned.
__device__ __forceinline__ void load_chunk(uint8_t *sm, const uint8_t *__restrict__ seq, int64_t c0,
                                           int64_t total, int k) {
    int64_t len = (int64_t)KM_CHUNK + k - 1;
    if (c0 + len > total) len = total - c0;
    int64_t done = 0;
    if ((((uintptr_t)(seq + c0)) & 15) == 0) {
        const int64_t nv = len >> 4;
        const uint4 *src = reinterpret_cast<const uint4 *>(seq + c0);
        uint4 *dst = reinterpret_cast<uint4 *>(sm);
        for (int64_t i = threadIdx.x; i < nv; i += KM_NT) dst[i] = __ldcs(src + i);
        done = nv << 4;
    }
    for (int64_t i = done + threadIdx.x; i < len; i += KM_NT) sm[i] = __ldcs(seq + c0 + i);
    __syncthreads();
}

// One walk over the reads: wc[q] = canonical code of the window starting at global position q
// (with the job prefix in a batch) | strand << 63, or ~0 when no valid window starts at q. The
// later passes stream this array instead of walking the reads again.
constexpr uint64_t WC_NONE = ~0ull;
constexpr uint64_t WC_STRAND = 1ull << 63;

template <int K>
__global__ void __launch_bounds__(KM_NT) window_codes_kernel(const uint8_t *__restrict__ seq, int64_t total,
                                                            const int64_t *__restrict__ off, int64_t n, int k,
                                                            JobMap jm, uint64_t *__restrict__ wc) {
    extern __shared__ __align__(16) unsigned char wc_raw[];
    uint64_t *s_wc = reinterpret_cast<uint64_t *>(wc_raw);
    uint8_t *sm = wc_raw + KM_CHUNK * sizeof(uint64_t);
    const int64_t c0 = (int64_t)blockIdx.x * KM_CHUNK;
    for (int i = threadIdx.x; i < KM_CHUNK; i += KM_NT) s_wc[i] = WC_NONE;
    load_chunk(sm, seq, c0, total, k);  // ends with __syncthreads
    JobCursor jc{jm};
    for_each_window<K>(sm, c0, total, off, n, k,
                       [&](uint64_t code0, uint32_t strand, int64_t r, uint32_t, int lw) {
        if (SG_IN_BOUNDS(lw >= 0 && lw < KM_CHUNK, 101, lw)) s_wc[lw] = jc.key(code0, r) | ((uint64_t)strand << 63);
    });
    __syncthreads();
    const int64_t cnt = total - c0 < KM_CHUNK ? total - c0 : KM_CHUNK;
    for (int64_t i = threadIdx.x; i < cnt; i += KM_NT) wc[c0 + i] = s_wc[i];
}

// One launch per slice [w_lo, w_hi) of B1's words: every launch streams all window codes but only
// the k-mers whose B1 word lies in its slice touch the filter, so the slice stays in L2.
__global__ void __launch_bounds__(KM_NT) bloom_insert_kernel(const uint64_t *__restrict__ wc, int64_t total,
                                                            Bloom b1, Bloom b2, uint32_t w_lo, uint32_t w_hi) {
    for (int64_t q = (int64_t)blockIdx.x * KM_NT + threadIdx.x; q < total; q += (int64_t)gridDim.x * KM_NT) {
        const uint64_t x = __ldcs(wc + q);
        if (x == WC_NONE) continue;
        const uint64_t code = x & ~WC_STRAND;
        uint32_t i1, m1;
        b1.probe(code, &i1, &m1);
        if (i1 < w_lo || i1 >= w_hi) continue;  // another slice's launch handles this k-mer
        const uint32_t old = atomicOr(b1.words + i1, m1);
        if ((old & m1) == m1) {
            uint32_t i2, m2;
            b2.probe(code, &i2, &m2);
            if ((b2.words[i2] & m2) != m2) atomicOr(b2.words + i2, m2);
        }
    }
}

// Candidates: windows whose code tests positive in B2 (every occurrence of a k-mer seen at least
// twice; false positives only add singletons, which the exact count drops). use_bloom == 0 keeps
// every window (lo == 1: singletons may be reliable). Thread t of block b owns the KM_W
// consecutive windows starting at b * KM_CHUNK + t * KM_W, so candidates keep position order.
__device__ __forceinline__ bool is_candidate(uint64_t x, const Bloom &b2, int use_bloom) {
    if (x == WC_NONE) return false;
    if (!use_bloom) return true;
    uint32_t i2, m2;
    b2.probe(x & ~WC_STRAND, &i2, &m2);
    return (b2.words[i2] & m2) == m2;
}

__global__ void __launch_bounds__(KM_NT) cand_count_kernel(const uint64_t *__restrict__ wc, int64_t total, Bloom b2,
                                                          int use_bloom, uint32_t *__restrict__ cnt) {
    const int64_t q0 = (int64_t)blockIdx.x * KM_CHUNK + (int64_t)threadIdx.x * KM_W;
    uint32_t c = 0;
    for (int w = 0; w < KM_W; w++) {
        const int64_t q = q0 + w;
        if (q >= total) break;
        c += is_candidate(__ldcs(wc + q), b2, use_bloom) ? 1u : 0u;
    }
    cnt[(int64_t)blockIdx.x * KM_NT + threadIdx.x] = c;
}

// keys = code (job prefix included), shifted left by ib with the candidate's index below it when
// ib > 0 (keys-only sort); vals = q | strand << 63 (global window start).
__global__ void __launch_bounds__(KM_NT) cand_emit_kernel(const uint64_t *__restrict__ wc, int64_t total, Bloom b2,
                                                         int use_bloom, const int64_t *__restrict__ pos_of_thread,
                                                         int ib, uint64_t *__restrict__ keys,
                                                         uint64_t *__restrict__ vals, int64_t nc) {
    const int64_t q0 = (int64_t)blockIdx.x * KM_CHUNK + (int64_t)threadIdx.x * KM_W;
    int64_t o = pos_of_thread[(int64_t)blockIdx.x * KM_NT + threadIdx.x];
    for (int w = 0; w < KM_W; w++) {
        const int64_t q = q0 + w;
        if (q >= total) break;
        const uint64_t x = __ldcs(wc + q);
        if (!is_candidate(x, b2, use_bloom)) continue;
        if (!SG_IN_BOUNDS(o >= 0 && o < nc, 102, o)) break;
        keys[o] = ib ? (((x & ~WC_STRAND) << ib) | (uint64_t)o) : (x & ~WC_STRAND);
        vals[o] = (uint64_t)q | (x & WC_STRAND);
        o++;
    }
}

__device__ __forceinline__ uint64_t resolve_pos(uint64_t v, const int64_t *__restrict__ off, int64_t n) {
    const int64_t q = (int64_t)(v & ~WC_STRAND);
    int64_t lo = 0, hi = n;  // last read r with off[r] <= q
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= q) lo = mid; else hi = mid;
    }
    return ((uint64_t)lo << 32) | (uint64_t)(uint32_t)(q - off[lo]) | ((v >> 63) << 31);
}

// Keys-only sort: packed (code << ib | index) -> code, and the indexed value resolved.
__global__ void unpack_kernel(const uint64_t *__restrict__ packed, const uint64_t *__restrict__ vals, int64_t nc,
                              int ib, const int64_t *__restrict__ off, int64_t n, uint64_t *__restrict__ key,
                              uint64_t *__restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const uint64_t p = packed[i];
    const int64_t src = (int64_t)(p & ((1ull << ib) - 1));
    key[i] = p >> ib;
    if (SG_IN_BOUNDS(src < nc, 103, src)) val[i] = resolve_pos(vals[src], off, n);
}

// After the pairs sort: val = q | strand << 63  ->  read << 32 | pos | strand << 31.
__global__ void resolve_kernel(uint64_t *__restrict__ val, int64_t nc, const int64_t *__restrict__ off,
                               int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const uint64_t v = val[i];
    const int64_t q = (int64_t)(v & ~WC_STRAND);
    int64_t lo = 0, hi = n;  // last read r with off[r] <= q
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= q) lo = mid; else hi = mid;
    }
    val[i] = ((uint64_t)lo << 32) | (uint64_t)(uint32_t)(q - off[lo]) | ((v >> 63) << 31);
}

__global__ void validate_offsets_kernel(const int64_t *__restrict__ off, int64_t n, int64_t total,
                                        uint32_t *__restrict__ err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    int64_t a = off[i];
    bool bad = false;
    if (i == 0 && a != 0) bad = true;
    if (i == n && a != total) bad = true;
    if (i < n) {
        int64_t b = off[i + 1];
        if (b < a || b - a >= ((int64_t)1 << 31)) bad = true;
    }
    if (bad) atomicOr(err, (uint32_t)DEV_INVALID);
}

// head[i] = 1 where a new code starts.
__global__ void seg_head_kernel(const uint64_t *__restrict__ key, int64_t nc, uint32_t *__restrict__ head) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) head[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

// seg_start[s] = first index of segment s; seg_start[nseg] = nc.
__global__ void seg_start_kernel(const uint32_t *__restrict__ head, const int64_t *__restrict__ seg_excl,
                                 int64_t nc, int64_t *__restrict__ seg_start) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc && head[i] && SG_IN_BOUNDS(seg_excl[i] >= 0 && seg_excl[i] <= nc, 104, seg_excl[i]))
        seg_start[seg_excl[i]] = i;
    if (i == nc - 1 && SG_IN_BOUNDS(seg_excl[nc] >= 0 && seg_excl[nc] <= nc, 104, seg_excl[nc]))
        seg_start[seg_excl[nc]] = nc;
}

// lohi (batches): the reliable range of each job, [2 * job] = lo, [2 * job + 1] = hi.
// Launched over at least nc threads; rel has nc + 1 slots.
__global__ void seg_reliable_kernel(const int64_t *__restrict__ seg_start, const int64_t *__restrict__ nseg_p,
                                    uint32_t lo, uint32_t hi, const uint64_t *__restrict__ key,
                                    const uint32_t *__restrict__ lohi, int kbits, int64_t nc,
                                    uint32_t *__restrict__ rel) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nc) return;
    int64_t nseg = *nseg_p;
    if (s >= nseg) {  // slots past the last segment still feed the scan below: make them 0
        rel[s] = 0u;
        return;
    }
    if (lohi) {
        const uint64_t job = key[seg_start[s]] >> kbits;
        lo = lohi[2 * job];
        hi = lohi[2 * job + 1];
    }
    int64_t len = seg_start[s + 1] - seg_start[s];
    rel[s] = (len >= (int64_t)lo && len <= (int64_t)hi) ? 1u : 0u;
}

// keep[i]: i lies in a reliable segment and is the first (lowest position) entry of its read.
__global__ void keep_kernel(const uint32_t *__restrict__ head, const int64_t *__restrict__ seg_excl,
                            const uint32_t *__restrict__ rel, const uint64_t *__restrict__ val, int64_t nc,
                            uint32_t *__restrict__ keep) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    int64_t s = seg_excl[i] + head[i] - 1;
    bool first = head[i] || ((val[i] >> 32) != (val[i - 1] >> 32));
    keep[i] = (rel[s] && first) ? 1u : 0u;
}

// Writes At's entries, its row pointers, the column codes, and the (read, col|val) pairs that
// are sorted into A.
__global__ void emit_at_kernel(const uint32_t *__restrict__ head, const int64_t *__restrict__ seg_excl,
                               const uint32_t *__restrict__ rel, const int64_t *__restrict__ col_of_seg,
                               const uint32_t *__restrict__ keep, const int64_t *__restrict__ out_pos,
                               const uint64_t *__restrict__ key, const uint64_t *__restrict__ val, int64_t nc,
                               int64_t m, int64_t nnz, int32_t *__restrict__ at_col, uint32_t *__restrict__ at_val,
                               int64_t *__restrict__ at_rp, uint64_t *__restrict__ codes,
                               uint32_t *__restrict__ a_key, uint64_t *__restrict__ a_val, int kbits,
                               unsigned long long *__restrict__ job_ncols) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) at_rp[m] = nnz;
    if (i >= nc) return;
    int64_t s = seg_excl[i] + head[i] - 1;
    if (head[i] && rel[s]) {
        int64_t j = col_of_seg[s];
        if (!SG_IN_BOUNDS(j >= 0 && j < m, 105, j)) return;
        at_rp[j] = out_pos[i];
        codes[j] = kbits < 64 ? key[i] & ((1ull << kbits) - 1) : key[i];
        if (job_ncols) atomicAdd(job_ncols + (key[i] >> kbits), 1ull);
    }
    if (keep[i]) {
        int64_t o = out_pos[i];
        if (!SG_IN_BOUNDS(o >= 0 && o < nnz, 106, o)) return;
        uint32_t r = (uint32_t)(val[i] >> 32), v = (uint32_t)val[i];
        at_col[o] = (int32_t)r;
        at_val[o] = v;
        a_key[o] = r;
        a_val[o] = ((uint64_t)col_of_seg[s] << 32) | v;
    }
}

// Row pointers of A from the read ids of its entries, sorted ascending.
__global__ void rowptr_from_sorted_kernel(const uint32_t *__restrict__ rows, int64_t nnz, int64_t n,
                                          int64_t *__restrict__ rp) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > nnz) return;
    int64_t prev = (e == 0) ? -1 : (int64_t)rows[e - 1];
    int64_t cur = (e == nnz) ? n : (int64_t)rows[e];
    if (!SG_IN_BOUNDS(prev >= -1 && cur <= n && prev <= cur, 107, cur)) return;
    for (int64_t r = prev + 1; r <= cur; r++) rp[r] = e;
}

__global__ void split_pairs_kernel(const uint64_t *__restrict__ pv, int64_t nnz, int32_t *__restrict__ col,
                                   uint32_t *__restrict__ val) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    uint64_t x = pv[e];
    col[e] = (int32_t)(x >> 32);
    val[e] = (uint32_t)x;
}

static inline int64_t blocks_for(int64_t n, int nt) { return (n + nt - 1) / nt; }

// Runs f with k as a compile-time constant for the common k (17 is the paper's), else 0.
template <class F>
static sg_status dispatch_k(int k, F &&f) {
    switch (k) {
        case 17: return f(std::integral_constant<int, 17>{});
        case 21: return f(std::integral_constant<int, 21>{});
        case 31: return f(std::integral_constant<int, 31>{});
        default: return f(std::integral_constant<int, 0>{});
    }
}

// jm.ro == nullptr: one read set with range [lo, hi]. Otherwise a batch: lohi (device) holds
// each job's range and job_ncols (device, zeroed, njobs entries) receives each job's column count.
sg_status build_impl(const uint8_t *seq, const int64_t *off, int64_t n, int64_t total, int k,
                     uint32_t lo, uint32_t hi, sg_csr_u32 *A, sg_csr_u32 *At, uint64_t **codes_out,
                     cudaStream_t s, Scratch &sc, JobMap jm, const uint32_t *lohi,
                     unsigned long long *job_ncols) {
    const int NT = 256;
    uint32_t *err = sc.get<uint32_t>(1);
    if (!err) return SG_ERR_OOM;
    SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    SG_LAUNCH("validate_offsets", validate_offsets_kernel, blocks_for(n + 1, NT), NT, 0, s, off, n, total, err);

    const int64_t nblk = blocks_for(total, KM_CHUNK);
    const int use_bloom = lo >= 2 ? 1 : 0;
    Bloom b1{nullptr, 0, 0x9e3779b9u}, b2{nullptr, 0, 0x7f4a7c15u};
    if (use_bloom && total > 0) {
        // B1: 8 bits per window; B2 ("seen twice"): 2 bits per window; 32-bit words
        const int64_t w1 = total / 4 + 1024, w2 = total / 16 + 1024;
        b1.nwords = (uint32_t)(w1 < 0xFFFFFFF0LL ? w1 : 0xFFFFFFF0LL);
        b2.nwords = (uint32_t)(w2 < 0xFFFFFFF0LL ? w2 : 0xFFFFFFF0LL);
        b1.words = sc.get<uint32_t>(b1.nwords);
        b2.words = sc.get<uint32_t>(b2.nwords);
        if (!b1.words || !b2.words) return SG_ERR_OOM;
        SG_CUDA_TRY(cudaMemsetAsync(b1.words, 0, (size_t)b1.nwords * 4, s));
        SG_CUDA_TRY(cudaMemsetAsync(b2.words, 0, (size_t)b2.nwords * 4, s));
    }
    // 0. window codes
    uint64_t *wc = sc.get<uint64_t>(total + 1);
    if (!wc) return SG_ERR_OOM;
    {
        const size_t smem = (size_t)KM_CHUNK * sizeof(uint64_t) + KM_CHUNK + 48;
        SG_TRY(dispatch_k(k, [&](auto kc) -> sg_status {
            SG_CUDA_TRY(ensure_smem(window_codes_kernel<decltype(kc)::value>, smem));
            SG_LAUNCH("window_codes", window_codes_kernel<decltype(kc)::value>, nblk, KM_NT, smem, s, seq, total,
                      off, n, k, jm, wc);
            return SG_OK;
        }));
    }
    if (use_bloom) {
        // slices of at most bloom_slice_mb of B1, so each launch's atomics stay in L2
        const uint64_t slice_words = ((uint64_t)tune("bloom_slice_mb") << 20) / 4;
        const uint64_t nsl = (b1.nwords + slice_words - 1) / slice_words;
        const int64_t grid = blocks_for(total, KM_NT) < 152 * 16 ? blocks_for(total, KM_NT) : 152 * 16;
        for (uint64_t q = 0; q < nsl; q++) {
            const uint32_t lo_w = (uint32_t)((uint64_t)b1.nwords * q / nsl);
            const uint32_t hi_w = (uint32_t)((uint64_t)b1.nwords * (q + 1) / nsl);
            SG_LAUNCH("bloom_insert", bloom_insert_kernel, grid, KM_NT, 0, s, (const uint64_t *)wc, total, b1, b2,
                      lo_w, hi_w);
        }
    }
    uint32_t *tcnt = sc.get<uint32_t>(nblk * KM_NT + 1);
    int64_t *tpos = sc.get<int64_t>(nblk * KM_NT + 1);
    if (!tcnt || !tpos) return SG_ERR_OOM;
    SG_LAUNCH("cand_count", cand_count_kernel, nblk, KM_NT, 0, s, (const uint64_t *)wc, total, b2, use_bloom, tcnt);
    SG_TRY(exclusive_scan<uint32_t>(tcnt, tpos, nblk * KM_NT, s));
    int64_t nc = 0;
    uint32_t herr = 0;
    SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(read_back(&nc, tpos + nblk * KM_NT, sizeof(int64_t), s));
    if (herr) {  // the passes above stayed in bounds; their results are discarded
        set_error("build_kmer_matrix: offsets are not a valid partition of the sequence");
        return SG_ERR_INVALID;
    }

    uint64_t *key0 = sc.get<uint64_t>(nc), *val0 = sc.get<uint64_t>(nc);
    uint64_t *key1 = sc.get<uint64_t>(nc), *val1 = sc.get<uint64_t>(nc);
    if (!key0 || !val0 || !key1 || !val1) return SG_ERR_OOM;
    int job_bits = 0;
    while (jm.ro && ((int64_t)1 << job_bits) < jm.njobs) job_bits++;
    const int code_bits = 2 * k + job_bits;
    int ib = 1;
    while (((int64_t)1 << ib) < nc) ib++;
    if (code_bits + ib > 64) ib = 0;  // too wide to pack: sort (key, value) pairs
    SG_LAUNCH("cand_emit", cand_emit_kernel, nblk, KM_NT, 0, s, (const uint64_t *)wc, total, b2, use_bloom,
              (const int64_t *)tpos, ib, key0, val0, nc);
    bool alt = false;
    const uint64_t *key;
    uint64_t *val;
    if (ib) {  // 8-byte keys through the radix passes, values gathered once afterwards
        SG_TRY(radix_sort_keys(key0, key1, nc, ib, ib + code_bits, &alt, s));
        uint64_t *ks = alt ? key1 : key0, *kfree = alt ? key0 : key1;
        SG_LAUNCH("unpack", unpack_kernel, blocks_for(nc, NT), NT, 0, s, (const uint64_t *)ks, (const uint64_t *)val0,
                  nc, ib, off, n, kfree, val1);
        key = kfree;
        val = val1;
    } else {
        SG_TRY((radix_sort_pairs<uint64_t, uint64_t>(key0, val0, key1, val1, nc, code_bits, &alt, s)));
        key = alt ? key1 : key0;
        val = alt ? val1 : val0;
        SG_LAUNCH("resolve", resolve_kernel, blocks_for(nc, NT), NT, 0, s, val, nc, off, n);
    }

    uint32_t *head = sc.get<uint32_t>(nc + 1);
    int64_t *seg_excl = sc.get<int64_t>(nc + 1);
    int64_t *seg_start = sc.get<int64_t>(nc + 1);
    uint32_t *rel = sc.get<uint32_t>(nc + 1);
    int64_t *col_of_seg = sc.get<int64_t>(nc + 1);
    uint32_t *keep = sc.get<uint32_t>(nc + 1);
    int64_t *out_pos = sc.get<int64_t>(nc + 1);
    if (!head || !seg_excl || !seg_start || !rel || !col_of_seg || !keep || !out_pos) return SG_ERR_OOM;
    SG_LAUNCH("seg_head", seg_head_kernel, blocks_for(nc, NT), NT, 0, s, key, nc, head);
    SG_TRY(exclusive_scan<uint32_t>(head, seg_excl, nc, s));
    SG_LAUNCH("seg_start", seg_start_kernel, blocks_for(nc, NT), NT, 0, s, head, seg_excl, nc, seg_start);
    // number of segments lives on the device at seg_excl[nc]; launch over the upper bound nc
    SG_LAUNCH("seg_reliable", seg_reliable_kernel, blocks_for(nc, NT), NT, 0, s, seg_start, seg_excl + nc, lo,
              hi, key, lohi, 2 * k, nc, rel);
    SG_TRY(exclusive_scan<uint32_t>(rel, col_of_seg, nc, s));
    SG_LAUNCH("keep", keep_kernel, blocks_for(nc, NT), NT, 0, s, head, seg_excl, rel, val, nc, keep);
    SG_TRY(exclusive_scan<uint32_t>(keep, out_pos, nc, s));
    int64_t sizes[2] = {0, 0};  // m, nnz
    // m = reliable segments = col_of_seg[nc] (rel is 0 past the last segment)
    SG_CUDA_TRY(cudaMemcpyAsync(&sizes[0], col_of_seg + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaMemcpyAsync(&sizes[1], out_pos + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t m = sizes[0], nnz = sizes[1];
    if (m >= ((int64_t)1 << 31)) {
        set_error("build_kmer_matrix: %lld reliable k-mers exceed the int32 column range", (long long)m);
        return SG_ERR_OVERFLOW;
    }

    // outputs
    SG_ALLOC(At->row_ptr, int64_t, m + 1, s);
    SG_ALLOC(At->col, int32_t, nnz, s);
    SG_ALLOC(At->val, uint32_t, nnz, s);
    SG_ALLOC(A->row_ptr, int64_t, n + 1, s);
    SG_ALLOC(A->col, int32_t, nnz, s);
    SG_ALLOC(A->val, uint32_t, nnz, s);
    SG_ALLOC(*codes_out, uint64_t, m, s);
    At->n_rows = m; At->n_cols = n; At->nnz = nnz;
    A->n_rows = n; A->n_cols = m; A->nnz = nnz;

    uint32_t *ak0 = sc.get<uint32_t>(nnz), *ak1 = sc.get<uint32_t>(nnz);
    uint64_t *av0 = sc.get<uint64_t>(nnz), *av1 = sc.get<uint64_t>(nnz);
    if (!ak0 || !ak1 || !av0 || !av1) return SG_ERR_OOM;
    SG_LAUNCH("emit_at", emit_at_kernel, blocks_for(nc > 0 ? nc : 1, NT), NT, 0, s, head, seg_excl, rel, col_of_seg,
              keep, out_pos, key, val, nc, m, nnz, At->col, At->val, At->row_ptr, *codes_out, ak0, av0, 2 * k,
              job_ncols);
    int rbits = 0;
    while (rbits < 32 && ((int64_t)1 << rbits) < n) rbits++;
    bool aalt = false;
    SG_TRY((radix_sort_pairs<uint32_t, uint64_t>(ak0, av0, ak1, av1, nnz, rbits, &aalt, s)));
    const uint32_t *arow = aalt ? ak1 : ak0;
    const uint64_t *apv = aalt ? av1 : av0;
    SG_LAUNCH("rowptr_from_sorted", rowptr_from_sorted_kernel, blocks_for(nnz + 1, NT), NT, 0, s, arow, nnz, n,
              A->row_ptr);
    SG_LAUNCH("split_pairs", split_pairs_kernel, blocks_for(nnz, NT), NT, 0, s, apv, nnz, A->col, A->val);
    return SG_OK;
}

}  // namespace sg

extern "C" sg_status sg_build_kmer_matrix(const uint8_t *d_seq, const int64_t *d_offsets, int64_t n_reads,
                                          int64_t total_len, int32_t k, uint32_t lo, uint32_t hi,
                                          sg_csr_u32 *A, sg_csr_u32 *At, uint64_t **d_kmer_codes,
                                          sg_stream_t stream) {
    if (!A || !At || !d_kmer_codes) {
        sg::set_error("build_kmer_matrix: NULL output struct");
        return SG_ERR_INVALID;
    }
    *A = sg_csr_u32{};
    *At = sg_csr_u32{};
    *d_kmer_codes = nullptr;
    if (k < 1 || k > 31 || (k & 1) == 0 || lo < 1 || lo > hi || n_reads < 0 || n_reads >= ((int64_t)1 << 31) ||
        total_len < 0 || !d_offsets || (total_len > 0 && !d_seq) || (n_reads == 0 && total_len != 0)) {
        sg::set_error("build_kmer_matrix: invalid arguments (k=%d lo=%u hi=%u n=%lld total=%lld)", k, lo, hi,
                      (long long)n_reads, (long long)total_len);
        return SG_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    sg_status st;
    {
        sg::Scratch sc(s);
        st = sg::build_impl(d_seq, d_offsets, n_reads, total_len, k, lo, hi, A, At, d_kmer_codes, s, sc,
                            sg::JobMap{nullptr, 1, 2 * k}, nullptr, nullptr);
    }
    if (st != SG_OK) {
        sg_free_csr_u32(A, stream);
        sg_free_csr_u32(At, stream);
        sg::dfree(*d_kmer_codes, s);
        *d_kmer_codes = nullptr;
    }
    return st;
}

extern "C" void sg_free_csr_u32(sg_csr_u32 *m, sg_stream_t stream) {
    if (!m) return;
    cudaStream_t s = (cudaStream_t)stream;
    sg::dfree(m->row_ptr, s);
    sg::dfree(m->col, s);
    sg::dfree(m->val, s);
    *m = sg_csr_u32{};
}
