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
//  0. pack           one walk over the reads packs the bases (2 bits each) and stores each
//                    window's 32-bit filter hash (H_NONE where no valid window starts); later
//                    passes recompute a window's canonical code and strand from two packed words.
//  1. bloom_insert   every code is OR-ed into the blocked Bloom filter B1 (all probe bits in one
//                    32-bit word, so "already present" is decided by one atomic); a code found
//                    present is OR-ed into B2 ("seen at least twice"). Where they fit, the hashes
//                    are first grouped by filter bin and each bin's filters live in shared memory.
//                    Skipped when lo == 1.
//  2. cand_count     per warp, a ballot mask of the windows whose code tests positive in B2.
//                    Every occurrence of a k-mer with frequency >= 2 passes (false positives only
//                    add singletons, which the exact count below drops).
//  3. cand_emit      writes (code, position | strand) at scanned offsets, so the candidates stay
//                    in position order, i.e. (read, pos) order.
//  4. radix sort by code (stable): equal codes form segments in (read, pos) order.
//  5. segments -> exact frequency (segment length) -> reliable flag -> column = rank of the
//     reliable code; within a reliable segment the first entry of each read is its lowest
//     position: those entries are At's row, already sorted by read. For position-and-code keys
//     this runs on the sorted keys themselves (seg_mark, scans of its tile totals, seg_emit,
//     which resolves the kept windows to (read, pos)); other key forms are unpacked first.
//  6. A = At transposed by a stable radix sort on the read id (columns stay ascending); its last
//     pass writes A's column and value arrays.
#include <optional>
#include <type_traits>

#include "check.cuh"
#include "ops.cuh"

namespace sg {

constexpr int KM_NT = 256;
constexpr int KM_W = 32;                  // windows per thread
constexpr int KM_CHUNK = KM_NT * KM_W;    // windows per block
constexpr int KM_WARPS = KM_NT / 32;

// 32-bit mix of a 64-bit k-mer code (multiply-xorshift finaliser).
__device__ __forceinline__ uint32_t fmix(uint32_t h) {
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}

__device__ __forceinline__ uint32_t hash32(uint64_t code, uint32_t seed) {
    uint32_t h = (uint32_t)code * 0x9E3779B1u + seed;
    h ^= (uint32_t)(code >> 32) * 0x85EBCA77u;
    return fmix(h);
}

// Blocked Bloom filter: a key sets 4 bits of one 32-bit word, so whether all of them were
// already set is decided by the single atomicOr that sets them. Word and bits come from the key's
// 32-bit hash h (B1: h = hash32(key); B2: h = fmix(that hash ^ B2 seed), so both filters work
// from one stored hash per window).
struct Bloom {
    uint32_t *words;
    uint32_t nwords;
    __device__ __forceinline__ void probe(uint32_t h, uint32_t *idx, uint32_t *mask) const {
        *idx = __umulhi(h, nwords);
        const uint32_t g = h * 0x85EBCA6Bu;  // bit positions from a second mix
        *mask = (1u << (g >> 27)) | (1u << ((g >> 22) & 31u)) | (1u << ((g >> 17) & 31u)) |
                (1u << ((g >> 12) & 31u));
    }
};

// Batches: the job prefix of a window, from the base offset of each job's first read (jpos[b] =
// off[ro[b]], jpos[njobs] = total). A window lies in the last job b with jpos[b] <= its position
// (windows never cross reads, and empty jobs start where the next one does). The cursor keeps the
// last job's range, so increasing positions search only when they leave it.
struct JobPos {
    const int64_t *jpos;  // nullptr: one read set, no prefix
    int64_t njobs;
    int kbits;  // 2k
};

struct JobPosCursor {
    JobPos m;
    int64_t jb = 0, jlo = 0, jhi = -1;
    __device__ __forceinline__ uint64_t prefix(int64_t q) {
        if (!m.jpos) return 0;
        if (q < jlo || q >= jhi) {
            int64_t lo = 0, hi = m.njobs;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (m.jpos[mid] <= q) lo = mid; else hi = mid;
            }
            jb = lo;
            jlo = m.jpos[lo];
            jhi = m.jpos[lo + 1];
        }
        return (uint64_t)jb << m.kbits;
    }
};

__global__ void job_pos_kernel(const int64_t *__restrict__ ro, int64_t njobs, const int64_t *__restrict__ off,
                               int64_t n, int64_t *__restrict__ jpos) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > njobs) return;
    int64_t r = ro[b];
    r = r < 0 ? 0 : (r > n ? n : r);
    jpos[b] = off[r];
}

// Staged bases: the block's chunk as 32-bit words (4 bases each), one pad word after every 8, so
// that thread t's 32-base segment starts at word 9t and a warp reading the j-th word of its
// segments hits 32 distinct banks. Bytes past the end of the sequence read as 'N'.
constexpr int KM_SWORDS = KM_CHUNK / 4 + 16;           // covers 32 + k - 1 bases past the last segment
constexpr int KM_SPAD = KM_SWORDS + KM_SWORDS / 8 + 1;
__device__ __forceinline__ int spad(int w) { return w + (w >> 3); }

__device__ __forceinline__ void load_chunk(uint32_t *smw, const uint8_t *__restrict__ seq, int64_t c0,
                                           int64_t total) {
    const int64_t len = total - c0;  // bytes of the sequence from c0 on
    const bool al4 = (((uintptr_t)(seq + c0)) & 3) == 0;
    for (int w = threadIdx.x; w < KM_SWORDS; w += KM_NT) {
        const int64_t b = 4 * (int64_t)w;
        uint32_t v;
        if (al4 && b + 3 < len) {
            v = __ldcs(reinterpret_cast<const unsigned int *>(seq + c0 + b));
        } else {
            v = 0;
#pragma unroll
            for (int u = 0; u < 4; u++) v |= (uint32_t)(b + u < len ? seq[c0 + b + u] : (uint8_t)'N') << (8 * u);
        }
        smw[spad(w)] = v;
    }
    __syncthreads();
}

// One walk over the reads. Every window q gets H[q] = the 32-bit hash of its canonical key (code,
// with the job prefix in a batch), or H_NONE when no valid window starts at q (a non-ACGT base, or
// the window crosses a read end); the Bloom passes and the candidate test work from H alone. P[g]
// holds bases 32g .. 32g + 31 as 2-bit codes (A=0 C=1 G=2 T=3), base 32g + j at bits 2j, from which
// the emit pass recomputes the code and strand of the few windows that are candidates
// (window_key). Thread t of block b covers windows and bases b * KM_CHUNK + t * KM_W + j, j < KM_W,
// reading bases [t * KM_W, t * KM_W + KM_W + k - 1) of the block's chunk. K > 0 makes k a
// compile-time constant (K == 0: k taken from k_rt).
constexpr uint64_t WC_STRAND = 1ull << 63;
constexpr uint32_t H_NONE = 0xFFFFFFFFu;
constexpr uint32_t B1_SEED = 0x9e3779b9u, B2_SEED = 0x7f4a7c15u;
static_assert(KM_W == 32, "one packed word per thread");

__device__ __forceinline__ uint32_t b2_hash(uint32_t h1) { return fmix(h1 ^ B2_SEED); }

template <int K>
__global__ void __launch_bounds__(KM_NT) pack_kernel(const uint8_t *__restrict__ seq, int64_t total,
                                                    const int64_t *__restrict__ off, int64_t n, int k_rt, JobPos jp,
                                                    uint64_t *__restrict__ P, uint32_t *__restrict__ H) {
    __shared__ uint32_t smw[KM_SPAD];
    const int k = K > 0 ? K : k_rt;
    const int64_t c0 = (int64_t)blockIdx.x * KM_CHUNK;
    load_chunk(smw, seq, c0, total);  // ends with __syncthreads
    const int ls = threadIdx.x * KM_W;
    const int64_t qs = c0 + ls;  // first window (and base) of this thread; a multiple of 32
    if (qs >= total || n <= 0) return;
    // read containing qs: last r with off[r] <= qs (off[n] = total > qs)
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= qs) lo = mid; else hi = mid;
    }
    int64_t r = lo;
    int64_t next = off[r + 1] - qs;  // start of read r + 1, relative to qs
    JobPosCursor jc{jp};
    const uint64_t mask = (1ull << (2 * k)) - 1;
    const int rs = 2 * (k - 1);
    uint64_t fw = 0, rc = 0, pw = 0;
    int run = 0;  // ACGT bases ending here inside the current read
    uint32_t hb[4];
    const uint32_t *mine = smw + 9 * threadIdx.x;  // spad(8t + i) = 9t + i + (i >> 3)
    const int nb = KM_W + k - 1;                   // bases this thread reads
#pragma unroll
    for (int wi = 0; wi < (K > 0 ? (KM_W + K - 1 + 3) / 4 : (KM_W + 31 - 1 + 3) / 4); wi++) {
        const uint32_t word = mine[wi + (wi >> 3)];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int qi = 4 * wi + u;
            if (qi >= nb) break;
            // crossed into the next read (skips empty reads); r + 1 < n keeps every access in
            // bounds even when the offsets turn out to be invalid (reported after this pass)
            while (qi >= next && r + 1 < n) {
                r++;
                next = off[r + 1] - qs;
                run = 0;
            }
            const uint32_t c = (word >> (8 * u)) & 0xffu;
            const bool ok = (c == 'A') | (c == 'C') | (c == 'G') | (c == 'T');
            const uint32_t t = (c >> 1) & 3u;
            const uint32_t b = t ^ (t >> 1);  // A=0 C=1 G=2 T=3
            if (qi < KM_W) pw |= (uint64_t)b << (2 * qi);
            fw = ((fw << 2) | b) & mask;
            rc = (rc >> 2) | ((uint64_t)(3u - b) << rs);
            run = ok ? run + 1 : 0;  // bases past the end read as 'N'
            const int j = qi - (k - 1);
            if (j >= 0) {
                uint32_t h = H_NONE;
                if (run >= k) {
                    h = hash32(jc.prefix(qs + j) | (fw < rc ? fw : rc), B1_SEED);
                    h = h == H_NONE ? H_NONE - 1 : h;
                }
                if (K > 0) {  // j is a compile-time index: buffer 4 windows, one 16-byte store
                    hb[j & 3] = h;
                    if ((j & 3) == 3) *reinterpret_cast<uint4 *>(H + qs + j - 3) = make_uint4(hb[0], hb[1], hb[2], hb[3]);
                } else {
                    H[qs + j] = h;
                }
            }
        }
    }
    P[qs >> 5] = pw;
}

// Key of window q = 32g + lane from P[g] = w0 and P[g + 1] = w1 (a valid window): the canonical
// code (with the job prefix) | strand << 63. The 2k bits from
// bit 2 * lane of w1:w0 hold the window's bases, first base lowest; complementing them gives the
// reverse complement's code (last base's complement highest), and reversing the order of the
// 2-bit groups gives the forward code (first base highest).
__device__ __forceinline__ uint64_t window_key(uint64_t w0, uint64_t w1, int lane, int k, JobPosCursor &jc,
                                               int64_t q) {
    const int sh = 2 * lane;
    const uint64_t x = sh ? (w0 >> sh) | (w1 << (64 - sh)) : w0;
    const uint64_t rc = ~x & ((1ull << (2 * k)) - 1);  // k <= 31
    uint64_t y = __brevll(x);
    y = ((y >> 1) & 0x5555555555555555ull) | ((y & 0x5555555555555555ull) << 1);
    const uint64_t fw = y >> (64 - 2 * k);
    return jc.prefix(q) | (fw < rc ? fw : rc) | (rc < fw ? WC_STRAND : 0ull);
}

// One launch per slice [w_lo, w_hi) of B1's words: every launch streams all window hashes but
// only the k-mers whose B1 word lies in its slice touch the filter, so the slice stays in L2.
template <int BI_U>
__global__ void __launch_bounds__(KM_NT) bloom_insert_kernel(const uint32_t *__restrict__ H, int64_t nvec, Bloom b1,
                                                            Bloom b2, uint32_t w_lo, uint32_t w_hi) {
    // BI_U / 4 16-byte loads (4 windows each) per thread per step, coalesced across the warp and
    // all issued before any is used, so that BI_U atomics per thread are in flight together
    constexpr int NV = BI_U / 4;
    const int64_t stride = (int64_t)gridDim.x * KM_NT;
    const uint4 *H4 = reinterpret_cast<const uint4 *>(H);
    for (int64_t v0 = (int64_t)blockIdx.x * KM_NT + threadIdx.x; v0 < nvec; v0 += NV * stride) {
        uint32_t h[BI_U], i1[BI_U], m1[BI_U], old[BI_U];
        bool mine[BI_U];
#pragma unroll
        for (int u = 0; u < NV; u++) {
            const int64_t v = v0 + u * stride;
            const uint4 x = v < nvec ? __ldcs(H4 + v) : make_uint4(H_NONE, H_NONE, H_NONE, H_NONE);
            h[4 * u] = x.x;
            h[4 * u + 1] = x.y;
            h[4 * u + 2] = x.z;
            h[4 * u + 3] = x.w;
        }
#pragma unroll
        for (int u = 0; u < BI_U; u++) {
            b1.probe(h[u], &i1[u], &m1[u]);
            mine[u] = h[u] != H_NONE && i1[u] >= w_lo && i1[u] < w_hi;
        }
#pragma unroll
        for (int u = 0; u < BI_U; u++) old[u] = mine[u] ? atomicOr(b1.words + i1[u], m1[u]) : 0u;
#pragma unroll
        for (int u = 0; u < BI_U; u++) {
            if (mine[u] && (old[u] & m1[u]) == m1[u]) {
                uint32_t i2, m2;
                b2.probe(b2_hash(h[u]), &i2, &m2);
                if ((b2.words[i2] & m2) != m2) atomicOr(b2.words + i2, m2);
            }
        }
    }
}

// Binned Bloom insertion (when the filters split into at most BB_MAXBINS bins): B1 and B2 are cut
// into bins of w1b and w2b words; a key's bin is that of its B1 word (idx1 / w1b), and its B2 word
// lies in the same bin (bin * w2b + a word from its B2 hash). bin_scatter groups the window hashes
// by bin (order within a bin is arbitrary: insertion into a filter is order-free); bin_insert runs
// one block per bin with the bin's two slices in shared memory, so every filter update is a
// shared-memory atomic, and writes the B2 slice out. B1 itself is never stored.
struct BinnedBloom {
    uint32_t nbins = 0;  // 0: the sliced global-memory filters
    uint32_t w1b = 0, w2b = 0;  // powers of two
    uint32_t lw1b = 0;          // log2(w1b)
    uint32_t nwords1 = 0;       // nbins * w1b
    uint32_t cap = 0;      // hashes a bin can hold in the scatter buffer
};

constexpr int BB_MAXBINS = 1 << 20;  // one pass up to 4096 bins, two beyond
constexpr int BB_CSTRIDE = 32;  // bin cursors 128 bytes apart
constexpr int BI_NT = 1024;

__device__ __forceinline__ uint32_t bloom_mask(uint32_t h) {
    const uint32_t g = h * 0x85EBCA6Bu;
    return (1u << (g >> 27)) | (1u << ((g >> 22) & 31u)) | (1u << ((g >> 17) & 31u)) | (1u << ((g >> 12) & 31u));
}

// B2 word and bits of a key (B1 hash h1) in the binned layout
__device__ __forceinline__ void b2_binned(uint32_t h1, const BinnedBloom &bb, uint32_t *idx, uint32_t *mask) {
    const uint32_t h2 = b2_hash(h1);
    *idx = (__umulhi(h1, bb.nwords1) >> bb.lw1b) * bb.w2b + __umulhi(h2, bb.w2b);
    *mask = bloom_mask(h2);
}

// One pass of grouping hashes by bin. The source is flat (n hashes), or grouped by an earlier pass
// (group g: src + g * cap_src, min(fill[g], cap_src) hashes). A hash's bin within its group is
// (umulhi(h, nwords1) >> shift) - g * nb; it goes to output bin g * nb + that, whose room is
// cap_out. One pass (shift = log2 w1b) groups straight into filter bins; two passes first into
// superbins of nb filter bins, then each superbin into its bins, so that every pass has few
// enough bins per tile to write long runs.
struct ScatterLevel {
    const uint32_t *src;
    int64_t n;
    const uint32_t *fill;  // nullptr: flat source
    uint32_t cap_src;
    uint32_t tiles_per_group;
    uint32_t shift;
    uint32_t nb;
    uint32_t cap_out;
};

// One tile of NT * ITEMS hashes per block: count per bin, reserve each bin's run in its global
// buffer (one atomic per bin and tile, on a cursor of its own 128-byte line), order the tile by bin
// in shared memory, then write it out so that consecutive threads fill consecutive slots of a run.
template <int NT, int ITEMS>
__global__ void __launch_bounds__(NT, 1024 / NT) bloom_bin_scatter_kernel(ScatterLevel L, uint32_t nwords1,
                                                                         uint32_t *__restrict__ cursor,
                                                                         uint32_t *__restrict__ out,
                                                                         uint32_t *__restrict__ ovf) {
    constexpr int TILE = NT * ITEMS;
    extern __shared__ uint32_t bs_sm[];
    uint32_t *cnt = bs_sm;             // [nb] tile count per bin
    uint32_t *lofs = cnt + L.nb;       // [nb] the bin's first slot in the ordered tile
    uint32_t *gbase = lofs + L.nb;     // [nb] the bin's run in its global buffer
    uint32_t *tile = gbase + L.nb;     // [TILE] the tile ordered by bin
    __shared__ uint32_t s_tmp[NT / 32 + 1];
    const uint32_t g = L.fill ? blockIdx.x / L.tiles_per_group : 0u;
    const int64_t t0 = (int64_t)(L.fill ? blockIdx.x % L.tiles_per_group : blockIdx.x) * TILE;
    const uint32_t *src = L.fill ? L.src + (int64_t)g * L.cap_src : L.src;
    int64_t n = L.n;
    if (L.fill) {
        const uint32_t f = L.fill[(size_t)g * BB_CSTRIDE];
        n = f < L.cap_src ? f : L.cap_src;
    }
    if (t0 >= n) return;  // the whole block: past its group's hashes
    const uint32_t gb0 = g * L.nb;
    for (uint32_t b = threadIdx.x; b < L.nb; b += NT) cnt[b] = 0u;
    __syncthreads();
    uint32_t h[ITEMS], rk[ITEMS];
#pragma unroll
    for (int u = 0; u < ITEMS; u++) {
        const int64_t q = t0 + u * NT + threadIdx.x;
        h[u] = q < n ? __ldcs(src + q) : H_NONE;
        rk[u] = h[u] != H_NONE ? atomicAdd(cnt + ((__umulhi(h[u], nwords1) >> L.shift) - gb0), 1u) : 0u;
    }
    __syncthreads();
    // thread t owns bins [t * per, t * per + per): their prefix, and their global runs
    const uint32_t per = (L.nb + NT - 1) / NT;
    const uint32_t b0 = threadIdx.x * per;
    uint32_t mine = 0;
    for (uint32_t b = b0; b < b0 + per && b < L.nb; b++) mine += cnt[b];
    uint32_t ntot;
    uint32_t run = block_exclusive_scan<NT>(mine, s_tmp, &ntot);
    for (uint32_t b = b0; b < b0 + per && b < L.nb; b++) {
        const uint32_t c = cnt[b];
        lofs[b] = run;
        run += c;
        gbase[b] = c ? atomicAdd(cursor + (size_t)(gb0 + b) * BB_CSTRIDE, c) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < ITEMS; u++)
        if (h[u] != H_NONE) tile[lofs[(__umulhi(h[u], nwords1) >> L.shift) - gb0] + rk[u]] = h[u];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < ntot; i += NT) {
        const uint32_t hv = tile[i];
        const uint32_t b = (__umulhi(hv, nwords1) >> L.shift) - gb0;
        const uint32_t pos = gbase[b] + (i - lofs[b]);
        if (pos < L.cap_out) out[(int64_t)(gb0 + b) * L.cap_out + pos] = hv;
        else *ovf = 1u;  // the bin is fuller than its room: the caller redoes the filters sliced
    }
}

__global__ void __launch_bounds__(BI_NT) bloom_bin_insert_kernel(const uint32_t *__restrict__ Hb,
                                                                const uint32_t *__restrict__ cursor, BinnedBloom bb,
                                                                uint32_t *__restrict__ b2words) {
    extern __shared__ uint32_t bi_sm[];
    uint32_t *s1 = bi_sm, *s2 = bi_sm + bb.w1b;
    const uint32_t bin = blockIdx.x;
    for (uint32_t x = threadIdx.x; x < bb.w1b + bb.w2b; x += BI_NT) bi_sm[x] = 0u;
    __syncthreads();
    const uint32_t fill = cursor[(size_t)bin * BB_CSTRIDE];
    const uint32_t c = fill < bb.cap ? fill : bb.cap;
    const uint32_t *hb = Hb + (int64_t)bin * bb.cap;
    const uint32_t lo1 = bin * bb.w1b;
    constexpr int U = 4;  // loads in flight per thread
    for (uint32_t i0 = threadIdx.x; i0 < c; i0 += U * BI_NT) {
        uint32_t h[U];
#pragma unroll
        for (int u = 0; u < U; u++) h[u] = i0 + u * BI_NT < c ? __ldcs(hb + i0 + u * BI_NT) : H_NONE;
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (h[u] == H_NONE) continue;
            const uint32_t w1 = __umulhi(h[u], bb.nwords1) - lo1;  // < w1b: the bin is that of the word
            const uint32_t m1 = bloom_mask(h[u]);
            if ((atomicOr(s1 + w1, m1) & m1) == m1) {
                const uint32_t h2 = b2_hash(h[u]);
                const uint32_t w2 = __umulhi(h2, bb.w2b), m2 = bloom_mask(h2);
                if ((s2[w2] & m2) != m2) atomicOr(s2 + w2, m2);
            }
        }
    }
    __syncthreads();
    uint32_t *out = b2words + (int64_t)bin * bb.w2b;
    for (uint32_t x = threadIdx.x; x < bb.w2b; x += BI_NT) out[x] = s2[x];
}

// Candidates: windows whose code tests positive in B2 (every occurrence of a k-mer seen at least
// twice; false positives only add singletons, which the exact count drops). use_bloom == 0 keeps
// every window (lo == 1: singletons may be reliable).
//
// Both passes are warp-cooperative: warp w of block b owns the KM_GW groups of 32 consecutive
// windows starting at group (b * KM_WARPS + w) * KM_GW, and handles one group (lane l: window
// 32g + l, from the group's two packed words) per step. The count pass stores each group's
// candidate ballot in cmask and the warp's total in wcnt; the emit pass writes each group's
// candidates contiguously at the scanned offset, so candidates keep position order.
constexpr int KM_GW = KM_CHUNK / KM_NT;  // groups per warp (32: one mask word per lane)
static_assert(KM_GW == 32, "one mask word per lane");

__device__ __forceinline__ bool is_candidate(uint32_t h, const Bloom &b2, int use_bloom, const BinnedBloom &bb) {
    if (h == H_NONE) return false;
    if (!use_bloom) return true;
    uint32_t i2, m2;
    if (bb.nbins)
        b2_binned(h, bb, &i2, &m2);
    else
        b2.probe(b2_hash(h), &i2, &m2);
    return (b2.words[i2] & m2) == m2;
}

// Candidate buckets by the top bits of the code (PK_POS with nb > 1): the candidates of bucket b
// go to one contiguous range, in position order, so that each range is sorted on the code's low
// `shift` bits only -- fewer radix passes, and on large inputs an 8-byte key where the whole code
// and position would need 16 bytes. wcnt / wpos are bucket-major: [b * nwarp + warp].
struct Buckets {
    const uint64_t *P;
    int k;
    JobPos jp;
    int nb;     // 1: no buckets
    int shift;  // code bits below the bucket bits
    uint64_t kmask;
    int64_t nwarp;
};

__device__ __forceinline__ uint32_t bucket_of(const Buckets &bk, uint64_t x) {
    return (uint32_t)((x & bk.kmask) >> bk.shift);
}

template <bool BKT>
__global__ void __launch_bounds__(KM_NT) cand_count_kernel(const uint32_t *__restrict__ H, int64_t nwin, Bloom b2,
                                                          int use_bloom, BinnedBloom bb, Buckets bk,
                                                          uint32_t *__restrict__ cmask, uint32_t *__restrict__ wcnt) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warp = (int64_t)blockIdx.x * KM_WARPS + w;
    const int64_t g0 = warp * KM_GW;
    JobPosCursor jc{bk.jp};
    uint32_t mine = 0, c = 0, cb = 0;  // cb: lane b's count of bucket b
    constexpr int CC_U = 8;  // groups whose hashes (and then filter words) are loaded together
    for (int g0u = 0; g0u < KM_GW; g0u += CC_U) {
        uint32_t h[CC_U];
#pragma unroll
        for (int u = 0; u < CC_U; u++) {
            const int64_t q = (g0 + g0u + u) * 32 + lane;
            h[u] = q < nwin ? __ldcs(H + q) : H_NONE;
        }
#pragma unroll
        for (int u = 0; u < CC_U; u++) {
            const uint32_t m = __ballot_sync(0xffffffffu, is_candidate(h[u], b2, use_bloom, bb));
            if (lane == g0u + u) mine = m;
            c += __popc(m);
            if (BKT && m) {  // lane j < nb counts the candidates of bucket j, one ballot per bucket bit
                const int64_t g = g0 + g0u + u;
                const bool cand = (m >> lane) & 1u;
                const uint32_t b = cand ? bucket_of(bk, window_key(bk.P[g], bk.P[g + 1], lane, bk.k, jc, g * 32 + lane))
                                        : 0u;
                uint32_t own = m;
                for (int t = 0; (1 << t) < bk.nb; t++) {
                    const uint32_t bt = __ballot_sync(0xffffffffu, cand && ((b >> t) & 1u));
                    own &= ((lane >> t) & 1) ? bt : ~bt;
                }
                if (lane < bk.nb) cb += __popc(own);
            }
        }
    }
    cmask[g0 + lane] = mine;
    if (BKT) {
        if (lane < bk.nb) wcnt[(int64_t)lane * bk.nwarp + warp] = cb;
    } else if (lane == 0) {
        wcnt[warp] = c;
    }
}

// Sort records of the candidates. The code (job prefix included) is the sort key; below it:
//   PK_POS   key = code << pb | q << 1 | strand  (pb = bits of q + 1): the window itself rides in the
//            key, nothing else is written and no gather follows the sort;
//   PK_IDX   key = code << pb | candidate index, vals = q | strand << 63, gathered after the sort;
//   PK_PAIRS key = code, vals = q | strand << 63, sorted as pairs (nothing fits in 64 bits).
enum : int { PK_POS = 0, PK_IDX = 1, PK_PAIRS = 2 };

template <bool BKT>
__global__ void __launch_bounds__(KM_NT) cand_emit_kernel(Buckets bk, const uint32_t *__restrict__ cmask,
                                                         const int64_t *__restrict__ wpos, int mode, int pb,
                                                         uint64_t *__restrict__ keys, uint64_t *__restrict__ vals,
                                                         int64_t nc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warp = (int64_t)blockIdx.x * KM_WARPS + w;
    const int64_t g0 = warp * KM_GW;
    JobPosCursor jc{bk.jp};
    const uint32_t mine = cmask[g0 + lane];
    const uint32_t below = (1u << lane) - 1u;
    const uint64_t lowmask = bk.shift < 64 ? (1ull << bk.shift) - 1 : ~0ull;
    // next free slot: of the warp (one bucket), or of bucket `lane` (lane < nb)
    int64_t o = BKT ? (lane < bk.nb ? wpos[(int64_t)lane * bk.nwarp + warp] : 0) : wpos[warp];
    for (int g = 0; g < KM_GW; g++) {
        const uint32_t m = __shfl_sync(0xffffffffu, mine, g);
        if (m == 0) continue;  // no candidate: also every group past the sequence
        const bool cand = (m >> lane) & 1u;
        if (!BKT) {  // one bucket: the candidates of a group go out in lane order
            if (cand) {
                const int64_t q = (g0 + g) * 32 + lane;
                const uint64_t x = window_key(bk.P[g0 + g], bk.P[g0 + g + 1], lane, bk.k, jc, q);
                const int64_t p = o + __popc(m & below);
                if (SG_IN_BOUNDS(p >= 0 && p < nc, 102, p)) {
                    const uint64_t code = x & bk.kmask;
                    if (mode == PK_POS) {
                        keys[p] = ((code & lowmask) << pb) | ((uint64_t)q << 1) | (x >> 63);
                    } else {
                        keys[p] = mode == PK_IDX ? ((code << pb) | (uint64_t)p) : code;
                        vals[p] = (uint64_t)q | (x & WC_STRAND);
                    }
                }
            }
            o += __popc(m);
            continue;
        }
        const int64_t q = (g0 + g) * 32 + lane;
        const uint64_t x = cand ? window_key(bk.P[g0 + g], bk.P[g0 + g + 1], lane, bk.k, jc, q) : 0ull;
        int64_t p;
        {
            // peers (the lanes of this lane's bucket) and own (the lanes of bucket `lane`, for
            // lane < nb) from one ballot per bucket bit; this lane's slot follows the base of its
            // bucket (held by lane b) and the lanes below it in the bucket
            const uint32_t b = cand ? bucket_of(bk, x) : 0u;
            uint32_t peers = m, own = m;
            for (int t = 0; (1 << t) < bk.nb; t++) {
                const uint32_t bt = __ballot_sync(0xffffffffu, cand && ((b >> t) & 1u));
                peers &= ((b >> t) & 1u) ? bt : ~bt;
                own &= ((lane >> t) & 1) ? bt : ~bt;
            }
            p = __shfl_sync(0xffffffffu, o, (int)b) + __popc(peers & below);
            if (lane < bk.nb) o += __popc(own);
        }
        if (cand && SG_IN_BOUNDS(p >= 0 && p < nc, 102, p))  // buckets: always PK_POS
            keys[p] = (((x & bk.kmask) & lowmask) << pb) | ((uint64_t)q << 1) | (x >> 63);
    }
}

// Read lookup: lut[b] = the read containing base b << LUT_SHIFT (the last r with off[r] <= it), so
// that finding a position's read is a binary search over the few reads of one bucket.
constexpr int LUT_SHIFT = 12;

__global__ void read_lut_kernel(const int64_t *__restrict__ off, int64_t n, int64_t nb, int32_t *__restrict__ lut) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int64_t q = b << LUT_SHIFT;
    int64_t lo = 0, hi = n;  // last read r with off[r] <= q
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= q) lo = mid; else hi = mid;
    }
    lut[b] = (int32_t)lo;
}

// v = q | strand << 63  ->  read << 32 | pos | strand << 31
__device__ __forceinline__ uint64_t resolve_pos(uint64_t v, const int64_t *__restrict__ off, int64_t n,
                                                const int32_t *__restrict__ lut, int64_t nb) {
    const int64_t q = (int64_t)(v & ~WC_STRAND);
    const int64_t b = q >> LUT_SHIFT;
    int64_t lo = lut[b], hi = b + 1 < nb ? (int64_t)lut[b + 1] + 1 : n;  // the read lies in [lo, hi)
    if (hi > n) hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= q) lo = mid; else hi = mid;
    }
    return ((uint64_t)lo << 32) | (uint64_t)(uint32_t)(q - off[lo]) | ((v >> 63) << 31);
}

// Bucket ranges of the candidate keys: bucket b holds [start[b], start[b + 1]).
struct BucketStarts {
    int64_t start[9];
    int nb;
    int shift;
};

// After a keys-only sort (PK_POS, PK_IDX): the code, and the window resolved to its read.
__global__ void unpack_kernel(const uint64_t *__restrict__ packed, const uint64_t *__restrict__ vals, int64_t nc,
                              int mode, int pb, BucketStarts bs, const int64_t *__restrict__ off, int64_t n,
                              const int32_t *__restrict__ lut, int64_t nb, uint64_t *__restrict__ key,
                              uint64_t *__restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const uint64_t p = packed[i];
    const uint64_t low = p & ((1ull << pb) - 1);
    uint64_t b = 0;  // the bucket's bits above the sorted code bits
#pragma unroll
    for (int j = 1; j < 8; j++)  // constant indices: the ranges stay in parameter space
        if (j < bs.nb) b += (uint64_t)(i >= bs.start[j]);
    key[i] = (b << bs.shift) | (p >> pb);
    if (mode == PK_POS) {
        val[i] = resolve_pos((low >> 1) | (low << 63), off, n, lut, nb);
    } else if (SG_IN_BOUNDS((int64_t)low < nc, 103, low)) {
        val[i] = resolve_pos(vals[low], off, n, lut, nb);
    }
}

// After the pairs sort: val = q | strand << 63  ->  read << 32 | pos | strand << 31.
__global__ void resolve_kernel(uint64_t *__restrict__ val, int64_t nc, const int64_t *__restrict__ off, int64_t n,
                               const int32_t *__restrict__ lut, int64_t nb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    val[i] = resolve_pos(val[i], off, n, lut, nb);
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

// Fused segment pass (used when every reliable range has hi <= SEG_WALK_MAX): each position walks
// its run of equal keys at most hmax + 1 steps each way. A run that is still equal after that is
// longer than any hi, hence unreliable; otherwise the walks give its exact length. Output per
// position: headrel (it heads a reliable segment) | keep (it lies in a reliable segment and is the
// first entry of its read there) << 31, so that one scan yields both the column ids and the
// positions in At.
constexpr int SEG_WALK_MAX = 64;
constexpr int PK_SHIFT = 31;

// nkeep receives the number of kept entries (nnz), which must stay below 2^31 for the packed
// scan.
__global__ void seg_flags_kernel(const uint64_t *__restrict__ key, const uint64_t *__restrict__ val, int64_t nc,
                                 uint32_t lo, uint32_t hi, const uint32_t *__restrict__ lohi, int kbits, int hmax,
                                 uint64_t *__restrict__ packed, unsigned long long *__restrict__ nkeep) {
    __shared__ unsigned int s_kept;
    if (threadIdx.x == 0) s_kept = 0u;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool kept = false;
    if (i < nc) {
        const uint64_t k = key[i];
        int64_t h = i, e = i + 1;
        int back = 0, fwd = 0;
        while (back <= hmax && h > 0 && key[h - 1] == k) {
            h--;
            back++;
        }
        while (fwd <= hmax && e < nc && key[e] == k) {
            e++;
            fwd++;
        }
        uint32_t lo_i = lo, hi_i = hi;
        if (lohi) {
            const uint64_t job = k >> kbits;
            lo_i = lohi[2 * job];
            hi_i = lohi[2 * job + 1];
        }
        const int64_t len = e - h;
        const bool rel = back <= hmax && fwd <= hmax && len >= (int64_t)lo_i && len <= (int64_t)hi_i;
        const bool head = h == i;
        const bool first = head || (val[i] >> 32) != (val[i - 1] >> 32);
        packed[i] = (uint64_t)(rel && head) | ((uint64_t)(rel && first) << PK_SHIFT);
        kept = rel && first;
    }
    const unsigned m = __ballot_sync(0xffffffffu, kept);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&s_kept, (unsigned)__popc(m));
    __syncthreads();
    if (threadIdx.x == 0 && s_kept) atomicAdd(nkeep, (unsigned long long)s_kept);
}

// Writes At's entries, its row pointers, the column codes and the (read, col|val) pairs sorted
// into A, from the exclusive scan of the fused flags (low 31 bits: reliable segments before, high
// bits: kept entries before; pre[nc] = the totals). Entry i's own flags are pre[i + 1] - pre[i].
__global__ void emit_fused_kernel(const uint64_t *__restrict__ pre,
                                  const uint64_t *__restrict__ key, const uint64_t *__restrict__ val, int64_t nc,
                                  int64_t m, int64_t nnz, int32_t *__restrict__ at_col, uint32_t *__restrict__ at_val,
                                  int64_t *__restrict__ at_rp, uint64_t *__restrict__ codes,
                                  uint32_t *__restrict__ a_key, uint64_t *__restrict__ a_val, int kbits,
                                  unsigned long long *__restrict__ job_ncols) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) at_rp[m] = nnz;
    if (i >= nc) return;
    const uint64_t x = pre[i];
    const uint64_t f = pre[i + 1] - x;
    if (f == 0) return;
    const uint64_t lowmask = (1ull << PK_SHIFT) - 1;
    const int64_t before = (int64_t)(x & lowmask), o = (int64_t)(x >> PK_SHIFT);
    const int64_t col = before + (int64_t)(f & 1) - 1;  // the segment's column (its head counted)
    if (!SG_IN_BOUNDS(col >= 0 && col < m, 108, col)) return;
    if (f & 1) {
        at_rp[col] = o;
        codes[col] = kbits < 64 ? key[i] & ((1ull << kbits) - 1) : key[i];
        if (job_ncols) atomicAdd(job_ncols + (key[i] >> kbits), 1ull);
    }
    if (f >> PK_SHIFT) {
        if (!SG_IN_BOUNDS(o >= 0 && o < nnz, 109, o)) return;
        const uint32_t r = (uint32_t)(val[i] >> 32), v = (uint32_t)val[i];
        at_col[o] = (int32_t)r;
        at_val[o] = v;
        a_key[o] = r;
        a_val[o] = ((uint64_t)col << 32) | v;
    }
}

// Segments straight from the sorted keys of the PK_POS form, in two passes over tiles of
// DS_TILE sorted candidates (DS_ITEMS consecutive ones per thread), with no unpacked key/value
// arrays and no per-candidate prefix array:
//   mark: each tile stages its keys (and DS_HALO neighbours on each side) in shared memory, walks
//         each candidate's run of equal keys there (as seg_flags_kernel does), and stores two bits
//         per candidate -- heads a reliable segment | kept (first of its read in a reliable
//         segment) << 1 -- and the tile's two totals;
//   emit: after exclusive scans of the tile totals, each tile recovers every candidate's column
//         and At slot from its tile's prefixes and a block scan of its flags, and writes At, the
//         codes and the pairs sorted into A (emit_fused_kernel's outputs).
// Keys are equal when they lie in the same bucket range and agree in their code bits. "First of
// its read" tests whether the previous candidate's window lies in the extent [off[r], off[r + 1])
// of the read r holding this one; the reads are found by searches that run for DS_GROUP
// candidates at once, so that their loads overlap.
constexpr int DS_NT = 256;
constexpr int DS_ITEMS = 16;
constexpr int DS_TILE = DS_NT * DS_ITEMS;
constexpr int DS_HALO = SEG_WALK_MAX + 16;  // a walk reads at most SEG_WALK_MAX + 1 neighbours
constexpr int DS_GROUP = 2;  // 2: 20.6 / 34.8 ms for mark / emit, 4: 26.2 / 37.9 ms (registers, occupancy)
// Staged keys are padded by one slot every 16, so that the 32 lanes of a warp, reading 8-byte
// keys DS_ITEMS apart, hit distinct banks.
__device__ __forceinline__ int ds_pad(int j) { return j + (j >> 4); }
constexpr int DS_SMEM = DS_TILE + 2 * DS_HALO + (DS_TILE + 2 * DS_HALO) / 16 + 1;

// The bucket holding sorted index i, and the bucket's index range [s0, s1).
__device__ __forceinline__ uint64_t bucket_range(const BucketStarts &bs, int64_t i, int64_t nc, int64_t &s0,
                                                 int64_t &s1) {
    uint64_t b = 0;
    s0 = 0;
    s1 = nc;
#pragma unroll
    for (int j = 1; j < 8; j++)  // constant indices: the ranges stay in parameter space
        if (j < bs.nb) {
            const int64_t st = bs.start[j];
            if (i >= st) {
                b++;
                s0 = st;
            } else if (st < s1) {
                s1 = st;
            }
        }
    return b;
}

// r[u] = the read holding window q[u] (the last r with off[r] <= q[u]) for the active u, found
// together: every step issues the loads of all unfinished searches before using any.
template <int G>
__device__ __forceinline__ void reads_of(const int64_t (&q)[G], const bool (&act)[G], int64_t (&r)[G],
                                         const int64_t *__restrict__ off, int64_t n,
                                         const int32_t *__restrict__ lut, int64_t nb) {
    int64_t lo[G], hi[G];
#pragma unroll
    for (int u = 0; u < G; u++) {
        lo[u] = 0;
        hi[u] = 1;
        if (act[u]) {
            const int64_t b = q[u] >> LUT_SHIFT;
            lo[u] = lut[b];
            hi[u] = b + 1 < nb ? (int64_t)lut[b + 1] + 1 : n;  // the read lies in [lo, hi)
            if (hi[u] > n) hi[u] = n;
        }
    }
    for (;;) {
        bool any = false;
        int64_t mid[G], om[G];
#pragma unroll
        for (int u = 0; u < G; u++) {
            mid[u] = (lo[u] + hi[u]) >> 1;
            if (hi[u] - lo[u] > 1) {
                om[u] = off[mid[u]];
                any = true;
            }
        }
        if (!any) break;
#pragma unroll
        for (int u = 0; u < G; u++)
            if (hi[u] - lo[u] > 1) {
                if (om[u] <= q[u]) lo[u] = mid[u]; else hi[u] = mid[u];
            }
    }
#pragma unroll
    for (int u = 0; u < G; u++) r[u] = lo[u];
}

// Stages sorted keys [base - DS_HALO, base + DS_TILE + DS_HALO) in sk, key base - DS_HALO + j at
// sk[ds_pad(j)] (0 outside [0, nc)).
__device__ __forceinline__ void stage_keys(uint64_t *sk, const uint64_t *__restrict__ packed, int64_t base,
                                           int64_t nc) {
    for (int j = threadIdx.x; j < DS_TILE + 2 * DS_HALO; j += DS_NT) {
        const int64_t g = base - DS_HALO + j;
        sk[ds_pad(j)] = (g >= 0 && g < nc) ? __ldg(packed + g) : 0ull;
    }
}

struct SegArgs {
    const uint64_t *packed;
    int64_t nc;
    int pb;
    BucketStarts bs;
    uint32_t lo, hi;
    const uint32_t *lohi;
    int kbits;
    int hmax;
    const int64_t *off;
    int64_t n;
    const int32_t *lut;
    int64_t nb;
};

__global__ void __launch_bounds__(DS_NT) seg_mark_kernel(SegArgs a, uint32_t *__restrict__ flags,
                                                        uint32_t *__restrict__ tseg, uint32_t *__restrict__ tkeep) {
    __shared__ uint64_t sk[DS_SMEM];
    __shared__ uint32_t red[2][DS_NT / 32];
    const int64_t tile = blockIdx.x, base = tile * DS_TILE;
    stage_keys(sk, a.packed, base, a.nc);
    __syncthreads();
    // indices below are local: candidate base - DS_HALO + x is staged at sk[ds_pad(x)]
    const int l0 = DS_HALO + threadIdx.x * DS_ITEMS;
    const int64_t g0 = base - DS_HALO;
    const int64_t lrest = a.nc - g0;
    const int lend = lrest < (int64_t)(l0 + DS_ITEMS) ? (int)lrest : l0 + DS_ITEMS;  // past this thread's last item
    const uint64_t lowmask = (1ull << a.pb) - 1, codemask = ~lowmask;
    uint32_t fw = 0, need = 0;
    // the bucket range [b0, b1) of the current item, clipped to the staged keys
    int b0 = 0, b1 = 0;
    uint64_t bkt = 0;
    // the run of equal keys [rh, re) holding the last walked item, and whether it is a reliable
    // segment; the items after it inside the run share both (a run cut short by the walk bound is
    // longer than any hi, hence unreliable for all of its items)
    int rh = 0, re = 0;
    bool rrel = false;
#pragma unroll 1
    for (int li = l0; li < lend; li++) {
        if (li >= re) {
            if (li >= b1) {
                int64_t s0, s1;
                bkt = bucket_range(a.bs, g0 + li, a.nc, s0, s1);
                b0 = s0 - g0 > 0 ? (int)(s0 - g0) : 0;
                b1 = s1 - g0 < (int64_t)(DS_TILE + 2 * DS_HALO) ? (int)(s1 - g0) : DS_TILE + 2 * DS_HALO;
            }
            const uint64_t key = sk[ds_pad(li)];
            int h = li, e = li + 1;
            while (li - h <= a.hmax && h > b0 && ((sk[ds_pad(h - 1)] ^ key) & codemask) == 0) h--;
            while (e - li - 1 <= a.hmax && e < b1 && ((sk[ds_pad(e)] ^ key) & codemask) == 0) e++;
            uint32_t lo_i = a.lo, hi_i = a.hi;
            if (a.lohi) {
                const uint64_t job = ((bkt << a.bs.shift) | (key >> a.pb)) >> a.kbits;
                lo_i = a.lohi[2 * job];
                hi_i = a.lohi[2 * job + 1];
            }
            const int len = e - h;
            rrel = li - h <= a.hmax && e - li - 1 <= a.hmax && len >= (int)lo_i && (uint32_t)len <= hi_i;
            rh = h;
            re = e;
        }
        const int u = li - l0;
        if (rrel && rh == li) fw |= 3u << (2 * u);  // heads its segment: first of its read too
        else if (rrel) need |= 1u << u;            // kept if the previous window is of another read
    }
    // the previous window qp < q (position order within a segment) lies in another read when a
    // read starts in (qp, q]: decided from the read table alone when the read holding q's bucket
    // start comes after the read holding the start of the bucket after qp's; else searched
#pragma unroll 1
    for (int u0 = 0; u0 < DS_ITEMS; u0 += DS_GROUP) {
        if (((need >> u0) & ((1u << DS_GROUP) - 1)) == 0) continue;
        int64_t q[DS_GROUP], qp[DS_GROUP], r[DS_GROUP];
        bool act[DS_GROUP];
#pragma unroll
        for (int u = 0; u < DS_GROUP; u++) {
            act[u] = (need >> (u0 + u)) & 1u;
            q[u] = (int64_t)((sk[ds_pad(l0 + u0 + u)] & lowmask) >> 1);
            qp[u] = (int64_t)((sk[ds_pad(l0 + u0 + u - 1)] & lowmask) >> 1);
            if (act[u]) {
                const int64_t bq = q[u] >> LUT_SHIFT, bp = (qp[u] >> LUT_SHIFT) + 1;
                if (bp < a.nb && bq >= bp && a.lut[bq] > a.lut[bp]) {
                    act[u] = false;
                    fw |= 2u << (2 * (u0 + u));
                }
            }
        }
        reads_of<DS_GROUP>(q, act, r, a.off, a.n, a.lut, a.nb);
#pragma unroll
        for (int u = 0; u < DS_GROUP; u++)
            if (act[u] && !(qp[u] >= a.off[r[u]] && qp[u] < a.off[r[u] + 1])) fw |= 2u << (2 * (u0 + u));
    }
    flags[tile * DS_NT + threadIdx.x] = fw;
    uint32_t ns = __popc(fw & 0x55555555u), nk = __popc(fw & 0xAAAAAAAAu);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ns += __shfl_xor_sync(0xffffffffu, ns, o);
        nk += __shfl_xor_sync(0xffffffffu, nk, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = ns;
        red[1][threadIdx.x >> 5] = nk;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ts = 0, tk = 0;
        for (int w = 0; w < DS_NT / 32; w++) {
            ts += red[0][w];
            tk += red[1][w];
        }
        tseg[tile] = ts;
        tkeep[tile] = tk;
    }
}

// pseg / pkeep: exclusive prefixes of the tile totals (reliable segments, kept entries). The
// tile's candidates are taken in DS_ITEMS rows of DS_NT (candidate base + row * DS_NT + thread),
// so that a warp's outputs of one row are consecutive; a candidate's column and At slot are its
// tile's prefix plus the counts of the rows before it and of the lanes before it (ballots).
__global__ void __launch_bounds__(DS_NT, 4) seg_emit_kernel(SegArgs a, const uint32_t *__restrict__ flags,
                                                        const int64_t *__restrict__ pseg,
                                                        const int64_t *__restrict__ pkeep, int64_t m, int64_t nnz,
                                                        int32_t *__restrict__ at_col, uint32_t *__restrict__ at_val,
                                                        int64_t *__restrict__ at_rp, uint64_t *__restrict__ codes,
                                                        uint32_t *__restrict__ a_key, uint64_t *__restrict__ a_val,
                                                        unsigned long long *__restrict__ job_ncols) {
    constexpr int NW = DS_NT / 32;
    __shared__ uint64_t sk[DS_SMEM];
    __shared__ uint32_t sf[DS_NT];                       // the tile's flag words (DS_ITEMS candidates each)
    __shared__ uint32_t hmask[DS_ITEMS][NW], kmask[DS_ITEMS][NW];  // per row and warp: heads, kept
    __shared__ uint32_t hpre[DS_ITEMS * NW], kpre[DS_ITEMS * NW];  // their exclusive prefixes in the tile
    const int64_t tile = blockIdx.x, base = tile * DS_TILE;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (tile == 0 && threadIdx.x == 0) at_rp[m] = nnz;
    stage_keys(sk, a.packed, base, a.nc);
    sf[threadIdx.x] = flags[tile * DS_NT + threadIdx.x];
    __syncthreads();
    auto flag_of = [&](int j) { return (sf[j >> 4] >> (2 * (j & 15))) & 3u; };  // candidate base + j
#pragma unroll
    for (int u = 0; u < DS_ITEMS; u++) {
        const uint32_t f = flag_of(u * DS_NT + threadIdx.x);
        const uint32_t hb = __ballot_sync(0xffffffffu, f & 1u), kb = __ballot_sync(0xffffffffu, f & 2u);
        if (lane == 0) {
            hmask[u][w] = hb;
            kmask[u][w] = kb;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scans of the DS_ITEMS * NW counts, row-major
        constexpr int PER = DS_ITEMS * NW / 32;
        uint32_t hc[PER], kc[PER], hs = 0, ks = 0;
#pragma unroll
        for (int x = 0; x < PER; x++) {
            const int idx = lane * PER + x;
            hc[x] = __popc(hmask[idx / NW][idx % NW]);
            kc[x] = __popc(kmask[idx / NW][idx % NW]);
            hs += hc[x];
            ks += kc[x];
        }
        uint32_t hi = hs, ki = ks;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t hy = __shfl_up_sync(0xffffffffu, hi, o), ky = __shfl_up_sync(0xffffffffu, ki, o);
            if (lane >= o) {
                hi += hy;
                ki += ky;
            }
        }
        uint32_t hr = hi - hs, kr = ki - ks;
#pragma unroll
        for (int x = 0; x < PER; x++) {
            hpre[lane * PER + x] = hr;
            kpre[lane * PER + x] = kr;
            hr += hc[x];
            kr += kc[x];
        }
    }
    __syncthreads();
    const int64_t seg0 = pseg[tile], keep0 = pkeep[tile];
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t lowmask = (1ull << a.pb) - 1;
    int64_t s0 = 0, s1 = 0;  // the bucket range of the last head, and its bucket
    uint64_t bkt = 0;
#pragma unroll 1
    for (int u0 = 0; u0 < DS_ITEMS; u0 += DS_GROUP) {
        int64_t q[DS_GROUP], r[DS_GROUP];
        bool act[DS_GROUP];
        bool any = false;
#pragma unroll
        for (int u = 0; u < DS_GROUP; u++) {
            const int j = (u0 + u) * DS_NT + threadIdx.x;
            act[u] = (flag_of(j) & 2u) != 0;
            any |= act[u];
            q[u] = (int64_t)((sk[ds_pad(DS_HALO + j)] & lowmask) >> 1);
        }
        if (any) reads_of<DS_GROUP>(q, act, r, a.off, a.n, a.lut, a.nb);
#pragma unroll
        for (int u = 0; u < DS_GROUP; u++) {
            const int row = u0 + u, j = row * DS_NT + threadIdx.x;
            const uint32_t f = flag_of(j);
            if (!f) continue;
            const int64_t i = base + j;
            const uint64_t p = sk[ds_pad(DS_HALO + j)];
            // heads up to and including this candidate: its segment's column is that count - 1
            const int64_t segs = seg0 + hpre[row * NW + w] + __popc(hmask[row][w] & lt) + (f & 1u);
            const int64_t col = segs - 1;
            const int64_t o = keep0 + kpre[row * NW + w] + __popc(kmask[row][w] & lt);
            if (!SG_IN_BOUNDS(col >= 0 && col < m, 110, col)) continue;
            if (f & 1u) {
                if (i < s0 || i >= s1) bkt = bucket_range(a.bs, i, a.nc, s0, s1);
                const uint64_t key = (bkt << a.bs.shift) | (p >> a.pb);
                at_rp[col] = o;
                codes[col] = a.kbits < 64 ? key & ((1ull << a.kbits) - 1) : key;
                if (job_ncols) atomicAdd(job_ncols + (key >> a.kbits), 1ull);
            }
            if (f & 2u) {
                if (!SG_IN_BOUNDS(o >= 0 && o < nnz, 111, o)) continue;
                const uint32_t rr = (uint32_t)r[u];
                const uint32_t v = (uint32_t)(q[u] - a.off[r[u]]) | (uint32_t)((p & 1u) << 31);
                at_col[o] = (int32_t)rr;
                at_val[o] = v;
                a_key[o] = rr;
                a_val[o] = ((uint64_t)col << 32) | v;
            }
        }
    }
}

// Row pointers of A from the read ids of its entries, sorted ascending.
__global__ void rowptr_from_sorted_kernel(const uint32_t *__restrict__ rows, int64_t nnz, int64_t n,
                                          int64_t *__restrict__ rp) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > nnz) return;
    int64_t prev = (e == 0) ? -1 : (int64_t)rows[e - 1];
    int64_t cur = (e == nnz) ? n : (int64_t)rows[e];
    // always in bounds, even for rows that a failed sort left unsorted (the call then fails)
    if (!SG_IN_BOUNDS(prev >= -1 && cur <= n && prev <= cur, 107, cur) || prev < -1 || cur > n) return;
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
                     unsigned long long *job_ncols, uint32_t hmax) {
    const int NT = 256;
    uint32_t *err = sc.get<uint32_t>(1);
    if (!err) return SG_ERR_OOM;
    SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    SG_LAUNCH("validate_offsets", validate_offsets_kernel, blocks_for(n + 1, NT), NT, 0, s, off, n, total, err);

    const int64_t nblk = blocks_for(total, KM_CHUNK);
    const int use_bloom = lo >= 2 ? 1 : 0;
    int job_bits = 0;
    while (jm.ro && ((int64_t)1 << job_bits) < jm.njobs) job_bits++;
    const int code_bits = 2 * k + job_bits;
    const uint64_t kmask = (1ull << code_bits) - 1;  // code_bits <= 62
    Bloom b1{nullptr, 0}, b2{nullptr, 0};
    // packed bases, filters and candidate masks: released (stream-ordered) once the candidates
    // are emitted, before the sort allocates its buffers
    std::optional<Scratch> early;
    early.emplace(s);
    BinnedBloom bb{};
    // B1: bloom_bits (8) bits per window; B2 ("seen twice"): a quarter of B1; 32-bit words. Binned
    // (shared-memory) filters when they cut into at most BB_MAXBINS bins of bloom_bin_kb KB of B1,
    // else sliced global-memory filters.
    auto sliced_filters = [&]() -> sg_status {
        const int64_t w1 = total * tune("bloom_bits") / 32 + 1024, w2 = w1 / 4 + 256;
        b1.nwords = (uint32_t)(w1 < 0xFFFFFFF0LL ? w1 : 0xFFFFFFF0LL);
        b2.nwords = (uint32_t)(w2 < 0xFFFFFFF0LL ? w2 : 0xFFFFFFF0LL);
        b1.words = early->get<uint32_t>(b1.nwords);
        b2.words = early->get<uint32_t>(b2.nwords);
        if (!b1.words || !b2.words) return SG_ERR_OOM;
        SG_CUDA_TRY(cudaMemsetAsync(b1.words, 0, (size_t)b1.nwords * 4, s));
        SG_CUDA_TRY(cudaMemsetAsync(b2.words, 0, (size_t)b2.nwords * 4, s));
        return SG_OK;
    };
    if (use_bloom && total > 0) {
        const int64_t w1 = total * tune("bloom_bits") / 32 + 1024;
        int lw1b = 0;  // bins of a power of two of words: a word's bin is a shift
        while (((int64_t)2 << lw1b) <= tune("bloom_bin_kb") * 256) lw1b++;
        const int64_t w1b = (int64_t)1 << lw1b;
        const int64_t nbins = (w1 + w1b - 1) / w1b;
        if (tune("bloom_binned") && nbins <= BB_MAXBINS && nbins * w1b < ((int64_t)1 << 32)) {
            bb.nbins = (uint32_t)nbins;
            bb.w1b = (uint32_t)w1b;
            bb.lw1b = (uint32_t)lw1b;
            bb.w2b = (uint32_t)(w1b / 4);
            bb.nwords1 = (uint32_t)(nbins * w1b);
            // a bin's expected hashes and room for repeats (bloom_bin_room_pct % of the mean, and
            // 16 K more when that is at least 100 %)
            const int64_t mean = total / nbins + 1, pct = tune("bloom_bin_room_pct");
            bb.cap = (uint32_t)(mean * pct / 100 + (pct >= 100 ? 16384 : 0) + 1);
            b1.nwords = bb.nwords1;  // never allocated in this form
            b2.nwords = bb.nbins * bb.w2b;
            b2.words = early->get<uint32_t>(b2.nwords);  // every word written by the bin pass
            if (!b2.words) return SG_ERR_OOM;
        } else {
            SG_TRY(sliced_filters());
        }
    }
    std::optional<StageScope> stage;
    stage.emplace("CountKmer", s);  // a1-a4: codes, Bloom, exact count, columns
    // 0. packed bases and window hashes (job prefixes by base position in a batch)
    const int64_t ngroups = (total + 31) / 32;
    JobPos jp{nullptr, 0, 2 * k};
    if (jm.ro) {
        int64_t *jpos = early->get<int64_t>(jm.njobs + 1);
        if (!jpos) return SG_ERR_OOM;
        SG_LAUNCH("job_pos", job_pos_kernel, blocks_for(jm.njobs + 1, NT), NT, 0, s, jm.ro, jm.njobs, off, n, jpos);
        jp = JobPos{jpos, jm.njobs, jm.kbits};
    }
    uint64_t *P = early->get<uint64_t>(ngroups + 1);
    uint32_t *H = early->get<uint32_t>(ngroups * 32);
    if (!P || !H) return SG_ERR_OOM;
    SG_CUDA_TRY(cudaMemsetAsync(P + ngroups, 0, sizeof(uint64_t), s));
    SG_TRY(dispatch_k(k, [&](auto kc) -> sg_status {
        SG_LAUNCH("pack", pack_kernel<decltype(kc)::value>, nblk, KM_NT, 0, s, seq, total, off, n, k, jp, P, H);
        return SG_OK;
    }));
    if (use_bloom && bb.nbins) {
        std::optional<Scratch> bins;
        bins.emplace(s);
        const int64_t nwin = ngroups * 32;
        // one grouping pass, or two (superbins of 2^lsup filter bins first): two where the filter
        // has more bins than one pass can count in shared memory (4096), or when asked
        const int64_t lv = tune("bloom_scatter_levels");
        const int levels = bb.nbins > 4096 ? 2 : (lv ? (int)lv : 1);
        int lsup = 0;
        if (levels == 2)
            while (((int64_t)1 << (2 * lsup)) < (int64_t)bb.nbins) lsup++;  // 2^lsup >= sqrt(nbins)
        const uint32_t nsup = levels == 2 ? (uint32_t)((bb.nbins + (1u << lsup) - 1) >> lsup) : 0u;
        const int64_t pct = tune("bloom_bin_room_pct");
        auto room = [&](int64_t groups) {  // hashes a group can hold: pct % of the mean, plus slack
            const int64_t mean = total / groups + 1;
            return (uint32_t)(mean * pct / 100 + (pct >= 100 ? 16384 : 0) + 1);
        };
        const uint32_t cap1 = levels == 2 ? room(nsup) : 0u;
        const size_t ncur = (size_t)bb.nbins * BB_CSTRIDE, ncur1 = (size_t)nsup * BB_CSTRIDE;
        uint32_t *cursor = bins->get<uint32_t>(ncur + ncur1 + 1);  // bins | superbins | overflow flag
        uint32_t *Hs = levels == 2 ? bins->get<uint32_t>((size_t)nsup * cap1) : nullptr;
        uint32_t *Hb = bins->get<uint32_t>((size_t)bb.nbins * bb.cap);
        if (!cursor || !Hb || (levels == 2 && !Hs)) return SG_ERR_OOM;
        SG_CUDA_TRY(cudaMemsetAsync(cursor, 0, (ncur + ncur1 + 1) * sizeof(uint32_t), s));
        uint32_t *ovf_flag = cursor + ncur + ncur1;
        const int64_t cfg = tune("bloom_scatter_cfg");
        const int nt = cfg == 0 ? 512 : 256, tile = cfg == 1 ? 4096 : 8192;
        auto scatter = [&](ScatterLevel L, uint32_t *cur, uint32_t *dst, int64_t grid) -> sg_status {
            const size_t ssm = ((size_t)3 * L.nb + tile) * sizeof(uint32_t);
            auto run = [&](auto kern) -> sg_status {
                SG_CUDA_TRY(ensure_smem(kern, ssm));
                SG_LAUNCH("bloom_bin_scatter", kern, grid, nt, ssm, s, L, bb.nwords1, cur, dst, ovf_flag);
                return SG_OK;
            };
            switch (cfg) {  // threads x hashes per thread
                case 0: return run(bloom_bin_scatter_kernel<512, 16>);
                case 1: return run(bloom_bin_scatter_kernel<256, 16>);
                default: return run(bloom_bin_scatter_kernel<256, 32>);
            }
        };
        if (levels == 2) {
            const ScatterLevel l1{(const uint32_t *)H, nwin, nullptr, 0u, 0u, bb.lw1b + lsup, nsup, cap1};
            SG_TRY(scatter(l1, cursor + ncur, Hs, blocks_for(nwin, tile)));
            const uint32_t tpg = (uint32_t)blocks_for(cap1, tile);
            const ScatterLevel l2{(const uint32_t *)Hs, 0, (const uint32_t *)(cursor + ncur), cap1, tpg, bb.lw1b,
                                  1u << lsup, bb.cap};
            SG_TRY(scatter(l2, cursor, Hb, (int64_t)nsup * tpg));
        } else {
            const ScatterLevel l1{(const uint32_t *)H, nwin, nullptr, 0u, 0u, bb.lw1b, bb.nbins, bb.cap};
            SG_TRY(scatter(l1, cursor, Hb, blocks_for(nwin, tile)));
        }
        const size_t ism = (size_t)(bb.w1b + bb.w2b) * sizeof(uint32_t);
        SG_CUDA_TRY(ensure_smem(bloom_bin_insert_kernel, ism));
        SG_LAUNCH("bloom_insert", bloom_bin_insert_kernel, bb.nbins, BI_NT, ism, s, (const uint32_t *)Hb,
                  (const uint32_t *)cursor, bb, b2.words);
        uint32_t ovf = 0;
        SG_CUDA_TRY(read_back(&ovf, ovf_flag, sizeof(uint32_t), s));
        if (ovf) {  // a bin outgrew its room (a hash value shared by very many windows): sliced filters
            bb = BinnedBloom{};
            SG_TRY(sliced_filters());
        }
    }
    if (use_bloom && !bb.nbins) {
        // slices of at most bloom_slice_mb of B1, so each launch's atomics stay in L2
        uint64_t slice_words = ((uint64_t)tune("bloom_slice_mb") << 20) / 4;
        uint64_t nsl = (b1.nwords + slice_words - 1) / slice_words;
        // every slice streams all window codes: beyond bloom_max_slices, slices grow instead
        const uint64_t max_sl = (uint64_t)tune("bloom_max_slices");
        if (nsl > max_sl) nsl = max_sl;
        const int64_t nvec = ngroups * 8;  // 16-byte vectors of 4 hashes
        const int64_t gmax = (int64_t)sm_count() * 16;
        const int64_t grid = blocks_for(nvec, KM_NT) < gmax ? blocks_for(nvec, KM_NT) : gmax;
        const int64_t u = tune("bloom_unroll");
        for (uint64_t q = 0; q < nsl; q++) {
            const uint32_t lo_w = (uint32_t)((uint64_t)b1.nwords * q / nsl);
            const uint32_t hi_w = (uint32_t)((uint64_t)b1.nwords * (q + 1) / nsl);
            if (u >= 8)
                SG_LAUNCH("bloom_insert", bloom_insert_kernel<8>, grid, KM_NT, 0, s, (const uint32_t *)H, nvec, b1, b2, lo_w,
                          hi_w);
            else
                SG_LAUNCH("bloom_insert", bloom_insert_kernel<4>, grid, KM_NT, 0, s, (const uint32_t *)H, nvec, b1, b2, lo_w,
                          hi_w);
        }
    }
    // Candidate records: PK_POS (code, position and strand in one 8-byte key) where the code's low
    // bits fit beside the position once its top 0..3 bits become buckets (the fewest that fit:
    // buckets cost a code per candidate in the count pass and per-bucket sort launches, so they
    // are used only to make the key fit), else PK_IDX or PK_PAIRS, chosen once nc is known.
    int qbits = 1;
    while (((int64_t)1 << qbits) < total) qbits++;
    int bbits = -1;
    for (int b = 0; b <= (int)tune("kmer_sort_buckets") && b < code_bits && bbits < 0; b++)
        if ((code_bits - b) + qbits + 1 <= 64) bbits = b;
    const int64_t nwarp = nblk * KM_WARPS;
    Buckets bk{P, k, jp, bbits > 0 ? 1 << bbits : 1, code_bits - (bbits > 0 ? bbits : 0), kmask, nwarp};
    uint32_t *cmask = early->get<uint32_t>(nwarp * KM_GW);
    uint32_t *wcnt = early->get<uint32_t>(nwarp * bk.nb + 1);
    int64_t *wpos = early->get<int64_t>(nwarp * bk.nb + 1);
    if (!cmask || !wcnt || !wpos) return SG_ERR_OOM;
    if (bk.nb > 1)
        SG_LAUNCH("cand_count", cand_count_kernel<true>, nblk, KM_NT, 0, s, (const uint32_t *)H, ngroups * 32, b2,
                  use_bloom, bb, bk, cmask, wcnt);
    else
        SG_LAUNCH("cand_count", cand_count_kernel<false>, nblk, KM_NT, 0, s, (const uint32_t *)H, ngroups * 32, b2,
                  use_bloom, bb, bk, cmask, wcnt);
    SG_TRY(exclusive_scan<uint32_t>(wcnt, wpos, nwarp * bk.nb, s, err));
    BucketStarts bs{};
    bs.nb = bk.nb;
    bs.shift = bk.shift;
    for (int b = 0; b <= bk.nb; b++)
        SG_CUDA_TRY(cudaMemcpyAsync(&bs.start[b], wpos + (int64_t)b * nwarp, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    uint32_t herr = 0;
    SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t nc = bs.start[bk.nb];
    if (herr & DEV_TIMEOUT) return timeout_error("build_kmer_matrix");
    if (herr) {  // the passes above stayed in bounds; their results are discarded
        set_error("build_kmer_matrix: offsets are not a valid partition of the sequence");
        return SG_ERR_INVALID;
    }

    int ibits = 1;
    while (((int64_t)1 << ibits) < nc) ibits++;
    const int mode = bbits >= 0 ? PK_POS : (code_bits + ibits <= 64 ? PK_IDX : PK_PAIRS);
    const int pb = mode == PK_POS ? qbits + 1 : (mode == PK_IDX ? ibits : 0);
    // buffers live only as long as they are needed, so that the pool can hand their memory to the
    // next phase: the emitted records, then (once the window hashes and filters are gone) the
    // sort's second buffers
    uint64_t *key0 = sc.get<uint64_t>(nc);
    uint64_t *val0 = mode == PK_POS ? nullptr : sc.get<uint64_t>(nc);
    if (!key0 || (mode != PK_POS && !val0)) return SG_ERR_OOM;
    if (bk.nb > 1)
        SG_LAUNCH("cand_emit", cand_emit_kernel<true>, nblk, KM_NT, 0, s, bk, (const uint32_t *)cmask,
                  (const int64_t *)wpos, mode, pb, key0, val0, nc);
    else
        SG_LAUNCH("cand_emit", cand_emit_kernel<false>, nblk, KM_NT, 0, s, bk, (const uint32_t *)cmask,
                  (const int64_t *)wpos, mode, pb, key0, val0, nc);
    early.reset();
    uint64_t *key1 = sc.get<uint64_t>(nc), *val1 = mode == PK_PAIRS ? sc.get<uint64_t>(nc) : nullptr;
    if (!key1 || (mode == PK_PAIRS && !val1)) return SG_ERR_OOM;
    bool alt = false;
    const uint64_t *key = nullptr;
    uint64_t *val = nullptr;
    // direct: segments, columns and At straight from the sorted PK_POS keys (seg_mark, scans of
    // its tile totals, seg_emit); needs the walk bound of the fused flags
    const bool direct = mode == PK_POS && nc > 0 && tune("kmer_direct_seg") && hmax <= (uint32_t)SEG_WALK_MAX;
    const uint64_t *sorted = nullptr;  // direct: the sorted keys
    uint32_t *dflags = nullptr;        // direct: two flag bits per candidate
    int64_t *dpre = nullptr;           // direct: [ntiles + 1] segments before each tile, then kept entries
    SegArgs dargs{};
    uint64_t *pre = nullptr;
    int64_t sizes[2] = {0, 0};  // m, nnz
    {
        sg_kmer_stats &ks = kmer_stats();
        ks = sg_kmer_stats{};
        ks.windows = total;
        ks.candidates = nc;
        ks.sort_key_bytes = 8;
        ks.sort_val_bytes = mode == PK_PAIRS ? 8 : 0;
        ks.sort_passes = nc > 1 ? (bk.shift + 7) / 8 : 0;
        ks.bloom_bins = bb.nbins;
        ks.bloom_b2_bytes = use_bloom ? (int64_t)b2.nwords * 4 : 0;
    }
    const int64_t nlut = (total >> LUT_SHIFT) + 1;
    int32_t *lut = sc.get<int32_t>(nlut);
    if (!lut) return SG_ERR_OOM;
    SG_LAUNCH("read_lut", read_lut_kernel, blocks_for(nlut, NT), NT, 0, s, off, n, nlut, lut);
    if (mode != PK_PAIRS) {  // 8-byte keys through the radix passes, then one unpacking pass
        // each bucket sorted on its `shift` code bits; buckets of 0 or 1 keys need no pass, but
        // must end in the same buffer as the others
        const int npass = (bk.shift + 7) / 8;
        bool any = false;
        for (int b = 0; b < bk.nb; b++) any |= bs.start[b + 1] - bs.start[b] > 1;
        alt = any && (npass & 1);
        for (int b = 0; b < bk.nb; b++) {
            const int64_t s0 = bs.start[b], nbk = bs.start[b + 1] - s0;
            if (nbk > 1) {
                bool a = false;
                SG_TRY(radix_sort_keys(key0 + s0, key1 + s0, nbk, pb, pb + bk.shift, &a, s, err));
            } else if (nbk == 1 && alt) {
                SG_CUDA_TRY(cudaMemcpyAsync(key1 + s0, key0 + s0, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
            }
        }
        uint64_t *ks = alt ? key1 : key0, *kfree = alt ? key0 : key1;
        if (direct) {
            sc.release(kfree);
            sorted = ks;
            const int64_t ntiles = (nc + DS_TILE - 1) / DS_TILE;
            dflags = sc.get<uint32_t>(ntiles * DS_NT);
            uint32_t *tcount = sc.get<uint32_t>(2 * ntiles);
            dpre = sc.get<int64_t>(2 * (ntiles + 1));
            if (!dflags || !tcount || !dpre) return SG_ERR_OOM;
            dargs = SegArgs{sorted, nc, pb, bs, lo, hi, lohi, 2 * k, (int)hmax, off, n, (const int32_t *)lut, nlut};
            SG_LAUNCH("seg_mark", seg_mark_kernel, ntiles, DS_NT, 0, s, dargs, dflags, tcount, tcount + ntiles);
            SG_TRY(exclusive_scan<uint32_t>(tcount, dpre, ntiles, s, err));
            SG_TRY(exclusive_scan<uint32_t>(tcount + ntiles, dpre + ntiles + 1, ntiles, s, err));
            SG_CUDA_TRY(cudaMemcpyAsync(&sizes[0], dpre + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            SG_CUDA_TRY(cudaMemcpyAsync(&sizes[1], dpre + 2 * ntiles + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            SG_CUDA_TRY(cudaStreamSynchronize(s));
            sc.release(tcount);
        }
        if (!direct) {
            val1 = sc.get<uint64_t>(nc);
            if (!val1) return SG_ERR_OOM;
            SG_LAUNCH("unpack", unpack_kernel, blocks_for(nc, NT), NT, 0, s, (const uint64_t *)ks,
                      (const uint64_t *)val0, nc, mode, pb, bs, off, n, (const int32_t *)lut, nlut, kfree, val1);
            key = kfree;
            val = val1;
            sc.release(ks);
        }
        if (val0) sc.release(val0);
    } else {
        SG_TRY((radix_sort_pairs<uint64_t, uint64_t>(key0, val0, key1, val1, nc, code_bits, &alt, s, err)));
        key = alt ? key1 : key0;
        val = alt ? val1 : val0;
        sc.release(alt ? key0 : key1);
        sc.release(alt ? val0 : val1);
        SG_LAUNCH("resolve", resolve_kernel, blocks_for(nc, NT), NT, 0, s, val, nc, off, n, (const int32_t *)lut,
                  nlut);
    }

    // segments -> exact frequency -> reliable -> columns; kept entries -> At
    // The fused form packs (reliable segments, kept entries) into one scanned 64-bit word whose
    // look-back keeps 62 bits: segments < 2^31 (at most nc / 2 with the Bloom filter, each reliable
    // segment holding >= lo >= 2 entries) and kept entries < 2^31 (counted first).
    bool fused = !direct && hmax <= (uint32_t)SEG_WALK_MAX && nc < ((int64_t)1 << 32) &&
                 (use_bloom || nc < ((int64_t)1 << PK_SHIFT));
    uint32_t *head = nullptr, *rel = nullptr, *keep = nullptr;
    int64_t *seg_excl = nullptr, *seg_start = nullptr, *col_of_seg = nullptr, *out_pos = nullptr;
    if (fused) {
        pre = sc.get<uint64_t>(nc + 1);
        unsigned long long *nkeep = sc.get<unsigned long long>(1);
        if (!pre || !nkeep) return SG_ERR_OOM;
        SG_CUDA_TRY(cudaMemsetAsync(nkeep, 0, sizeof(unsigned long long), s));
        SG_LAUNCH("seg_flags", seg_flags_kernel, blocks_for(nc, NT), NT, 0, s, key, (const uint64_t *)val, nc, lo, hi,
                  lohi, 2 * k, (int)hmax, pre, nkeep);
        unsigned long long hk = 0;
        SG_CUDA_TRY(read_back(&hk, nkeep, sizeof(hk), s));
        if (hk >= (1ull << PK_SHIFT)) {  // too many kept entries for the packed scan
            sc.release(pre);
            pre = nullptr;
            fused = false;
        }
    }
    if (fused) {
        // flags scanned in place: each tile reads its items before it writes them
        SG_TRY(exclusive_scan<int64_t>((const int64_t *)pre, (int64_t *)pre, nc, s, err));
        uint64_t tot = 0;
        SG_CUDA_TRY(cudaMemcpyAsync(&tot, pre + nc, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaStreamSynchronize(s));
        sizes[0] = (int64_t)(tot & ((1ull << PK_SHIFT) - 1));
        sizes[1] = (int64_t)(tot >> PK_SHIFT);
    } else if (!direct) {  // (direct: sizes and the error word were read back after its scan)
        head = sc.get<uint32_t>(nc + 1);
        seg_excl = sc.get<int64_t>(nc + 1);
        seg_start = sc.get<int64_t>(nc + 1);
        rel = sc.get<uint32_t>(nc + 1);
        col_of_seg = sc.get<int64_t>(nc + 1);
        keep = sc.get<uint32_t>(nc + 1);
        out_pos = sc.get<int64_t>(nc + 1);
        if (!head || !seg_excl || !seg_start || !rel || !col_of_seg || !keep || !out_pos) return SG_ERR_OOM;
        SG_LAUNCH("seg_head", seg_head_kernel, blocks_for(nc, NT), NT, 0, s, key, nc, head);
        SG_TRY(exclusive_scan<uint32_t>(head, seg_excl, nc, s, err));
        SG_LAUNCH("seg_start", seg_start_kernel, blocks_for(nc, NT), NT, 0, s, head, seg_excl, nc, seg_start);
        // number of segments lives on the device at seg_excl[nc]; launch over the upper bound nc
        SG_LAUNCH("seg_reliable", seg_reliable_kernel, blocks_for(nc, NT), NT, 0, s, seg_start, seg_excl + nc, lo,
                  hi, key, lohi, 2 * k, nc, rel);
        SG_TRY(exclusive_scan<uint32_t>(rel, col_of_seg, nc, s, err));
        SG_LAUNCH("keep", keep_kernel, blocks_for(nc, NT), NT, 0, s, head, seg_excl, rel, val, nc, keep);
        SG_TRY(exclusive_scan<uint32_t>(keep, out_pos, nc, s, err));
        // m = reliable segments = col_of_seg[nc] (rel is 0 past the last segment)
        SG_CUDA_TRY(cudaMemcpyAsync(&sizes[0], col_of_seg + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaMemcpyAsync(&sizes[1], out_pos + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (herr) return timeout_error("build_kmer_matrix");
    const int64_t m = sizes[0], nnz = sizes[1];
    if (m >= ((int64_t)1 << 31)) {
        set_error("build_kmer_matrix: %lld reliable k-mers exceed the int32 column range", (long long)m);
        return SG_ERR_OVERFLOW;
    }

    // outputs: At and the column codes now, A once the candidate records are gone
    SG_ALLOC(At->row_ptr, int64_t, m + 1, s);
    SG_ALLOC(At->col, int32_t, nnz, s);
    SG_ALLOC(At->val, uint32_t, nnz, s);
    SG_ALLOC(*codes_out, uint64_t, m, s);
    At->n_rows = m; At->n_cols = n; At->nnz = nnz;

    stage.emplace("CreateSpMat", s);  // a5: At, then A by a sort on the read
    uint32_t *ak0 = sc.get<uint32_t>(nnz);
    uint64_t *av0 = sc.get<uint64_t>(nnz);
    if (!ak0 || !av0) return SG_ERR_OOM;
    if (direct) {
        const int64_t ntiles = (nc + DS_TILE - 1) / DS_TILE;
        SG_LAUNCH("emit_at", seg_emit_kernel, ntiles, DS_NT, 0, s, dargs, (const uint32_t *)dflags,
                  (const int64_t *)dpre, (const int64_t *)(dpre + ntiles + 1), m, nnz, At->col, At->val,
                  At->row_ptr, *codes_out, ak0, av0, job_ncols);
    } else if (fused)
        SG_LAUNCH("emit_at", emit_fused_kernel, blocks_for(nc > 0 ? nc : 1, NT), NT, 0, s, (const uint64_t *)pre, key,
                  (const uint64_t *)val, nc, m, nnz, At->col, At->val, At->row_ptr, *codes_out, ak0, av0, 2 * k,
                  job_ncols);
    else
        SG_LAUNCH("emit_at", emit_at_kernel, blocks_for(nc > 0 ? nc : 1, NT), NT, 0, s, head, seg_excl, rel,
                  col_of_seg, keep, out_pos, key, val, nc, m, nnz, At->col, At->val, At->row_ptr, *codes_out, ak0,
                  av0, 2 * k, job_ncols);
    for (const void *p : {(const void *)key, (const void *)val, (const void *)pre, (const void *)sorted,
                          (const void *)dflags, (const void *)dpre,
                          (const void *)head, (const void *)seg_excl, (const void *)seg_start, (const void *)rel,
                          (const void *)col_of_seg, (const void *)keep, (const void *)out_pos})
        if (p) sc.release(p);
    SG_ALLOC(A->row_ptr, int64_t, n + 1, s);
    SG_ALLOC(A->col, int32_t, nnz, s);
    SG_ALLOC(A->val, uint32_t, nnz, s);
    A->n_rows = n; A->n_cols = m; A->nnz = nnz;
    uint32_t *ak1 = sc.get<uint32_t>(nnz);
    uint64_t *av1 = sc.get<uint64_t>(nnz);
    if (!ak1 || !av1) return SG_ERR_OOM;
    int rbits = 0;
    while (rbits < 32 && ((int64_t)1 << rbits) < n) rbits++;
    kmer_stats().m = m;
    kmer_stats().nnz = nnz;
    kmer_stats().a_sort_passes = nnz > 1 ? (rbits + 7) / 8 : 0;
    bool aalt = false;
    const bool split = nnz > 1 && rbits > 0;  // the sort's last pass writes A's columns and values
    if (split)
        SG_TRY(radix_sort_pairs_split(ak0, av0, ak1, av1, nnz, rbits, &aalt, (uint32_t *)A->col, A->val, s, err));
    const uint32_t *arow = aalt ? ak1 : ak0;
    const uint64_t *apv = aalt ? av1 : av0;
    SG_LAUNCH("rowptr_from_sorted", rowptr_from_sorted_kernel, blocks_for(nnz + 1, NT), NT, 0, s, arow, nnz, n,
              A->row_ptr);
    if (!split) SG_LAUNCH("split_pairs", split_pairs_kernel, blocks_for(nnz, NT), NT, 0, s, apv, nnz, A->col, A->val);
    SG_CUDA_TRY(read_back(&herr, err, sizeof(uint32_t), s));  // the sort of A waits between tiles
    if (herr) return timeout_error("build_kmer_matrix");
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
                            sg::JobMap{nullptr, 1, 2 * k}, nullptr, nullptr, hi);
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
