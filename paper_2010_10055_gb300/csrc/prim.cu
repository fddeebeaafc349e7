// prim.cu -- single-pass exclusive scan and stable LSD radix sort, both with decoupled look-back
// between tiles (the radix sort: one upfront digit count for all passes, then one kernel per pass
// that ranks keys per warp with ballots and scatters from shared memory in digit order).
#include <algorithm>

#include "check.cuh"
#include "prim.cuh"

namespace sg {

// -------------------------------------------------------------------- decoupled look-back
// A tile publishes a 64-bit status word per counter: flag in the top two bits (0 = nothing yet,
// LB_A = this tile's own aggregate, LB_P = inclusive prefix through this tile), value in the low 62
// bits. Tiles take their ids from an atomic counter in launch order, so every tile waited on has
// already started and never waits on a later one. Each wait is bounded: after LB_SPIN_LIMIT polls
// the waiter records DEV_TIMEOUT in *err (read back by the caller) and goes on with a zero.
constexpr unsigned long long LB_A = 1ull << 62, LB_P = 2ull << 62, LB_VAL = (1ull << 62) - 1;
constexpr int LB_SPIN_LIMIT = 1 << 20;  // at least 64 ms of polling; a real wait takes microseconds

__device__ __forceinline__ void lb_store(unsigned long long *p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long *>(p) = v;
}

__device__ __forceinline__ unsigned long long lb_wait(const unsigned long long *p, uint32_t *err) {
    unsigned long long v = *reinterpret_cast<const volatile unsigned long long *>(p);
    for (int it = 0; (v >> 62) == 0; it++) {
        if (it >= LB_SPIN_LIMIT) {
            if (err) atomicOr(err, (uint32_t)DEV_TIMEOUT);
            return LB_P;
        }
        __nanosleep(64);
        v = *reinterpret_cast<const volatile unsigned long long *>(p);
    }
    return v;
}

// ------------------------------------------------------------------------------- scan
// One pass: each tile loads its items once, publishes its sum, finds the sum of all earlier tiles
// by look-back (warp 0, 32 predecessors per step) and writes its outputs.
constexpr int SCAN_NT = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_NT * SCAN_ITEMS;

// stall != 0 (test hook, sg_debug_stall_lookback): tile 0 withholds its prefix, so the waits of
// the tiles after it run out.
template <class T>
__global__ void __launch_bounds__(SCAN_NT) scan_kernel(const T *in, int64_t n, int64_t *out,
                                                      unsigned long long *status, unsigned int *tile_ctr,
                                                      uint32_t *err, int stall) {
    __shared__ int64_t vals[SCAN_TILE + SCAN_TILE / 32];
    __shared__ int64_t tmp[SCAN_NT / 32 + 1];
    __shared__ int64_t s_excl;
    __shared__ unsigned int s_tile;
    if (threadIdx.x == 0) s_tile = tile_ctr ? atomicAdd(tile_ctr, 1u) : 0u;
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * SCAN_TILE;
    auto pad = [](int i) { return i + (i >> 5); };  // break the bank conflicts of blocked reads
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        const int idx = i * SCAN_NT + threadIdx.x;
        vals[pad(idx)] = (base + idx < n) ? (int64_t)in[base + idx] : 0;
    }
    __syncthreads();
    int64_t loc[SCAN_ITEMS];
    int64_t sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        loc[i] = sum;
        sum += vals[pad(threadIdx.x * SCAN_ITEMS + i)];
    }
    int64_t total;
    const int64_t pre = block_exclusive_scan<SCAN_NT>(sum, tmp, &total);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int64_t excl = 0;
        if (tile > 0) {
            if (lane == 0) lb_store(status + tile, LB_A | (unsigned long long)total);
            for (int64_t t = tile - 1;; t -= 32) {
                const int64_t idx = t - lane;
                const unsigned long long v = idx >= 0 ? lb_wait(status + idx, err) : LB_P;
                const unsigned pm = __ballot_sync(0xffffffffu, (v >> 62) == 2);
                const int stop = pm ? __ffs(pm) - 1 : 31;  // nearest inclusive prefix
                int64_t c = lane <= stop ? (int64_t)(v & LB_VAL) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                excl += c;
                if (pm) break;
            }
        }
        if (lane == 0) {
            if (status && !(stall && tile == 0)) lb_store(status + tile, LB_P | (unsigned long long)(excl + total));
            s_excl = excl;
        }
    }
    __syncthreads();
    const int64_t off = s_excl + pre;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) vals[pad(threadIdx.x * SCAN_ITEMS + i)] = loc[i] + off;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        const int idx = i * SCAN_NT + threadIdx.x;
        if (base + idx < n) out[base + idx] = vals[pad(idx)];
    }
    if (base + SCAN_TILE >= n && threadIdx.x == 0) out[n] = s_excl + total;
}

template <class T>
sg_status exclusive_scan(const T *in, int64_t *out, int64_t n, cudaStream_t s, uint32_t *err) {
    if (n <= 0) {
        SG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return SG_OK;
    }
    const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nt == 1) {
        SG_LAUNCH("scan", scan_kernel<T>, 1, SCAN_NT, 0, s, in, n, out, (unsigned long long *)nullptr,
                  (unsigned int *)nullptr, err, 0);
        return SG_OK;
    }
    Scratch sc(s);
    unsigned long long *status = sc.get<unsigned long long>(nt + 1);  // [nt] status, then the tile counter
    if (!status) return SG_ERR_OOM;
    SG_CUDA_TRY(cudaMemsetAsync(status, 0, (size_t)(nt + 1) * sizeof(unsigned long long), s));
    SG_LAUNCH("scan", scan_kernel<T>, nt, SCAN_NT, 0, s, in, n, out, status, (unsigned int *)(status + nt), err,
              debug_stall_lookback());
    return SG_OK;
}

template sg_status exclusive_scan<int64_t>(const int64_t *, int64_t *, int64_t, cudaStream_t, uint32_t *);
template sg_status exclusive_scan<uint32_t>(const uint32_t *, int64_t *, int64_t, cudaStream_t, uint32_t *);
template sg_status exclusive_scan<int32_t>(const int32_t *, int64_t *, int64_t, cudaStream_t, uint32_t *);
template sg_status exclusive_scan<uint8_t>(const uint8_t *, int64_t *, int64_t, cudaStream_t, uint32_t *);

// ------------------------------------------------------------------------- radix sort
// LSD, 8-bit digits. One upfront pass counts the digits of every pass; then each pass is one
// kernel: a tile ranks its keys per warp (peer masks from one ballot per digit bit), publishes its
// digit counts, finds each
// digit's count in all earlier tiles by look-back (one thread per digit), stages its keys in
// shared memory in digit order and writes every digit's run contiguously.
constexpr int RS_BITS = 8;
constexpr int RS_RADIX = 1 << RS_BITS;
constexpr int RS_NT = 256;
constexpr int RS_WARPS = RS_NT / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_NT * RS_ITEMS;
constexpr int RS_MAXP = 8;
constexpr int RS_LBW = 8;  // predecessors read per look-back step, at most

template <class K>
__global__ void __launch_bounds__(RS_NT) radix_upfront_kernel(const K *__restrict__ keys, int64_t n, int lo_bit,
                                                             int npass, unsigned long long *__restrict__ ghist) {
    __shared__ uint32_t h[RS_MAXP * RS_RADIX];
    for (int i = threadIdx.x; i < npass * RS_RADIX; i += RS_NT) h[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * RS_NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RS_NT) {
        const K key = keys[i];
        for (int p = 0; p < npass; p++)
            atomicAdd(&h[p * RS_RADIX + ((uint32_t)(key >> (lo_bit + RS_BITS * p)) & (RS_RADIX - 1))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * RS_RADIX; i += RS_NT)
        if (h[i]) atomicAdd(ghist + i, (unsigned long long)h[i]);
}

template <class K, class V, bool HAS_V>
struct RsSmem {
    K keys[RS_TILE];
    V vals[HAS_V ? RS_TILE : 1];
    int64_t gbase[RS_RADIX];
    int64_t tmp64[RS_WARPS + 1];
    uint32_t wcnt[RS_WARPS][RS_RADIX];
    uint32_t tstart[RS_RADIX];
    uint32_t tmp[RS_WARPS + 1];
    unsigned int tile;
};

// ghist: this pass's 256 digit totals; status: [ntiles][256] look-back words, zeroed; tile_ctr:
// zeroed. Without values (HAS_V == false) vin / vout are not touched.
template <class K, class V, bool HAS_V, bool MATCH>
__global__ void __launch_bounds__(RS_NT, HAS_V ? 3 : 4) radix_onesweep_kernel(const K *__restrict__ kin, const V *__restrict__ vin,
                                                              K *__restrict__ kout, V *__restrict__ vout,
                                                              int64_t n, int shift,
                                                              const unsigned long long *__restrict__ ghist,
                                                              unsigned long long *status, unsigned int *tile_ctr,
                                                              uint32_t *err, int lbw) {
    extern __shared__ __align__(16) unsigned char rs_raw[];
    RsSmem<K, V, HAS_V> &sm = *reinterpret_cast<RsSmem<K, V, HAS_V> *>(rs_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) sm.tile = atomicAdd(tile_ctr, 1u);
    for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_NT) (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile = sm.tile;
    const int64_t tbase = tile * RS_TILE;
    const int64_t wbase = tbase + (int64_t)w * 32 * RS_ITEMS;
    const uint32_t lt = (1u << lane) - 1u;
    K key[RS_ITEMS];
    V val[HAS_V ? RS_ITEMS : 1];
    uint32_t local[RS_ITEMS];
#pragma unroll
    for (int it = 0; it < RS_ITEMS; it++) {
        const int64_t idx = wbase + it * 32 + lane;
        const bool valid = idx < n;
        key[it] = valid ? kin[idx] : K(0);
        if (HAS_V) val[HAS_V ? it : 0] = valid ? vin[idx] : V(0);
        const uint32_t d = (uint32_t)(key[it] >> shift) & (RS_RADIX - 1);
        // lanes holding the same digit: one match instruction, or the intersection of the ballots
        // of the digit's 8 bits (invalid lanes carry a digit value no valid lane has)
        uint32_t peers;
        if (MATCH) {
            peers = __match_any_sync(0xffffffffu, valid ? d : RS_RADIX);
        } else {
            peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int b = 0; b < RS_BITS; b++) {
                const bool bit = (d >> b) & 1u;
                const uint32_t bb = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bb : ~bb;
            }
        }
        const uint32_t base_cnt = valid ? sm.wcnt[w][d] : 0u;
        __syncwarp();
        if (valid) {
            local[it] = base_cnt + __popc(peers & lt);
            if ((peers >> lane) == 1u) sm.wcnt[w][d] = base_cnt + __popc(peers);  // highest peer lane
        }
        __syncwarp();
    }
    __syncthreads();
    // thread d: digit d's offsets across warps and its count in this tile
    const int d = threadIdx.x;  // RS_NT == RS_RADIX
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ww++) {
        const uint32_t c = sm.wcnt[ww][d];
        sm.wcnt[ww][d] = tot;
        tot += c;
    }
    // publish this tile's count of digit d, then look back for the count in all earlier tiles
    unsigned long long *mine = status + tile * RS_RADIX + d;
    int64_t excl = 0;
    if (tile == 0) {
        lb_store(mine, LB_P | tot);
    } else {
        lb_store(mine, LB_A | tot);
        // walk back lbw predecessors at a time: their words are read together, and only a word not
        // yet published is waited on
        bool done = false;
        for (int64_t t = tile - 1; t >= 0 && !done; t -= lbw) {
            unsigned long long v[RS_LBW];
#pragma unroll
            for (int q = 0; q < RS_LBW; q++)
                v[q] = (q < lbw && t - q >= 0)
                           ? *reinterpret_cast<const volatile unsigned long long *>(status + (t - q) * RS_RADIX + d)
                           : 0ull;
#pragma unroll
            for (int q = 0; q < RS_LBW; q++) {
                if (done || q >= lbw || t - q < 0) continue;
                unsigned long long x = v[q];
                if ((x >> 62) == 0) x = lb_wait(status + (t - q) * RS_RADIX + d, err);
                excl += (int64_t)(x & LB_VAL);
                if ((x >> 62) == 2) done = true;
            }
        }
        lb_store(mine, LB_P | (unsigned long long)(excl + tot));
    }
    uint32_t total;
    const uint32_t st = block_exclusive_scan<RS_NT>(tot, sm.tmp, &total);
    int64_t gtotal;
    const int64_t dstart = block_exclusive_scan<RS_NT>((int64_t)ghist[d], sm.tmp64, &gtotal);
    sm.tstart[d] = st;
    sm.gbase[d] = dstart + excl - (int64_t)st;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; it++) {
        const int64_t idx = wbase + it * 32 + lane;
        if (idx < n) {
            const uint32_t dd = (uint32_t)(key[it] >> shift) & (RS_RADIX - 1);
            const uint32_t p = sm.tstart[dd] + sm.wcnt[w][dd] + local[it];
            if (!SG_IN_BOUNDS(p < RS_TILE, 201, p)) continue;
            sm.keys[p] = key[it];
            if (HAS_V) sm.vals[HAS_V ? p : 0] = val[HAS_V ? it : 0];
        }
    }
    __syncthreads();
    const int64_t cnt = n - tbase < RS_TILE ? n - tbase : RS_TILE;
    for (int i = threadIdx.x; i < cnt; i += RS_NT) {
        const K kk = sm.keys[i];
        const uint32_t dd = (uint32_t)(kk >> shift) & (RS_RADIX - 1);
        const int64_t o = sm.gbase[dd] + i;
        if (!SG_IN_BOUNDS(o >= 0 && o < n, 202, o)) continue;
        kout[o] = kk;
        if (HAS_V) vout[o] = sm.vals[HAS_V ? i : 0];
    }
}

template <class K, class V, bool HAS_V>
static sg_status radix_sort_impl(K *k0, V *v0, K *k1, V *v1, int64_t n, int lo_bit, int hi_bit, bool *in_alt,
                                 cudaStream_t s, uint32_t *err) {
    static_assert(RS_NT == RS_RADIX, "one thread per digit");
    *in_alt = false;
    if (n <= 1 || hi_bit <= lo_bit) return SG_OK;
    const int npass = (hi_bit - lo_bit + RS_BITS - 1) / RS_BITS;
    if (npass > RS_MAXP) {
        set_error("internal: radix sort of %d bits", hi_bit - lo_bit);
        return SG_ERR_INVALID;
    }
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    Scratch sc(s);
    // [npass][256] digit totals | [npass][ntiles][256] look-back words | [npass] tile counters
    const size_t words = (size_t)npass * RS_RADIX + (size_t)npass * ntiles * RS_RADIX + (size_t)npass;
    unsigned long long *ws = sc.get<unsigned long long>(words);
    if (!ws) return SG_ERR_OOM;
    unsigned long long *ghist = ws, *status = ws + (size_t)npass * RS_RADIX;
    unsigned int *ctr = (unsigned int *)(status + (size_t)npass * ntiles * RS_RADIX);
    SG_CUDA_TRY(cudaMemsetAsync(ws, 0, words * sizeof(unsigned long long), s));
    const int64_t hmax = (int64_t)sm_count() * 8;
    const int64_t hgrid = ntiles < hmax ? ntiles : hmax;
    SG_LAUNCH("radix_upfront", radix_upfront_kernel<K>, hgrid, RS_NT, 0, s, (const K *)k0, n, lo_bit, npass, ghist);
    const size_t smem = sizeof(RsSmem<K, V, HAS_V>);
    const bool match = tune("radix_match") != 0;
    const int lbw = (int)std::min<int64_t>(std::max<int64_t>(tune("radix_lookback"), 1), RS_LBW);
    if (match) SG_CUDA_TRY(ensure_smem(radix_onesweep_kernel<K, V, HAS_V, true>, smem));
    else SG_CUDA_TRY(ensure_smem(radix_onesweep_kernel<K, V, HAS_V, false>, smem));
    K *ki = k0, *ko = k1;
    V *vi = v0, *vo = v1;
    for (int p = 0; p < npass; p++) {
        if (match)
            SG_LAUNCH("radix_onesweep", (radix_onesweep_kernel<K, V, HAS_V, true>), ntiles, RS_NT, smem, s,
                      (const K *)ki, (const V *)vi, ko, vo, n, lo_bit + RS_BITS * p,
                      (const unsigned long long *)(ghist + p * RS_RADIX), status + (size_t)p * ntiles * RS_RADIX,
                      ctr + p, err, lbw);
        else
            SG_LAUNCH("radix_onesweep", (radix_onesweep_kernel<K, V, HAS_V, false>), ntiles, RS_NT, smem, s,
                      (const K *)ki, (const V *)vi, ko, vo, n, lo_bit + RS_BITS * p,
                      (const unsigned long long *)(ghist + p * RS_RADIX), status + (size_t)p * ntiles * RS_RADIX,
                      ctr + p, err, lbw);
        K *tk = ki; ki = ko; ko = tk;
        V *tv = vi; vi = vo; vo = tv;
        *in_alt = !*in_alt;
    }
    return SG_OK;
}

template <class K, class V>
sg_status radix_sort_pairs(K *k0, V *v0, K *k1, V *v1, int64_t n, int key_bits, bool *in_alt, cudaStream_t s,
                           uint32_t *err) {
    return radix_sort_impl<K, V, true>(k0, v0, k1, v1, n, 0, key_bits, in_alt, s, err);
}

sg_status radix_sort_keys(uint64_t *k0, uint64_t *k1, int64_t n, int lo_bit, int hi_bit, bool *in_alt,
                          cudaStream_t s, uint32_t *err) {
    return radix_sort_impl<uint64_t, uint64_t, false>(k0, nullptr, k1, nullptr, n, lo_bit, hi_bit, in_alt, s, err);
}

template sg_status radix_sort_pairs<uint64_t, uint64_t>(uint64_t *, uint64_t *, uint64_t *, uint64_t *, int64_t,
                                                        int, bool *, cudaStream_t, uint32_t *);
template sg_status radix_sort_pairs<uint32_t, uint64_t>(uint32_t *, uint64_t *, uint32_t *, uint64_t *, int64_t,
                                                        int, bool *, cudaStream_t, uint32_t *);
template sg_status radix_sort_pairs<uint32_t, uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *, int64_t,
                                                        int, bool *, cudaStream_t, uint32_t *);

}  // namespace sg
