// prim.cu -- single-pass exclusive scan and stable LSD radix sort, both with decoupled look-back
// between tiles (the radix sort: one upfront digit count for all passes, then one kernel per pass
// that ranks keys per warp with ballots and scatters from shared memory in digit order).
#include <algorithm>

#include "check.cuh"
#include "prim.cuh"

namespace sg {

template <class T>
sg_status exclusive_scan(const T *in, int64_t *out, int64_t n, cudaStream_t s, uint32_t *err) {
    return exclusive_scan_fn(ScanLoad<T>{in}, out, n, s, err);
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
                                                              uint32_t *err, int lbw, uint32_t *__restrict__ vhi,
                                                              uint32_t *__restrict__ vlo) {
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
        if (HAS_V) {
            const V v = sm.vals[HAS_V ? i : 0];
            if (vhi) {  // 64-bit values written as their two halves
                vhi[o] = (uint32_t)((uint64_t)v >> 32);
                vlo[o] = (uint32_t)v;
            } else {
                vout[o] = v;
            }
        }
    }
}

template <class K, class V, bool HAS_V>
static sg_status radix_sort_impl(K *k0, V *v0, K *k1, V *v1, int64_t n, int lo_bit, int hi_bit, bool *in_alt,
                                 cudaStream_t s, uint32_t *err, uint32_t *vhi = nullptr, uint32_t *vlo = nullptr) {
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
        uint32_t *hi = p == npass - 1 ? vhi : nullptr, *lo = p == npass - 1 ? vlo : nullptr;
        if (match)
            SG_LAUNCH("radix_onesweep", (radix_onesweep_kernel<K, V, HAS_V, true>), ntiles, RS_NT, smem, s,
                      (const K *)ki, (const V *)vi, ko, vo, n, lo_bit + RS_BITS * p,
                      (const unsigned long long *)(ghist + p * RS_RADIX), status + (size_t)p * ntiles * RS_RADIX,
                      ctr + p, err, lbw, hi, lo);
        else
            SG_LAUNCH("radix_onesweep", (radix_onesweep_kernel<K, V, HAS_V, false>), ntiles, RS_NT, smem, s,
                      (const K *)ki, (const V *)vi, ko, vo, n, lo_bit + RS_BITS * p,
                      (const unsigned long long *)(ghist + p * RS_RADIX), status + (size_t)p * ntiles * RS_RADIX,
                      ctr + p, err, lbw, hi, lo);
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

sg_status radix_sort_pairs_split(uint32_t *k0, uint64_t *v0, uint32_t *k1, uint64_t *v1, int64_t n, int key_bits,
                                 bool *in_alt, uint32_t *vhi, uint32_t *vlo, cudaStream_t s, uint32_t *err) {
    if (n <= 1 || key_bits <= 0) {
        set_error("internal: split radix sort of %lld pairs on %d bits", (long long)n, key_bits);
        return SG_ERR_INVALID;
    }
    return radix_sort_impl<uint32_t, uint64_t, true>(k0, v0, k1, v1, n, 0, key_bits, in_alt, s, err, vhi, vlo);
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
