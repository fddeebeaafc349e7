// prim.cu -- exclusive scan (reduce, scan partials, downsweep) and stable LSD radix sort
// (per-tile digit histograms, scan, stable per-warp ranking with __match_any_sync, then a
// shared-memory staged scatter so that each digit's run is written contiguously).
#include "check.cuh"
#include "prim.cuh"

namespace sg {

// ------------------------------------------------------------------------------- scan
constexpr int SCAN_NT = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_NT * SCAN_ITEMS;

template <class T>
__global__ void __launch_bounds__(SCAN_NT) scan_reduce_kernel(const T *__restrict__ in, int64_t n,
                                                             int64_t *__restrict__ partial) {
    __shared__ int64_t tmp[SCAN_NT / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t acc = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int64_t idx = base + i * SCAN_NT + threadIdx.x;
        if (idx < n) acc += (int64_t)in[idx];
    }
    int64_t total;
    block_exclusive_scan<SCAN_NT>(acc, tmp, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Scans one tile per block; adds the block's exclusive offset from `partial` (nullptr for a
// single block). The last block also writes out[n], the grand total.
template <class T>
__global__ void __launch_bounds__(SCAN_NT) scan_down_kernel(const T *in, int64_t n,
                                                           const int64_t *__restrict__ partial,
                                                           int64_t *out) {
    __shared__ int64_t vals[SCAN_TILE + SCAN_TILE / 32];
    __shared__ int64_t tmp[SCAN_NT / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    auto pad = [](int i) { return i + (i >> 5); };  // break the 8-way bank conflict of blocked reads
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int idx = i * SCAN_NT + threadIdx.x;
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
    int64_t off = partial ? partial[blockIdx.x] : 0;
    int64_t pre = block_exclusive_scan<SCAN_NT>(sum, tmp, &total) + off;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) vals[pad(threadIdx.x * SCAN_ITEMS + i)] = loc[i] + pre;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int idx = i * SCAN_NT + threadIdx.x;
        if (base + idx < n) out[base + idx] = vals[pad(idx)];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + total;
}

template <class T>
sg_status exclusive_scan(const T *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        SG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return SG_OK;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        SG_LAUNCH("scan_down", scan_down_kernel<T>, 1, SCAN_NT, 0, s, in, n, (const int64_t *)nullptr, out);
        return SG_OK;
    }
    Scratch sc(s);
    int64_t *partial = sc.get<int64_t>(nb + 1);
    if (!partial) return SG_ERR_OOM;
    SG_LAUNCH("scan_reduce", scan_reduce_kernel<T>, nb, SCAN_NT, 0, s, in, n, partial);
    SG_TRY(exclusive_scan<int64_t>(partial, partial, nb, s));
    SG_LAUNCH("scan_down", scan_down_kernel<T>, nb, SCAN_NT, 0, s, in, n, (const int64_t *)partial, out);
    return SG_OK;
}

template sg_status exclusive_scan<int64_t>(const int64_t *, int64_t *, int64_t, cudaStream_t);
template sg_status exclusive_scan<uint32_t>(const uint32_t *, int64_t *, int64_t, cudaStream_t);
template sg_status exclusive_scan<int32_t>(const int32_t *, int64_t *, int64_t, cudaStream_t);
template sg_status exclusive_scan<uint8_t>(const uint8_t *, int64_t *, int64_t, cudaStream_t);

// ------------------------------------------------------------------------- radix sort
constexpr int RS_BITS = 8;
constexpr int RS_RADIX = 1 << RS_BITS;
constexpr int RS_NT = 256;
constexpr int RS_WARPS = RS_NT / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_NT * RS_ITEMS;

template <class K>
__global__ void __launch_bounds__(RS_NT) radix_hist_kernel(const K *__restrict__ keys, int64_t n, int shift,
                                                          uint32_t *__restrict__ counts, int64_t ntiles) {
    __shared__ uint32_t hist[RS_RADIX];
    for (int d = threadIdx.x; d < RS_RADIX; d += RS_NT) hist[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t idx = base + i * RS_NT + threadIdx.x;
        if (idx < n) atomicAdd(&hist[(uint32_t)(keys[idx] >> shift) & (RS_RADIX - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_RADIX; d += RS_NT) counts[(int64_t)d * ntiles + blockIdx.x] = hist[d];
}

template <class K, class V, bool HAS_V>
struct RsSmem {
    K keys[RS_TILE];
    V vals[HAS_V ? RS_TILE : 1];
    uint32_t wcnt[RS_WARPS][RS_RADIX];
    uint32_t tstart[RS_RADIX];
    uint32_t tmp[RS_WARPS + 1];
};

// offsets[d * ntiles + t] = first output position of digit d's keys from tile t. Without values
// (HAS_V == false) vin / vout are not touched.
template <class K, class V, bool HAS_V>
__global__ void __launch_bounds__(RS_NT) radix_scatter_kernel(const K *__restrict__ kin, const V *__restrict__ vin,
                                                             K *__restrict__ kout, V *__restrict__ vout,
                                                             int64_t n, int shift,
                                                             const int64_t *__restrict__ offsets,
                                                             int64_t ntiles) {
    extern __shared__ __align__(16) unsigned char rs_raw[];
    RsSmem<K, V, HAS_V> &sm = *reinterpret_cast<RsSmem<K, V, HAS_V> *>(rs_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_NT) (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
    const int64_t wbase = tbase + (int64_t)w * 32 * RS_ITEMS;
    const uint32_t lt = (1u << lane) - 1u;
    K key[RS_ITEMS];
    V val[HAS_V ? RS_ITEMS : 1];
    uint32_t local[RS_ITEMS];
#pragma unroll
    for (int it = 0; it < RS_ITEMS; it++) {
        int64_t idx = wbase + it * 32 + lane;
        bool valid = idx < n;
        key[it] = valid ? kin[idx] : K(0);
        if (HAS_V) val[HAS_V ? it : 0] = valid ? vin[idx] : V(0);
        uint32_t d = (uint32_t)(key[it] >> shift) & (RS_RADIX - 1);
        uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : (RS_RADIX + lane));
        uint32_t base_cnt = valid ? sm.wcnt[w][d] : 0u;
        __syncwarp();
        if (valid) {
            local[it] = base_cnt + __popc(peers & lt);
            if ((peers >> lane) == 1u) sm.wcnt[w][d] = base_cnt + __popc(peers);  // highest peer lane
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive offsets across warps, then the tile's digit starts
    uint32_t tot = 0;
    for (int d = threadIdx.x; d < RS_RADIX; d += RS_NT) {
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ww++) {
            uint32_t c = sm.wcnt[ww][d];
            sm.wcnt[ww][d] = run;
            run += c;
        }
        tot = run;
    }
    uint32_t total;
    uint32_t st = block_exclusive_scan<RS_NT>(tot, sm.tmp, &total);  // RS_NT == RS_RADIX
    sm.tstart[threadIdx.x] = st;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; it++) {
        int64_t idx = wbase + it * 32 + lane;
        if (idx < n) {
            uint32_t d = (uint32_t)(key[it] >> shift) & (RS_RADIX - 1);
            uint32_t p = sm.tstart[d] + sm.wcnt[w][d] + local[it];
            if (!SG_IN_BOUNDS(p < RS_TILE, 201, p)) continue;
            sm.keys[p] = key[it];
            if (HAS_V) sm.vals[HAS_V ? p : 0] = val[HAS_V ? it : 0];
        }
    }
    __syncthreads();
    int64_t cnt = n - tbase < RS_TILE ? n - tbase : RS_TILE;
    for (int i = threadIdx.x; i < cnt; i += RS_NT) {
        K kk = sm.keys[i];
        uint32_t d = (uint32_t)(kk >> shift) & (RS_RADIX - 1);
        int64_t o = offsets[(int64_t)d * ntiles + blockIdx.x] + (i - (int64_t)sm.tstart[d]);
        if (!SG_IN_BOUNDS(o >= 0 && o < n, 202, o)) continue;
        kout[o] = kk;
        if (HAS_V) vout[o] = sm.vals[HAS_V ? i : 0];
    }
}

template <class K, class V, bool HAS_V>
static sg_status radix_sort_impl(K *k0, V *v0, K *k1, V *v1, int64_t n, int lo_bit, int hi_bit, bool *in_alt,
                                 cudaStream_t s) {
    static_assert(RS_NT == RS_RADIX, "one thread per digit in the scatter's digit scan");
    *in_alt = false;
    if (n <= 1 || hi_bit <= lo_bit) return SG_OK;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    Scratch sc(s);
    uint32_t *counts = sc.get<uint32_t>((size_t)RS_RADIX * ntiles);
    int64_t *offs = sc.get<int64_t>((size_t)RS_RADIX * ntiles + 1);
    if (!counts || !offs) return SG_ERR_OOM;
    size_t smem = sizeof(RsSmem<K, V, HAS_V>);
    SG_CUDA_TRY(ensure_smem(radix_scatter_kernel<K, V, HAS_V>, smem));
    K *ki = k0, *ko = k1;
    V *vi = v0, *vo = v1;
    for (int shift = lo_bit; shift < hi_bit; shift += RS_BITS) {
        SG_LAUNCH("radix_hist", radix_hist_kernel<K>, ntiles, RS_NT, 0, s, ki, n, shift, counts, ntiles);
        SG_TRY(exclusive_scan<uint32_t>(counts, offs, (int64_t)RS_RADIX * ntiles, s));
        SG_LAUNCH("radix_scatter", (radix_scatter_kernel<K, V, HAS_V>), ntiles, RS_NT, smem, s, ki, vi, ko, vo, n,
                  shift, (const int64_t *)offs, ntiles);
        K *tk = ki; ki = ko; ko = tk;
        V *tv = vi; vi = vo; vo = tv;
        *in_alt = !*in_alt;
    }
    return SG_OK;
}

template <class K, class V>
sg_status radix_sort_pairs(K *k0, V *v0, K *k1, V *v1, int64_t n, int key_bits, bool *in_alt, cudaStream_t s) {
    return radix_sort_impl<K, V, true>(k0, v0, k1, v1, n, 0, key_bits, in_alt, s);
}

sg_status radix_sort_keys(uint64_t *k0, uint64_t *k1, int64_t n, int lo_bit, int hi_bit, bool *in_alt,
                          cudaStream_t s) {
    return radix_sort_impl<uint64_t, uint64_t, false>(k0, nullptr, k1, nullptr, n, lo_bit, hi_bit, in_alt, s);
}

template sg_status radix_sort_pairs<uint64_t, uint64_t>(uint64_t *, uint64_t *, uint64_t *, uint64_t *, int64_t,
                                                        int, bool *, cudaStream_t);
template sg_status radix_sort_pairs<uint32_t, uint64_t>(uint32_t *, uint64_t *, uint32_t *, uint64_t *, int64_t,
                                                        int, bool *, cudaStream_t);
template sg_status radix_sort_pairs<uint32_t, uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *, int64_t,
                                                        int, bool *, cudaStream_t);

}  // namespace sg
