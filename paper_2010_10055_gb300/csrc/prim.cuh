// prim.cuh -- device primitives: exclusive scan and stable LSD radix sort of key/value pairs.
#pragma once

#include "common.cuh"

namespace sg {

// Both primitives coordinate their tiles by bounded waits; if one ever gives up it ORs
// DEV_TIMEOUT into *err (a device word the caller reads back; may be nullptr) and the results are
// not valid. Enqueued on `s`; temporaries come from the stream-ordered allocator.

// out[0..n] = exclusive prefix sums of in[0..n-1]; out[n] = total (< 2^62). `out` may alias `in`
// only when T is int64_t.
template <class T>
sg_status exclusive_scan(const T *in, int64_t *out, int64_t n, cudaStream_t s, uint32_t *err);

// The same scan over values computed on the fly: item i is ld(i) (a device functor returning a
// non-negative int64_t, called once per item, consecutive threads on consecutive items).
template <class Ld>
sg_status exclusive_scan_fn(Ld ld, int64_t *out, int64_t n, cudaStream_t s, uint32_t *err);

// Stable LSD radix sort of (keys, vals) by the low `key_bits` bits of the key. Buffers are
// ping-ponged between (k0, v0) and (k1, v1); on return *in_alt says whether the sorted data is
// in (k1, v1). Key bits above the last 8-bit digit that covers key_bits must be zero.
template <class K, class V>
sg_status radix_sort_pairs(K *k0, V *v0, K *k1, V *v1, int64_t n, int key_bits, bool *in_alt,
                           cudaStream_t s, uint32_t *err);

// radix_sort_pairs for 32-bit keys and 64-bit values whose last pass writes each value as two
// 32-bit halves, vhi[i] = v >> 32 and vlo[i] = (uint32_t)v (n entries each), instead of to v0/v1;
// the sorted keys end as radix_sort_pairs says. Needs n > 1 and key_bits > 0 (at least one pass).
sg_status radix_sort_pairs_split(uint32_t *k0, uint64_t *v0, uint32_t *k1, uint64_t *v1, int64_t n, int key_bits,
                                 bool *in_alt, uint32_t *vhi, uint32_t *vlo, cudaStream_t s, uint32_t *err);

// Stable LSD radix sort of 64-bit keys by their bits [lo_bit, hi_bit) (other bits ride along;
// bits above hi_bit up to the last digit's end must be zero).
sg_status radix_sort_keys(uint64_t *k0, uint64_t *k1, int64_t n, int lo_bit, int hi_bit, bool *in_alt,
                          cudaStream_t s, uint32_t *err);

// Block-wide exclusive scan of one value per thread (blockDim.x = NT, a multiple of 32).
// `tmp` must hold NT/32 + 1 values. Returns the exclusive prefix; *total gets the block total.
template <int NT, class T>
__device__ __forceinline__ T block_exclusive_scan(T x, T *tmp, T *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) tmp[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = (lane < NT / 32) ? tmp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NT / 32) tmp[lane] = t;  // inclusive warp totals
        if (lane == NT / 32 - 1) tmp[NT / 32] = t;
    }
    __syncthreads();
    T excl = v - x + (w > 0 ? tmp[w - 1] : T(0));
    *total = tmp[NT / 32];
    __syncthreads();
    return excl;
}

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

// Item loader of the plain scan: in[i] widened to int64_t.
template <class T>
struct ScanLoad {
    const T *in;
    __device__ __forceinline__ int64_t operator()(int64_t i) const { return (int64_t)in[i]; }
};

// stall != 0 (test hook, sg_debug_stall_lookback): tile 0 withholds its prefix, so the waits of
// the tiles after it run out.
template <class Ld>
__global__ void __launch_bounds__(SCAN_NT) scan_kernel(Ld ld, int64_t n, int64_t *out, unsigned long long *status,
                                                      unsigned int *tile_ctr, uint32_t *err, int stall) {
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
        vals[pad(idx)] = (base + idx < n) ? ld(base + idx) : 0;
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

template <class Ld>
sg_status exclusive_scan_fn(Ld ld, int64_t *out, int64_t n, cudaStream_t s, uint32_t *err) {
    if (n <= 0) {
        SG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return SG_OK;
    }
    const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nt == 1) {
        SG_LAUNCH("scan", scan_kernel<Ld>, 1, SCAN_NT, 0, s, ld, n, out, (unsigned long long *)nullptr,
                  (unsigned int *)nullptr, err, 0);
        return SG_OK;
    }
    Scratch sc(s);
    unsigned long long *status = sc.get<unsigned long long>(nt + 1);  // [nt] status, then the tile counter
    if (!status) return SG_ERR_OOM;
    SG_CUDA_TRY(cudaMemsetAsync(status, 0, (size_t)(nt + 1) * sizeof(unsigned long long), s));
    SG_LAUNCH("scan", scan_kernel<Ld>, nt, SCAN_NT, 0, s, ld, n, out, status, (unsigned int *)(status + nt), err,
              debug_stall_lookback());
    return SG_OK;
}

}  // namespace sg
