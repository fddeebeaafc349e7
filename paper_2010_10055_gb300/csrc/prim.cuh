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

// Stable LSD radix sort of (keys, vals) by the low `key_bits` bits of the key. Buffers are
// ping-ponged between (k0, v0) and (k1, v1); on return *in_alt says whether the sorted data is
// in (k1, v1). Key bits above the last 8-bit digit that covers key_bits must be zero.
template <class K, class V>
sg_status radix_sort_pairs(K *k0, V *v0, K *k1, V *v1, int64_t n, int key_bits, bool *in_alt,
                           cudaStream_t s, uint32_t *err);

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

}  // namespace sg
