// check.cuh -- device-side bounds checks of the checked build.
//
// In a build compiled with -DSG_CHECKED, SG_IN_BOUNDS(cond, site) evaluates `cond`; when it is
// false the kernel records (site, index) in a per-file device word and the guarded access is
// skipped, so a bad index is reported instead of faulting. sg_debug_check() reads and clears the
// words of every file. In the normal build SG_IN_BOUNDS is `true` and compiles away.
#pragma once

#include <stdint.h>

namespace sg {

// first violation seen in this translation unit: site << 40 | (index & (2^40 - 1)), 0 = none
static __device__ unsigned long long g_check_word;

__device__ __forceinline__ bool check_ok(bool cond, int site, int64_t idx) {
    if (!cond) atomicCAS(&g_check_word, 0ull, ((unsigned long long)site << 40) | ((unsigned long long)idx & ((1ull << 40) - 1)));
    return cond;
}

// Host side: every file that includes this header registers a reader of its own word.
typedef unsigned long long (*check_reader_fn)();
void register_check_reader(check_reader_fn f);

static unsigned long long read_and_clear_check_word() {
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_check_word, sizeof(v)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_check_word, &z, sizeof(z));
    return v;
}

namespace {
struct CheckRegistrar {
    CheckRegistrar() { register_check_reader(&read_and_clear_check_word); }
};
static CheckRegistrar g_check_registrar;
}  // namespace

}  // namespace sg

#ifdef SG_CHECKED
#define SG_IN_BOUNDS(cond, site, idx) ::sg::check_ok((cond), (site), (int64_t)(idx))
#else
#define SG_IN_BOUNDS(cond, site, idx) true
#endif
