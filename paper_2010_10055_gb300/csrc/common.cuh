// common.cuh -- shared runtime pieces of the sm_103a library: status plumbing, stream-ordered
// allocation, launch accounting and per-kernel event timing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/sgraph.h"

namespace sg {

// Record a printf-style description of the current error for sg_last_error().
void set_error(const char *fmt, ...);

// Device allocation through the installed allocator (default cudaMallocAsync on `s`).
// Returns nullptr and records an error on failure. bytes == 0 allocates 16 bytes so that the
// result is always a valid, distinct pointer.
void *dalloc(size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);

// Launch bookkeeping: counts launches and, while profiling is on, brackets them with events.
struct LaunchScope {
    const char *name;
    cudaStream_t stream;
    int slot;
    LaunchScope(const char *name, cudaStream_t s);
    ~LaunchScope();
};

// A stage of the method (the paper's stage names: CountKmer, CreateSpMat, SpGEMMSymbolic,
// SpGEMMNumeric, TrReduction, TrRound): an NVTX range on the host, and while profiling is on, a
// pair of events on `s` reported by sg_prof_collect as "stage/<name>".
struct StageScope {
    cudaStream_t stream;
    int slot;
    StageScope(const char *name, cudaStream_t s);
    ~StageScope();
    StageScope(const StageScope &) = delete;
    StageScope &operator=(const StageScope &) = delete;
};

// Scoped set of temporary device buffers, released (stream-ordered) in reverse order on scope
// exit. Not copyable: a copy would free the same buffers twice.
struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) { ptrs.reserve(32); }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    template <class T> T *get(size_t count) {
        void *p = dalloc(count * sizeof(T), s);
        if (p) ptrs.push_back(p);
        return (T *)p;
    }
    // releases one buffer before scope exit (stream-ordered: later work may reuse its memory)
    void release(const void *p) {
        for (size_t i = ptrs.size(); i-- > 0;)
            if (ptrs[i] == p) {
                dfree(ptrs[i], s);
                ptrs.erase(ptrs.begin() + (std::ptrdiff_t)i);
                return;
            }
    }
    ~Scratch() { for (size_t i = ptrs.size(); i-- > 0;) dfree(ptrs[i], s); }
};

// Records that a bounded wait between thread blocks gave up during `what` and returns
// SG_ERR_TIMEOUT.
sg_status timeout_error(const char *what);

// Test hook (sg_debug_stall_lookback): nonzero makes multi-tile scans withhold tile 0's prefix.
int debug_stall_lookback();

// Multiprocessors of the current device, for grid sizes.
int sm_count();

// Device memory a call can still obtain (driver free + unused memory held by the library's pool).
size_t device_bytes_available();

// The calling thread's last k-mer build sizes (sg_last_kmer_stats).
sg_kmer_stats &kmer_stats();

// Test hook (sg_debug_record_classes): whether to record, and the calling thread's record of,
// the numeric launch that handled each row of the last fused overlap product.
bool debug_record_classes();
std::vector<int32_t> &debug_classes();

// Current value of a tunable parameter (see sg_tune_set).
int64_t tune(const char *name);

// Copy one device value to the host and wait for it.
cudaError_t read_back(void *host, const void *dev, size_t bytes, cudaStream_t s);

// Makes sure `kernel` may be launched with `bytes` of dynamic shared memory. The cap is a
// process-wide function attribute: it is raised once per kernel under a lock (never lowered, never
// rewritten while other host threads may be launching the kernel), and later calls only consult
// a registry.
cudaError_t ensure_smem_cap(const void *kernel, size_t bytes);
template <class K>
inline cudaError_t ensure_smem(K kernel, size_t bytes) {
    return ensure_smem_cap(reinterpret_cast<const void *>(kernel), bytes);
}

// Whether a launch grid has any blocks.
inline bool grid_ok(int64_t g) { return g > 0; }
inline bool grid_ok(dim3 g) { return g.x > 0 && g.y > 0 && g.z > 0; }

// The device-side error word used by validation kernels (one per call, zeroed first).
// DEV_TIMEOUT: a bounded wait between thread blocks gave up (never expected; the call fails
// instead of hanging).
enum : uint32_t { DEV_OK = 0, DEV_INVALID = 1, DEV_OVERFLOW = 2, DEV_TIMEOUT = 4 };

}  // namespace sg

#define SG_CUDA_TRY(call)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            sg::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #call,                    \
                          cudaGetErrorString(e_));                                              \
            return SG_ERR_CUDA;                                                                 \
        }                                                                                       \
    } while (0)

// Launch `kernel<<<grid, block, smem, stream>>>(args...)` with accounting; returns SG_ERR_CUDA
// from the enclosing function if the launch is rejected.
#define SG_LAUNCH(name, kernel, grid, block, smem, stream, ...)                                 \
    do {                                                                                        \
        if (sg::grid_ok(grid)) {                                                                \
            sg::LaunchScope ls_(name, stream);                                                  \
            kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                         \
        }                                                                                       \
        cudaError_t e_ = cudaGetLastError();                                                    \
        if (e_ != cudaSuccess) {                                                                \
            sg::set_error("%s:%d: launch of %s failed: %s", __FILE__, __LINE__, name,           \
                          cudaGetErrorString(e_));                                              \
            return SG_ERR_CUDA;                                                                 \
        }                                                                                       \
    } while (0)

#define SG_TRY(expr)                                                                            \
    do {                                                                                        \
        sg_status st_ = (expr);                                                                 \
        if (st_ != SG_OK) return st_;                                                           \
    } while (0)

#define SG_ALLOC(ptr, type, count, stream)                                                      \
    do {                                                                                        \
        ptr = (type *)sg::dalloc((size_t)(count) * sizeof(type), stream);                       \
        if (!ptr) return SG_ERR_OOM;                                                            \
    } while (0)
