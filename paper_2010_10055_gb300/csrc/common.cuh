// common.cuh -- shared runtime pieces of the sm_103a library: status plumbing, stream-ordered
// allocation, launch accounting and per-kernel event timing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

// Scoped set of temporary device buffers, released in reverse order on scope exit.
struct Scratch {
    cudaStream_t s;
    void *ptrs[128];
    int n = 0;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <class T> T *get(size_t count) {
        if (n == 128) { set_error("internal: scratch table full"); return nullptr; }
        void *p = dalloc(count * sizeof(T), s);
        if (p) ptrs[n++] = p;
        return (T *)p;
    }
    ~Scratch() { for (int i = n - 1; i >= 0; --i) dfree(ptrs[i], s); }
};

// Current value of a tunable parameter (see sg_tune_set).
int64_t tune(const char *name);

// Copy one device value to the host and wait for it.
cudaError_t read_back(void *host, const void *dev, size_t bytes, cudaStream_t s);

// Whether a launch grid has any blocks.
inline bool grid_ok(int64_t g) { return g > 0; }
inline bool grid_ok(dim3 g) { return g.x > 0 && g.y > 0 && g.z > 0; }

// The device-side error word used by validation kernels (one per call, zeroed first).
enum : uint32_t { DEV_OK = 0, DEV_INVALID = 1, DEV_OVERFLOW = 2 };

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
