// runtime.cu -- error strings, allocation, launch counting and per-kernel event timing.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "check.cuh"

namespace sg {

static thread_local char g_err[1024] = "";
static thread_local sg_kmer_stats g_kstats = {};
sg_kmer_stats &kmer_stats() { return g_kstats; }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

sg_status timeout_error(const char *what) {
    set_error("%s: a bounded wait between thread blocks gave up (internal error); results discarded", what);
    return SG_ERR_TIMEOUT;
}

static std::atomic<int> g_debug_stall{0};
int debug_stall_lookback() { return g_debug_stall.load(); }

static sg_alloc_fn g_alloc = nullptr;
static sg_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;
static std::atomic<int64_t> g_fail_after{0};

// The library's own stream-ordered pool on each device. Its release threshold is unbounded, so
// memory freed at the end of one call is reused by the next instead of being unmapped at every
// synchronisation (the default pool's threshold of 0 returns it to the driver each time). The
// pool belongs to this process and disappears with it.
int64_t tune(const char *name);
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[256];
static bool g_pool_tried[256];

static cudaMemPool_t library_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_tried[dev]) {
        g_pool_tried[dev] = true;
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            int reuse = tune("pool_cross_stream_reuse") ? 1 : 0;
            cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowOpportunistic, &reuse);
            cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &reuse);
            g_pools[dev] = pool;
        } else {
            cudaGetLastError();
        }
    }
    return g_pools[dev];
}

// Multiprocessors of the current device (152 on a GB300), for grid sizes; read once per device.
int sm_count() {
    static std::atomic<int> cache[256];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return 152;
    }
    int v = cache[dev].load();
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        v = 152;
    }
    cache[dev].store(v);
    return v;
}

// Device memory a call can still obtain: free in the driver plus what the library's pool holds
// unused (the pool keeps freed memory reserved).
size_t device_bytes_available() {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaMemPool_t pool = g_alloc ? nullptr : library_pool();
    if (pool) {
        uint64_t reserved = 0, used = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            free_b += (size_t)(reserved - used);
        cudaGetLastError();
    }
    return free_b;
}

void *dalloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    int64_t f = g_fail_after.load();
    if (f > 0) {
        if (g_fail_after.fetch_sub(1) == 1) {
            set_error("device allocation of %zu bytes failed (injected)", bytes);
            return nullptr;
        }
    }
    void *p = nullptr;
    if (g_alloc) {
        p = g_alloc(bytes, (sg_stream_t)s, g_alloc_ctx);
        if (!p) set_error("device allocation of %zu bytes failed (user allocator)", bytes);
        if (p && ((uintptr_t)p & 255)) {
            set_error("user allocator returned %p, which is not 256-byte aligned", p);
            if (g_free) g_free(p, (sg_stream_t)s, g_alloc_ctx);
            return nullptr;
        }
        return p;
    }
    cudaMemPool_t pool = library_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess && pool) {
        // the pool keeps freed memory reserved; blocks freed by earlier calls may not fit this
        // request. Once this stream's frees have completed, give the unused part back and retry.
        cudaGetLastError();
        if (cudaStreamSynchronize(s) == cudaSuccess && cudaMemPoolTrimTo(pool, 0) == cudaSuccess)
            e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        size_t free_b = 0, total_b = 0;
        uint64_t reserved = 0, used = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) cudaGetLastError();
        if (pool && (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
                     cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess))
            cudaGetLastError();
        set_error("cudaMallocAsync(%zu bytes) failed: %s (device: %.1f of %.1f GB free; library pool: %.1f GB "
                  "reserved, %.1f GB in use)",
                  bytes, cudaGetErrorString(e), free_b / 1e9, total_b / 1e9, reserved / 1e9, used / 1e9);
        return nullptr;
    }
    return p;
}

void dfree(void *p, cudaStream_t s) {
    if (!p) return;
    if (g_free) {
        g_free(p, (sg_stream_t)s, g_alloc_ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

static std::mutex g_check_mu;
static std::vector<check_reader_fn> *g_check_readers;

void register_check_reader(check_reader_fn f) {
    std::lock_guard<std::mutex> lk(g_check_mu);
    if (!g_check_readers) g_check_readers = new std::vector<check_reader_fn>();
    g_check_readers->push_back(f);
}

static std::mutex g_smem_mu;
static std::map<const void *, size_t> g_smem_caps;

static std::map<const void *, size_t> g_smem_static;

// The default cap of 48 KB covers a kernel's static and dynamic shared memory together.
cudaError_t ensure_smem_cap(const void *kernel, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    auto st = g_smem_static.find(kernel);
    if (st == g_smem_static.end()) {
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
        if (e != cudaSuccess) return e;
        st = g_smem_static.emplace(kernel, fa.sharedSizeBytes).first;
    }
    if (bytes + st->second <= 48 * 1024) return cudaSuccess;
    auto it = g_smem_caps.find(kernel);
    if (it != g_smem_caps.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g_smem_caps[kernel] = bytes;
    return e;
}

cudaError_t read_back(void *host, const void *dev, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// ---------------------------------------------------------------- launch accounting
static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_prof_on{0};
static std::string g_prof_prefix;  // only kernels whose name starts with this are timed
struct PendingEvent { std::string name; cudaEvent_t a, b; };
static std::mutex g_prof_mu;
static std::vector<PendingEvent> g_pending;
static std::vector<cudaEvent_t> g_event_pool;
struct ProfTotal { int64_t launches = 0; double ms = 0.0; };
static std::map<std::string, ProfTotal> g_totals;
static std::vector<std::pair<std::string, ProfTotal>> g_snapshot;

static cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

LaunchScope::LaunchScope(const char *n, cudaStream_t s) : name(n), stream(s), slot(-1) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_prof_on.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_prof_prefix.empty() && strncmp(name, g_prof_prefix.c_str(), g_prof_prefix.size()) != 0) return;
        PendingEvent pe{name, take_event(), take_event()};
        cudaEventRecord(pe.a, s);
        g_pending.push_back(pe);
        slot = (int)g_pending.size() - 1;
    }
}

LaunchScope::~LaunchScope() {
    if (slot >= 0) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (slot < (int)g_pending.size()) cudaEventRecord(g_pending[slot].b, stream);  // unless reset meanwhile
    }
}

StageScope::StageScope(const char *name, cudaStream_t s) : stream(s), slot(-1) {
    nvtxRangePushA(name);
    if (g_prof_on.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        const std::string full = std::string("stage/") + name;
        if (!g_prof_prefix.empty() && full.compare(0, g_prof_prefix.size(), g_prof_prefix) != 0) return;
        PendingEvent pe{full, take_event(), take_event()};
        cudaEventRecord(pe.a, s);
        g_pending.push_back(pe);
        slot = (int)g_pending.size() - 1;
    }
}

StageScope::~StageScope() {
    if (slot >= 0) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (slot < (int)g_pending.size()) cudaEventRecord(g_pending[slot].b, stream);  // unless reset meanwhile
    }
    nvtxRangePop();
}

// ------------------------------------------------------------------------- tunables
struct Tunable { const char *name; int64_t value; int64_t lo, hi; };
static Tunable g_tunables[] = {
    // defaults: the autotuner's choice on a GB300 for the bacterial-scale read set
    {"bloom_bits", 8, 2, 32},             // bits of the first Bloom filter per window
    {"bloom_slice_mb", 64, 1, 1 << 20},   // B1 megabytes updated per Bloom launch
    {"bloom_max_slices", 8, 1, 1024},     // at most this many Bloom launches (slices grow beyond)
    {"bloom_unroll", 4, 4, 8},            // windows (atomics in flight) per thread per Bloom step: 4 or 8
    {"bloom_binned", 1, 0, 1},            // 1: shared-memory filter bins where they fit (else sliced)
    {"bloom_bin_kb", 128, 16, 176},       // B1 kilobytes per bin, rounded down to a power of two
                                          // (B2: a quarter of it)
    {"bloom_scatter_cfg", 0, 0, 2},       // bin scatter tile: 0 512x16, 1 256x16, 2 256x32 hashes
    {"bloom_scatter_levels", 0, 0, 2},    // passes grouping hashes by bin (0: two beyond 4096 bins)
    {"kmer_sort_buckets", 3, 0, 3},       // at most this many top code bits become candidate buckets
    {"kmer_direct_seg", 1, 0, 1},         // 1: segments and At straight from the sorted packed keys
    {"radix_match", 0, 0, 1},             // radix sort ranking: 1 one match instruction per key, 0 ballots
    {"radix_lookback", 8, 1, 8},          // radix sort look-back: predecessors read per step
    {"bloom_bin_room_pct", 112, 1, 1000}, // a bin's hash buffer, % of the mean (overflow: sliced)
    {"spgemm_fused", 1, 0, 1},            // 1: numeric pass with guessed tables, no symbolic pass
    {"spgemm_upper", 1, 0, 1},            // 1: the fused pass tabulates partners k > i only and
                                          // mirrors them (C is symmetric); 0: whole rows
    {"spgemm_at_records", 1, 0, 1},       // 1: the fused pass reads At rows as 32-byte records
    {"spgemm_smem_carveout", -1, -1, 100},// fused-pass shared-memory carveout, % (-1: the driver's)
    {"spgemm_escalate", 1, 0, 8},         // a guessed table that overflows is tried once more
                                          // 2^this times larger in shared memory (0: global memory)
    {"spgemm_mirror_rec", 1, 0, 1},       // 1: (mirror sort) U's entries copied into 32-byte records that
                                          // the mirror reads, instead of C's arrays (max_seeds <= 3)
    {"spgemm_mirror_sort", 1, 0, 1},      // 1: mirrored entries ordered by a stable radix sort by column;
                                          // 0: scattered by atomics and sorted per row
    {"spgemm_lower_smem", 4096, 1, 4096}, // (0 above) parts up to this long are sorted in shared memory
    {"spgemm_tab_warps", 64, 0, 64},      // fused-pass blocks: threads for about this many warps per SM
                                          // across the blocks that fit (0: fixed threads per table size)
    {"spgemm_tab_warps_big", 32, 1, 64},  // ... the same for tables of 4 K slots and more
    {"spgemm_sample_rows", 256, 0, 1 << 20},  // rows sampled for the fused tables' guesses (0: none)
    {"spgemm_guess_pct", 200, 1, 10000},  // guess = pct / 100 x sampled partners per A entry x entries
    {"spgemm_tmp_pct", 125, 1, 10000},    // fused temporary region = pct / 100 x sampled kept entries
                                          // (+ 4 per row); rows that find it full are redone
    {"spgemm_fused_max_mb", 65536, 0, 1 << 30},  // temporary C region above which the two passes run
                                                  // (also when it exceeds half the free memory)
    {"spgemm_filter_mode", 0, 0, 2},      // seen-twice filter: 0 never, 1 where the sample finds it
                                          // pays, 2 always (rows of spgemm_filter_work products or more)
    {"spgemm_filter_work", 1024, 0, (int64_t)1 << 40},  // fused rows with this many A entries or more
                                          // may first mark partners seen twice (0: never)
    {"spgemm_filter_log2", 17, 10, 19},   // at most 2^this bits per seen-once / seen-twice filter
    {"sym_guess_shift", 2, 0, 8},         // symbolic table guess = products >> shift
    {"spgemm_blocks_per_sm", 16, 1, 64},  // grid of each SpGEMM class launch
    {"spgemm_big_threads", 1024, 512, 1024},  // threads of numeric blocks with 4 K table slots or more
    {"tr_blocks_per_sm", 32, 1, 64},      // grid of the min-plus launch
    {"tr_warp_rows", 1, 0, 1},            // 1: min-plus products of staged rows by a warp per neighbour
    {"pool_cross_stream_reuse", 1, 0, 1}, // pool may hand memory freed on one stream to another
    {"batch_alone_kb", 64000, 0, 1 << 30},  // batched items of this many kilobases or more run on their
                                            // own (0: every item shares the union)
    {"batch_group_kb", 250000, 1, 1 << 30}, // ... the others share unions of at most this many kilobases
};
static std::mutex g_tune_mu;

int64_t tune(const char *name) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &t : g_tunables)
        if (strcmp(t.name, name) == 0) return t.value;
    return 0;
}

}  // namespace sg

namespace sg {
static thread_local bool t_record_classes = false;
static thread_local std::vector<int32_t> t_classes;
static thread_local bool t_classes_valid = false;
bool debug_record_classes() { return t_record_classes; }
std::vector<int32_t> &debug_classes() {
    t_classes_valid = true;
    return t_classes;
}
}  // namespace sg

extern "C" {

int sg_tune_set(const char *name, int64_t value) {
    std::lock_guard<std::mutex> lk(sg::g_tune_mu);
    for (auto &t : sg::g_tunables)
        if (name && strcmp(t.name, name) == 0) {
            if (value < t.lo || value > t.hi) return 0;
            t.value = value;
            return 1;
        }
    return 0;
}

int64_t sg_tune_get(const char *name) { return name ? sg::tune(name) : 0; }

const char *sg_tune_name(int idx) {
    const int n = (int)(sizeof(sg::g_tunables) / sizeof(sg::g_tunables[0]));
    return (idx >= 0 && idx < n) ? sg::g_tunables[idx].name : nullptr;
}

const char *sg_last_error(void) { return sg::g_err; }

void sg_set_allocator(sg_alloc_fn alloc, sg_free_fn release, void *ctx) {
    sg::g_alloc = alloc;
    sg::g_free = release;
    sg::g_alloc_ctx = ctx;
}

void sg_debug_fail_alloc_after(int64_t n) { sg::g_fail_after.store(n > 0 ? n : 0); }

void sg_debug_stall_lookback(int on) { sg::g_debug_stall.store(on ? 1 : 0); }

void sg_debug_record_classes(int on) {
    sg::t_record_classes = on != 0;
    sg::t_classes_valid = false;
    sg::t_classes.clear();
}

int64_t sg_debug_spgemm_classes(int32_t *host_out, int64_t n) {
    if (!sg::t_classes_valid) return -1;
    const int64_t m = std::min<int64_t>(n, (int64_t)sg::t_classes.size());
    if (host_out && m > 0) memcpy(host_out, sg::t_classes.data(), (size_t)m * sizeof(int32_t));
    return (int64_t)sg::t_classes.size();
}

void sg_free(void *d_ptr, sg_stream_t stream) { sg::dfree(d_ptr, (cudaStream_t)stream); }

uint64_t sg_launch_count(void) { return sg::g_launches.load(); }

sg_status sg_memory_stats(uint64_t *reserved, uint64_t *in_use, uint64_t *in_use_peak) {
    uint64_t r = 0, u = 0, h = 0;
    cudaMemPool_t pool = sg::g_alloc ? nullptr : sg::library_pool();
    if (pool && (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess ||
                 cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess ||
                 cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &h) != cudaSuccess)) {
        cudaGetLastError();
        sg::set_error("memory_stats: the pool cannot be queried");
        return SG_ERR_CUDA;
    }
    if (reserved) *reserved = r;
    if (in_use) *in_use = u;
    if (in_use_peak) *in_use_peak = h;
    return SG_OK;
}

void sg_memory_reset_peak(void) {
    cudaMemPool_t pool = sg::g_alloc ? nullptr : sg::library_pool();
    uint64_t zero = 0;
    if (pool && cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess) cudaGetLastError();
}

void sg_last_kmer_stats(sg_kmer_stats *out) {
    if (out) *out = sg::g_kstats;
}

uint64_t sg_debug_check(void) {
    std::lock_guard<std::mutex> lk(sg::g_check_mu);
    uint64_t first = 0;
    if (sg::g_check_readers)
        for (auto f : *sg::g_check_readers) {
            uint64_t v = f();
            if (v && !first) first = v;
        }
    return first;
}

void sg_prof_enable(int on) { sg::g_prof_on.store(on ? 1 : 0); }

void sg_prof_select(const char *name_prefix) {
    std::lock_guard<std::mutex> lk(sg::g_prof_mu);
    sg::g_prof_prefix = name_prefix ? name_prefix : "";
}

void sg_prof_reset(void) {
    std::lock_guard<std::mutex> lk(sg::g_prof_mu);
    for (auto &p : sg::g_pending) {
        sg::g_event_pool.push_back(p.a);
        sg::g_event_pool.push_back(p.b);
    }
    sg::g_pending.clear();
    sg::g_totals.clear();
    sg::g_snapshot.clear();
}

int sg_prof_collect(void) {
    std::lock_guard<std::mutex> lk(sg::g_prof_mu);
    for (auto &p : sg::g_pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto &t = sg::g_totals[p.name];
            t.launches += 1;
            t.ms += ms;
        }
        sg::g_event_pool.push_back(p.a);
        sg::g_event_pool.push_back(p.b);
    }
    sg::g_pending.clear();
    sg::g_snapshot.assign(sg::g_totals.begin(), sg::g_totals.end());
    return (int)sg::g_snapshot.size();
}

int sg_prof_entry(int idx, const char **name, int64_t *launches, double *total_ms) {
    std::lock_guard<std::mutex> lk(sg::g_prof_mu);
    if (idx < 0 || idx >= (int)sg::g_snapshot.size()) return 0;
    *name = sg::g_snapshot[idx].first.c_str();
    *launches = sg::g_snapshot[idx].second.launches;
    *total_ms = sg::g_snapshot[idx].second.ms;
    return 1;
}

}  // extern "C"
