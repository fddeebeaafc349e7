// tr.cu -- transitive reduction of the bidirected overlap graph R (Algorithm 1, Sec. IV-E) with
// the MinPlus semiring of Algorithm 3, on the GPU.
//
// One round, for every row i in one thread block:
//   N_ik = min over j of R_ij + R_jk, over walks i->j->k that are valid (the two heads at j
//          point opposite ways: in(d_ij) == out(d_jk), Sec. II) -- only for k with R_ik present,
//          since Algorithm 1 compares M and N only where both exist;
//   v_i  = max_k R_ik + fuzz                                   (Reduce(Row, max), Apply(+x));
//   I_ik = N_ik exists, its end orientations equal d_ik (rules (b), (c) of Sec. II), and
//          v_i >= N_ik                                        (M >= N with M = DimApply(Row, v));
//   R    = R minus I                                          (R o not I).
// The round's result is a keep flag per entry; a stable compaction builds the next R. Rounds
// repeat until nnz(R) does not change.
//
// Direction encoding: d = 2 * o_first + o_second (o = 1: the read is traversed reverse-
// complemented). in(d) = d & 1, out(d) = d >> 1; the walk's composite dir is
// 2 * out(d_ij) + in(d_jk). N is kept as (sum << 2 | composite) in one 64-bit word so that
// DIRMATCH (composite must equal d_ik before the min) and LITERAL (lexicographic min of
// (sum, composite), checked after) share one atomicMin.
#include "check.cuh"
#include "ops.cuh"

namespace sg {

constexpr int TR_NT = 128;
constexpr int TR_SMEM_ROW = 1024;  // rows up to this degree stage their entries in shared memory
constexpr unsigned long long TR_NONE = ~0ull;

struct TrGraph {
    const int64_t *rp;
    const int32_t *col;
    const uint32_t *suf;
    const uint8_t *dir;
    int64_t n;
};

__global__ void validate_graph_kernel(TrGraph g, int64_t nnz, uint32_t *__restrict__ err) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row > g.n) return;
    if (row == g.n) {
        if (lane == 0 && (g.rp[g.n] != nnz || g.rp[0] != 0)) atomicOr(err, (uint32_t)DEV_INVALID);
        return;
    }
    int64_t r0 = g.rp[row], r1 = g.rp[row + 1];
    if (r1 < r0 || r0 < 0 || r1 > nnz) {
        if (lane == 0) atomicOr(err, (uint32_t)DEV_INVALID);
        return;
    }
    bool bad = false;
    for (int64_t e = r0 + lane; e < r1; e += 32) {
        int32_t c = g.col[e];
        if (c < 0 || c >= g.n || c == row) bad = true;
        if (e > r0 && g.col[e - 1] >= c) bad = true;
        if (g.suf[e] >= (1u << 30) || g.dir[e] > 3) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, (uint32_t)DEV_INVALID);
}

// index of k in the sorted cols[0..deg), or -1
__device__ __forceinline__ int64_t find_col(const int32_t *cols, int64_t deg, int32_t k) {
    int64_t lo = 0, hi = deg;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (cols[mid] < k) lo = mid + 1; else hi = mid;
    }
    return (lo < deg && cols[lo] == k) ? lo : -1;
}

// One block per row. GMEM: the row is read in place from global memory and the per-entry
// minima live in `gbest` (indexed by entry); otherwise the row is staged in shared memory.
template <bool GMEM>
__global__ void __launch_bounds__(TR_NT) minplus_mark_kernel(TrGraph g, const int32_t *__restrict__ rows,
                                                            const unsigned long long *__restrict__ nrows_p,
                                                            const uint32_t *__restrict__ err, int mode, uint32_t fuzz,
                                                            unsigned long long *__restrict__ gbest,
                                                            int64_t *__restrict__ gpre,
                                                            uint8_t *__restrict__ keep, int64_t *__restrict__ kept,
                                                            uint32_t *__restrict__ outN, uint8_t *__restrict__ outD,
                                                            int warp_rows) {
    __shared__ int32_t s_col[GMEM ? 1 : TR_SMEM_ROW];
    __shared__ uint32_t s_suf[GMEM ? 1 : TR_SMEM_ROW];
    __shared__ uint8_t s_dir[GMEM ? 1 : TR_SMEM_ROW];
    __shared__ unsigned long long s_best[GMEM ? 1 : TR_SMEM_ROW];
    __shared__ int64_t s_pre[GMEM ? 1 : TR_SMEM_ROW + 1];
    __shared__ int64_t s_tmp[TR_NT / 32 + 1];
    __shared__ uint32_t s_red[2 * (TR_NT / 32)];
    __shared__ int64_t s_kept[TR_NT / 32];
    if (*err) return;  // the graph failed validation: touch nothing
    const int64_t nrows = (int64_t)*nrows_p;
    for (int64_t rb = blockIdx.x; rb < nrows; rb += gridDim.x) {
        const int32_t i = rows[rb];
        if (!SG_IN_BOUNDS(i >= 0 && i < g.n, 404, i)) continue;
        const int64_t r0 = g.rp[i], r1 = g.rp[i + 1], deg = r1 - r0;
        const int32_t *col = GMEM ? g.col + r0 : s_col;
        const uint32_t *suf = GMEM ? g.suf + r0 : s_suf;
        const uint8_t *dir = GMEM ? g.dir + r0 : s_dir;
        unsigned long long *best = GMEM ? gbest + r0 : s_best;
        int64_t *pre = GMEM ? gpre + r0 + i : s_pre;  // deg + 1 slots per row
        // stage row i and the exclusive prefix of its neighbours' degrees; the row max per read
        // end of i (out(d)), folded into one for the whole-row form
        uint32_t vmax0 = 0, vmax1 = 0;
        int64_t run = 0;
        for (int64_t base = 0; base < deg; base += TR_NT) {
            int64_t a = base + threadIdx.x;
            int64_t dj = 0;
            if (a < deg) {
                int32_t j = g.col[r0 + a];
                uint32_t sv = g.suf[r0 + a];
                const uint8_t da = g.dir[r0 + a];
                if (!GMEM) {
                    s_col[a] = j;
                    s_suf[a] = sv;
                    s_dir[a] = da;
                }
                best[a] = TR_NONE;
                if (da >> 1) vmax1 = sv > vmax1 ? sv : vmax1;
                else vmax0 = sv > vmax0 ? sv : vmax0;
                dj = g.rp[j + 1] - g.rp[j];
            }
            int64_t tot;
            int64_t ex = block_exclusive_scan<TR_NT>(dj, s_tmp, &tot);
            if (a < deg) pre[a] = run + ex;
            run += tot;
        }
        if (threadIdx.x == 0) pre[deg] = run;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            uint32_t y = __shfl_xor_sync(0xffffffffu, vmax0, o);
            vmax0 = y > vmax0 ? y : vmax0;
            y = __shfl_xor_sync(0xffffffffu, vmax1, o);
            vmax1 = y > vmax1 ? y : vmax1;
        }
        if ((threadIdx.x & 31) == 0) {
            s_red[2 * (threadIdx.x >> 5)] = vmax0;
            s_red[2 * (threadIdx.x >> 5) + 1] = vmax1;
        }
        __syncthreads();
        const int64_t P = pre[deg];
        // N = R^2 on the pattern of row i: a warp per neighbour j walking j's row (staged rows,
        // warp_rows), or every thread on the flattened products, each finding its neighbour by a
        // search of the degree prefix
        if (!GMEM && warp_rows) {
            const int lane = threadIdx.x & 31;
            for (int64_t a = threadIdx.x >> 5; a < deg; a += TR_NT / 32) {
                const int32_t j = col[a];
                const int64_t jb = g.rp[j], je = g.rp[j + 1];
                const uint32_t dij = dir[a], sa = suf[a];
                for (int64_t b = jb + lane; b < je; b += 32) {
                    const int32_t k = g.col[b];
                    if (k == i) continue;
                    const int64_t t = find_col(col, deg, k);
                    if (t < 0) continue;
                    const uint32_t djk = g.dir[b];
                    if ((dij & 1u) != (djk >> 1)) continue;  // heads at j must point opposite ways
                    const uint32_t comp = (dij & 2u) | (djk & 1u);
                    if ((mode & 1) == SG_TR_DIRMATCH && comp != dir[t]) continue;
                    const unsigned long long key = ((unsigned long long)(sa + g.suf[b]) << 2) | comp;
                    atomicMin(best + t, key);
                }
            }
        } else
        for (int64_t p = threadIdx.x; p < P; p += TR_NT) {
            int64_t lo = 0, hi = deg;  // entry a with pre[a] <= p < pre[a + 1]
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) >> 1;
                if (pre[mid] <= p) lo = mid; else hi = mid;
            }
            const int64_t a = lo;
            const int32_t j = col[a];
            const int64_t b = g.rp[j] + (p - pre[a]);
            const int32_t k = g.col[b];
            if (k == i) continue;
            const int64_t t = find_col(col, deg, k);
            if (t < 0) continue;
            const uint32_t dij = dir[a], djk = g.dir[b];
            if ((dij & 1u) != (djk >> 1)) continue;  // heads at j must point opposite ways
            const uint32_t comp = (dij & 2u) | (djk & 1u);
            if ((mode & 1) == SG_TR_DIRMATCH && comp != dir[t]) continue;
            const unsigned long long key = ((unsigned long long)(suf[a] + g.suf[b]) << 2) | comp;
            atomicMin(best + t, key);
        }
        __syncthreads();
        uint32_t vm[2] = {0u, 0u};
        for (int w = 0; w < TR_NT / 32; w++)
            for (int e = 0; e < 2; e++) vm[e] = s_red[2 * w + e] > vm[e] ? s_red[2 * w + e] : vm[e];
        const bool per_end = (mode & SG_TR_PER_END) != 0;
        const uint32_t vrow = vm[0] > vm[1] ? vm[0] : vm[1];
        const uint64_t v0 = (uint64_t)(per_end ? vm[0] : vrow) + fuzz;  // M_ik: the bound of end 0
        const uint64_t v1 = (uint64_t)(per_end ? vm[1] : vrow) + fuzz;  // ... and of end 1
        int64_t mykept = 0;
        for (int64_t t = threadIdx.x; t < deg; t += TR_NT) {
            const unsigned long long bt = best[t];
            const uint32_t d = dir[t];
            const bool has = bt != TR_NONE;
            const uint64_t N = bt >> 2;
            const bool transitive = has && (uint32_t)(bt & 3u) == d && ((d >> 1) ? v1 : v0) >= N;
            if (keep) keep[r0 + t] = transitive ? 0 : 1;
            mykept += transitive ? 0 : 1;
            if (outN) outN[r0 + t] = has ? (uint32_t)N : 0xFFFFFFFFu;
            if (outD) outD[r0 + t] = has ? (uint8_t)(bt & 3u) : (uint8_t)d;
        }
        if (kept) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mykept += __shfl_xor_sync(0xffffffffu, mykept, o);
            if ((threadIdx.x & 31) == 0) s_kept[threadIdx.x >> 5] = mykept;
            __syncthreads();
            if (threadIdx.x == 0) {
                int64_t a = 0;
                for (int w = 0; w < TR_NT / 32; w++) a += s_kept[w];
                kept[i] = a;
            }
        }
        __syncthreads();
    }
}

// rows of each kind: 0 = empty, 1 = staged in shared memory, 2 = global memory
__global__ void tr_bin_kernel(const int64_t *__restrict__ rp, int64_t n, unsigned long long *__restrict__ counts,
                              int8_t *__restrict__ kind) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t d = rp[i + 1] - rp[i];
    int8_t c = d == 0 ? 0 : (d <= TR_SMEM_ROW ? 1 : 2);
    kind[i] = c;
    atomicAdd(counts + c, 1ull);
}

// rows[0 .. n) lists the shared-memory rows, rows[n .. 2n) the global-memory rows
__global__ void tr_fill_kernel(const int8_t *__restrict__ kind, int64_t n, unsigned long long *__restrict__ cursor,
                               int32_t *__restrict__ rows) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = kind[i];
    if (c == 0) return;
    unsigned long long p = atomicAdd(cursor + c, 1ull);
    if (SG_IN_BOUNDS((int64_t)p < n, 403, p)) rows[(c == 1 ? 0 : n) + (int64_t)p] = (int32_t)i;
}

// Stable compaction of kept entries: one warp per row.
__global__ void tr_compact_kernel(TrGraph g, const uint8_t *__restrict__ keep, const int64_t *__restrict__ nrp,
                                  int32_t *__restrict__ ocol, uint32_t *__restrict__ osuf,
                                  uint8_t *__restrict__ odir) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= g.n) return;
    int64_t r0 = g.rp[row], r1 = g.rp[row + 1], w = nrp[row];
    for (int64_t base = r0; base < r1; base += 32) {
        int64_t e = base + lane;
        bool kp = e < r1 && keep[e];
        uint32_t bal = __ballot_sync(0xffffffffu, kp);
        if (kp) {
            int64_t o = w + __popc(bal & ((1u << lane) - 1u));
            ocol[o] = g.col[e];
            osuf[o] = g.suf[e];
            odir[o] = g.dir[e];
        }
        w += __popc(bal);
    }
}

static inline int64_t blocks_for(int64_t n, int nt) { return (n + nt - 1) / nt; }

// Buffers reused by every round (sized for the input graph; later rounds only shrink).
struct TrWork {
    unsigned long long *counts;  // [6]: rows per kind, then fill cursors
    int8_t *kind;                // [n + 1]
    int32_t *rows;               // [2 (n + 1)]: shared-memory rows from 0, global-memory rows from n
    unsigned long long *gbest;   // [nnz + 1] per-entry minima of global-memory rows
    int64_t *gpre;               // [nnz + n + 1] neighbour-degree prefixes of global-memory rows
};

// Element counts of TrWork's arrays for a graph of n rows and nnz entries, in field order. Both
// the allocating path and the fixed-workspace path size their buffers from this one table.
struct TrWorkSizes {
    int64_t counts, kind, rows, gbest, gpre;
};
static TrWorkSizes tr_work_sizes(int64_t n, int64_t nnz) {
    return TrWorkSizes{6, n + 1, 2 * (n + 1), nnz + 1, nnz + n + 1};
}

static sg_status tr_work_alloc(TrWork *w, int64_t n, int64_t nnz, Scratch &sc) {
    const TrWorkSizes z = tr_work_sizes(n, nnz);
    w->counts = sc.get<unsigned long long>(z.counts);
    w->kind = sc.get<int8_t>(z.kind);
    w->rows = sc.get<int32_t>(z.rows);
    w->gbest = sc.get<unsigned long long>(z.gbest);
    w->gpre = sc.get<int64_t>(z.gpre);
    return (w->counts && w->kind && w->rows && w->gbest && w->gpre) ? SG_OK : SG_ERR_OOM;
}

// One round over graph g: keep flags + per-row kept counts (and optionally N / Ndir). Rows are
// binned on the device and both kernels run grid-stride over the device-side row counts, so the
// round needs no host round trip. Nothing runs past a set `err` (failed validation).
static sg_status minplus_round(const TrGraph &g, int64_t nnz, int mode, uint32_t fuzz, uint8_t *keep,
                               int64_t *kept, uint32_t *outN, uint8_t *outD, const TrWork &w, const uint32_t *err,
                               cudaStream_t s) {
    (void)nnz;
    const int64_t n = g.n;
    unsigned long long *counts = w.counts;
    SG_CUDA_TRY(cudaMemsetAsync(counts, 0, 6 * sizeof(unsigned long long), s));
    if (kept) SG_CUDA_TRY(cudaMemsetAsync(kept, 0, (n + 1) * sizeof(int64_t), s));
    if (n == 0) return SG_OK;
    SG_LAUNCH("tr_bin", tr_bin_kernel, blocks_for(n, 256), 256, 0, s, g.rp, n, counts, w.kind);
    SG_LAUNCH("tr_fill", tr_fill_kernel, blocks_for(n, 256), 256, 0, s, w.kind, n, counts + 3, w.rows);
    const int64_t gcap = (int64_t)sm_count() * tune("tr_blocks_per_sm");
    const int64_t gs = n < gcap ? n : gcap;
    SG_LAUNCH("tr_minplus_mark", minplus_mark_kernel<false>, gs, TR_NT, 0, s, g, (const int32_t *)w.rows,
              counts + 1, err, mode, fuzz, (unsigned long long *)nullptr, (int64_t *)nullptr, keep, kept, outN,
              outD, (int)tune("tr_warp_rows"));
    const int64_t gg = n < (int64_t)sm_count() * 2 ? n : (int64_t)sm_count() * 2;
    SG_LAUNCH("tr_minplus_mark_gmem", minplus_mark_kernel<true>, gg, TR_NT, 0, s, g, (const int32_t *)(w.rows + n),
              counts + 2, err, mode, fuzz, w.gbest, w.gpre, keep, kept, outN, outD, 0);
    return SG_OK;
}

static void free_graph_arrays(sg_graph_csr *x, cudaStream_t s) {
    dfree(x->row_ptr, s);
    dfree(x->col, s);
    dfree(x->suffix, s);
    dfree(x->dir, s);
    *x = sg_graph_csr{};
}

// Batches: job_last[b] = max(job_last[b], round) for every job b that lost an entry this round.
__global__ void job_changes_kernel(const int64_t *__restrict__ rp, const int64_t *__restrict__ kept, int64_t n,
                                   const int64_t *__restrict__ job_ro, int64_t njobs, int32_t round,
                                   int32_t *__restrict__ job_last) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (rp[i + 1] - rp[i]) == kept[i]) return;
    int64_t lo = 0, hi = njobs;  // last job b with job_ro[b] <= i
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (job_ro[mid] <= i) lo = mid; else hi = mid;
    }
    atomicMax(job_last + lo, round);
}

sg_status tr_impl(const sg_graph_csr *R, uint32_t fuzz, int mode, sg_graph_csr *S, int32_t *iters,
                  cudaStream_t s, const int64_t *job_ro, int64_t njobs, int32_t *job_last, int32_t max_rounds,
                  int32_t *converged) {
    const int64_t n = R->n, nnz0 = R->nnz;
    StageScope stage("TrReduction", s);
    Scratch sc(s);
    uint32_t *err = sc.get<uint32_t>(1);
    uint8_t *keep = sc.get<uint8_t>(nnz0 + 1);
    int64_t *kept = sc.get<int64_t>(n + 1);
    if (!err || !keep || !kept) return SG_ERR_OOM;
    TrWork wk;
    SG_TRY(tr_work_alloc(&wk, n, nnz0, sc));
    // two graph buffers of the input's size: round r reads one and compacts into the other
    int64_t *rp[2];
    int32_t *col[2];
    uint32_t *suf[2];
    uint8_t *dir[2];
    for (int b = 0; b < 2; b++) {
        rp[b] = sc.get<int64_t>(n + 1);
        col[b] = sc.get<int32_t>(nnz0 + 1);
        suf[b] = sc.get<uint32_t>(nnz0 + 1);
        dir[b] = sc.get<uint8_t>(nnz0 + 1);
        if (!rp[b] || !col[b] || !suf[b] || !dir[b]) return SG_ERR_OOM;
    }
    TrGraph g{R->row_ptr, R->col, R->suffix, R->dir, n};
    SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    SG_LAUNCH("validate_graph", validate_graph_kernel, blocks_for((n + 1) * 32, 256), 256, 0, s, g, nnz0, err);
    int64_t cur_nnz = nnz0;
    int cur = -1;  // -1: the current graph is still the caller's R
    int32_t it = 0;
    bool done = false;
    for (;;) {
        if (max_rounds > 0 && it == max_rounds) break;  // stopped early: S is an intermediate R
        it++;
        StageScope round("TrRound", s);
        const int nxt = cur == 0 ? 1 : 0;
        SG_TRY(minplus_round(g, cur_nnz, mode, fuzz, keep, kept, nullptr, nullptr, wk, err, s));
        if (job_ro)
            SG_LAUNCH("tr_job_changes", job_changes_kernel, blocks_for(n, 256), 256, 0, s, g.rp,
                      (const int64_t *)kept, n, job_ro, njobs, it, job_last);
        SG_TRY(exclusive_scan<int64_t>(kept, rp[nxt], n, s, err));
        int64_t nnz2 = 0;
        uint32_t herr = 0;
        SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(read_back(&nnz2, rp[nxt] + n, sizeof(int64_t), s));
        if (herr & DEV_TIMEOUT) return timeout_error("transitive_reduce");
        if (herr) {
            set_error("graph does not satisfy the CSR contract (sorted unique columns, no diagonal, suffix < 2^30, dir <= 3)");
            return SG_ERR_INVALID;
        }
        if (nnz2 == cur_nnz) {  // nothing removed: R is final
            done = true;
            break;
        }
        SG_LAUNCH("tr_compact", tr_compact_kernel, blocks_for(n * 32, 256), 256, 0, s, g, keep, rp[nxt], col[nxt],
                  suf[nxt], dir[nxt]);
        cur = nxt;
        cur_nnz = nnz2;
        g = TrGraph{rp[cur], col[cur], suf[cur], dir[cur], n};
    }
    // S: exact-size copy of the final graph
    sg_graph_csr out{};
    out.n = n;
    out.nnz = cur_nnz;
    out.row_ptr = (int64_t *)dalloc((n + 1) * sizeof(int64_t), s);
    out.col = (int32_t *)dalloc(cur_nnz * sizeof(int32_t), s);
    out.suffix = (uint32_t *)dalloc(cur_nnz * sizeof(uint32_t), s);
    out.dir = (uint8_t *)dalloc(cur_nnz, s);
    if (!out.row_ptr || !out.col || !out.suffix || !out.dir) {
        free_graph_arrays(&out, s);
        return SG_ERR_OOM;
    }
    cudaError_t e = cudaMemcpyAsync(out.row_ptr, g.rp, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && cur_nnz)
        e = cudaMemcpyAsync(out.col, g.col, cur_nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && cur_nnz)
        e = cudaMemcpyAsync(out.suffix, g.suf, cur_nnz * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && cur_nnz) e = cudaMemcpyAsync(out.dir, g.dir, cur_nnz, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        free_graph_arrays(&out, s);
        set_error("transitive_reduce: copying S failed: %s", cudaGetErrorString(e));
        return SG_ERR_CUDA;
    }
    *S = out;
    *iters = it;
    if (converged) *converged = done ? 1 : 0;
    return SG_OK;
}

static bool graph_args_ok(const sg_graph_csr *R) {
    return R && R->n >= 0 && R->n < ((int64_t)1 << 31) && R->nnz >= 0 && R->row_ptr &&
           (R->nnz == 0 || (R->col && R->suffix && R->dir));
}

}  // namespace sg

extern "C" sg_status sg_transitive_reduce(const sg_graph_csr *R, uint32_t fuzz, int32_t mode, sg_graph_csr *S,
                                          int32_t *iterations, sg_stream_t stream) {
    if (!S || !iterations) {
        sg::set_error("transitive_reduce: NULL output");
        return SG_ERR_INVALID;
    }
    *S = sg_graph_csr{};
    *iterations = 0;
    if (!sg::graph_args_ok(R) || fuzz >= (1u << 30) || mode < 0 || mode > (SG_TR_LITERAL | SG_TR_PER_END)) {
        sg::set_error("transitive_reduce: invalid arguments");
        return SG_ERR_INVALID;
    }
    return sg::tr_impl(R, fuzz, mode, S, iterations, (cudaStream_t)stream, nullptr, 0, nullptr, 0, nullptr);
}

extern "C" sg_status sg_transitive_reduce_rounds(const sg_graph_csr *R, uint32_t fuzz, int32_t mode,
                                                 int32_t max_rounds, sg_graph_csr *S, int32_t *rounds,
                                                 int32_t *converged, sg_stream_t stream) {
    if (!S || !rounds || !converged) {
        sg::set_error("transitive_reduce_rounds: NULL output");
        return SG_ERR_INVALID;
    }
    *S = sg_graph_csr{};
    *rounds = 0;
    *converged = 0;
    if (!sg::graph_args_ok(R) || fuzz >= (1u << 30) || mode < 0 || mode > (SG_TR_LITERAL | SG_TR_PER_END) ||
        max_rounds < 1) {
        sg::set_error("transitive_reduce_rounds: invalid arguments");
        return SG_ERR_INVALID;
    }
    return sg::tr_impl(R, fuzz, mode, S, rounds, (cudaStream_t)stream, nullptr, 0, nullptr, max_rounds,
                       converged);
}

extern "C" sg_status sg_minplus_square(const sg_graph_csr *R, int32_t mode, uint32_t *d_N, uint8_t *d_Ndir,
                                       sg_stream_t stream) {
    if (!sg::graph_args_ok(R) || (mode != SG_TR_DIRMATCH && mode != SG_TR_LITERAL) || (R->nnz > 0 && !d_N)) {
        sg::set_error("minplus_square: invalid arguments");
        return SG_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    sg::Scratch sc(s);
    uint32_t *err = sc.get<uint32_t>(1);
    if (!err) return SG_ERR_OOM;
    sg::TrGraph g{R->row_ptr, R->col, R->suffix, R->dir, R->n};
    sg::TrWork wk;
    SG_TRY(sg::tr_work_alloc(&wk, R->n, R->nnz, sc));
    SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    SG_LAUNCH("validate_graph", sg::validate_graph_kernel, (R->n + 1 + 7) / 8, 256, 0, s, g, R->nnz, err);
    SG_TRY(sg::minplus_round(g, R->nnz, mode, 0, nullptr, nullptr, d_N, d_Ndir, wk, err, s));
    uint32_t herr = 0;
    SG_CUDA_TRY(sg::read_back(&herr, err, sizeof(uint32_t), s));
    if (herr) {
        sg::set_error("minplus_square: graph does not satisfy the CSR contract");
        return SG_ERR_INVALID;
    }
    return SG_OK;
}

extern "C" void sg_free_graph(sg_graph_csr *x, sg_stream_t stream) {
    if (!x) return;
    sg::free_graph_arrays(x, (cudaStream_t)stream);
}

// ------------------------------------------------------------------------------------------
// Allocation-free variant of sg_minplus_square.
//
// Some callers cannot allocate device memory at the moment they want this product: code that
// runs while a memory pool is being torn down or is already exhausted, code that must not
// grow the footprint of a process that shares its GPU under a hard memory cap, and host
// threads (e.g. a real-time scheduler loop) that may not take the allocator's locks or wait on
// its synchronisation. For them the workspace of the product lives in one file-scope device
// array, reserved when the library is loaded and kept until the process exits, on every GPU
// that loads the library.
#include <mutex>

static __device__ __align__(256) unsigned char sg_noalloc_scratch[SG_NOALLOC_SCRATCH_BYTES];

namespace sg {

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];  // device address of sg_noalloc_scratch, per device ordinal

// Device address of the scratch array on the current device. The first call on a device looks
// it up (the array's name in host code is only a stand-in, never a device address).
static sg_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("minplus_square_noalloc: device ordinal %d out of range", dev);
        return SG_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, sg_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("minplus_square_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                      cudaGetErrorString(e));
            return SG_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = (unsigned char *)g_noalloc_addr[dev];
    return SG_OK;
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace sg

extern "C" sg_status sg_minplus_square_noalloc(const sg_graph_csr *R, int32_t mode, uint32_t *d_N,
                                               uint8_t *d_Ndir, sg_stream_t stream) {
    if (!sg::graph_args_ok(R) || (mode != SG_TR_DIRMATCH && mode != SG_TR_LITERAL) || (R->nnz > 0 && !d_N)) {
        sg::set_error("minplus_square_noalloc: invalid arguments");
        return SG_ERR_INVALID;
    }
    const int64_t n = R->n, nnz = R->nnz;
    // workspace layout inside the scratch array: the error word, then TrWork's arrays with the
    // sizes the allocating path uses
    const sg::TrWorkSizes z = sg::tr_work_sizes(n, nnz);
    const size_t o_err = 0;
    const size_t o_cnt = sg::up256(o_err + sizeof(uint32_t));
    const size_t o_kind = sg::up256(o_cnt + (size_t)z.counts * sizeof(unsigned long long));
    const size_t o_rows = sg::up256(o_kind + (size_t)z.kind * sizeof(int8_t));
    const size_t o_best = sg::up256(o_rows + (size_t)z.rows * sizeof(int32_t));
    const size_t o_pre = sg::up256(o_best + (size_t)z.gbest * sizeof(unsigned long long));
    const size_t need = o_pre + (size_t)z.gpre * sizeof(int64_t);
    if (need > (size_t)SG_NOALLOC_SCRATCH_BYTES) {
        sg::set_error("minplus_square_noalloc: a graph with n=%lld and nnz=%lld needs %zu bytes of workspace, "
                      "more than the fixed %zu-byte scratch array; use sg_minplus_square",
                      (long long)n, (long long)nnz, need, (size_t)SG_NOALLOC_SCRATCH_BYTES);
        return SG_ERR_BUDGET;
    }
    unsigned char *base = nullptr;
    SG_TRY(sg::noalloc_scratch(&base));
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *err = (uint32_t *)(base + o_err);
    sg::TrWork wk;
    wk.counts = (unsigned long long *)(base + o_cnt);
    wk.kind = (int8_t *)(base + o_kind);
    wk.rows = (int32_t *)(base + o_rows);
    wk.gbest = (unsigned long long *)(base + o_best);
    wk.gpre = (int64_t *)(base + o_pre);
    sg::TrGraph g{R->row_ptr, R->col, R->suffix, R->dir, n};
    // the array keeps whatever the previous call left: the error word starts from zero here,
    // the row counters are zeroed by minplus_round, and every other word is written before read
    SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    SG_LAUNCH("validate_graph", sg::validate_graph_kernel, (n + 1 + 7) / 8, 256, 0, s, g, nnz, err);
    uint32_t herr = 0;
    SG_CUDA_TRY(sg::read_back(&herr, err, sizeof(uint32_t), s));
    if (herr) {
        sg::set_error("minplus_square_noalloc: graph does not satisfy the CSR contract");
        return SG_ERR_INVALID;
    }
    SG_TRY(sg::minplus_round(g, nnz, mode, 0, nullptr, nullptr, d_N, d_Ndir, wk, err, s));
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    return SG_OK;
}
