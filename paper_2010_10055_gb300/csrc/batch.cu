// batch.cu -- many independent read sets in one pass.
//
// The read sets of a batch are laid end to end as one block-diagonal problem: reads of set b
// are rows read_off[b] .. read_off[b+1] of every matrix, and its k-mers carry b above their 2k
// code bits, so k-mer frequencies, the reliable range and the column order are per set and no
// k-mer is shared across sets. C = A A^T and the transitive reduction then never connect two
// sets, so every set's slice of the results equals what the three calls give for that set alone,
// while the whole batch costs one pass of launches.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ops.cuh"

namespace sg {

struct ItemDesc {
    const uint8_t *seq;
    const int64_t *off;
    int64_t n, total, read0, base0;
    const int64_t *rrp;
    const int32_t *rcol;
    const uint32_t *rsuf;
    const uint8_t *rdir;
    int64_t rnnz, rnnz0;
};

// Item-local contract: offsets start at 0 and end at total; R (if any) has n + 1 row pointers
// from 0 to rnnz and columns in [0, n). Checked before the union is formed.
__global__ void batch_check_kernel(const ItemDesc *__restrict__ items, int nitems, uint32_t *__restrict__ err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nitems) return;
    const ItemDesc it = items[b];
    bool bad = it.off[0] != 0 || it.off[it.n] != it.total;
    if (it.rrp) bad = bad || it.rrp[0] != 0 || it.rrp[it.n] != it.rnnz;
    if (bad) atomicOr(err, (uint32_t)DEV_INVALID);
}

// blockIdx.y = item; x-blocks stride over the item's elements.
__global__ void batch_concat_kernel(const ItemDesc *__restrict__ items, uint8_t *__restrict__ seq,
                                    int64_t *__restrict__ off, int64_t *__restrict__ rrp, int32_t *__restrict__ rcol,
                                    uint32_t *__restrict__ rsuf, uint8_t *__restrict__ rdir, uint32_t *__restrict__ err) {
    const ItemDesc it = items[blockIdx.y];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < it.total; i += stride)
        seq[it.base0 + i] = it.seq[i];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= it.n; i += stride) {
        // entry n of set b and entry 0 of set b + 1 land on the same slot with the same value
        off[it.read0 + i] = it.off[i] + it.base0;
        if (rrp) rrp[it.read0 + i] = (it.rrp ? it.rrp[i] : 0) + it.rnnz0;
    }
    if (it.rrp) {
        bool bad = false;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < it.rnnz; e += stride) {
            const int32_t c = it.rcol[e];
            bad |= c < 0 || c >= it.n;
            rcol[it.rnnz0 + e] = (int32_t)(c + it.read0);
            rsuf[it.rnnz0 + e] = it.rsuf[e];
            rdir[it.rnnz0 + e] = it.rdir[e];
        }
        if (bad) atomicOr(err, (uint32_t)DEV_INVALID);
    }
}

// One group of items as one block-diagonal union (the whole batch when it is one group).
static sg_status union_impl(const sg_batch_item *items, int32_t nitems, const sg_batch_params *p,
                            sg_batch_result *out, cudaStream_t s, Scratch &sc) {
    std::vector<ItemDesc> d(nitems);
    std::vector<int64_t> ro(nitems + 1, 0), co(nitems + 1, 0);
    std::vector<uint32_t> lohi(2 * (size_t)nitems);
    int64_t N = 0, T = 0, RN = 0;
    uint32_t min_lo = 0xFFFFFFFFu, max_hi = 0;
    bool any_r = false;
    for (int b = 0; b < nitems; b++) {
        const sg_batch_item &x = items[b];
        if (x.n_reads < 0 || x.total_len < 0 || !x.d_offsets || (x.total_len > 0 && !x.d_seq) || x.lo < 1 ||
            x.lo > x.hi || (x.n_reads == 0 && x.total_len != 0)) {
            set_error("run_batch: item %d is invalid", b);
            return SG_ERR_INVALID;
        }
        if (x.R && (x.R->n != x.n_reads || x.R->nnz < 0 || !x.R->row_ptr ||
                    (x.R->nnz > 0 && (!x.R->col || !x.R->suffix || !x.R->dir)))) {
            set_error("run_batch: item %d has an R that does not match its reads", b);
            return SG_ERR_INVALID;
        }
        d[b] = ItemDesc{x.d_seq, x.d_offsets, x.n_reads, x.total_len, N, T,
                        x.R ? x.R->row_ptr : nullptr, x.R ? x.R->col : nullptr, x.R ? x.R->suffix : nullptr,
                        x.R ? x.R->dir : nullptr, x.R ? x.R->nnz : 0, RN};
        lohi[2 * b] = x.lo;
        min_lo = x.lo < min_lo ? x.lo : min_lo;
        max_hi = x.hi > max_hi ? x.hi : max_hi;
        lohi[2 * b + 1] = x.hi;
        any_r |= x.R != nullptr;
        N += x.n_reads;
        T += x.total_len;
        RN += x.R ? x.R->nnz : 0;
        ro[b + 1] = N;
    }
    if (N >= ((int64_t)1 << 31)) {
        set_error("run_batch: %lld reads exceed the int32 index range", (long long)N);
        return SG_ERR_OVERFLOW;
    }
    ItemDesc *d_items = sc.get<ItemDesc>(nitems);
    int64_t *d_ro = sc.get<int64_t>(nitems + 1);
    uint32_t *d_lohi = sc.get<uint32_t>(2 * (size_t)nitems);
    unsigned long long *d_ncols = sc.get<unsigned long long>(nitems);
    int32_t *d_last = sc.get<int32_t>(nitems);
    uint32_t *err = sc.get<uint32_t>(1);
    uint8_t *seq = sc.get<uint8_t>(T + 16);
    int64_t *off = sc.get<int64_t>(N + 1);
    if (!d_items || !d_ro || !d_lohi || !d_ncols || !d_last || !err || !seq || !off) return SG_ERR_OOM;
    int64_t *rrp = nullptr;
    int32_t *rcol = nullptr;
    uint32_t *rsuf = nullptr;
    uint8_t *rdir = nullptr;
    if (any_r) {
        rrp = sc.get<int64_t>(N + 1);
        rcol = sc.get<int32_t>(RN + 1);
        rsuf = sc.get<uint32_t>(RN + 1);
        rdir = sc.get<uint8_t>(RN + 1);
        if (!rrp || !rcol || !rsuf || !rdir) return SG_ERR_OOM;
    }
    SG_CUDA_TRY(cudaMemcpyAsync(d_items, d.data(), sizeof(ItemDesc) * nitems, cudaMemcpyHostToDevice, s));
    SG_CUDA_TRY(cudaMemcpyAsync(d_ro, ro.data(), sizeof(int64_t) * (nitems + 1), cudaMemcpyHostToDevice, s));
    SG_CUDA_TRY(cudaMemcpyAsync(d_lohi, lohi.data(), sizeof(uint32_t) * 2 * nitems, cudaMemcpyHostToDevice, s));
    SG_CUDA_TRY(cudaMemsetAsync(d_ncols, 0, sizeof(unsigned long long) * nitems, s));
    SG_CUDA_TRY(cudaMemsetAsync(d_last, 0, sizeof(int32_t) * nitems, s));
    SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
    SG_LAUNCH("batch_check", batch_check_kernel, (nitems + 127) / 128, 128, 0, s, (const ItemDesc *)d_items, nitems,
              err);
    uint32_t herr = 0;
    SG_CUDA_TRY(read_back(&herr, err, sizeof(uint32_t), s));
    if (herr) {
        set_error("run_batch: an item's offsets or R row pointers are inconsistent with its sizes");
        return SG_ERR_INVALID;
    }
    const dim3 cgrid(64, (unsigned)nitems);
    SG_LAUNCH("batch_concat", batch_concat_kernel, cgrid, 256, 0, s, (const ItemDesc *)d_items, seq, off, rrp, rcol,
              rsuf, rdir, err);

    {  // each stage's temporaries are released before the next stage starts
        Scratch sc1(s);
        // the scalar range only decides whether the Bloom pass may drop singletons: every set needs lo >= 2
    SG_TRY(build_impl(seq, off, N, T, p->k, min_lo, min_lo, &out->A, &out->At, &out->d_kmer_codes, s, sc1,
                          JobMap{d_ro, nitems, 2 * p->k}, d_lohi, d_ncols, max_hi));
    }
    {
        Scratch sc2(s);
        SG_TRY(overlap_impl(&out->A, &out->At, p->min_shared, p->max_seeds, &out->C, s, sc2));
    }
    if (any_r) {
        const sg_graph_csr R{N, RN, rrp, rcol, rsuf, rdir};
        SG_TRY(tr_impl(&R, p->fuzz, p->tr_mode, &out->S, &out->iterations_all, s, d_ro, nitems, d_last));
    }
    // per-item sizes back to the host
    std::vector<unsigned long long> ncols(nitems);
    std::vector<int32_t> last(nitems);
    SG_CUDA_TRY(cudaMemcpyAsync(ncols.data(), d_ncols, sizeof(unsigned long long) * nitems, cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaMemcpyAsync(last.data(), d_last, sizeof(int32_t) * nitems, cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(read_back(&herr, err, sizeof(uint32_t), s));
    if (herr) {
        set_error("run_batch: an item's R has a column outside its own reads");
        return SG_ERR_INVALID;
    }
    for (int b = 0; b < nitems; b++) co[b + 1] = co[b] + (int64_t)ncols[b];
    out->n_items = nitems;
    out->read_off = (int64_t *)malloc(sizeof(int64_t) * (nitems + 1));
    out->col_off = (int64_t *)malloc(sizeof(int64_t) * (nitems + 1));
    out->iterations = (int32_t *)malloc(sizeof(int32_t) * (nitems > 0 ? nitems : 1));
    if (!out->read_off || !out->col_off || !out->iterations) {
        set_error("run_batch: host allocation failed");
        return SG_ERR_OOM;
    }
    memcpy(out->read_off, ro.data(), sizeof(int64_t) * (nitems + 1));
    memcpy(out->col_off, co.data(), sizeof(int64_t) * (nitems + 1));
    for (int b = 0; b < nitems; b++) out->iterations[b] = items[b].R ? last[b] + 1 : 0;
    return SG_OK;
}

// dst[i] = src[i] + add (i < n): a group's indices moved to their place in the whole batch
template <class T>
__global__ void copy_add_kernel(const T *__restrict__ src, int64_t n, T add, T *__restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + add;
}

template <class T>
__global__ void fill_kernel(T *__restrict__ dst, int64_t n, T v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = v;
}

template <class T>
static sg_status copy_add(const T *src, int64_t n, T add, T *dst, cudaStream_t s) {
    if (n <= 0) return SG_OK;
    if (add == T(0)) {
        SG_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        return SG_OK;
    }
    SG_LAUNCH("batch_merge", copy_add_kernel<T>, (n + 255) / 256, 256, 0, s, src, n, add, dst);
    return SG_OK;
}

// Runs of the batch: an item of at least batch_alone_kb kilobases runs on its own (alone it
// already fills the GPU, and in a union its k-mer keys would carry more bits); consecutive
// smaller items share a union of at most batch_group_kb kilobases, which saves their per-call
// launches. Every group's results are then moved, indices offset, into the one batch result,
// so the result is the same whatever the grouping.
static sg_status batch_impl(const sg_batch_item *items, int32_t nitems, const sg_batch_params *p,
                            sg_batch_result *out, cudaStream_t s, Scratch &sc) {
    const int64_t alone = tune("batch_alone_kb") * 1000, gmax = tune("batch_group_kb") * 1000;
    std::vector<int32_t> cut{0};  // group g = items cut[g] .. cut[g + 1]
    int64_t acc = 0;
    for (int32_t b = 0; b < nitems; b++) {
        const int64_t t = items[b].total_len;
        const bool big = alone > 0 && t >= alone;
        if (b > cut.back() && (big || acc + t > gmax || (alone > 0 && items[b - 1].total_len >= alone))) {
            cut.push_back(b);
            acc = 0;
        }
        acc += t;
    }
    cut.push_back(nitems);
    const int ng = (int)cut.size() - 1;
    if (ng == 1) return union_impl(items, nitems, p, out, s, sc);
    std::vector<sg_batch_result> gr(ng);
    for (int g = 0; g < ng; g++) {
        Scratch sg_(s);
        const sg_status st = union_impl(items + cut[g], cut[g + 1] - cut[g], p, &gr[g], s, sg_);
        if (st != SG_OK) {
            for (int h = 0; h <= g; h++) sg_free_batch(&gr[h], (sg_stream_t)s);
            return st;
        }
    }
    // sizes and bases of every group in the whole batch
    int64_t N = 0, M = 0, nA = 0, nC = 0, nS = 0;
    bool any_s = false;
    std::vector<int64_t> RB(ng), CB(ng), AB(ng), CCB(ng), SB(ng);
    for (int g = 0; g < ng; g++) {
        RB[g] = N; CB[g] = M; AB[g] = nA; CCB[g] = nC; SB[g] = nS;
        N += gr[g].A.n_rows;
        M += gr[g].A.n_cols;
        nA += gr[g].A.nnz;
        nC += gr[g].C.nnz;
        nS += gr[g].S.nnz;
        any_s |= gr[g].S.row_ptr != nullptr;
    }
    const int S = p->max_seeds;
    sg_status st = SG_OK;
    auto fail = [&](sg_status e) {
        for (int g = 0; g < ng; g++) sg_free_batch(&gr[g], (sg_stream_t)s);
        return e;
    };
#define SG_MERGE_TRY(expr)                  \
    do {                                    \
        st = (expr);                        \
        if (st != SG_OK) return fail(st);   \
    } while (0)
#define SG_MERGE_ALLOC(ptr, type, count)                                \
    do {                                                                \
        ptr = (type *)dalloc((size_t)(count) * sizeof(type), s);        \
        if (!ptr) return fail(SG_ERR_OOM);                              \
    } while (0)
    out->A = sg_csr_u32{N, M, nA, nullptr, nullptr, nullptr};
    out->At = sg_csr_u32{M, N, nA, nullptr, nullptr, nullptr};
    SG_MERGE_ALLOC(out->A.row_ptr, int64_t, N + 1);
    SG_MERGE_ALLOC(out->A.col, int32_t, nA);
    SG_MERGE_ALLOC(out->A.val, uint32_t, nA);
    SG_MERGE_ALLOC(out->At.row_ptr, int64_t, M + 1);
    SG_MERGE_ALLOC(out->At.col, int32_t, nA);
    SG_MERGE_ALLOC(out->At.val, uint32_t, nA);
    SG_MERGE_ALLOC(out->d_kmer_codes, uint64_t, M);
    out->C = sg_overlap_csr{N, nC, S, nullptr, nullptr, nullptr, nullptr, nullptr};
    SG_MERGE_ALLOC(out->C.row_ptr, int64_t, N + 1);
    SG_MERGE_ALLOC(out->C.col, int32_t, nC);
    SG_MERGE_ALLOC(out->C.count, uint32_t, nC);
    SG_MERGE_ALLOC(out->C.seed_i, uint32_t, (int64_t)S * nC);
    SG_MERGE_ALLOC(out->C.seed_k, uint32_t, (int64_t)S * nC);
    if (any_s) {
        out->S = sg_graph_csr{N, nS, nullptr, nullptr, nullptr, nullptr};
        SG_MERGE_ALLOC(out->S.row_ptr, int64_t, N + 1);
        SG_MERGE_ALLOC(out->S.col, int32_t, nS);
        SG_MERGE_ALLOC(out->S.suffix, uint32_t, nS);
        SG_MERGE_ALLOC(out->S.dir, uint8_t, nS);
    }
    for (int g = 0; g < ng; g++) {
        const sg_batch_result &r = gr[g];
        const int64_t n = r.A.n_rows, m = r.A.n_cols;
        SG_MERGE_TRY(copy_add<int64_t>(r.A.row_ptr, n, AB[g], out->A.row_ptr + RB[g], s));
        SG_MERGE_TRY(copy_add<int32_t>(r.A.col, r.A.nnz, (int32_t)CB[g], out->A.col + AB[g], s));
        SG_MERGE_TRY(copy_add<uint32_t>(r.A.val, r.A.nnz, 0u, out->A.val + AB[g], s));
        SG_MERGE_TRY(copy_add<int64_t>(r.At.row_ptr, m, AB[g], out->At.row_ptr + CB[g], s));
        SG_MERGE_TRY(copy_add<int32_t>(r.At.col, r.At.nnz, (int32_t)RB[g], out->At.col + AB[g], s));
        SG_MERGE_TRY(copy_add<uint32_t>(r.At.val, r.At.nnz, 0u, out->At.val + AB[g], s));
        SG_MERGE_TRY(copy_add<uint64_t>(r.d_kmer_codes, m, 0ull, out->d_kmer_codes + CB[g], s));
        SG_MERGE_TRY(copy_add<int64_t>(r.C.row_ptr, n, CCB[g], out->C.row_ptr + RB[g], s));
        SG_MERGE_TRY(copy_add<int32_t>(r.C.col, r.C.nnz, (int32_t)RB[g], out->C.col + CCB[g], s));
        SG_MERGE_TRY(copy_add<uint32_t>(r.C.count, r.C.nnz, 0u, out->C.count + CCB[g], s));
        for (int q = 0; q < S; q++) {
            SG_MERGE_TRY(copy_add<uint32_t>(r.C.seed_i + (int64_t)q * r.C.nnz, r.C.nnz, 0u,
                                            out->C.seed_i + (int64_t)q * nC + CCB[g], s));
            SG_MERGE_TRY(copy_add<uint32_t>(r.C.seed_k + (int64_t)q * r.C.nnz, r.C.nnz, 0u,
                                            out->C.seed_k + (int64_t)q * nC + CCB[g], s));
        }
        if (any_s) {
            if (r.S.row_ptr) {
                SG_MERGE_TRY(copy_add<int64_t>(r.S.row_ptr, n, SB[g], out->S.row_ptr + RB[g], s));
                SG_MERGE_TRY(copy_add<int32_t>(r.S.col, r.S.nnz, (int32_t)RB[g], out->S.col + SB[g], s));
                SG_MERGE_TRY(copy_add<uint32_t>(r.S.suffix, r.S.nnz, 0u, out->S.suffix + SB[g], s));
                SG_MERGE_TRY(copy_add<uint8_t>(r.S.dir, r.S.nnz, (uint8_t)0, out->S.dir + SB[g], s));
            } else if (n > 0) {  // no item of this group has R: its rows of S are empty
                SG_LAUNCH("batch_merge", fill_kernel<int64_t>, (n + 255) / 256, 256, 0, s, out->S.row_ptr + RB[g],
                          n, SB[g]);
            }
        }
    }
    // the closing row pointers
    SG_CUDA_TRY(cudaMemcpyAsync(out->A.row_ptr + N, &nA, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    SG_CUDA_TRY(cudaMemcpyAsync(out->At.row_ptr + M, &nA, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    SG_CUDA_TRY(cudaMemcpyAsync(out->C.row_ptr + N, &nC, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (any_s) SG_CUDA_TRY(cudaMemcpyAsync(out->S.row_ptr + N, &nS, sizeof(int64_t), cudaMemcpyHostToDevice, s));
#undef SG_MERGE_ALLOC
#undef SG_MERGE_TRY
    out->n_items = nitems;
    out->read_off = (int64_t *)malloc(sizeof(int64_t) * (nitems + 1));
    out->col_off = (int64_t *)malloc(sizeof(int64_t) * (nitems + 1));
    out->iterations = (int32_t *)malloc(sizeof(int32_t) * (nitems > 0 ? nitems : 1));
    if (!out->read_off || !out->col_off || !out->iterations) {
        set_error("run_batch: host allocation failed");
        return fail(SG_ERR_OOM);
    }
    out->iterations_all = 0;
    for (int g = 0; g < ng; g++) {
        const sg_batch_result &r = gr[g];
        for (int32_t b = cut[g]; b < cut[g + 1]; b++) {
            const int32_t lb = b - cut[g];
            out->read_off[b] = RB[g] + r.read_off[lb];
            out->col_off[b] = CB[g] + r.col_off[lb];
            out->iterations[b] = r.iterations[lb];
        }
        out->iterations_all = std::max(out->iterations_all, r.iterations_all);
    }
    out->read_off[nitems] = N;
    out->col_off[nitems] = M;
    // the host copies of the closing row pointers must outlive the copies: wait for them
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    for (int g = 0; g < ng; g++) sg_free_batch(&gr[g], (sg_stream_t)s);
    return SG_OK;
}

}  // namespace sg

extern "C" sg_status sg_run_batch(const sg_batch_item *items, int32_t n_items, const sg_batch_params *params,
                                  sg_batch_result *out, sg_stream_t stream) {
    if (!out) {
        sg::set_error("run_batch: NULL output");
        return SG_ERR_INVALID;
    }
    memset(out, 0, sizeof(*out));
    if (!params || n_items < 1 || !items || params->k < 1 || params->k > 31 || (params->k & 1) == 0 ||
        params->min_shared < 1 || params->max_seeds < 0 || params->max_seeds > 8 || params->fuzz >= (1u << 30) ||
        params->tr_mode < 0 || params->tr_mode > (SG_TR_LITERAL | SG_TR_PER_END)) {
        sg::set_error("run_batch: invalid parameters");
        return SG_ERR_INVALID;
    }
    int job_bits = 0;
    while (((int64_t)1 << job_bits) < n_items) job_bits++;
    if (2 * params->k + job_bits > 64) {
        sg::set_error("run_batch: %d items with k = %d do not fit a 64-bit k-mer key", n_items, params->k);
        return SG_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    sg_status st;
    {
        sg::Scratch sc(s);
        st = sg::batch_impl(items, n_items, params, out, s, sc);
    }
    if (st != SG_OK) sg_free_batch(out, stream);
    return st;
}

extern "C" void sg_free_batch(sg_batch_result *r, sg_stream_t stream) {
    if (!r) return;
    sg_free_csr_u32(&r->A, stream);
    sg_free_csr_u32(&r->At, stream);
    sg::dfree(r->d_kmer_codes, (cudaStream_t)stream);
    sg_free_overlap(&r->C, stream);
    sg_free_graph(&r->S, stream);
    free(r->read_off);
    free(r->col_off);
    free(r->iterations);
    memset(r, 0, sizeof(*r));
}
