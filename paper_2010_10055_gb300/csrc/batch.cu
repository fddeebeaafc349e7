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

static sg_status batch_impl(const sg_batch_item *items, int32_t nitems, const sg_batch_params *p,
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
