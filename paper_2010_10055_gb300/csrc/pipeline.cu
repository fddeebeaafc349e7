// pipeline.cu -- the whole hot path of Algorithm 2 (KmerCounter, GenerateA, Transpose, C = A At,
// TransitiveReduction) behind one call that takes and returns HOST buffers. Device inputs and
// host results live in a caller-held arena (pinned host memory + device memory, grow-only),
// so steady-state calls allocate only what the three device operations allocate themselves.
#include <stdlib.h>
#include <string.h>

#include <new>

#include "prim.cuh"

struct sg_host_arena {
    void *h = nullptr;  // pinned host block
    size_t h_cap = 0;
    void *d = nullptr;  // device block for the inputs
    size_t d_cap = 0;
    cudaStream_t cs = nullptr;  // copies C to the host while the reduction runs
    cudaEvent_t ev = nullptr;   // C complete on the call's stream
};

namespace sg {

__global__ void products_kernel(const int64_t *__restrict__ rp, int64_t m, unsigned long long *__restrict__ out) {
    unsigned long long acc = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long a = (unsigned long long)(rp[j + 1] - rp[j]);
        acc += a * a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static sg_status grow_host(sg_host_arena *a, size_t bytes) {
    if (a->h_cap >= bytes) return SG_OK;
    if (a->h) cudaFreeHost(a->h);
    a->h = nullptr;
    a->h_cap = 0;
    size_t cap = bytes + bytes / 4;
    if (cudaHostAlloc(&a->h, cap, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        set_error("pipeline: pinned host allocation of %zu bytes failed", cap);
        return SG_ERR_OOM;
    }
    a->h_cap = cap;
    return SG_OK;
}

static sg_status grow_dev(sg_host_arena *a, size_t bytes) {
    if (a->d_cap >= bytes) return SG_OK;
    if (a->d) cudaFree(a->d);
    a->d = nullptr;
    a->d_cap = 0;
    size_t cap = bytes + bytes / 4;
    if (cudaMalloc(&a->d, cap) != cudaSuccess) {
        cudaGetLastError();
        set_error("pipeline: device allocation of %zu bytes failed", cap);
        return SG_ERR_OOM;
    }
    a->d_cap = cap;
    return SG_OK;
}

static sg_status pipeline_impl(const sg_pipeline_job *j, sg_host_arena *ar, sg_pipeline_result *out, cudaStream_t s) {
    const int64_t n = j->n_reads;
    const bool do_tr = j->r_nnz >= 0 && j->r_row_ptr != nullptr;
    // device inputs: seq | offsets | R arrays | products counter
    size_t o_seq = 0, o_off = align256(o_seq + (size_t)j->total_len);
    size_t o_rp = align256(o_off + (size_t)(n + 1) * 8);
    size_t o_rc = align256(o_rp + (do_tr ? (size_t)(n + 1) * 8 : 0));
    size_t o_rs = align256(o_rc + (do_tr ? (size_t)j->r_nnz * 4 : 0));
    size_t o_rd = align256(o_rs + (do_tr ? (size_t)j->r_nnz * 4 : 0));
    size_t o_pr = align256(o_rd + (do_tr ? (size_t)j->r_nnz : 0));
    size_t dbytes = o_pr + 8;
    SG_TRY(grow_dev(ar, dbytes));
    unsigned char *d = (unsigned char *)ar->d;
    SG_CUDA_TRY(cudaMemcpyAsync(d + o_seq, j->seq, (size_t)j->total_len, cudaMemcpyHostToDevice, s));
    SG_CUDA_TRY(cudaMemcpyAsync(d + o_off, j->offsets, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, s));
    sg_graph_csr R{};
    if (do_tr) {
        SG_CUDA_TRY(cudaMemcpyAsync(d + o_rp, j->r_row_ptr, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, s));
        if (j->r_nnz) {
            SG_CUDA_TRY(cudaMemcpyAsync(d + o_rc, j->r_col, (size_t)j->r_nnz * 4, cudaMemcpyHostToDevice, s));
            SG_CUDA_TRY(cudaMemcpyAsync(d + o_rs, j->r_suffix, (size_t)j->r_nnz * 4, cudaMemcpyHostToDevice, s));
            SG_CUDA_TRY(cudaMemcpyAsync(d + o_rd, j->r_dir, (size_t)j->r_nnz, cudaMemcpyHostToDevice, s));
        }
        R = sg_graph_csr{n, j->r_nnz, (int64_t *)(d + o_rp), (int32_t *)(d + o_rc), (uint32_t *)(d + o_rs),
                         (uint8_t *)(d + o_rd)};
    }
    sg_csr_u32 A{}, At{};
    uint64_t *codes = nullptr;
    SG_TRY(sg_build_kmer_matrix(d + o_seq, (const int64_t *)(d + o_off), n, j->total_len, j->k, j->lo, j->hi, &A, &At,
                                &codes, (sg_stream_t)s));
    unsigned long long *prod = (unsigned long long *)(d + o_pr);
    sg_status st = SG_OK;
    sg_overlap_csr C{};
    sg_graph_csr S{};
    int32_t iters = 0;
    do {
        if (cudaMemsetAsync(prod, 0, 8, s) != cudaSuccess) { st = SG_ERR_CUDA; break; }
        {
            LaunchScope ls("products", s);
            int grid = (int)((At.n_rows + 255) / 256);
            if (grid > sm_count() * 8) grid = sm_count() * 8;
            if (grid > 0) products_kernel<<<grid, 256, 0, s>>>(At.row_ptr, At.n_rows, prod);
        }
        st = sg_overlap_spgemm(&A, &At, j->min_shared, j->max_seeds, &C, (sg_stream_t)s);
        if (st != SG_OK) break;
        // host results: C then S (at most nnz(R) entries: S is a subgraph of R), packed in the
        // pinned arena; C is copied on the arena's copy stream while the reduction runs
        const int64_t cn = C.nnz, Sd = C.max_seeds, smax = do_tr ? j->r_nnz : 0;
        size_t h_crp = 0, h_ccol = align256(h_crp + (size_t)(n + 1) * 8);
        size_t h_ccnt = align256(h_ccol + (size_t)cn * 4);
        size_t h_csi = align256(h_ccnt + (size_t)cn * 4);
        size_t h_csk = align256(h_csi + (size_t)cn * Sd * 4);
        size_t h_srp = align256(h_csk + (size_t)cn * Sd * 4);
        size_t h_scol = align256(h_srp + (do_tr ? (size_t)(n + 1) * 8 : 0));
        size_t h_ssuf = align256(h_scol + (size_t)smax * 4);
        size_t h_sdir = align256(h_ssuf + (size_t)smax * 4);
        size_t hbytes = h_sdir + (size_t)smax + 8;
        st = grow_host(ar, hbytes);  // no copy into the arena is in flight between calls
        if (st != SG_OK) break;
        if (!ar->cs && cudaStreamCreateWithFlags(&ar->cs, cudaStreamNonBlocking) != cudaSuccess) {
            ar->cs = nullptr;
            set_error("pipeline: copy stream creation failed");
            st = SG_ERR_CUDA;
            break;
        }
        if (!ar->ev && cudaEventCreateWithFlags(&ar->ev, cudaEventDisableTiming) != cudaSuccess) {
            ar->ev = nullptr;
            set_error("pipeline: event creation failed");
            st = SG_ERR_CUDA;
            break;
        }
        unsigned char *h = (unsigned char *)ar->h;
        unsigned long long hprod = 0;
        cudaError_t e = cudaMemcpyAsync(&hprod, prod, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(ar->ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ar->cs, ar->ev, 0);
        cudaStream_t cs = ar->cs;
        if (e == cudaSuccess) e = cudaMemcpyAsync(h + h_crp, C.row_ptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && cn) e = cudaMemcpyAsync(h + h_ccol, C.col, (size_t)cn * 4, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && cn) e = cudaMemcpyAsync(h + h_ccnt, C.count, (size_t)cn * 4, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && cn && Sd)
            e = cudaMemcpyAsync(h + h_csi, C.seed_i, (size_t)cn * Sd * 4, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && cn && Sd)
            e = cudaMemcpyAsync(h + h_csk, C.seed_k, (size_t)cn * Sd * 4, cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(cs);  // nothing of C is freed while a copy may still read it
            set_error("pipeline: copying C to the host failed: %s", cudaGetErrorString(e));
            st = SG_ERR_CUDA;
            break;
        }
        if (do_tr) {
            st = sg_transitive_reduce(&R, j->fuzz, j->tr_mode, &S, &iters, (sg_stream_t)s);
            if (st != SG_OK) {
                cudaStreamSynchronize(cs);
                break;
            }
        }
        const int64_t sn = S.nnz;
        if (do_tr) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(h + h_srp, S.row_ptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && sn) e = cudaMemcpyAsync(h + h_scol, S.col, (size_t)sn * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && sn) e = cudaMemcpyAsync(h + h_ssuf, S.suffix, (size_t)sn * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && sn) e = cudaMemcpyAsync(h + h_sdir, S.dir, (size_t)sn, cudaMemcpyDeviceToHost, s);
        }
        const cudaError_t ec = cudaStreamSynchronize(cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = ec;
        if (e != cudaSuccess) {
            set_error("pipeline: copying results to the host failed: %s", cudaGetErrorString(e));
            st = SG_ERR_CUDA;
            break;
        }
        out->m = A.n_cols;
        out->nnz_a = A.nnz;
        out->nnz_c = cn;
        out->nnz_s = do_tr ? sn : 0;
        out->iterations = iters;
        out->products = hprod;
        out->max_seeds = (int32_t)Sd;
        out->c_row_ptr = (int64_t *)(h + h_crp);
        out->c_col = (int32_t *)(h + h_ccol);
        out->c_count = (uint32_t *)(h + h_ccnt);
        out->c_seed_i = (uint32_t *)(h + h_csi);
        out->c_seed_k = (uint32_t *)(h + h_csk);
        out->s_row_ptr = do_tr ? (int64_t *)(h + h_srp) : nullptr;
        out->s_col = (int32_t *)(h + h_scol);
        out->s_suffix = (uint32_t *)(h + h_ssuf);
        out->s_dir = (uint8_t *)(h + h_sdir);
    } while (0);
    sg_free_graph(&S, (sg_stream_t)s);
    sg_free_overlap(&C, (sg_stream_t)s);
    sg_free_csr_u32(&A, (sg_stream_t)s);
    sg_free_csr_u32(&At, (sg_stream_t)s);
    dfree(codes, s);
    return st;
}

}  // namespace sg

extern "C" sg_status sg_host_arena_create(sg_host_arena **arena) {
    if (!arena) return SG_ERR_INVALID;
    *arena = new (std::nothrow) sg_host_arena();
    return *arena ? SG_OK : SG_ERR_OOM;
}

extern "C" void sg_host_arena_destroy(sg_host_arena *a) {
    if (!a) return;
    if (a->cs) {
        cudaStreamSynchronize(a->cs);
        cudaStreamDestroy(a->cs);
    }
    if (a->ev) cudaEventDestroy(a->ev);
    if (a->h) cudaFreeHost(a->h);
    if (a->d) cudaFree(a->d);
    delete a;
}

extern "C" sg_status sg_pipeline_host(const sg_pipeline_job *job, sg_host_arena *arena, sg_pipeline_result *out,
                                      sg_stream_t stream) {
    if (!out || !job || !arena) {
        sg::set_error("pipeline_host: NULL argument");
        return SG_ERR_INVALID;
    }
    memset(out, 0, sizeof(*out));
    if (job->n_reads < 0 || job->total_len < 0 || !job->offsets || (job->total_len > 0 && !job->seq) ||
        (job->r_row_ptr && job->r_nnz > 0 && (!job->r_col || !job->r_suffix || !job->r_dir))) {
        sg::set_error("pipeline_host: invalid job");
        return SG_ERR_INVALID;
    }
    return sg::pipeline_impl(job, arena, out, (cudaStream_t)stream);
}
