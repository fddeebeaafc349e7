// ops.cuh -- the three operations' implementations, shared with the batched entry point.
#pragma once

#include "prim.cuh"

namespace sg {

// Read -> job map of a batch: the k-mers of job b get b in the bits above the 2k code bits, so
// counting, the reliable range and the column order are all per job. ro == nullptr: one job.
struct JobMap {
    const int64_t *ro;  // [njobs + 1] first read of each job (device)
    int64_t njobs;
    int kbits;          // 2k
};

// Reads -> A, At, column codes (kmer.cu). For a batch, lohi (device, 2 per job) holds each job's
// reliable range and job_ncols (device, zeroed, njobs) receives each job's number of columns.
sg_status build_impl(const uint8_t *seq, const int64_t *off, int64_t n, int64_t total, int k, uint32_t lo,
                     uint32_t hi, sg_csr_u32 *A, sg_csr_u32 *At, uint64_t **codes_out, cudaStream_t s,
                     Scratch &sc, JobMap jm, const uint32_t *lohi, unsigned long long *job_ncols, uint32_t hmax);

// Options of the overlap product. A row range of a larger A (memory-bounded tiles): A holds rows
// row0 .. row0 + A->n_rows of the full matrix with its row pointers rebased to 0, partners are
// all At->n_cols reads, and C's rows are the range's (columns stay read ids).
struct OverlapOpts {
    int64_t row0 = 0;
    bool whole_rows = false;  // fused pass on whole rows, no mirror, never the two-pass form
    size_t gmem_bytes = 0;    // > 0: cap on the global-memory table pool of the redo pass
    int64_t tmp_cap = 0;      // > 0: entries of the fused pass's temporary region (else from a sample)
};

// C = A At over the overlap semiring (spgemm.cu).
sg_status overlap_impl(const sg_csr_u32 *A, const sg_csr_u32 *At, uint32_t min_shared, int S, sg_overlap_csr *C,
                       cudaStream_t s, Scratch &sc, const OverlapOpts &opt = OverlapOpts{});

// Transitive reduction (tr.cu). With job_ro (device, njobs + 1 read offsets), job_last (device,
// njobs, zeroed) receives for each job the last round that removed one of its entries.
// max_rounds > 0 stops after that many rounds (*converged, if given, says whether the last round
// removed nothing); 0 runs to the fixpoint.
sg_status tr_impl(const sg_graph_csr *R, uint32_t fuzz, int mode, sg_graph_csr *S, int32_t *iters,
                  cudaStream_t s, const int64_t *job_ro, int64_t njobs, int32_t *job_last, int32_t max_rounds = 0,
                  int32_t *converged = nullptr);

}  // namespace sg
