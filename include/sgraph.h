/*
 * sgraph.h -- C ABI of the GB300 (sm_103a) library for the overlap-and-layout hot path of
 * diBELLA 2D, "Parallel String Graph Construction and Transitive Reduction for De Novo Genome
 * Assembly" (arXiv 2010.10055).
 *
 * Three operations, each one call, each run entirely by the library's own CUDA kernels:
 *   sg_build_kmer_matrix   reads -> A (reads x reliable k-mers) and its transpose
 *                          (Algorithm 2 steps KmerCounter, GenerateA, Transpose; Sec. IV-C, IV-D)
 *   sg_overlap_spgemm      C = A A^T over the overlap semiring (Algorithm 2 step "C <- A A^T";
 *                          Sec. IV-D)
 *   sg_transitive_reduce   S = TransitiveReduction(R) (Algorithm 1 with the MinPlus semiring of
 *                          Algorithm 3; Sec. IV-E)
 * plus sg_minplus_square, the single N = R^2 product of Algorithm 1 exposed on its own.
 *
 * Conventions shared by every call
 *  - Pointers named d_* and the array members of the CSR structs are DEVICE pointers (the
 *    current CUDA device); the structs themselves and the scalars live on the host.
 *  - Inputs are borrowed and never modified.
 *  - Outputs are allocated by the library with stream-ordered allocation (cudaMallocAsync) on
 *    the caller's stream, or with the allocator installed by sg_set_allocator, and are released
 *    with the matching sg_free_* call. On any error every output pointer is left NULL and no
 *    memory stays allocated.
 *  - All work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream). Each
 *    compute call validates its device inputs on the device and synchronises the stream to read
 *    that outcome and its output sizes back, so outputs are complete when it returns.
 *  - Errors: a non-SG_OK status; sg_last_error() describes it (per host thread). There is no
 *    CPU fallback: if the GPU cannot run the call, it fails.
 *  - Sizes are int64. Row pointers are int64, column indices int32 (so n and m < 2^31).
 */
#ifndef SGRAPH_H
#define SGRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *sg_stream_t; /* cudaStream_t */

typedef enum {
    SG_OK = 0,
    SG_ERR_INVALID = 1,  /* an argument or input array breaks the documented contract */
    SG_ERR_OOM = 2,      /* device (or host staging) allocation failed */
    SG_ERR_CUDA = 3,     /* a CUDA runtime call failed; sg_last_error() has the CUDA message */
    SG_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
    SG_ERR_BUDGET = 5,   /* a job does not fit the memory budget it was given */
    SG_ERR_OVERFLOW = 6, /* an intermediate exceeded a documented limit (e.g. nnz >= 2^31 per row) */
    SG_ERR_CANCELLED = 7 /* a served job was cancelled before it ran (sg_server_cancel) */
} sg_status;

/* Sparse matrix in CSR with a 32-bit payload: A (n x m) and At (m x n).
 * val = pos | strand << 31: pos = 0-based start of the k-mer in the read, strand = 1 when the
 * read holds the reverse complement of the canonical k-mer. Columns ascend within each row. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    int64_t *row_ptr; /* [n_rows + 1] */
    int32_t *col;     /* [nnz] */
    uint32_t *val;    /* [nnz] */
} sg_csr_u32;

/* Candidate overlap matrix C (n x n). count = number of shared reliable k-mers. Seed arrays are
 * slot-major, [max_seeds][nnz]: seed_i[s*nnz+e] = position of the s-th seed k-mer in read i (the
 * row), seed_k[s*nnz+e] = its position in read k (the column) | (strand_i xor strand_k) << 31.
 * Seeds are the shared k-mers with the smallest column index of A, ascending; unused slots hold
 * 0xFFFFFFFF. No diagonal entries; columns ascend within each row. */
typedef struct {
    int64_t n, nnz;
    int32_t max_seeds;
    int64_t *row_ptr; /* [n + 1] */
    int32_t *col;     /* [nnz] */
    uint32_t *count;  /* [nnz] */
    uint32_t *seed_i; /* [max_seeds * nnz] */
    uint32_t *seed_k; /* [max_seeds * nnz] */
} sg_overlap_csr;

/* Bidirected overlap / string graph R or S (n x n). Entry (i, k) is the walk i -> k:
 * suffix = overhang of read k beyond read i (< 2^30); dir = 2 * o_i + o_k where o = 0 when the
 * read is traversed as given and 1 when traversed reverse-complemented (Sec. II, Fig. 1).
 * No diagonal entries; columns strictly ascend within each row. */
typedef struct {
    int64_t n, nnz;
    int64_t *row_ptr; /* [n + 1] */
    int32_t *col;     /* [nnz] */
    uint32_t *suffix; /* [nnz] */
    uint8_t *dir;     /* [nnz] */
} sg_graph_csr;

/* Transitive-reduction semiring readings (Algorithm 3 keeps one min per entry; the paper does
 * not say which orientation that min carries when walks with different end orientations tie). */
enum {
    SG_TR_DIRMATCH = 0, /* N_ik = min over valid walks i->j->k whose end orientations match d_ik */
    SG_TR_LITERAL = 1,  /* N_ik = lexicographic min of (sum, composite dir) over valid walks; the
                           end-orientation check is applied to that one min afterwards */
    SG_TR_PER_END = 2   /* flag, or-ed with either: the row max of Algorithm 1's Reduce is taken
                           per read end (over the entries i -> k that leave read i through the
                           same end, out(d_ik)), and each entry is bounded by its own end's max,
                           instead of the whole row's (the transitive reduction) */
};

/*
 * Reads -> A and At (Sec. II canonical k-mers; Sec. IV-C k-mer counting and reliable range;
 * Sec. IV-D "A_ij stores the position of the j-th k-mer in the i-th sequence").
 *   d_seq      [total_len] ASCII bases of all reads back to back. Only 'A','C','G','T' form
 *              k-mers; a window holding any other byte is skipped.
 *   d_offsets  [n_reads + 1] int64; read i is d_seq[d_offsets[i] .. d_offsets[i+1]);
 *              d_offsets[0] = 0, non-decreasing, d_offsets[n_reads] = total_len, each read
 *              shorter than 2^31.
 *   k          odd, 1..31 (odd k: no k-mer equals its reverse complement).
 *   lo, hi     a canonical k-mer is reliable iff lo <= (occurrences over all windows) <= hi;
 *              1 <= lo <= hi. (The paper drops singletons and k-mers seen at least d times:
 *              lo = 2, hi = d - 1.)
 * Outputs: *A (n_reads x m), *At (m x n_reads), *d_kmer_codes [m] = canonical 2k-bit code of each
 * column (first base in the most significant bits, A=0 C=1 G=2 T=3); columns are numbered by
 * ascending code. A_ij = pos | strand << 31 at the LOWEST position of k-mer j in read i.
 * Errors: SG_ERR_INVALID for bad k/lo/hi/n_reads or inconsistent offsets (checked on the device),
 * SG_ERR_OOM, SG_ERR_CUDA.
 */
sg_status sg_build_kmer_matrix(const uint8_t *d_seq, const int64_t *d_offsets, int64_t n_reads,
                               int64_t total_len, int32_t k, uint32_t lo, uint32_t hi,
                               sg_csr_u32 *A, sg_csr_u32 *At, uint64_t **d_kmer_codes,
                               sg_stream_t stream);

/*
 * C = A At over the overlap semiring (Sec. IV-D: multiply = take the positions of the k-mer in
 * both reads; add = count the shared k-mer and keep up to max_seeds positions).
 *   A, At      as produced by sg_build_kmer_matrix (At must be the transpose of A, rows of both
 *              sorted by column).
 *   min_shared entries of C with count < min_shared are dropped (>= 1).
 *   max_seeds  0..8 seed slots per entry.
 * Output *C as documented at sg_overlap_csr. C is symmetric in pattern and count.
 * Errors: SG_ERR_INVALID (shape mismatch, bad scalars), SG_ERR_OOM, SG_ERR_CUDA.
 */
sg_status sg_overlap_spgemm(const sg_csr_u32 *A, const sg_csr_u32 *At, uint32_t min_shared,
                            int32_t max_seeds, sg_overlap_csr *C, sg_stream_t stream);

/*
 * Receives one tile of C from sg_overlap_spgemm_tiled: rows row_begin .. row_begin + tile->n of C
 * as a CSR of tile->n rows (row_ptr from 0; columns are read ids 0 .. n - 1; seeds slot-major with
 * stride tile->nnz). The arrays are device memory owned by the library, complete when the
 * callback runs and freed when it returns (copy what you keep). Any status other than SG_OK
 * stops the call, which returns that status.
 */
typedef sg_status (*sg_overlap_tile_fn)(const sg_overlap_csr *tile, int64_t row_begin, void *user);

/*
 * C = A At as sg_overlap_spgemm, formed in row tiles under a device-memory budget (the paper's
 * closing remark, Sec. VIII: forming C partially, under a memory bound, instead of all at once).
 * Rows of C are independent; each tile is a range of consecutive rows, sized so that what the
 * call holds at once -- the tile's intermediates, one global-memory hash table for its largest
 * row, and the tile of C -- stays within budget_bytes (on top of A and At, which the caller
 * holds). Tiles are handed to fn in row order, one at a time, on the calling thread; the
 * concatenated tiles equal sg_overlap_spgemm's C bit for bit.
 *   budget_bytes  device bytes the call may hold at once (> 0).
 *   n_tiles       out (may be NULL): tiles delivered.
 * Errors: as sg_overlap_spgemm; SG_ERR_BUDGET when one row alone does not fit the budget (no tile
 * delivered); the callback's own status if it stops the call.
 */
sg_status sg_overlap_spgemm_tiled(const sg_csr_u32 *A, const sg_csr_u32 *At, uint32_t min_shared,
                                  int32_t max_seeds, size_t budget_bytes, sg_overlap_tile_fn fn, void *user,
                                  int64_t *n_tiles, sg_stream_t stream);

/*
 * N = R^2 over the MinPlus semiring of Algorithm 3 (add = min, multiply = R_ij + R_jk when the
 * walk i->j->k is valid, i.e. the two heads at j point opposite ways, Sec. II and IV-E),
 * evaluated on the pattern of R only (Algorithm 1 compares M and N only where both exist).
 *   d_N    [R->nnz] caller-allocated; N for entry e of R, 0xFFFFFFFF when no walk qualifies.
 *   d_Ndir [R->nnz] caller-allocated; the composite dir of the minimising walk (LITERAL), or the
 *          entry's own dir (DIRMATCH). May be NULL.
 * R must satisfy the sg_graph_csr contract (checked on the device; SG_ERR_INVALID otherwise).
 */
sg_status sg_minplus_square(const sg_graph_csr *R, int32_t mode, uint32_t *d_N, uint8_t *d_Ndir,
                            sg_stream_t stream);

/*
 * Allocation-free form of sg_minplus_square (the paper has no counterpart; this is a library
 * convenience). Same inputs, outputs, result and errors, but it never allocates device memory:
 * its workspace is one fixed device array of SG_NOALLOC_SCRATCH_BYTES that every GPU which
 * loads the library reserves until the process exits. It is meant for callers that cannot call
 * cudaMalloc when they need the product -- e.g. code running under a hard per-process memory
 * cap, while a memory pool is exhausted or being torn down, or on a host thread that may not
 * take the allocator's locks.
 *  - Limit: the workspace needs 17 n + 16 nnz bytes plus about 1.3 KB (row kinds 1 B, two row
 *    lists 8 B and one prefix 8 B per row; one minimum and one prefix, 16 B, per entry); larger
 *    graphs are rejected with SG_ERR_BUDGET and a message naming the sizes (use
 *    sg_minplus_square for them).
 *  - The first call on each device looks up the array's device address (cudaGetSymbolAddress);
 *    make that first call before any stream capture.
 *  - Every call on a device shares the one array, and it keeps the previous call's contents
 *    (the call clears what must start at zero itself). Calls whose work overlaps on the GPU
 *    (other streams, other host threads) race on it: serialise them.
 *  - Synchronises `stream`.
 */
#define SG_NOALLOC_SCRATCH_BYTES (16u << 20)
sg_status sg_minplus_square_noalloc(const sg_graph_csr *R, int32_t mode, uint32_t *d_N, uint8_t *d_Ndir,
                                    sg_stream_t stream);

/*
 * The overlap graph R estimated from C's seeds: the role the alignment plays between C and R in
 * Algorithm 2 (Sec. IV-D), read from the positions C keeps. Entry C_ik's first seed (slot 0, the
 * shared k-mer with the smallest column) places read k in read i's frame: with s_i, s_k the
 * k-mer's positions and rc = strand_i xor strand_k (bit 31 of seed_k),
 *     o = s_i - s_k  (rc = 0)      o = s_i - (L_k - s_k - k)  (rc = 1),
 * so i spans [0, L_i) and k spans [o, o + L_k). The pair is an edge iff the overlap is at least
 * min_overlap bases and neither interval contains the other (contained overlaps are not part of R;
 * equal starts count as contained). Row i keeps R_ik = (o + L_k - L_i, rc) if o > 0 and
 * (-o, 3 - rc) if o < 0: the bidirected rule (suffix = overhang of the walk's second read; dir bit
 * 1 = orientation of the walk's first read, bit 0 = of its second) with read i forward.
 *   C          as produced by sg_overlap_spgemm (device arrays), max_seeds >= 1.
 *   d_offsets  the reads' offsets (device, n + 1 entries; L_i = d_offsets[i + 1] - d_offsets[i]).
 *   k          the k-mer length C was built with.
 * Output *R (library-owned device arrays, release with sg_free_graph) has C's row order; it can be
 * passed to sg_transitive_reduce (suffixes stay below 2^30 for reads shorter than 2^30).
 * Errors: SG_ERR_INVALID (bad arguments; a column of C outside [0, n)), SG_ERR_OOM, SG_ERR_CUDA.
 * Synchronises once (R's size).
 */
sg_status sg_overlap_graph_from_seeds(const sg_overlap_csr *C, const int64_t *d_offsets, int32_t k,
                                      uint32_t min_overlap, sg_graph_csr *R, sg_stream_t stream);

/*
 * Algorithm 1: repeat { N = R^2 (Algorithm 3); v = rowmax(R) + fuzz; I = (v_i >= N_ik, with the
 * end-orientation rule); R = R minus I } until nnz(R) stops changing; S = R.
 *   fuzz        < 2^30 (the scalar x of Sec. IV-E).
 *   mode        SG_TR_DIRMATCH or SG_TR_LITERAL, optionally | SG_TR_PER_END.
 *   *iterations rounds run, including the last round that removed nothing.
 * Output *S keeps the surviving entries of R with their values, in R's order.
 * Errors: SG_ERR_INVALID (R breaks the sg_graph_csr contract, fuzz or mode out of range),
 * SG_ERR_OOM, SG_ERR_CUDA.
 */
sg_status sg_transitive_reduce(const sg_graph_csr *R, uint32_t fuzz, int32_t mode, sg_graph_csr *S,
                               int32_t *iterations, sg_stream_t stream);

/*
 * Checkpoint / resume of Algorithm 1. The loop's whole state is the current R, so the reduction
 * can stop after at most max_rounds (>= 1) rounds and be resumed later by passing the returned
 * S as R: the final graph is the same as sg_transitive_reduce's, and the rounds of the pieces add
 * up to its iteration count.
 *   *rounds     rounds run by this call.
 *   *converged  1 if the last of them removed nothing (S is final), else 0 (S is an
 *               intermediate R).
 * Errors as sg_transitive_reduce; max_rounds < 1 is SG_ERR_INVALID.
 */
sg_status sg_transitive_reduce_rounds(const sg_graph_csr *R, uint32_t fuzz, int32_t mode, int32_t max_rounds,
                                      sg_graph_csr *S, int32_t *rounds, int32_t *converged, sg_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Batched form: many independent read sets in one pass. The sets are laid end to end as one
 * block-diagonal problem (set b's reads are rows read_off[b] .. read_off[b+1] of A, C and S; its
 * k-mers are columns col_off[b] .. col_off[b+1] of A, ordered by code within the set), so each
 * set's slice of the results equals what the three calls above give for that set alone --
 * indices in the slice are offset by read_off[b] (rows of A, C, S; columns of C, S, At) and
 * col_off[b] (columns of A, rows of At) -- while the batch runs as one sequence of launches.
 */
typedef struct {
    const uint8_t *d_seq;      /* device, as sg_build_kmer_matrix */
    const int64_t *d_offsets;  /* device [n_reads + 1] */
    int64_t n_reads, total_len;
    uint32_t lo, hi;           /* this set's reliable range */
    const sg_graph_csr *R;     /* device graph over this set's reads, or NULL (no reduction) */
} sg_batch_item;

typedef struct {
    int32_t k;                 /* shared by all sets */
    uint32_t min_shared;
    int32_t max_seeds;
    uint32_t fuzz;
    int32_t tr_mode;           /* as sg_transitive_reduce's mode */
} sg_batch_params;

typedef struct {
    int32_t n_items;
    int64_t *read_off;         /* host [n_items + 1] */
    int64_t *col_off;          /* host [n_items + 1] */
    int32_t *iterations;       /* host [n_items]: rounds the set alone would take (0 without R) */
    int32_t iterations_all;    /* rounds run for the whole batch */
    sg_csr_u32 A, At;          /* device, union */
    uint64_t *d_kmer_codes;    /* device [A.n_cols], codes without the set prefix */
    sg_overlap_csr C;          /* device, union (column indices are union read ids) */
    sg_graph_csr S;            /* device, union; empty when no item has R */
} sg_batch_result;

/* Errors: SG_ERR_INVALID (an item or the parameters break the contract, e.g. an R column outside
 * its own set), SG_ERR_OVERFLOW (more than 2^31 reads, or set prefix + 2k > 64 bits), SG_ERR_OOM,
 * SG_ERR_CUDA. Synchronises. Release with sg_free_batch. */
sg_status sg_run_batch(const sg_batch_item *items, int32_t n_items, const sg_batch_params *params,
                       sg_batch_result *out, sg_stream_t stream);
void sg_free_batch(sg_batch_result *r, sg_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Served form: a continuous-batching server. Jobs (host buffers, copied at submit) queue in
 * arrival order; each of `workers` threads owns a CUDA stream and, whenever idle, admits the
 * longest prefix of the queue that fits max_batch and the free part of hbm_budget, runs it as one
 * sg_run_batch and publishes each job's C and S. Jobs arriving while batches run are admitted as
 * workers and memory free up, and batches of different workers overlap on the device. A job's
 * result is the same alone and in any mix (the batch is block-diagonal). A job whose own device
 * estimate (about 64 B per base + 48 B per R entry) exceeds hbm_budget waits until nothing else
 * is admitted and runs alone with C formed in row tiles (sg_overlap_spgemm_tiled) under what the
 * budget leaves once its inputs, A, At and R are resident (about 24 B per base + 48 B per R
 * entry); its result is the same. A job that does not fit even so (the k-mer stage, about 40 B
 * per base, or the resident part plus 64 MB of tiles, above hbm_budget) completes with
 * SG_ERR_BUDGET. All calls are thread-safe.
 */
typedef struct sg_server sg_server;

typedef struct {
    size_t hbm_budget;        /* device bytes the server may commit to admitted jobs */
    int32_t max_batch;        /* jobs fused into one batch at most */
    int32_t workers;          /* batches in flight at most (one stream each) */
    int32_t device;           /* CUDA device ordinal */
    sg_batch_params params;   /* shared by all jobs */
} sg_server_config;

typedef struct {              /* host buffers, copied by sg_server_submit */
    const uint8_t *seq;
    const int64_t *offsets;   /* [n_reads + 1] */
    int64_t n_reads, total_len;
    uint32_t lo, hi;
    const int64_t *r_row_ptr; /* R over the same reads, or NULL */
    const int32_t *r_col;
    const uint32_t *r_suffix;
    const uint8_t *r_dir;
    int64_t r_nnz;
} sg_job;

typedef struct {
    sg_status status;
    int64_t n, m, nnz_c, nnz_s;
    int32_t iterations, max_seeds, batch_size;
    double t_submit, t_start, t_done;  /* steady-clock seconds: submitted, batch started, results ready */
    int64_t *c_row_ptr;                /* host (malloc), layouts as sg_overlap_csr / sg_graph_csr */
    int32_t *c_col;
    uint32_t *c_count, *c_seed_i, *c_seed_k;
    int64_t *s_row_ptr;                /* NULL when the job had no R */
    int32_t *s_col;
    uint32_t *s_suffix;
    uint8_t *s_dir;
    char error[192];                   /* when status != SG_OK: what went wrong, NUL-terminated */
} sg_job_result;

sg_status sg_server_create(const sg_server_config *cfg, sg_server **out);
/* Copies the job and queues it; *ticket identifies it. SG_ERR_INVALID for a malformed job. */
sg_status sg_server_submit(sg_server *srv, const sg_job *job, uint64_t *ticket);
/* SG_OK and the result (ownership passes to the caller: sg_job_result_free) if the job is done,
 * SG_ERR_TIMEOUT if not yet. A result is handed out once. The job's own status is out->status. */
sg_status sg_server_poll(sg_server *srv, uint64_t ticket, sg_job_result *out);
/* As poll, waiting up to timeout_s seconds. */
sg_status sg_server_wait(sg_server *srv, uint64_t ticket, double timeout_s, sg_job_result *out);
void sg_job_result_free(sg_job_result *r);
/* Cancels a job that is still queued: it never runs, its budget share is never taken, and its
 * result (poll / wait) has status SG_ERR_CANCELLED. SG_ERR_INVALID if the ticket is unknown or the
 * job has already been admitted to a batch (it then completes normally). */
sg_status sg_server_cancel(sg_server *srv, uint64_t ticket);
/* Stops the workers after their current batches; queued jobs are dropped. */
void sg_server_destroy(sg_server *srv);

/* ---------------------------------------------------------------------------------------
 * The whole path on HOST buffers: Algorithm 2 from the reads to S (KmerCounter, GenerateA,
 * Transpose, C = A A^T, TransitiveReduction; the alignment/prune steps that turn C into R are not
 * part of this library, so R is an input). Copies the inputs to the device, runs the three
 * operations above, and copies C, S and the sizes back.
 */
typedef struct {
    const uint8_t *seq;       /* [total_len] host, ASCII bases */
    const int64_t *offsets;   /* [n_reads + 1] host */
    int64_t n_reads, total_len;
    int32_t k;                /* as sg_build_kmer_matrix */
    uint32_t lo, hi;
    uint32_t min_shared;      /* as sg_overlap_spgemm */
    int32_t max_seeds;
    const int64_t *r_row_ptr; /* host R over the same n_reads reads; NULL skips the reduction */
    const int32_t *r_col;
    const uint32_t *r_suffix;
    const uint8_t *r_dir;
    int64_t r_nnz;
    uint32_t fuzz;            /* as sg_transitive_reduce */
    int32_t tr_mode;          /* as sg_transitive_reduce's mode */
} sg_pipeline_job;

/* Host results. The arrays point into the arena passed to sg_pipeline_host and stay valid until
 * that arena's next use or its destruction. Layouts as sg_overlap_csr (c_*) and sg_graph_csr (s_*).
 * products = sum over k-mers j of nnz(At_j)^2, the number of semiring multiplications in A A^T. */
typedef struct {
    int64_t m, nnz_a, nnz_c, nnz_s;
    int32_t iterations, max_seeds;
    uint64_t products;
    int64_t *c_row_ptr;
    int32_t *c_col;
    uint32_t *c_count, *c_seed_i, *c_seed_k;
    int64_t *s_row_ptr;
    int32_t *s_col;
    uint32_t *s_suffix;
    uint8_t *s_dir;
} sg_pipeline_result;

/* Grow-only pinned host + device staging owned by one caller (not thread-safe). */
typedef struct sg_host_arena sg_host_arena;
sg_status sg_host_arena_create(sg_host_arena **arena);
void sg_host_arena_destroy(sg_host_arena *arena);
/* Errors: as the three operations, plus SG_ERR_OOM when staging cannot grow. Synchronises. */
sg_status sg_pipeline_host(const sg_pipeline_job *job, sg_host_arena *arena, sg_pipeline_result *out,
                           sg_stream_t stream);

/* Release outputs (stream-ordered on `stream`); the struct is zeroed. NULL-safe. */
void sg_free_csr_u32(sg_csr_u32 *m, sg_stream_t stream);
void sg_free_overlap(sg_overlap_csr *c, sg_stream_t stream);
void sg_free_graph(sg_graph_csr *g, sg_stream_t stream);
void sg_free(void *d_ptr, sg_stream_t stream);

/* Description of the last non-OK status returned on this host thread. */
const char *sg_last_error(void);

/* Optional device allocator (e.g. a framework's caching allocator). alloc returns NULL on
 * failure, else a pointer aligned to 256 bytes as cudaMalloc's are (the kernels use 16-byte
 * vector accesses; a less aligned pointer fails the call with SG_ERR_OOM and a message). Pass
 * NULLs to restore cudaMallocAsync / cudaFreeAsync. Not thread-safe to change while calls are
 * running. */
typedef void *(*sg_alloc_fn)(size_t bytes, sg_stream_t stream, void *ctx);
typedef void (*sg_free_fn)(void *ptr, sg_stream_t stream, void *ctx);
void sg_set_allocator(sg_alloc_fn alloc, sg_free_fn release, void *ctx);

/* Test hook: make the n-th device allocation from now fail (n >= 1); 0 disables. */
void sg_debug_fail_alloc_after(int64_t n);

/* Test hook for the bounded waits between thread blocks. While on, every scan of more than one
 * tile has its first tile withhold its prefix: the waits of the later tiles give up after their
 * poll limit (well under a second each), set the call's device error word, and the call returns
 * SG_ERR_TIMEOUT with its outputs freed. Nothing hangs and the context stays usable. Off by
 * default; affects all threads. */
void sg_debug_stall_lookback(int on);

/* Checked builds (compiled with -DSG_CHECKED): the first out-of-bounds index any kernel detected
 * and skipped since the last call, as site << 40 | index, or 0. Always 0 in normal builds. */
uint64_t sg_debug_check(void);

/* Test hook: while on, each fused overlap product (sg_overlap_spgemm) on the calling thread
 * records which numeric launch handled each row of C, for parity tests that sample rows per
 * launch. sg_debug_spgemm_classes copies the last record (n entries) to host memory and returns
 * the number of rows recorded, or -1 if there is none (off, or the two-pass form ran). Codes:
 * log2 of the shared-memory table size (6..14), 16 + log2 for a filtered table, 32 for a row sent
 * straight to a global-memory table, 33 for a filtered one, plus 64 when a guessed table overflowed
 * and the row was redone in global memory; 96 + log2 for a row redone in a larger shared-memory
 * table after an overflow (128: in global memory; plus 64 if that one overflowed too); -1 for a
 * row with no products. */
void sg_debug_record_classes(int on);
int64_t sg_debug_spgemm_classes(int32_t *host_out, int64_t n);

/* Sizes of the calling thread's last k-mer matrix build (sg_build_kmer_matrix or a batch), for
 * profiling: windows = sequence positions, candidates = windows that passed the Bloom filters and
 * were sorted, sort_key_bytes / sort_val_bytes = bytes per candidate through each radix pass
 * (val 0 when the window rides in the key), sort_passes = 8-bit passes over the candidates,
 * a_sort_passes = passes of the (read, entry) sort that forms A, m and nnz as in the outputs,
 * bloom_bins = shared-memory filter bins (0: the filters were sliced global-memory arrays),
 * bloom_b2_bytes = size of the seen-twice filter. */
typedef struct {
    int64_t windows, candidates, m, nnz;
    int32_t sort_key_bytes, sort_val_bytes, sort_passes, a_sort_passes;
    int64_t bloom_bins, bloom_b2_bytes;
} sg_kmer_stats;
void sg_last_kmer_stats(sg_kmer_stats *out);

/* Number of kernels this library has launched in this process. */
uint64_t sg_launch_count(void);

/* Device memory of the library's pool on the current device, in bytes: reserved = held by the
 * pool (freed memory stays reserved for reuse), in_use = allocated and not yet freed (library
 * outputs the caller still holds, and work memory of calls in flight), in_use_peak = the largest
 * in_use since the pool was created or sg_memory_reset_peak. All 0 while an allocator installed by
 * sg_set_allocator is in use. NULL pointers are skipped. Returns SG_OK, or SG_ERR_CUDA if the pool
 * cannot be queried. */
sg_status sg_memory_stats(uint64_t *reserved, uint64_t *in_use, uint64_t *in_use_peak);
void sg_memory_reset_peak(void);

/* Tunable launch parameters (used by the autotuner; results never depend on them):
 *   bloom_bits            bits of the first-level Bloom filter per window (8): fewer bits, fewer
 *                         slices but more false positives (singletons that reach the exact count)
 *   bloom_slice_mb        megabytes of the first-level Bloom filter updated per launch (64)
 *   bloom_max_slices      at most this many Bloom launches, each streaming all window hashes;
 *                         for larger filters the slices grow instead (8)
 *   bloom_unroll          windows (independent atomics) per thread per Bloom step: 4 or 8 (4)
 *   bloom_binned          1: the window hashes are grouped by filter bin and each bin's filters
 *                         are built in shared memory (1); 0: sliced global-memory filters
 *   bloom_scatter_levels  passes that group the hashes: 1 straight into bins, 2 into superbins
 *                         first (0, and always beyond 4096 bins: two only where needed)
 *   bloom_bin_kb          first-filter kilobytes per bin, rounded down to a power of two (128;
 *                         the second filter gets a quarter)
 *   bloom_scatter_cfg     tile of the pass that groups hashes by bin: 0 512 x 16, 1 256 x 16,
 *                         2 256 x 32 threads x hashes (0)
 *   kmer_sort_buckets     at most this many top code bits may split the candidates into buckets
 *                         sorted apart, where that lets the rest of the code fit beside the
 *                         position in an 8-byte key (3); 0: 16-byte pairs instead
 *   bloom_bin_room_pct    hash buffer per bin, % of the mean bin (112, plus 16 K); a bin that
 *                         overflows sends the whole build to the sliced filters
 *   spgemm_fused          1: C in one numeric pass whose tables are sized from a guess (rows that
 *                         overflow are redone in exact-size global-memory tables) and whose rows
 *                         go to a temporary region; 0: symbolic pass (exact sizes), then numeric (1)
 *   spgemm_sample_rows    rows sampled before the fused pass when nnz(A) >= spgemm_sample_min_nnz
 *                         (2^26) (256): their partners per product
 *                         (distinct, and seen at least twice) scale every row's table guess, and
 *                         the seen-twice filter is used only where it keeps under half the
 *                         partners; 0: no sample, guesses by the shifts below
 *   spgemm_guess_pct      sampled guess = pct / 100 x partners per product x products (300)
 *   num_guess_shift       fused numeric table guess without a sample = products >> shift (2)
 *   spgemm_fused_max_mb   largest temporary region of the fused pass, MB (65536); above it, or
 *                         above half the device memory free at the call, the two-pass form runs
 *   spgemm_filter_mode    seen-twice filter for fused rows of spgemm_filter_work products or
 *                         more: they first mark, in two bit filters, the partners seen once and
 *                         seen twice, and tabulate only the latter (count-1 partners cannot reach C
 *                         when min_shared >= 2). 0 never, 1 when the row sample finds that fewer
 *                         than half the partners recur (1), 2 always
 *   spgemm_filter_work    rows with at least this many products may be filtered; 0: none (2048)
 *   spgemm_filter_shift   table guess of those rows without a sample = products >> shift (2)
 *   spgemm_filter_log2    bits per filter: one per read up to 2^this, hashed beyond (17)
 *   sym_guess_shift       symbolic hash table guess = products of the row >> shift (2)
 *   spgemm_blocks_per_sm  blocks per SM of each SpGEMM class launch (16)
 *   spgemm_big_threads    threads per numeric block for tables of 4 K slots or more: 512 or 1024
 *                         (1024)
 *   tr_blocks_per_sm      blocks per SM of the min-plus launch (32)
 *   pool_cross_stream_reuse  1: the library's memory pool may reuse memory freed on one stream for
 *                         another (read once, when the pool is created) (1)
 * sg_tune_set returns 1 if the name is known and the value in range, else 0 (no change).
 * sg_tune_name(i) enumerates the names (NULL past the end). Not thread-safe against running calls. */
int sg_tune_set(const char *name, int64_t value);
int64_t sg_tune_get(const char *name);
const char *sg_tune_name(int idx);

/* Per-kernel CUDA-event timing. While enabled, each kernel launch is bracketed by two events on
 * its stream. sg_prof_collect synchronises on the recorded events and folds them into per-name
 * totals, readable with sg_prof_entry(idx, ...) for idx < sg_prof_collect()'s return value. */
void sg_prof_enable(int on);
/* Time only kernels whose name starts with name_prefix (NULL or "" = all). */
void sg_prof_select(const char *name_prefix);
void sg_prof_reset(void);
int sg_prof_collect(void);
int sg_prof_entry(int idx, const char **name, int64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif
#endif /* SGRAPH_H */
