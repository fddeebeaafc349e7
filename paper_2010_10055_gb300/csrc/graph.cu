// graph.cu -- the overlap graph R estimated from C's seeds (the alignment's role in Algorithm 2,
// Sec. IV-D), on the GPU.
//
// Entry C_ik's first seed (the shared k-mer with the smallest column) places read k in read i's
// frame: with s_i, s_k its positions and rc = strand_i xor strand_k, read k starts at
//   o = s_i - s_k                 (rc = 0)
//   o = s_i - (L_k - s_k - K)     (rc = 1: k's window, seen on k's reverse complement)
// so i = [0, L_i) and k = [o, o + L_k). The pair is an edge iff the overlap is >= min_overlap and
// neither interval contains the other; then, with read i forward and read k in orientation rc,
//   o > 0:  R_ik = (o + L_k - L_i, rc)          o < 0:  R_ik = (-o, 2 + 1 - rc)
// which is the bidirected rule of the coordinate-built graph (the read that starts first is a:
// R_ab = (e_b - e_a, 2 s_a + s_b), R_ba = (s_b - s_a, 2 (1 - s_b) + (1 - s_a))).
//
// Two warp-per-row passes over C: count each row's edges (ballot), scan, then write each row's
// edges contiguously (the same integer decision recomputed). R keeps C's row order.
#include "check.cuh"
#include "ops.cuh"

namespace sg {

struct SeedEdge {
    bool keep;
    uint32_t suffix;
    uint8_t dir;
};

__device__ __forceinline__ SeedEdge seed_edge(int64_t Li, int64_t Lk, uint32_t si_w, uint32_t sk_w, int K,
                                              int64_t min_ov) {
    SeedEdge r{false, 0u, 0};
    if (si_w == 0xFFFFFFFFu || sk_w == 0xFFFFFFFFu) return r;  // no seed (cannot happen for count >= 1)
    const int64_t si = si_w & 0x7FFFFFFFu, sk = sk_w & 0x7FFFFFFFu;
    const int rc = (int)(sk_w >> 31);
    const int64_t o = rc ? si - (Lk - sk - K) : si - sk;
    const int64_t lo = o > 0 ? o : 0, hi = (o + Lk < Li) ? o + Lk : Li;
    if (hi - lo < min_ov) return r;
    if (o >= 0 && o + Lk <= Li) return r;  // k within i (equal starts included)
    if (o <= 0 && o + Lk >= Li) return r;  // i within k
    r.keep = true;
    if (o > 0) {
        r.suffix = (uint32_t)(o + Lk - Li);
        r.dir = (uint8_t)rc;
    } else {
        r.suffix = (uint32_t)(-o);
        r.dir = (uint8_t)(3 - rc);
    }
    return r;
}

struct SeedArgs {
    const int64_t *c_rp;
    const int32_t *c_col;
    const uint32_t *c_si;  // slot 0 of the seeds
    const uint32_t *c_sk;
    const int64_t *off;
    int64_t n;
    int K;
    int64_t min_ov;
};

// One warp per row: number of edges of row i (WRITE == false), or the edges themselves at
// r_rp[i] (WRITE == true).
template <bool WRITE>
__global__ void seed_edges_kernel(SeedArgs a, int64_t *__restrict__ cnt, const int64_t *__restrict__ r_rp,
                                  int32_t *__restrict__ r_col, uint32_t *__restrict__ r_suf,
                                  uint8_t *__restrict__ r_dir, uint32_t *__restrict__ err) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= a.n) return;
    const int64_t Li = a.off[i + 1] - a.off[i];
    const int64_t r0 = a.c_rp[i], r1 = a.c_rp[i + 1];
    int64_t w = WRITE ? r_rp[i] : 0;
    for (int64_t b = r0; b < r1; b += 32) {
        const int64_t x = b + lane;
        SeedEdge e{false, 0u, 0};
        int32_t k = 0;
        if (x < r1) {
            k = a.c_col[x];
            if (k >= 0 && k < a.n) {
                e = seed_edge(Li, a.off[k + 1] - a.off[k], a.c_si[x], a.c_sk[x], a.K, a.min_ov);
            } else if (!WRITE) {
                atomicOr(err, (uint32_t)DEV_INVALID);
            }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, e.keep);
        if (WRITE && e.keep) {
            const int64_t o = w + __popc(m & ((1u << lane) - 1u));
            if (SG_IN_BOUNDS(o < r_rp[i + 1], 601, o)) {
                r_col[o] = k;
                r_suf[o] = e.suffix;
                r_dir[o] = e.dir;
            }
        }
        w += __popc(m);
    }
    if (!WRITE && lane == 0) cnt[i] = w;
}

static inline int64_t blocks_for(int64_t n, int nt) { return (n + nt - 1) / nt; }

}  // namespace sg

extern "C" sg_status sg_overlap_graph_from_seeds(const sg_overlap_csr *C, const int64_t *d_offsets, int32_t k,
                                                 uint32_t min_overlap, sg_graph_csr *R, sg_stream_t stream) {
    if (!R) {
        sg::set_error("overlap_graph_from_seeds: NULL output");
        return SG_ERR_INVALID;
    }
    *R = sg_graph_csr{};
    if (!C || !d_offsets || C->n < 0 || C->n >= ((int64_t)1 << 31) || C->nnz < 0 || !C->row_ptr ||
        (C->nnz > 0 && (!C->col || !C->seed_i || !C->seed_k)) || C->max_seeds < 1 || k < 1 || k > 31 ||
        (k & 1) == 0 || min_overlap < 1) {
        sg::set_error("overlap_graph_from_seeds: invalid arguments (C needs max_seeds >= 1; odd k in 1..31; "
                      "min_overlap >= 1)");
        return SG_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = C->n;
    sg_status st = SG_OK;
    {
        sg::Scratch sc(s);
        uint32_t *err = sc.get<uint32_t>(1);
        int64_t *cnt = sc.get<int64_t>(n + 1);
        if (!err || !cnt) return SG_ERR_OOM;
        sg::StageScope stage("GraphFromSeeds", s);
        st = [&]() -> sg_status {
            SG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), s));
            const sg::SeedArgs a{C->row_ptr, C->col, C->seed_i, C->seed_k, d_offsets, n, k, (int64_t)min_overlap};
            SG_LAUNCH("seed_edges_count", sg::seed_edges_kernel<false>, sg::blocks_for(n * 32, 256), 256, 0, s, a,
                      cnt, (const int64_t *)nullptr, (int32_t *)nullptr, (uint32_t *)nullptr, (uint8_t *)nullptr,
                      err);
            int64_t *rp = (int64_t *)sg::dalloc((n + 1) * sizeof(int64_t), s);
            if (!rp) return SG_ERR_OOM;
            R->row_ptr = rp;
            R->n = n;
            SG_TRY(sg::exclusive_scan<int64_t>(cnt, rp, n, s, err));
            int64_t nnz = 0;
            uint32_t herr = 0;
            SG_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            SG_CUDA_TRY(sg::read_back(&nnz, rp + n, sizeof(int64_t), s));
            if (herr & sg::DEV_TIMEOUT) return sg::timeout_error("overlap_graph_from_seeds");
            if (herr) {
                sg::set_error("overlap_graph_from_seeds: C has a column outside [0, n)");
                return SG_ERR_INVALID;
            }
            R->nnz = nnz;
            SG_ALLOC(R->col, int32_t, nnz, s);
            SG_ALLOC(R->suffix, uint32_t, nnz, s);
            SG_ALLOC(R->dir, uint8_t, nnz, s);
            SG_LAUNCH("seed_edges_write", sg::seed_edges_kernel<true>, sg::blocks_for(n * 32, 256), 256, 0, s, a,
                      (int64_t *)nullptr, (const int64_t *)rp, R->col, R->suffix, R->dir, err);
            return SG_OK;
        }();
    }
    if (st != SG_OK) sg_free_graph(R, stream);
    return st;
}
