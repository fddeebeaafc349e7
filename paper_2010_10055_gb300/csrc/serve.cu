// serve.cu -- continuous-batching server for overlap + transitive-reduction jobs.
//
// Jobs are submitted from host buffers (copied at submit) and queue in arrival order. Each of
// `workers` threads owns a CUDA stream; whenever one is idle it admits the longest prefix of the
// queue that fits both max_batch and the free part of the device-memory budget, runs the admitted
// jobs as one sg_run_batch (block-diagonal, so every job's result equals its result alone), copies
// the results back and publishes them. A job arriving while other batches are on the GPU is
// admitted by the next idle worker as soon as memory frees up, and batches on different workers
// overlap on the device. A job whose estimate alone exceeds the budget runs alone, once nothing
// else is on the device, with C formed in row tiles under what the budget leaves
// (sg_overlap_spgemm_tiled); one that does not fit even so completes with SG_ERR_BUDGET.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ops.cuh"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
    uint64_t ticket;
    std::vector<uint8_t> seq;
    std::vector<int64_t> off, rrp;
    std::vector<int32_t> rcol;
    std::vector<uint32_t> rsuf;
    std::vector<uint8_t> rdir;
    uint32_t lo, hi;
    bool has_r;
    size_t est, est_tiled;
    double t_submit;
};

struct Done {
    sg_job_result r;
};

// Device bytes a job may need while its batch runs (inputs, filters, candidates, matrices).
size_t estimate_bytes(const Job &j) {
    return (size_t)64 * j.seq.size() + (size_t)48 * j.rcol.size() + (size_t)64 * j.off.size() + (1u << 20);
}

// Device bytes of the parts of a job that are not C: inputs, A and At, R and the reduction.
size_t resident_bytes(const Job &j) {
    return (size_t)24 * j.seq.size() + (size_t)48 * j.rcol.size() + (size_t)64 * j.off.size() + (1u << 20);
}

// ... and with C formed in row tiles (sg_overlap_spgemm_tiled): the k-mer stage's peak (about
// 40 B per base) or the resident part plus the smallest useful tile budget, whichever is larger.
constexpr size_t MIN_TILE_BUDGET = (size_t)64 << 20;
size_t estimate_tiled_bytes(const Job &j) {
    const size_t kmer = (size_t)40 * j.seq.size() + (size_t)64 * j.off.size() + (1u << 20);
    const size_t rest = resident_bytes(j) + MIN_TILE_BUDGET;
    return kmer > rest ? kmer : rest;
}

}  // namespace

struct sg_server {
    sg_server_config cfg;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::unordered_map<uint64_t, Done *> done;
    size_t budget_used = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> threads;
};

namespace sg {

static void fill_error(sg_job_result *r, sg_status st, double t_sub, const char *msg) {
    memset(r, 0, sizeof(*r));
    r->status = st;
    r->t_submit = t_sub;
    r->t_start = r->t_done = now_s();
    snprintf(r->error, sizeof(r->error), "%s", msg);
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Runs one admitted batch on stream s and fills each job's result.
static void run_batch_on(sg_server *srv, std::vector<Job *> &jobs, cudaStream_t s, std::vector<Done *> &out) {
    const double t_start = now_s();
    const int nb = (int)jobs.size();
    out.assign(nb, nullptr);
    for (int b = 0; b < nb; b++) out[b] = new Done();
    sg_status st = SG_OK;
    std::vector<sg_batch_item> items(nb);
    std::vector<sg_graph_csr> Rs(nb);
    // every job's inputs in one device buffer, each array on a 256-byte boundary
    size_t bytes = 0;
    for (Job *jp : jobs) {
        bytes += up256(jp->seq.size() + 16) + up256(jp->off.size() * 8);
        if (jp->has_r)
            bytes += up256(jp->rrp.size() * 8) + up256((jp->rcol.size() + 1) * 4) * 2 + up256(jp->rcol.size() + 1);
    }
    Scratch sc(s);
    unsigned char *dbuf = sc.get<unsigned char>(bytes);
    if (!dbuf) st = SG_ERR_OOM;
    size_t at = 0;
    auto put = [&](const void *src, size_t n, size_t room) -> void * {
        void *dst = dbuf + at;
        at += up256(room);
        if (n && st == SG_OK && cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            set_error("server: input upload failed");
            st = SG_ERR_CUDA;
        }
        return dst;
    };
    for (int b = 0; b < nb && st == SG_OK; b++) {
        Job &j = *jobs[b];
        const int64_t n = (int64_t)j.off.size() - 1;
        const uint8_t *dseq = (const uint8_t *)put(j.seq.data(), j.seq.size(), j.seq.size() + 16);
        const int64_t *doff = (const int64_t *)put(j.off.data(), j.off.size() * 8, j.off.size() * 8);
        items[b] = sg_batch_item{dseq, doff, n, (int64_t)j.seq.size(), j.lo, j.hi, nullptr};
        if (j.has_r) {
            const int64_t nnz = (int64_t)j.rcol.size();
            int64_t *rp = (int64_t *)put(j.rrp.data(), j.rrp.size() * 8, j.rrp.size() * 8);
            int32_t *rc = (int32_t *)put(j.rcol.data(), nnz * 4, (nnz + 1) * 4);
            uint32_t *rs = (uint32_t *)put(j.rsuf.data(), nnz * 4, (nnz + 1) * 4);
            uint8_t *rd = (uint8_t *)put(j.rdir.data(), nnz, nnz + 1);
            Rs[b] = sg_graph_csr{n, nnz, rp, rc, rs, rd};
            items[b].R = &Rs[b];
        }
    }
    sg_batch_result br{};
    if (st == SG_OK) st = sg_run_batch(items.data(), nb, &srv->cfg.params, &br, (sg_stream_t)s);
    std::vector<int64_t> crp, srp;
    std::vector<int32_t> ccol, scol;
    std::vector<uint32_t> ccnt, csi, csk, ssuf;
    std::vector<uint8_t> sdir;
    if (st == SG_OK) {
        const int64_t N = br.read_off[nb], cn = br.C.nnz, S = br.C.max_seeds, sn = br.S.nnz;
        crp.resize(N + 1); ccol.resize(cn); ccnt.resize(cn); csi.resize(cn * S); csk.resize(cn * S);
        cudaError_t e = cudaMemcpyAsync(crp.data(), br.C.row_ptr, (N + 1) * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && cn) e = cudaMemcpyAsync(ccol.data(), br.C.col, cn * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && cn) e = cudaMemcpyAsync(ccnt.data(), br.C.count, cn * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && cn && S) e = cudaMemcpyAsync(csi.data(), br.C.seed_i, cn * S * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && cn && S) e = cudaMemcpyAsync(csk.data(), br.C.seed_k, cn * S * 4, cudaMemcpyDeviceToHost, s);
        if (br.S.row_ptr) {
            srp.resize(N + 1); scol.resize(sn); ssuf.resize(sn); sdir.resize(sn);
            if (e == cudaSuccess) e = cudaMemcpyAsync(srp.data(), br.S.row_ptr, (N + 1) * 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && sn) e = cudaMemcpyAsync(scol.data(), br.S.col, sn * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && sn) e = cudaMemcpyAsync(ssuf.data(), br.S.suffix, sn * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && sn) e = cudaMemcpyAsync(sdir.data(), br.S.dir, sn, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("server: result download failed: %s", cudaGetErrorString(e));
            st = SG_ERR_CUDA;
        }
    }
    const char *msg = st == SG_OK ? "" : sg_last_error();
    const double t_done = now_s();
    for (int b = 0; b < nb; b++) {
        sg_job_result &r = out[b]->r;
        memset(&r, 0, sizeof(r));
        r.status = st;
        r.t_submit = jobs[b]->t_submit;
        r.t_start = t_start;
        r.t_done = t_done;
        r.batch_size = nb;
        if (st != SG_OK) {
            snprintf(r.error, sizeof(r.error), "%s", msg);
            continue;
        }
        const int64_t r0 = br.read_off[b], r1 = br.read_off[b + 1], n = r1 - r0, S = br.C.max_seeds;
        const int64_t cb = crp[r0], ce = crp[r1], cn = ce - cb, cN = br.C.nnz;
        r.n = n;
        r.m = br.col_off[b + 1] - br.col_off[b];
        r.nnz_c = cn;
        r.max_seeds = (int32_t)S;
        r.c_row_ptr = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
        r.c_col = (int32_t *)malloc(sizeof(int32_t) * (cn ? cn : 1));
        r.c_count = (uint32_t *)malloc(sizeof(uint32_t) * (cn ? cn : 1));
        r.c_seed_i = (uint32_t *)malloc(sizeof(uint32_t) * (cn * S > 0 ? cn * S : 1));
        r.c_seed_k = (uint32_t *)malloc(sizeof(uint32_t) * (cn * S > 0 ? cn * S : 1));
        for (int64_t i = 0; i <= n; i++) r.c_row_ptr[i] = crp[r0 + i] - cb;
        for (int64_t e = 0; e < cn; e++) {
            r.c_col[e] = ccol[cb + e] - (int32_t)r0;
            r.c_count[e] = ccnt[cb + e];
        }
        for (int64_t q = 0; q < S; q++)
            for (int64_t e = 0; e < cn; e++) {
                r.c_seed_i[q * cn + e] = csi[q * cN + cb + e];
                r.c_seed_k[q * cn + e] = csk[q * cN + cb + e];
            }
        if (jobs[b]->has_r && !srp.empty()) {
            const int64_t sb = srp[r0], se = srp[r1], sn = se - sb;
            r.nnz_s = sn;
            r.iterations = br.iterations[b];
            r.s_row_ptr = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
            r.s_col = (int32_t *)malloc(sizeof(int32_t) * (sn ? sn : 1));
            r.s_suffix = (uint32_t *)malloc(sizeof(uint32_t) * (sn ? sn : 1));
            r.s_dir = (uint8_t *)malloc(sn ? sn : 1);
            for (int64_t i = 0; i <= n; i++) r.s_row_ptr[i] = srp[r0 + i] - sb;
            for (int64_t e = 0; e < sn; e++) {
                r.s_col[e] = scol[sb + e] - (int32_t)r0;
                r.s_suffix[e] = ssuf[sb + e];
                r.s_dir[e] = sdir[sb + e];
            }
        }
    }
    sg_free_batch(&br, (sg_stream_t)s);
}

// A job too large for the budget in one piece, run alone: A and At as usual, C formed in row
// tiles under what the budget leaves once the rest of the job is resident (each tile copied to
// the host as it completes), then the reduction of R.
struct TileSink {
    cudaStream_t s;
    int S;
    std::vector<int64_t> rp;
    std::vector<int32_t> col;
    std::vector<uint32_t> cnt;
    std::vector<std::vector<uint32_t>> si, sk;  // per seed slot
};

static sg_status tile_to_host(const sg_overlap_csr *t, int64_t row_begin, void *user) {
    TileSink &k = *(TileSink *)user;
    (void)row_begin;  // tiles arrive in row order
    const int64_t base = (int64_t)k.col.size(), nt = t->nnz;
    std::vector<int64_t> rp(t->n + 1);
    k.col.resize(base + nt);
    k.cnt.resize(base + nt);
    cudaError_t e = cudaMemcpyAsync(rp.data(), t->row_ptr, (t->n + 1) * 8, cudaMemcpyDeviceToHost, k.s);
    if (e == cudaSuccess && nt) e = cudaMemcpyAsync(k.col.data() + base, t->col, nt * 4, cudaMemcpyDeviceToHost, k.s);
    if (e == cudaSuccess && nt) e = cudaMemcpyAsync(k.cnt.data() + base, t->count, nt * 4, cudaMemcpyDeviceToHost, k.s);
    for (int q = 0; q < k.S && e == cudaSuccess; q++) {
        k.si[q].resize(base + nt);
        k.sk[q].resize(base + nt);
        if (nt) e = cudaMemcpyAsync(k.si[q].data() + base, t->seed_i + (int64_t)q * nt, nt * 4, cudaMemcpyDeviceToHost, k.s);
        if (e == cudaSuccess && nt)
            e = cudaMemcpyAsync(k.sk[q].data() + base, t->seed_k + (int64_t)q * nt, nt * 4, cudaMemcpyDeviceToHost, k.s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(k.s);
    if (e != cudaSuccess) {
        set_error("server: tile download failed: %s", cudaGetErrorString(e));
        return SG_ERR_CUDA;
    }
    for (int64_t i = 1; i <= t->n; i++) k.rp.push_back(base + rp[i]);
    return SG_OK;
}

static void run_large_on(sg_server *srv, Job *jp, cudaStream_t s, Done *&out) {
    const double t_start = now_s();
    out = new Done();
    Job &j = *jp;
    const sg_batch_params &p = srv->cfg.params;
    const int64_t n = (int64_t)j.off.size() - 1;
    sg_status st = SG_OK;
    sg_csr_u32 A{}, At{};
    uint64_t *codes = nullptr;
    sg_graph_csr Sg{};
    int32_t iters = 0;
    int64_t m_cols = 0;
    TileSink sink;
    sink.s = s;
    sink.S = p.max_seeds;
    sink.rp.push_back(0);
    sink.si.resize(p.max_seeds);
    sink.sk.resize(p.max_seeds);
    std::vector<int64_t> srp;
    std::vector<int32_t> scol;
    std::vector<uint32_t> ssuf;
    std::vector<uint8_t> sdir;
    {
        Scratch sc(s);
        uint8_t *dseq = sc.get<uint8_t>(j.seq.size() + 16);
        int64_t *doff = sc.get<int64_t>(j.off.size());
        if (!dseq || !doff) st = SG_ERR_OOM;
        if (st == SG_OK && (cudaMemcpyAsync(dseq, j.seq.data(), j.seq.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                            cudaMemcpyAsync(doff, j.off.data(), j.off.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)) {
            set_error("server: input upload failed");
            st = SG_ERR_CUDA;
        }
        if (st == SG_OK)
            st = sg_build_kmer_matrix(dseq, doff, n, (int64_t)j.seq.size(), p.k, j.lo, j.hi, &A, &At, &codes,
                                      (sg_stream_t)s);
        dfree(codes, s);
        codes = nullptr;
        if (st == SG_OK) {
            const size_t res = resident_bytes(j), budget = srv->cfg.hbm_budget;
            const size_t tb = budget > res + MIN_TILE_BUDGET ? budget - res : MIN_TILE_BUDGET;
            int64_t ntiles = 0;
            st = sg_overlap_spgemm_tiled(&A, &At, p.min_shared, p.max_seeds, tb, tile_to_host, &sink, &ntiles,
                                         (sg_stream_t)s);
        }
        m_cols = A.n_cols;
        sg_free_csr_u32(&A, (sg_stream_t)s);
        sg_free_csr_u32(&At, (sg_stream_t)s);
        if (st == SG_OK && j.has_r) {
            const int64_t nnz = (int64_t)j.rcol.size();
            int64_t *rp = sc.get<int64_t>(n + 1);
            int32_t *rc = sc.get<int32_t>(nnz + 1);
            uint32_t *rs = sc.get<uint32_t>(nnz + 1);
            uint8_t *rd = sc.get<uint8_t>(nnz + 1);
            if (!rp || !rc || !rs || !rd) st = SG_ERR_OOM;
            cudaError_t e = cudaSuccess;
            if (st == SG_OK) e = cudaMemcpyAsync(rp, j.rrp.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s);
            if (st == SG_OK && e == cudaSuccess && nnz) e = cudaMemcpyAsync(rc, j.rcol.data(), nnz * 4, cudaMemcpyHostToDevice, s);
            if (st == SG_OK && e == cudaSuccess && nnz) e = cudaMemcpyAsync(rs, j.rsuf.data(), nnz * 4, cudaMemcpyHostToDevice, s);
            if (st == SG_OK && e == cudaSuccess && nnz) e = cudaMemcpyAsync(rd, j.rdir.data(), nnz, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                set_error("server: R upload failed");
                st = SG_ERR_CUDA;
            }
            sg_graph_csr R{n, nnz, rp, rc, rs, rd};
            if (st == SG_OK) st = sg_transitive_reduce(&R, p.fuzz, p.tr_mode, &Sg, &iters, (sg_stream_t)s);
            if (st == SG_OK) {
                srp.resize(n + 1);
                scol.resize(Sg.nnz);
                ssuf.resize(Sg.nnz);
                sdir.resize(Sg.nnz);
                e = cudaMemcpyAsync(srp.data(), Sg.row_ptr, (n + 1) * 8, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess && Sg.nnz) e = cudaMemcpyAsync(scol.data(), Sg.col, Sg.nnz * 4, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess && Sg.nnz) e = cudaMemcpyAsync(ssuf.data(), Sg.suffix, Sg.nnz * 4, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess && Sg.nnz) e = cudaMemcpyAsync(sdir.data(), Sg.dir, Sg.nnz, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) {
                    set_error("server: result download failed: %s", cudaGetErrorString(e));
                    st = SG_ERR_CUDA;
                }
            }
            sg_free_graph(&Sg, (sg_stream_t)s);
        }
    }
    sg_job_result &r = out->r;
    memset(&r, 0, sizeof(r));
    r.status = st;
    r.t_submit = j.t_submit;
    r.t_start = t_start;
    r.t_done = now_s();
    r.batch_size = 1;
    if (st != SG_OK) {
        snprintf(r.error, sizeof(r.error), "%s", sg_last_error());
        return;
    }
    const int64_t cn = (int64_t)sink.col.size(), S = p.max_seeds;
    r.n = n;
    r.m = m_cols;
    r.nnz_c = cn;
    r.max_seeds = (int32_t)S;
    r.c_row_ptr = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    r.c_col = (int32_t *)malloc(sizeof(int32_t) * (cn ? cn : 1));
    r.c_count = (uint32_t *)malloc(sizeof(uint32_t) * (cn ? cn : 1));
    r.c_seed_i = (uint32_t *)malloc(sizeof(uint32_t) * (cn * S > 0 ? cn * S : 1));
    r.c_seed_k = (uint32_t *)malloc(sizeof(uint32_t) * (cn * S > 0 ? cn * S : 1));
    memcpy(r.c_row_ptr, sink.rp.data(), sizeof(int64_t) * (n + 1));
    if (cn) {
        memcpy(r.c_col, sink.col.data(), sizeof(int32_t) * cn);
        memcpy(r.c_count, sink.cnt.data(), sizeof(uint32_t) * cn);
        for (int64_t q = 0; q < S; q++) {
            memcpy(r.c_seed_i + q * cn, sink.si[q].data(), sizeof(uint32_t) * cn);
            memcpy(r.c_seed_k + q * cn, sink.sk[q].data(), sizeof(uint32_t) * cn);
        }
    }
    if (j.has_r) {
        const int64_t sn = (int64_t)scol.size();
        r.nnz_s = sn;
        r.iterations = iters;
        r.s_row_ptr = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
        r.s_col = (int32_t *)malloc(sizeof(int32_t) * (sn ? sn : 1));
        r.s_suffix = (uint32_t *)malloc(sizeof(uint32_t) * (sn ? sn : 1));
        r.s_dir = (uint8_t *)malloc(sn ? sn : 1);
        memcpy(r.s_row_ptr, srp.data(), sizeof(int64_t) * (n + 1));
        if (sn) {
            memcpy(r.s_col, scol.data(), sizeof(int32_t) * sn);
            memcpy(r.s_suffix, ssuf.data(), sizeof(uint32_t) * sn);
            memcpy(r.s_dir, sdir.data(), sn);
        }
    }
}

static void worker_main(sg_server *srv) {
    if (cudaSetDevice(srv->cfg.device) != cudaSuccess) return;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    const size_t budget = srv->cfg.hbm_budget;
    for (;;) {
        std::vector<Job *> batch;
        Job *large = nullptr;
        size_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                if (srv->stop) break;
                // jobs that can never fit, not even with C in tiles, are answered right away
                while (!srv->pending.empty() && srv->pending.front()->est > budget &&
                       srv->pending.front()->est_tiled > budget) {
                    Job *j = srv->pending.front();
                    srv->pending.pop_front();
                    Done *d = new Done();
                    char msg[160];
                    snprintf(msg, sizeof(msg),
                             "job needs about %zu bytes of device memory (%zu with C in tiles), the budget is %zu",
                             j->est, j->est_tiled, budget);
                    fill_error(&d->r, SG_ERR_BUDGET, j->t_submit, msg);
                    srv->done[j->ticket] = d;
                    delete j;
                    srv->cv_done.notify_all();
                }
                // a job that fits only with C in tiles runs alone, with the whole budget
                if (!srv->pending.empty() && srv->pending.front()->est > budget) {
                    if (srv->budget_used == 0) {
                        large = srv->pending.front();
                        srv->pending.pop_front();
                        bytes = budget;
                        break;
                    }
                    srv->cv_work.wait(lk);
                    continue;
                }
                while (!srv->pending.empty() && (int)batch.size() < srv->cfg.max_batch &&
                       srv->pending.front()->est <= budget &&
                       srv->budget_used + bytes + srv->pending.front()->est <= budget) {
                    bytes += srv->pending.front()->est;
                    batch.push_back(srv->pending.front());
                    srv->pending.pop_front();
                }
                if (!batch.empty()) break;
                srv->cv_work.wait(lk);
            }
            if (batch.empty() && !large) break;  // stopping
            srv->budget_used += bytes;
        }
        std::vector<Done *> res;
        if (large) {
            res.resize(1);
            run_large_on(srv, large, s, res[0]);
            batch.push_back(large);
        } else {
            run_batch_on(srv, batch, s, res);
        }
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->budget_used -= bytes;
            for (size_t b = 0; b < batch.size(); b++) srv->done[batch[b]->ticket] = res[b];
        }
        for (Job *j : batch) delete j;
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();  // memory freed: another worker may admit now
    }
    cudaStreamDestroy(s);
}

}  // namespace sg

extern "C" sg_status sg_server_create(const sg_server_config *cfg, sg_server **out) {
    if (!cfg || !out || cfg->workers < 1 || cfg->workers > 64 || cfg->max_batch < 1 || cfg->hbm_budget == 0 ||
        cfg->params.k < 1 || cfg->params.k > 31 || (cfg->params.k & 1) == 0) {
        sg::set_error("server_create: invalid configuration");
        return SG_ERR_INVALID;
    }
    sg_server *srv = new (std::nothrow) sg_server();
    if (!srv) return SG_ERR_OOM;
    srv->cfg = *cfg;
    for (int w = 0; w < cfg->workers; w++) srv->threads.emplace_back(sg::worker_main, srv);
    *out = srv;
    return SG_OK;
}

extern "C" sg_status sg_server_submit(sg_server *srv, const sg_job *job, uint64_t *ticket) {
    if (!srv || !job || !ticket || job->n_reads < 0 || job->total_len < 0 || !job->offsets ||
        (job->total_len > 0 && !job->seq) || job->lo < 1 || job->lo > job->hi ||
        (job->r_row_ptr && job->r_nnz > 0 && (!job->r_col || !job->r_suffix || !job->r_dir))) {
        sg::set_error("server_submit: invalid job");
        return SG_ERR_INVALID;
    }
    Job *j = new (std::nothrow) Job();
    if (!j) return SG_ERR_OOM;
    j->seq.assign(job->seq, job->seq + job->total_len);
    j->off.assign(job->offsets, job->offsets + job->n_reads + 1);
    j->lo = job->lo;
    j->hi = job->hi;
    j->has_r = job->r_row_ptr != nullptr;
    if (j->has_r) {
        j->rrp.assign(job->r_row_ptr, job->r_row_ptr + job->n_reads + 1);
        j->rcol.assign(job->r_col, job->r_col + job->r_nnz);
        j->rsuf.assign(job->r_suffix, job->r_suffix + job->r_nnz);
        j->rdir.assign(job->r_dir, job->r_dir + job->r_nnz);
    }
    j->est = estimate_bytes(*j);
    j->est_tiled = estimate_tiled_bytes(*j);
    j->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        j->ticket = srv->next_ticket++;
        *ticket = j->ticket;
        srv->pending.push_back(j);
    }
    srv->cv_work.notify_one();
    return SG_OK;
}

extern "C" sg_status sg_server_cancel(sg_server *srv, uint64_t ticket) {
    if (!srv) {
        sg::set_error("server_cancel: NULL server");
        return SG_ERR_INVALID;
    }
    Job *j = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (auto it = srv->pending.begin(); it != srv->pending.end(); ++it)
            if ((*it)->ticket == ticket) {
                j = *it;
                srv->pending.erase(it);
                break;
            }
        if (j) {
            Done *d = new Done();
            sg::fill_error(&d->r, SG_ERR_CANCELLED, j->t_submit, "cancelled before it ran");
            srv->done[ticket] = d;
        }
    }
    if (!j) {
        sg::set_error("server_cancel: job %llu is not queued (unknown, running or done)", (unsigned long long)ticket);
        return SG_ERR_INVALID;
    }
    delete j;
    srv->cv_done.notify_all();
    return SG_OK;
}

static sg_status take_done(sg_server *srv, uint64_t ticket, sg_job_result *out) {
    auto it = srv->done.find(ticket);
    if (it == srv->done.end()) return SG_ERR_TIMEOUT;
    *out = it->second->r;
    delete it->second;
    srv->done.erase(it);
    return SG_OK;
}

extern "C" sg_status sg_server_poll(sg_server *srv, uint64_t ticket, sg_job_result *out) {
    if (!srv || !out) return SG_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    return take_done(srv, ticket, out);
}

extern "C" sg_status sg_server_wait(sg_server *srv, uint64_t ticket, double timeout_s, sg_job_result *out) {
    if (!srv || !out) return SG_ERR_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        if (take_done(srv, ticket, out) == SG_OK) return SG_OK;
        if (srv->cv_done.wait_until(lk, until) == std::cv_status::timeout) return take_done(srv, ticket, out);
    }
}

extern "C" void sg_job_result_free(sg_job_result *r) {
    if (!r) return;
    free(r->c_row_ptr);
    free(r->c_col);
    free(r->c_count);
    free(r->c_seed_i);
    free(r->c_seed_k);
    free(r->s_row_ptr);
    free(r->s_col);
    free(r->s_suffix);
    free(r->s_dir);
    memset(r, 0, sizeof(*r));
}

extern "C" void sg_server_destroy(sg_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->threads) t.join();
    for (Job *j : srv->pending) delete j;
    for (auto &kv : srv->done) {
        sg_job_result_free(&kv.second->r);
        delete kv.second;
    }
    delete srv;
}
