/*
 * sgo.c -- ORACLE: plain, slow, obviously correct CPU definitions of the three operations of
 * the overlap-and-layout hot path of diBELLA 2D (arXiv 2010.10055).
 *
 * This is TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg call it; the library's product path never does. It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Everything here is integer arithmetic, done in the order the definitions state it:
 *   sgo_build_kmer_matrix  -- Sec. II (canonical form), Sec. IV-C (k-mer frequency and the
 *                             reliable range), Sec. IV-D (A_ij = position of k-mer j in read i)
 *   sgo_overlap_spgemm     -- Sec. IV-D: C = A A^T over the overlap semiring (count of shared
 *                             k-mers plus the positions of up to max_seeds of them)
 *   sgo_minplus            -- Algorithm 3 (MinPlus semiring with the walk-validity check of
 *                             Sec. II / IV-E), evaluated on the pattern of R
 *   sgo_transitive_reduce  -- Algorithm 1 (Reduce/Apply/DimApply, M >= N, R o not I, until
 *                             nnz(R) stops changing)
 *   sgo_graph_from_seeds   -- R estimated from C's first seeds (overlap interval, containment,
 *                             suffix and dir), the alignment's role in Algorithm 2
 *   sgo_kmer_census, sgo_read_windows, sgo_overlap_row -- single outputs of the same definitions
 *                             (a k-mer's frequency and occurrences, a read's windows, one row of
 *                             C), for sampled checks at sizes where the whole oracle is too slow
 *
 * Readings of places where the paper is silent (all shared with the CUDA path's spec):
 *  - A_ij keeps the LOWEST position of k-mer j in read i; every occurrence still counts
 *    toward the k-mer's frequency.
 *  - A k-mer is reliable iff lo <= freq <= hi (the paper's cut "at least d times" is hi = d-1).
 *  - The seeds kept in C_ik are those of the max_seeds shared k-mers with the smallest column
 *    index (= smallest canonical code); seed_i = position in read i, seed_k = position in read k
 *    with bit 31 = strand_i xor strand_k. Unused seed slots hold 0xFFFFFFFF.
 *  - Entries with fewer than min_shared shared k-mers are dropped; the diagonal is never stored.
 *  - Edge dir (2 bits): bit 1 = orientation of the walk's first read, bit 0 = orientation of its
 *    second read. A walk i->j->k is valid iff in(d_ij) == out(d_jk) (the two heads at j point
 *    opposite ways); its composite dir is 2*out(d_ij) + in(d_jk). The endpoint rules (b), (c)
 *    of Sec. II hold iff the composite equals d_ik.
 *  - mode 0 (DIRMATCH): N_ik is the min of R_ij + R_jk over valid walks whose composite dir is
 *    d_ik. mode 1 (LITERAL): N_ik is the lexicographic min of (R_ij + R_jk, composite) over all
 *    valid walks, and the endpoint check is applied to that single minimum afterwards.
 *  - The row maximum is over the whole row (0 for an empty row); M_ik >= N_ik removes on ties.
 *    With mode bit 1 (PER_END) it is taken per read end of the row's read instead, each entry
 *    bounded by the maximum of the entries that leave the read through the same end.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SGO_OK 0
#define SGO_INVALID 1
#define SGO_OOM 2
#define SGO_INF 0xFFFFFFFFu

typedef struct { int64_t n_rows, n_cols, nnz; int64_t *row_ptr; int32_t *col; uint32_t *val; } sgo_csr;
typedef struct {
    int64_t n, nnz; int32_t max_seeds;
    int64_t *row_ptr; int32_t *col; uint32_t *count;
    uint32_t *seed_i; uint32_t *seed_k; /* [max_seeds][nnz], slot-major */
} sgo_overlap;
typedef struct { int64_t n, nnz; int64_t *row_ptr; int32_t *col; uint32_t *suffix; uint8_t *dir; } sgo_graph;

void sgo_free(void *p) { free(p); }

/* ============================================================ k-mers and A */
static int base_code(uint8_t c) {
    switch (c) { case 'A': return 0; case 'C': return 1; case 'G': return 2; case 'T': return 3; }
    return -1;
}

/* Canonical k-mer of the window seq[p .. p+k-1] (Sec. II): f reads the window as a base-4
 * number, first base most significant; r does the same for its reverse complement. With
 * A<C<G<T, numeric order is lexicographic order, so the canonical form is min(f, r).
 * Returns 0 if the window holds a character other than A, C, G, T. */
static int window_code(const uint8_t *w, int k, uint64_t *code, uint32_t *strand) {
    uint64_t f = 0, r = 0;
    for (int t = 0; t < k; t++) {
        int b = base_code(w[t]);
        if (b < 0) return 0;
        f = f * 4 + (uint64_t)b;
    }
    for (int t = 0; t < k; t++) {
        int b = base_code(w[k - 1 - t]);
        r = r * 4 + (uint64_t)(3 - b);
    }
    *code = f < r ? f : r;
    *strand = (r < f) ? 1u : 0u;
    return 1;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}
typedef struct { int32_t col; uint32_t pos; uint32_t strand; } occ_t;
static int cmp_occ(const void *a, const void *b) {
    const occ_t *x = (const occ_t *)a, *y = (const occ_t *)b;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    return (x->pos > y->pos) - (x->pos < y->pos);
}

/*
 * A (n x m, CSR): row i lists the reliable k-mers of read i by ascending column; the value is
 * pos | strand << 31 at the lowest position pos where the k-mer occurs in read i.
 * At (m x n): the transpose, reads ascending within each row. codes[j] = canonical code of
 * column j; columns are numbered by ascending code.
 */
int sgo_build_kmer_matrix(const uint8_t *seq, const int64_t *offsets, int64_t n, int32_t k,
                          uint32_t lo, uint32_t hi, sgo_csr *A, sgo_csr *At,
                          uint64_t **codes_out, int64_t *m_out) {
    memset(A, 0, sizeof(*A)); memset(At, 0, sizeof(*At));
    *codes_out = NULL; *m_out = 0;
    if (k < 1 || k > 31 || (k % 2) == 0 || lo < 1 || lo > hi || n < 0) return SGO_INVALID;
    for (int64_t i = 0; i < n; i++)
        if (offsets[i + 1] < offsets[i] || offsets[i + 1] - offsets[i] >= ((int64_t)1 << 31)) return SGO_INVALID;
    if (n > 0 && offsets[0] != 0) return SGO_INVALID;

    /* 1. frequency of every canonical k-mer over all windows of all reads (Sec. IV-C) */
    int64_t nwin = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t len = offsets[i + 1] - offsets[i];
        if (len >= k) nwin += len - k + 1;
    }
    uint64_t *all = (uint64_t *)malloc((size_t)(nwin ? nwin : 1) * sizeof(uint64_t));
    if (!all) return SGO_OOM;
    int64_t na = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t p = 0; p + k <= offsets[i + 1] - offsets[i]; p++) {
            uint64_t c; uint32_t s;
            if (window_code(seq + offsets[i] + p, k, &c, &s)) all[na++] = c;
        }
    }
    qsort(all, (size_t)na, sizeof(uint64_t), cmp_u64);

    /* 2. reliable k-mers: lo <= freq <= hi; column id = rank by ascending code */
    int64_t m = 0;
    for (int64_t a = 0; a < na;) {
        int64_t b = a;
        while (b < na && all[b] == all[a]) b++;
        uint64_t freq = (uint64_t)(b - a);
        if (freq >= lo && freq <= hi) all[m++] = all[a];
        a = b;
    }
    uint64_t *codes = (uint64_t *)malloc((size_t)(m ? m : 1) * sizeof(uint64_t));
    if (!codes) { free(all); return SGO_OOM; }
    memcpy(codes, all, (size_t)m * sizeof(uint64_t));
    free(all);

    /* 3. A: per read, reliable occurrences sorted by (column, position); keep the first */
    int64_t *rp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    int64_t cap = 1024, nnz = 0;
    int32_t *acol = (int32_t *)malloc(cap * sizeof(int32_t));
    uint32_t *aval = (uint32_t *)malloc(cap * sizeof(uint32_t));
    int64_t maxlen = 0;
    for (int64_t i = 0; i < n; i++)
        if (offsets[i + 1] - offsets[i] > maxlen) maxlen = offsets[i + 1] - offsets[i];
    occ_t *occ = (occ_t *)malloc((size_t)(maxlen + 1) * sizeof(occ_t));
    if (!rp || !acol || !aval || !occ) { free(rp); free(acol); free(aval); free(occ); free(codes); return SGO_OOM; }
    for (int64_t i = 0; i < n; i++) {
        int64_t no = 0;
        for (int64_t p = 0; p + k <= offsets[i + 1] - offsets[i]; p++) {
            uint64_t c; uint32_t s;
            if (!window_code(seq + offsets[i] + p, k, &c, &s)) continue;
            uint64_t *hit = (uint64_t *)bsearch(&c, codes, (size_t)m, sizeof(uint64_t), cmp_u64);
            if (!hit) continue;
            occ[no].col = (int32_t)(hit - codes); occ[no].pos = (uint32_t)p; occ[no].strand = s;
            no++;
        }
        qsort(occ, (size_t)no, sizeof(occ_t), cmp_occ);
        for (int64_t e = 0; e < no; e++) {
            if (e > 0 && occ[e].col == occ[e - 1].col) continue;
            if (nnz == cap) {
                cap *= 2;
                int32_t *c2 = (int32_t *)realloc(acol, cap * sizeof(int32_t));
                if (c2) acol = c2;
                uint32_t *v2 = (uint32_t *)realloc(aval, cap * sizeof(uint32_t));
                if (v2) aval = v2;
                if (!c2 || !v2) { free(rp); free(acol); free(aval); free(occ); free(codes); return SGO_OOM; }
            }
            acol[nnz] = occ[e].col;
            aval[nnz] = occ[e].pos | (occ[e].strand << 31);
            nnz++;
        }
        rp[i + 1] = nnz;
    }
    free(occ);

    /* 4. At = transpose of A, filled row by row so each At row lists reads in order */
    int64_t *trp = (int64_t *)calloc((size_t)(m + 1), sizeof(int64_t));
    int32_t *tcol = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
    uint32_t *tval = (uint32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(uint32_t));
    int64_t *fill = (int64_t *)malloc((size_t)(m ? m : 1) * sizeof(int64_t));
    if (!trp || !tcol || !tval || !fill) {
        free(trp); free(tcol); free(tval); free(fill); free(rp); free(acol); free(aval); free(codes);
        return SGO_OOM;
    }
    for (int64_t e = 0; e < nnz; e++) trp[acol[e] + 1]++;
    for (int64_t j = 0; j < m; j++) trp[j + 1] += trp[j];
    for (int64_t j = 0; j < m; j++) fill[j] = trp[j];
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
            int64_t d = fill[acol[e]]++;
            tcol[d] = (int32_t)i;
            tval[d] = aval[e];
        }
    free(fill);

    A->n_rows = n; A->n_cols = m; A->nnz = nnz; A->row_ptr = rp; A->col = acol; A->val = aval;
    At->n_rows = m; At->n_cols = n; At->nnz = nnz; At->row_ptr = trp; At->col = tcol; At->val = tval;
    *codes_out = codes; *m_out = m;
    return SGO_OK;
}

/* ====================================================== C = A A^T (overlap) */
/*
 * Row-by-row Gustavson product over the overlap semiring (Sec. IV-D). For row i, the columns j
 * of A_i are visited in ascending order; each product with At_j contributes one shared k-mer to
 * C_ik. The first max_seeds contributions to C_ik are therefore the shared k-mers with the
 * smallest column index, and those are the ones whose positions are kept.
 */
int sgo_overlap_spgemm(const sgo_csr *A, const sgo_csr *At, uint32_t min_shared, int32_t max_seeds,
                       sgo_overlap *C) {
    memset(C, 0, sizeof(*C));
    if (max_seeds < 0 || max_seeds > 8 || min_shared < 1) return SGO_INVALID;
    if (A->n_cols != At->n_rows || A->n_rows != At->n_cols) return SGO_INVALID;
    int64_t n = A->n_rows;
    int S = max_seeds;
    uint32_t *cnt = (uint32_t *)calloc((size_t)(n ? n : 1), sizeof(uint32_t));
    uint32_t *si = (uint32_t *)malloc((size_t)(n ? n : 1) * (S ? S : 1) * sizeof(uint32_t));
    uint32_t *sk = (uint32_t *)malloc((size_t)(n ? n : 1) * (S ? S : 1) * sizeof(uint32_t));
    int64_t *touched = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *rp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    int64_t cap = 1024, nnz = 0;
    int32_t *ccol = (int32_t *)malloc(cap * sizeof(int32_t));
    uint32_t *ccnt = (uint32_t *)malloc(cap * sizeof(uint32_t));
    uint32_t *csi = (uint32_t *)malloc(cap * (S ? S : 1) * sizeof(uint32_t)); /* row-major [nnz][S] */
    uint32_t *csk = (uint32_t *)malloc(cap * (S ? S : 1) * sizeof(uint32_t));
    if (!cnt || !si || !sk || !touched || !rp || !ccol || !ccnt || !csi || !csk) goto oom;
    for (int64_t i = 0; i < n; i++) {
        int64_t nt = 0;
        for (int64_t a = A->row_ptr[i]; a < A->row_ptr[i + 1]; a++) {
            int64_t j = A->col[a];
            uint32_t vi = A->val[a];
            for (int64_t b = At->row_ptr[j]; b < At->row_ptr[j + 1]; b++) {
                int64_t kk = At->col[b];
                if (kk == i) continue;
                uint32_t vk = At->val[b];
                if (cnt[kk] == 0) touched[nt++] = kk;
                if (cnt[kk] < (uint32_t)S) {
                    si[kk * S + cnt[kk]] = vi & 0x7FFFFFFFu;
                    sk[kk * S + cnt[kk]] = (vk & 0x7FFFFFFFu) | ((vi ^ vk) & 0x80000000u);
                }
                cnt[kk]++;
            }
        }
        qsort(touched, (size_t)nt, sizeof(int64_t), cmp_u64); /* non-negative: u64 order is fine */
        for (int64_t q = 0; q < nt; q++) {
            int64_t kk = touched[q];
            if (cnt[kk] >= min_shared) {
                if (nnz == cap) {
                    cap *= 2;
                    int32_t *a1 = (int32_t *)realloc(ccol, cap * sizeof(int32_t)); if (a1) ccol = a1;
                    uint32_t *a2 = (uint32_t *)realloc(ccnt, cap * sizeof(uint32_t)); if (a2) ccnt = a2;
                    uint32_t *a3 = (uint32_t *)realloc(csi, cap * (S ? S : 1) * sizeof(uint32_t)); if (a3) csi = a3;
                    uint32_t *a4 = (uint32_t *)realloc(csk, cap * (S ? S : 1) * sizeof(uint32_t)); if (a4) csk = a4;
                    if (!a1 || !a2 || !a3 || !a4) goto oom;
                }
                ccol[nnz] = (int32_t)kk;
                ccnt[nnz] = cnt[kk];
                for (int s = 0; s < S; s++) {
                    int used = (uint32_t)s < cnt[kk];
                    csi[nnz * S + s] = used ? si[kk * S + s] : SGO_INF;
                    csk[nnz * S + s] = used ? sk[kk * S + s] : SGO_INF;
                }
                nnz++;
            }
            cnt[kk] = 0;
        }
        rp[i + 1] = nnz;
    }
    free(cnt); free(si); free(sk); free(touched);
    /* slot-major output layout: seed s of entry e at [s * nnz + e] */
    C->seed_i = (uint32_t *)malloc((size_t)(nnz * S ? nnz * S : 1) * sizeof(uint32_t));
    C->seed_k = (uint32_t *)malloc((size_t)(nnz * S ? nnz * S : 1) * sizeof(uint32_t));
    if (!C->seed_i || !C->seed_k) { free(C->seed_i); free(C->seed_k); free(rp); free(ccol); free(ccnt); free(csi); free(csk); return SGO_OOM; }
    for (int64_t e = 0; e < nnz; e++)
        for (int s = 0; s < S; s++) {
            C->seed_i[(int64_t)s * nnz + e] = csi[e * S + s];
            C->seed_k[(int64_t)s * nnz + e] = csk[e * S + s];
        }
    free(csi); free(csk);
    C->n = n; C->nnz = nnz; C->max_seeds = S; C->row_ptr = rp; C->col = ccol; C->count = ccnt;
    return SGO_OK;
oom:
    free(cnt); free(si); free(sk); free(touched); free(rp); free(ccol); free(ccnt); free(csi); free(csk);
    return SGO_OOM;
}

/* ====================================================== transitive reduction */
static int dir_in(uint8_t d) { return d & 1; }   /* orientation of the walk's second read */
static int dir_out(uint8_t d) { return d >> 1; } /* orientation of the walk's first read */

int sgo_validate_graph(const sgo_graph *R) {
    if (R->n < 0 || R->n >= ((int64_t)1 << 31)) return SGO_INVALID;
    if (R->row_ptr[0] != 0 || R->row_ptr[R->n] != R->nnz) return SGO_INVALID;
    for (int64_t i = 0; i < R->n; i++) {
        if (R->row_ptr[i + 1] < R->row_ptr[i]) return SGO_INVALID;
        for (int64_t e = R->row_ptr[i]; e < R->row_ptr[i + 1]; e++) {
            if (R->col[e] < 0 || R->col[e] >= R->n || R->col[e] == i) return SGO_INVALID;
            if (e > R->row_ptr[i] && R->col[e] <= R->col[e - 1]) return SGO_INVALID;
            if (R->suffix[e] >= (1u << 30) || R->dir[e] > 3) return SGO_INVALID;
        }
    }
    return SGO_OK;
}

/* index of entry (j, k) in R, or -1 (binary search over the sorted row j) */
static int64_t find_entry(const sgo_graph *R, int64_t j, int32_t k) {
    int64_t lo = R->row_ptr[j], hi = R->row_ptr[j + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (R->col[mid] < k) lo = mid + 1; else hi = mid;
    }
    return (lo < R->row_ptr[j + 1] && R->col[lo] == k) ? lo : -1;
}

/*
 * N = R^2 over the MinPlus semiring of Algorithm 3, evaluated only where R has an entry (the
 * element-wise M >= N step only looks at entries present in both). N[e] = 0xFFFFFFFF when no
 * walk qualifies. Ndir[e] = composite dir of the minimising walk (mode 1), or d_ik (mode 0).
 */
int sgo_minplus(const sgo_graph *R, int32_t mode, uint32_t *N, uint8_t *Ndir) {
    if (mode != 0 && mode != 1) return SGO_INVALID;
    for (int64_t i = 0; i < R->n; i++) {
        for (int64_t e = R->row_ptr[i]; e < R->row_ptr[i + 1]; e++) {
            int32_t kk = R->col[e];
            uint8_t dik = R->dir[e];
            uint64_t best = SGO_INF;
            uint8_t bestdir = dik;
            for (int64_t a = R->row_ptr[i]; a < R->row_ptr[i + 1]; a++) {
                int64_t j = R->col[a];
                if (j == kk) continue;
                int64_t b = find_entry(R, j, kk);
                if (b < 0) continue;
                uint8_t dij = R->dir[a], djk = R->dir[b];
                if (dir_in(dij) != dir_out(djk)) continue;            /* not a valid walk */
                uint8_t comp = (uint8_t)(2 * dir_out(dij) + dir_in(djk));
                uint64_t sum = (uint64_t)R->suffix[a] + (uint64_t)R->suffix[b];
                if (mode == 0) {
                    if (comp != dik) continue;
                    if (sum < best) best = sum;
                } else {
                    if (sum < best || (sum == best && comp < bestdir)) { best = sum; bestdir = comp; }
                }
            }
            N[e] = (uint32_t)best;
            Ndir[e] = (mode == 0) ? dik : bestdir;
        }
    }
    return SGO_OK;
}

/*
 * mode bit 0: the semiring reading (0 DIRMATCH, 1 LITERAL). mode bit 1 (PER_END): the row max of
 * Algorithm 1's Reduce is taken per read end instead of over the whole row -- v_i,e = max of R_ik
 * over the entries that leave read i through end e = out(d_ik), the orientation of read i in the
 * overlap -- and an entry is compared with the max of its own end (the per-end bound of the
 * string-graph reduction the paper builds on, as opposed to its literal whole-row Reduce).
 */
int sgo_transitive_reduce(const sgo_graph *R_in, uint32_t fuzz, int32_t mode, sgo_graph *S,
                          int32_t *iterations) {
    memset(S, 0, sizeof(*S));
    *iterations = 0;
    if (fuzz >= (1u << 30) || mode < 0 || mode > 3) return SGO_INVALID;
    const int32_t semiring = mode & 1, per_end = (mode >> 1) & 1;
    if (sgo_validate_graph(R_in) != SGO_OK) return SGO_INVALID;
    int64_t n = R_in->n, nnz = R_in->nnz;
    sgo_graph R;
    R.n = n; R.nnz = nnz;
    R.row_ptr = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    R.col = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
    R.suffix = (uint32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(uint32_t));
    R.dir = (uint8_t *)malloc((size_t)(nnz ? nnz : 1));
    uint32_t *N = (uint32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(uint32_t));
    uint8_t *Nd = (uint8_t *)malloc((size_t)(nnz ? nnz : 1));
    uint64_t *v = (uint64_t *)malloc((size_t)(n ? 2 * n : 2) * sizeof(uint64_t));  /* [i][end] */
    if (!R.row_ptr || !R.col || !R.suffix || !R.dir || !N || !Nd || !v) {
        free(R.row_ptr); free(R.col); free(R.suffix); free(R.dir); free(N); free(Nd); free(v);
        return SGO_OOM;
    }
    memcpy(R.row_ptr, R_in->row_ptr, (size_t)(n + 1) * sizeof(int64_t));
    memcpy(R.col, R_in->col, (size_t)nnz * sizeof(int32_t));
    memcpy(R.suffix, R_in->suffix, (size_t)nnz * sizeof(uint32_t));
    memcpy(R.dir, R_in->dir, (size_t)nnz);
    int64_t prev;
    do {
        prev = R.nnz;                                      /* prev <- R.nnz() */
        sgo_minplus(&R, semiring, N, Nd);                  /* N <- R^2 */
        for (int64_t i = 0; i < n; i++) {                  /* v <- R.Reduce(Row, 0, max) */
            uint64_t mx[2] = {0, 0};
            for (int64_t e = R.row_ptr[i]; e < R.row_ptr[i + 1]; e++) {
                const int end = per_end ? dir_out(R.dir[e]) : 0;
                if (R.suffix[e] > mx[end]) mx[end] = R.suffix[e];
            }
            v[2 * i] = mx[0] + fuzz;                       /* v <- v.Apply(x, add) */
            v[2 * i + 1] = mx[1] + fuzz;
        }
        /* M <- DimApply(Row, v); I <- M >= N (with the endpoint rule); R <- R o not I */
        int64_t w = 0;
        for (int64_t i = 0; i < n; i++) {
            int64_t b = R.row_ptr[i], e_end = R.row_ptr[i + 1];
            R.row_ptr[i] = w;
            for (int64_t e = b; e < e_end; e++) {
                const uint64_t vi = v[2 * i + (per_end ? dir_out(R.dir[e]) : 0)];
                int transitive = N[e] != SGO_INF && Nd[e] == R.dir[e] && vi >= (uint64_t)N[e];
                if (!transitive) {
                    R.col[w] = R.col[e]; R.suffix[w] = R.suffix[e]; R.dir[w] = R.dir[e];
                    w++;
                }
            }
        }
        R.row_ptr[n] = w;
        R.nnz = w;
        (*iterations)++;
    } while (R.nnz != prev);                               /* until nnz == prev */
    free(N); free(Nd); free(v);
    *S = R;
    return SGO_OK;
}

/* ============================================ single outputs at full size (sampled checks) */

/*
 * Census of given k-mers over the whole input (Sec. IV-C: the frequency of a k-mer is its number
 * of occurrences in the reads). query[0..nq) are canonical codes in ascending order. Every window
 * of every read is coded as in sgo_build_kmer_matrix; for each window whose code is a query,
 * freq[q] is incremented and, while fewer than occ_cap have been stored, the occurrence (q, read,
 * pos, strand) is appended in scan order (reads ascending, positions ascending).
 */
int sgo_kmer_census(const uint8_t *seq, const int64_t *offsets, int64_t n, int32_t k,
                    const uint64_t *query, int64_t nq, uint64_t *freq, int64_t occ_cap,
                    int64_t *occ_q, int32_t *occ_read, uint32_t *occ_pos, uint32_t *occ_strand,
                    int64_t *n_occ) {
    if (k < 1 || k > 31 || (k & 1) == 0 || n < 0) return SGO_INVALID;
    for (int64_t q = 0; q < nq; q++) freq[q] = 0;
    int64_t stored = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t len = offsets[i + 1] - offsets[i];
        for (int64_t p = 0; p + k <= len; p++) {
            uint64_t code;
            uint32_t strand;
            if (!window_code(seq + offsets[i] + p, k, &code, &strand)) continue;
            int64_t lo = 0, hi = nq;  /* binary search for code among the queries */
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (query[mid] < code) lo = mid + 1; else hi = mid;
            }
            if (lo == nq || query[lo] != code) continue;
            freq[lo]++;
            if (stored < occ_cap) {
                occ_q[stored] = lo;
                occ_read[stored] = (int32_t)i;
                occ_pos[stored] = (uint32_t)p;
                occ_strand[stored] = strand;
                stored++;
            }
        }
    }
    *n_occ = stored;
    return SGO_OK;
}

/* Every valid window of read i: canonical code, position and strand, by position. cap entries
 * at most (len - k + 1 suffice). */
int sgo_read_windows(const uint8_t *seq, const int64_t *offsets, int64_t i, int32_t k, int64_t cap,
                     uint64_t *code_out, uint32_t *pos_out, uint32_t *strand_out, int64_t *count) {
    if (k < 1 || k > 31 || (k & 1) == 0) return SGO_INVALID;
    int64_t len = offsets[i + 1] - offsets[i], c = 0;
    for (int64_t p = 0; p + k <= len && c < cap; p++) {
        uint64_t code;
        uint32_t strand;
        if (!window_code(seq + offsets[i] + p, k, &code, &strand)) continue;
        code_out[c] = code;
        pos_out[c] = (uint32_t)p;
        strand_out[c] = strand;
        c++;
    }
    *count = c;
    return SGO_OK;
}

/*
 * Row i of C = A At over the overlap semiring (Sec. IV-D), as in sgo_overlap_spgemm: the columns j
 * of A_i are visited in ascending order, so the first max_seeds contributions to C_ik are the
 * shared k-mers with the smallest column index. Writes the row's entries with count >= min_shared
 * by ascending k into col/count and seeds [e * max_seeds + s] (row-major); returns their number in
 * *nnz (at most A->n_rows - 1, which the arrays must hold).
 */
int sgo_overlap_row(const sgo_csr *A, const sgo_csr *At, int64_t i, uint32_t min_shared, int32_t max_seeds,
                    int32_t *col, uint32_t *count, uint32_t *seed_i, uint32_t *seed_k, int64_t *nnz) {
    if (max_seeds < 0 || max_seeds > 8 || min_shared < 1 || i < 0 || i >= A->n_rows) return SGO_INVALID;
    int64_t n = A->n_rows;
    int S = max_seeds;
    uint32_t *cnt = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
    uint32_t *si = (uint32_t *)malloc((size_t)n * (S ? S : 1) * sizeof(uint32_t));
    uint32_t *sk = (uint32_t *)malloc((size_t)n * (S ? S : 1) * sizeof(uint32_t));
    int64_t *touched = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!cnt || !si || !sk || !touched) { free(cnt); free(si); free(sk); free(touched); return SGO_OOM; }
    int64_t nt = 0;
    for (int64_t a = A->row_ptr[i]; a < A->row_ptr[i + 1]; a++) {
        int64_t j = A->col[a];
        uint32_t vi = A->val[a];
        for (int64_t b = At->row_ptr[j]; b < At->row_ptr[j + 1]; b++) {
            int64_t kk = At->col[b];
            if (kk == i) continue;
            uint32_t vk = At->val[b];
            if (cnt[kk] == 0) touched[nt++] = kk;
            if (cnt[kk] < (uint32_t)S) {
                si[kk * S + cnt[kk]] = vi & 0x7FFFFFFFu;
                sk[kk * S + cnt[kk]] = (vk & 0x7FFFFFFFu) | ((vi ^ vk) & 0x80000000u);
            }
            cnt[kk]++;
        }
    }
    qsort(touched, (size_t)nt, sizeof(int64_t), cmp_u64);
    int64_t e = 0;
    for (int64_t q = 0; q < nt; q++) {
        int64_t kk = touched[q];
        if (cnt[kk] < min_shared) continue;
        col[e] = (int32_t)kk;
        count[e] = cnt[kk];
        for (int s = 0; s < S; s++) {
            int used = (uint32_t)s < cnt[kk];
            seed_i[e * S + s] = used ? si[kk * S + s] : SGO_INF;
            seed_k[e * S + s] = used ? sk[kk * S + s] : SGO_INF;
        }
        e++;
    }
    *nnz = e;
    free(cnt); free(si); free(sk); free(touched);
    return SGO_OK;
}

/* ============================================================ R from C's seeds */

/*
 * Overlap graph R estimated from C (the alignment's role in Algorithm 2, read from the seeds):
 * entry C_ik's first seed (the shared k-mer with the smallest column, Sec. IV-D) places read k in
 * read i's frame. With s_i, s_k the k-mer's positions and rc = strand_i xor strand_k, read k
 * starts at  o = s_i - s_k  (same orientation)  or  o = s_i - (L_k - s_k - K)  (rc = 1; K = k-mer
 * length), so in i's frame i = [0, L_i) and k = [o, o + L_k). The pair is an edge iff the overlap
 * is at least min_overlap and neither interval contains the other (contained overlaps are not part
 * of R, Sec. IV-D; equal starts count as contained). With read i forward and read k in orientation
 * rc, the bidirected edge follows the rule of the coordinate-built R (the read that starts first is
 * a, the other b; R_ab = (e_b - e_a, 2 s_a + s_b), R_ba = (s_b - s_a, 2 (1 - s_b) + (1 - s_a))),
 * of which row i keeps R_ik:
 *   o > 0:  R_ik = (o + L_k - L_i, rc)
 *   o < 0:  R_ik = (-o, 2 + 1 - rc)
 * R has C's row order (ascending k).
 */
int sgo_graph_from_seeds(const sgo_overlap *C, const int64_t *offsets, int32_t K, int64_t min_overlap,
                         sgo_graph *R) {
    memset(R, 0, sizeof(*R));
    if (C->max_seeds < 1 || K < 1 || min_overlap < 1) return SGO_INVALID;
    int64_t n = C->n, nnz = C->nnz;
    R->row_ptr = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    R->col = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
    R->suffix = (uint32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(uint32_t));
    R->dir = (uint8_t *)malloc((size_t)(nnz ? nnz : 1));
    if (!R->row_ptr || !R->col || !R->suffix || !R->dir) {
        free(R->row_ptr); free(R->col); free(R->suffix); free(R->dir);
        memset(R, 0, sizeof(*R));
        return SGO_OOM;
    }
    int64_t e = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t Li = offsets[i + 1] - offsets[i];
        for (int64_t x = C->row_ptr[i]; x < C->row_ptr[i + 1]; x++) {
            int64_t k = C->col[x];
            int64_t Lk = offsets[k + 1] - offsets[k];
            int64_t si = C->seed_i[x] & 0x7FFFFFFF;       /* seed slot 0 */
            int64_t sk = C->seed_k[x] & 0x7FFFFFFF;
            int rc = (int)(C->seed_k[x] >> 31);
            int64_t o = rc ? si - (Lk - sk - K) : si - sk;
            int64_t lo = o > 0 ? o : 0, hi = (o + Lk < Li) ? o + Lk : Li;
            if (hi - lo < min_overlap) continue;
            if (o >= 0 && o + Lk <= Li) continue;         /* k within i (equal starts included) */
            if (o <= 0 && o + Lk >= Li) continue;         /* i within k */
            R->col[e] = (int32_t)k;
            if (o > 0) {
                R->suffix[e] = (uint32_t)(o + Lk - Li);
                R->dir[e] = (uint8_t)rc;
            } else {
                R->suffix[e] = (uint32_t)(-o);
                R->dir[e] = (uint8_t)(2 + 1 - rc);
            }
            e++;
        }
        R->row_ptr[i + 1] = e;
    }
    R->n = n;
    R->nnz = e;
    return SGO_OK;
}
