/*
 * synth.c -- seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.
 *
 * This module holds none of the method's arithmetic: it draws genomes, long reads with a
 * PacBio-CLR-like error model, their true genome coordinates, and overlap graphs R whose
 * suffix/orientation values follow from those coordinates (the input of the transitive
 * reduction, Sec. IV-D/IV-E: R is what alignment and pruning hand to Algorithm 1).
 *
 * Random numbers: splitmix64 seeds xoshiro256** (both as published by Blackman & Vigna).
 * Every floating-point step uses only +,-,*,/ and sqrt (all correctly rounded in IEEE-754),
 * and log/exp are computed here from their series, so the same seed gives the same bytes on
 * any IEEE machine when compiled with -ffp-contract=off.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ RNG */
static inline uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
typedef struct { uint64_t s[4]; } xo_t;
static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t xo_next(xo_t *r) {
    uint64_t *s = r->s;
    uint64_t out = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl64(s[3], 45);
    return out;
}
static void xo_seed(xo_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
/* uniform double in [0,1) with 53 random bits */
static inline double xo_unif(xo_t *r) { return (double)(xo_next(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, n) by the multiply-high method */
static inline uint64_t xo_below(xo_t *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)xo_next(r) * n) >> 64);
}

/* ------------------------------------------------------- deterministic log/exp */
static const double LN2_HI = 6.93147180369123816490e-01; /* ln2 split (Cody-Waite) */
static const double LN2_LO = 1.90821492927058770002e-10;
static double det_exp(double x) {
    if (x > 700.0) x = 700.0;
    if (x < -700.0) x = -700.0;
    double nd = floor(x / 0.69314718055994530942 + 0.5);
    double r = (x - nd * LN2_HI) - nd * LN2_LO;          /* |r| <= 0.35 */
    double term = 1.0, sum = 1.0;
    for (int i = 1; i <= 18; i++) { term = term * r / (double)i; sum += term; }
    return ldexp(sum, (int)nd);
}
static double det_log(double x) {                        /* x > 0 */
    int e;
    double m = frexp(x, &e);                              /* x = m 2^e, m in [0.5,1) */
    if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; } /* m in [0.707, 1.414) */
    double s = (m - 1.0) / (m + 1.0), s2 = s * s, p = s, sum = 0.0;
    for (int i = 1; i <= 41; i += 2) { sum += p / (double)i; p *= s2; }  /* atanh series */
    return 2.0 * sum + (double)e * LN2_HI + (double)e * LN2_LO;
}
/* standard normal by Marsaglia's polar method */
static double xo_normal(xo_t *r) {
    for (;;) {
        double u = 2.0 * xo_unif(r) - 1.0, v = 2.0 * xo_unif(r) - 1.0;
        double s = u * u + v * v;
        if (s > 0.0 && s < 1.0) return u * sqrt(-2.0 * det_log(s) / s);
    }
}

static const uint8_t BASES[4] = {'A', 'C', 'G', 'T'};
static inline uint8_t comp_base(uint8_t b) {
    switch (b) { case 'A': return 'T'; case 'C': return 'G'; case 'G': return 'C'; case 'T': return 'A'; }
    return b;
}
static void revcomp_inplace(uint8_t *s, int64_t n) {
    for (int64_t i = 0, j = n - 1; i < j; i++, j--) {
        uint8_t a = comp_base(s[i]), b = comp_base(s[j]);
        s[i] = b; s[j] = a;
    }
    if (n & 1) s[n / 2] = comp_base(s[n / 2]);
}

void synth_free(void *p) { free(p); }

/* ---------------------------------------------------------------- genome */
/*
 * Uniform i.i.d. ACGT genome of length G, then repeat families pasted at non-overlapping loci.
 * n_families > 0: that many families, each with a copy count drawn log-uniformly in
 *                 [copies_lo, copies_hi] (equal bounds give a fixed count).
 * n_families == 0 and repeat_fraction > 0: families are drawn until the pasted bases reach
 *                 repeat_fraction * G.
 * Each family has length U[fam_len_lo, fam_len_hi]; each copy substitutes every base with
 * probability U[div_lo, div_hi] (drawn per copy) and is pasted reverse-complemented with
 * probability 1/2. Returns the number of pasted bases, or -1 on allocation failure.
 */
int64_t synth_genome(uint8_t *out, int64_t G, uint64_t seed, int32_t n_families,
                     double repeat_fraction, double copies_lo, double copies_hi,
                     int64_t fam_len_lo, int64_t fam_len_hi, double div_lo, double div_hi) {
    xo_t r;
    xo_seed(&r, seed);
    for (int64_t i = 0; i < G; i += 32) {
        uint64_t w = xo_next(&r);
        for (int t = 0; t < 32 && i + t < G; t++) { out[i + t] = BASES[w & 3]; w >>= 2; }
    }
    if (n_families <= 0 && repeat_fraction <= 0.0) return 0;
    if (fam_len_hi < fam_len_lo || fam_len_lo < 1 || fam_len_hi >= G) return 0;
    uint8_t *occ = (uint8_t *)calloc((size_t)G, 1);
    uint8_t *fam = (uint8_t *)malloc((size_t)fam_len_hi);
    if (!occ || !fam) { free(occ); free(fam); return -1; }
    int64_t pasted = 0, target = (int64_t)(repeat_fraction * (double)G);
    for (int32_t f = 0;; f++) {
        if (n_families > 0 && f >= n_families) break;
        if (n_families <= 0 && pasted >= target) break;
        int64_t flen = fam_len_lo + (int64_t)xo_below(&r, (uint64_t)(fam_len_hi - fam_len_lo + 1));
        for (int64_t i = 0; i < flen; i++) fam[i] = BASES[xo_next(&r) >> 62];
        double lc = det_log(copies_lo), hc = det_log(copies_hi);
        int64_t copies = (int64_t)floor(det_exp(lc + (hc - lc) * xo_unif(&r)) + 0.5);
        if (copies < 1) copies = 1;
        for (int64_t c = 0; c < copies; c++) {
            int64_t pos = -1;
            for (int attempt = 0; attempt < 1000 && pos < 0; attempt++) {
                int64_t p = (int64_t)xo_below(&r, (uint64_t)(G - flen + 1));
                int ok = 1;
                for (int64_t i = 0; i < flen; i++) if (occ[p + i]) { ok = 0; break; }
                if (ok) pos = p;
            }
            if (pos < 0) continue; /* genome too full: skip this copy */
            double div = div_lo + (div_hi - div_lo) * xo_unif(&r);
            int rc = (int)(xo_next(&r) >> 63);
            for (int64_t i = 0; i < flen; i++) {
                uint8_t b = rc ? comp_base(fam[flen - 1 - i]) : fam[i];
                if (xo_unif(&r) < div) {
                    uint8_t nb;
                    do { nb = BASES[xo_next(&r) >> 62]; } while (nb == b);
                    b = nb;
                }
                out[pos + i] = b;
                occ[pos + i] = 1;
            }
            pasted += flen;
        }
    }
    free(occ);
    free(fam);
    return pasted;
}

/* ----------------------------------------------------------------- reads */
typedef struct {
    int64_t n;        /* reads */
    int64_t total;    /* bases in seq */
    uint8_t *seq;     /* ASCII concatenation */
    int64_t *offsets; /* n+1 */
    int64_t *start;   /* template start on the genome */
    int64_t *end;     /* template end (exclusive) */
    uint8_t *strand;  /* 1 = read is the reverse complement of the template */
} synth_reads_t;

/*
 * Reads are drawn until their template lengths sum to coverage * G. Length ~ lognormal with the
 * given mean and sd (sigma^2 = ln(1 + sd^2/mean^2), mu = ln(mean) - sigma^2/2), rounded and
 * clipped to [len_min, G]; start uniform in [0, G - L]; strand a fair coin. Each template base
 * is deleted with p_del, else substituted (uniform over the 3 other bases) with p_sub, else
 * copied; then a uniform random base is inserted after it with p_ins. Strand 1 reads are
 * reverse-complemented. Read i's errors use its own xoshiro stream seeded from (seed, i).
 * max_reads > 0 caps n. Returns 0, or -1 on allocation failure.
 */
int synth_reads(const uint8_t *genome, int64_t G, double coverage, double len_mean, double len_sd,
                int64_t len_min, double p_ins, double p_del, double p_sub, uint64_t seed,
                int64_t max_reads, synth_reads_t *out) {
    memset(out, 0, sizeof(*out));
    xo_t r;
    xo_seed(&r, seed ^ 0x5bd1e995a5a5a5a5ULL);
    double s2 = det_log(1.0 + (len_sd * len_sd) / (len_mean * len_mean));
    double sig = sqrt(s2), mu = det_log(len_mean) - 0.5 * s2;
    if (len_min > G) len_min = G;
    int64_t cap = 1024, n = 0;
    int64_t *st = (int64_t *)malloc(cap * sizeof(int64_t));
    int64_t *en = (int64_t *)malloc(cap * sizeof(int64_t));
    uint8_t *sd = (uint8_t *)malloc(cap);
    if (!st || !en || !sd) goto oom;
    double target = coverage * (double)G, sum = 0.0;
    while (sum < target && (max_reads <= 0 || n < max_reads)) {
        double lf = det_exp(mu + sig * xo_normal(&r));
        int64_t L = (int64_t)floor(lf + 0.5);
        if (L < len_min) L = len_min;
        if (L > G) L = G;
        int64_t s = (int64_t)xo_below(&r, (uint64_t)(G - L + 1));
        uint8_t strand = (uint8_t)(xo_next(&r) >> 63);
        if (n == cap) {
            cap *= 2;
            int64_t *a = (int64_t *)realloc(st, cap * sizeof(int64_t));
            if (a) st = a;
            int64_t *b = (int64_t *)realloc(en, cap * sizeof(int64_t));
            if (b) en = b;
            uint8_t *c = (uint8_t *)realloc(sd, cap);
            if (c) sd = c;
            if (!a || !b || !c) goto oom;
        }
        st[n] = s; en[n] = s + L; sd[n] = strand; n++;
        sum += (double)L;
    }
    int64_t seqcap = (int64_t)(sum * (1.0 + 2.0 * p_ins)) + 1024, tot = 0;
    uint8_t *seq = (uint8_t *)malloc((size_t)seqcap);
    int64_t *off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!seq || !off) { free(seq); free(off); goto oom; }
    uint64_t pd = (uint64_t)(p_del * 9007199254740992.0), ps = (uint64_t)(p_sub * 9007199254740992.0),
             pi = (uint64_t)(p_ins * 9007199254740992.0);
    for (int64_t i = 0; i < n; i++) {
        xo_t rr;
        xo_seed(&rr, seed * 0x9e3779b97f4a7c15ULL + (uint64_t)i + 1);
        off[i] = tot;
        int64_t need = tot + 2 * (en[i] - st[i]) + 16;
        if (need > seqcap) {
            seqcap = need + seqcap / 2;
            uint8_t *q = (uint8_t *)realloc(seq, (size_t)seqcap);
            if (!q) { free(seq); free(off); goto oom; }
            seq = q;
        }
        for (int64_t p = st[i]; p < en[i]; p++) {
            uint8_t b = genome[p];
            if ((xo_next(&rr) >> 11) < pd) {
                /* deleted */
            } else {
                if ((xo_next(&rr) >> 11) < ps) {
                    uint8_t nb;
                    do { nb = BASES[xo_next(&rr) >> 62]; } while (nb == b);
                    b = nb;
                }
                seq[tot++] = b;
            }
            if ((xo_next(&rr) >> 11) < pi) seq[tot++] = BASES[xo_next(&rr) >> 62];
        }
        if (sd[i]) revcomp_inplace(seq + off[i], tot - off[i]);
    }
    off[n] = tot;
    out->n = n; out->total = tot; out->seq = seq; out->offsets = off;
    out->start = st; out->end = en; out->strand = sd;
    return 0;
oom:
    free(st); free(en); free(sd);
    return -1;
}

/* ------------------------------------------------------- overlap graph R */
typedef struct {
    int64_t n, nnz;
    int64_t *row_ptr; /* n+1 */
    int32_t *col;
    uint32_t *suffix;
    uint8_t *dir;
} synth_graph_t;

typedef struct { int64_t row; int32_t col; uint32_t suffix; uint8_t dir; } quad_t;
static int cmp_quad(const void *a, const void *b) {
    const quad_t *x = (const quad_t *)a, *y = (const quad_t *)b;
    if (x->row != y->row) return x->row < y->row ? -1 : 1;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    if (x->suffix != y->suffix) return x->suffix < y->suffix ? -1 : 1;
    return (x->dir > y->dir) - (x->dir < y->dir);
}
static int quads_to_csr(quad_t *q, int64_t nq, int64_t n, synth_graph_t *g) {
    qsort(q, (size_t)nq, sizeof(quad_t), cmp_quad);
    g->n = n; g->nnz = nq;
    g->row_ptr = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    g->col = (int32_t *)malloc((size_t)(nq ? nq : 1) * sizeof(int32_t));
    g->suffix = (uint32_t *)malloc((size_t)(nq ? nq : 1) * sizeof(uint32_t));
    g->dir = (uint8_t *)malloc((size_t)(nq ? nq : 1));
    if (!g->row_ptr || !g->col || !g->suffix || !g->dir) return -1;
    for (int64_t e = 0; e < nq; e++) {
        g->row_ptr[q[e].row + 1]++;
        g->col[e] = q[e].col; g->suffix[e] = q[e].suffix; g->dir[e] = q[e].dir;
    }
    for (int64_t i = 0; i < n; i++) g->row_ptr[i + 1] += g->row_ptr[i];
    return 0;
}

/* reads in (start, end, index) order; the comparator reads only its two records, so concurrent
 * calls (the batched and served sets are drawn on several host threads) do not interfere */
typedef struct { int64_t start, end, idx; } span_t;
static int cmp_span(const void *a, const void *b) {
    const span_t *x = (const span_t *)a, *y = (const span_t *)b;
    if (x->start != y->start) return x->start < y->start ? -1 : 1;
    if (x->end != y->end) return x->end < y->end ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/*
 * Overlap graph from true template coordinates. A pair of reads is an edge iff the intervals
 * overlap by >= min_overlap bp and neither interval contains the other (contained overlaps are
 * not part of R, Sec. IV-D). With a the read that starts first and b the other:
 *   R[a][b] = (e_b - e_a,  2*strand_a + strand_b)          walk a -> b
 *   R[b][a] = (s_b - s_a,  2*(1-strand_b) + (1-strand_a))  walk b -> a
 * The suffix is the overhang of the walk's second read (Sec. II); the 2-bit dir holds the
 * orientation of the walk's first read in bit 1 and of its second read in bit 0.
 * jitter > 0 adds U[0, jitter] to every suffix (seeded), modelling coordinate noise.
 */
int synth_overlap_graph(const int64_t *start, const int64_t *end, const uint8_t *strand, int64_t n,
                        int64_t min_overlap, uint32_t jitter, uint64_t seed, synth_graph_t *g) {
    memset(g, 0, sizeof(*g));
    if (min_overlap < 1) min_overlap = 1;
    int64_t *ord = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    span_t *sp = (span_t *)malloc((size_t)(n ? n : 1) * sizeof(span_t));
    if (!ord || !sp) { free(ord); free(sp); return -1; }
    for (int64_t i = 0; i < n; i++) { sp[i].start = start[i]; sp[i].end = end[i]; sp[i].idx = i; }
    qsort(sp, (size_t)n, sizeof(span_t), cmp_span);
    for (int64_t i = 0; i < n; i++) ord[i] = sp[i].idx;
    free(sp);
    int64_t cap = 1024, nq = 0;
    quad_t *q = (quad_t *)malloc(cap * sizeof(quad_t));
    if (!q) { free(ord); return -1; }
    xo_t r;
    xo_seed(&r, seed ^ 0x243f6a8885a308d3ULL);
    for (int64_t x = 0; x < n; x++) {
        int64_t a = ord[x];
        for (int64_t y = x + 1; y < n; y++) {
            int64_t b = ord[y];
            if (start[b] >= end[a]) break;
            if (start[b] == start[a] || end[b] <= end[a]) continue; /* contained */
            if (end[a] - start[b] < min_overlap) continue;
            if (nq + 2 > cap) {
                cap *= 2;
                quad_t *qq = (quad_t *)realloc(q, cap * sizeof(quad_t));
                if (!qq) { free(q); free(ord); return -1; }
                q = qq;
            }
            uint32_t ja = jitter ? (uint32_t)xo_below(&r, (uint64_t)jitter + 1) : 0;
            uint32_t jb = jitter ? (uint32_t)xo_below(&r, (uint64_t)jitter + 1) : 0;
            q[nq].row = a; q[nq].col = (int32_t)b;
            q[nq].suffix = (uint32_t)(end[b] - end[a]) + ja;
            q[nq].dir = (uint8_t)(2 * strand[a] + strand[b]);
            nq++;
            q[nq].row = b; q[nq].col = (int32_t)a;
            q[nq].suffix = (uint32_t)(start[b] - start[a]) + jb;
            q[nq].dir = (uint8_t)(2 * (1 - strand[b]) + (1 - strand[a]));
            nq++;
        }
    }
    free(ord);
    int rc = quads_to_csr(q, nq, n, g);
    free(q);
    return rc;
}

/*
 * Random directed graph for transitive-reduction tests: about n*avg_deg distinct off-diagonal
 * entries; a fraction hub_frac of rows draw 8x as many entries (skewed degrees); suffix
 * U[0, max_suffix]; dir U{0..3}.
 */
int synth_random_graph(int64_t n, double avg_deg, double hub_frac, uint32_t max_suffix,
                       uint64_t seed, synth_graph_t *g) {
    memset(g, 0, sizeof(*g));
    xo_t r;
    xo_seed(&r, seed ^ 0x13198a2e03707344ULL);
    int64_t cap = 1024, nq = 0;
    quad_t *q = (quad_t *)malloc(cap * sizeof(quad_t));
    if (!q) return -1;
    for (int64_t i = 0; i < n && n > 1; i++) {
        double d = avg_deg * ((xo_unif(&r) < hub_frac) ? 8.0 : 1.0);
        int64_t deg = (int64_t)floor(d * 2.0 * xo_unif(&r));
        if (deg > n - 1) deg = n - 1;
        for (int64_t t = 0; t < deg; t++) {
            int64_t j = (int64_t)xo_below(&r, (uint64_t)(n - 1));
            if (j >= i) j++;
            if (nq == cap) {
                cap *= 2;
                quad_t *qq = (quad_t *)realloc(q, cap * sizeof(quad_t));
                if (!qq) { free(q); return -1; }
                q = qq;
            }
            q[nq].row = i; q[nq].col = (int32_t)j;
            q[nq].suffix = (uint32_t)xo_below(&r, (uint64_t)max_suffix + 1);
            q[nq].dir = (uint8_t)(xo_next(&r) >> 62);
            nq++;
        }
    }
    qsort(q, (size_t)nq, sizeof(quad_t), cmp_quad);
    int64_t w = 0; /* drop duplicate (row, col), keeping the smallest (suffix, dir) */
    for (int64_t e = 0; e < nq; e++)
        if (w == 0 || q[e].row != q[w - 1].row || q[e].col != q[w - 1].col) q[w++] = q[e];
    int rc = quads_to_csr(q, w, n, g);
    free(q);
    return rc;
}
