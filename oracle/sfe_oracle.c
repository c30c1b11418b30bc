/*
 * CPU oracle for spaced-seed hit generation, the per-diagonal skip and the
 * ungapped X-drop filter (the filter stage of the seed-filter-extend pipeline,
 * Section 1 and Section 2 of the paper; its loop shape is Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, serial statement of
 * what the CUDA library must compute bit for bit. It is used by the tests, by
 * the smoke check and by the benchmark's CPU-baseline leg, never by the product
 * path, and it shares no code, header or table with the CUDA library.
 *
 * Coding: A=0, C=1, G=2, T=3 (one byte per base). Complement x^3, transition
 * partner x^2 (A<->G, C<->T).
 *
 * Definitions (the paper names the steps but fixes none of these details; each
 * reading below is recorded in the design notes):
 *
 *  Seed (Section 7): a pattern of '1' (care) and '0' (don't care) positions,
 *  default 1110100110010101111 (weight 12, span 19). (s, t, q) is a hit iff at
 *  every care offset c, T[t+c] equals Qs[q+c], except that with transition
 *  tolerance (Section 2) at most one care offset may hold a transition
 *  (T[t+c] == Qs[q+c]^2). Q+ = Q; Q- = reverse complement of Q, and minus-strand
 *  coordinates index Q-. With a step s > 1 (Section 7: the spacing between
 *  seeds), only target positions t with t % s == 0 are in the position table,
 *  so only they start hits.
 *
 *  Skip (Algorithm 1, the IsContained test; the masking-list update): hits are
 *  processed per (strand, diagonal d = t - q) in increasing t. A hit with
 *  t < E is skipped, where E is the exclusive end of the last extended HSP on
 *  that diagonal (E starts below every t). E is updated after every extension,
 *  or only after extensions that reach the threshold when OR_SKIP_PASSING_ONLY
 *  is set.
 *
 *  X-drop (Section 2, Section 8: ungapped, 1-D): the HSP always holds the whole
 *  seed span [t, t+span). The right extension scores bases t+span, t+span+1, ...
 *  while both sequences last, keeping the running sum, its maximum (which
 *  starts at 0 for the empty extension) and the earliest length at which the
 *  maximum is reached; it stops right after the first base at which
 *  maximum - sum > X. The left extension is the mirror image from t-1 down.
 *  HSP = [t - lbest_len, t + span + rbest_len), score = span score + both
 *  maxima. E = t + span + rbest_len. cells = span + bases scored on both sides.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

#define OR_SKIP_PASSING_ONLY 1

typedef struct {
    int32_t strand, tpos, qpos, len, score;
} or_hsp;

typedef struct {
    int64_t hits;     /* seed hits enumerated */
    int64_t extended; /* hits not skipped, i.e. X-drop extensions run */
    int64_t cells;    /* span + bases scored, summed over extended hits */
    int64_t hsps;     /* extensions with score >= threshold */
} or_stats;

/* One extension, as a record (used for per-hit logs). */
typedef struct {
    int32_t strand, t, q, lext, rext, lscored, rscored;
    int64_t score;
} or_ext;

typedef struct {
    int span, weight;
    int care[32];
    int step; /* index stride: only target positions t with t % step == 0 are seeds */
} or_pattern;

/* ---------------------------------------------------------------- basics */

int or_encode(const uint8_t *ascii, int64_t n, uint8_t *codes)
{
    for (int64_t i = 0; i < n; i++) {
        switch (ascii[i]) {
        case 'A': case 'a': codes[i] = 0; break;
        case 'C': case 'c': codes[i] = 1; break;
        case 'G': case 'g': codes[i] = 2; break;
        case 'T': case 't': codes[i] = 3; break;
        default: return OR_EINVAL;
        }
    }
    return OR_OK;
}

void or_revcomp(const uint8_t *q, int64_t n, uint8_t *out)
{
    for (int64_t i = 0; i < n; i++)
        out[i] = (uint8_t)(q[n - 1 - i] ^ 3);
}

int or_parse_pattern(const char *s, or_pattern *p)
{
    int n = (int)strlen(s);
    if (n < 1 || n > 32)
        return OR_EINVAL;
    p->span = n;
    p->weight = 0;
    p->step = 1;
    for (int i = 0; i < n; i++) {
        if (s[i] == '1')
            p->care[p->weight++] = i;
        else if (s[i] != '0')
            return OR_EINVAL;
    }
    if (p->weight < 1 || p->weight > 16)
        return OR_EINVAL;
    return OR_OK;
}

/* The hit predicate, written out directly (Section 7 seed, Section 2 transitions). */
int or_is_hit(const uint8_t *T, const uint8_t *Qs, int64_t t, int64_t q,
              const or_pattern *p, int transition)
{
    int used = 0;
    for (int i = 0; i < p->weight; i++) {
        uint8_t a = T[t + p->care[i]], b = Qs[q + p->care[i]];
        if (a == b)
            continue;
        if (transition && (a ^ b) == 2 && !used) {
            used = 1;
            continue;
        }
        return 0;
    }
    return 1;
}

/* ------------------------------------------------------------- the index */

typedef struct {
    uint32_t key;
    int64_t pos;
} or_entry;

static int cmp_entry(const void *a, const void *b)
{
    const or_entry *x = (const or_entry *)a, *y = (const or_entry *)b;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    return (x->pos > y->pos) - (x->pos < y->pos);
}

static uint32_t seed_key(const uint8_t *S, int64_t pos, const or_pattern *p)
{
    uint32_t k = 0;
    for (int i = 0; i < p->weight; i++)
        k = (k << 2) | S[pos + p->care[i]];
    return k;
}

/* First index in the sorted table whose key is >= k. */
static int64_t lower_key(const or_entry *tab, int64_t n, uint32_t k)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (tab[mid].key < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

typedef struct {
    int64_t t, q;
} or_tq;

typedef struct {
    or_tq *v;
    int64_t n, cap;
} tq_vec;

static int tq_push(tq_vec *a, int64_t t, int64_t q)
{
    if (a->n == a->cap) {
        int64_t nc = a->cap ? a->cap * 2 : 1024;
        or_tq *nv = (or_tq *)realloc(a->v, (size_t)nc * sizeof(or_tq));
        if (!nv)
            return OR_ENOMEM;
        a->v = nv;
        a->cap = nc;
    }
    a->v[a->n].t = t;
    a->v[a->n].q = q;
    a->n++;
    return OR_OK;
}

static int cmp_diag_t(const void *a, const void *b)
{
    const or_tq *x = (const or_tq *)a, *y = (const or_tq *)b;
    int64_t dx = x->t - x->q, dy = y->t - y->q;
    if (dx != dy)
        return dx < dy ? -1 : 1;
    return (x->t > y->t) - (x->t < y->t);
}

/*
 * The position table of the target: (seed key, position) for every position
 * t in [0, tlen - span] with t % step == 0, sorted by key and then position.
 * With nthreads > 1
 * the entries are first split by the top bits of their key (a stable
 * counting pass) and each part is sorted on its own thread; the order of
 * (key, position) pairs is total, so the table is the same either way.
 */
static int build_table(const uint8_t *T, int64_t tlen, const or_pattern *p, int nthreads,
                       or_entry **tab_out, int64_t *nt_out)
{
    *tab_out = NULL;
    *nt_out = 0;
    if (tlen < p->span)
        return OR_OK;
    int64_t npos = tlen - p->span + 1;
    int64_t nt = (npos + p->step - 1) / p->step;
    or_entry *tab = (or_entry *)malloc((size_t)nt * sizeof(or_entry));
    if (!tab)
        return OR_ENOMEM;
    for (int64_t j = 0; j < nt; j++) {
        tab[j].key = seed_key(T, j * p->step, p);
        tab[j].pos = j * p->step;
    }
    if (nthreads <= 1) {
        qsort(tab, (size_t)nt, sizeof(or_entry), cmp_entry);
    } else {
        int shift = 2 * p->weight > 8 ? 2 * p->weight - 8 : 0; /* 256 parts by the top key bits */
        int64_t start[257] = {0};
        for (int64_t t = 0; t < nt; t++)
            start[(tab[t].key >> shift) + 1]++;
        for (int b = 0; b < 256; b++)
            start[b + 1] += start[b];
        or_entry *tmp = (or_entry *)malloc((size_t)nt * sizeof(or_entry));
        if (!tmp) {
            free(tab);
            return OR_ENOMEM;
        }
        int64_t fill[256];
        memcpy(fill, start, sizeof(fill));
        for (int64_t t = 0; t < nt; t++)
            tmp[fill[tab[t].key >> shift]++] = tab[t];
        free(tab);
        tab = tmp;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
        for (int b = 0; b < 256; b++)
            qsort(tab + start[b], (size_t)(start[b + 1] - start[b]), sizeof(or_entry), cmp_entry);
    }
    *tab_out = tab;
    *nt_out = nt;
    return OR_OK;
}

/*
 * Hits of query positions q0 <= q < q1 (and q <= qlen - span) against the
 * table, appended to out in query order: the exact key of Qs at q, then with
 * transition tolerance the weight keys with one care position's transition
 * partner (the 2-bit code x^2) in place of the query base.
 */
static int probe_range(const or_entry *tab, int64_t nt, const uint8_t *Qs, int64_t qlen,
                       int64_t q0, int64_t q1, const or_pattern *p, int transition, tq_vec *out)
{
    int nprobe = transition ? 1 + p->weight : 1;
    for (int64_t q = q0; q + p->span <= qlen && q < q1; q++) {
        uint32_t k = seed_key(Qs, q, p);
        for (int j = 0; j < nprobe; j++) {
            uint32_t pk = j == 0 ? k : k ^ (2u << (2 * (p->weight - j)));
            for (int64_t i = lower_key(tab, nt, pk); i < nt && tab[i].key == pk; i++) {
                if (tq_push(out, tab[i].pos, q))
                    return OR_ENOMEM;
            }
        }
    }
    return OR_OK;
}

/* Every hit of one strand, sorted by (diagonal t-q, t). */
static int enumerate_hits(const uint8_t *T, int64_t tlen, const uint8_t *Qs, int64_t qlen,
                          const or_pattern *p, int transition, tq_vec *out)
{
    out->v = NULL;
    out->n = out->cap = 0;
    if (tlen < p->span || qlen < p->span)
        return OR_OK;
    or_entry *tab;
    int64_t nt;
    if (build_table(T, tlen, p, 1, &tab, &nt))
        return OR_ENOMEM;
    int e = probe_range(tab, nt, Qs, qlen, 0, qlen, p, transition, out);
    free(tab);
    if (e)
        return e;
    qsort(out->v, (size_t)out->n, sizeof(or_tq), cmp_diag_t);
    return OR_OK;
}

/* ------------------------------------------------------------ extension */

void or_xdrop(const uint8_t *T, int64_t tlen, const uint8_t *Qs, int64_t qlen, int64_t t,
              int64_t q, int span, const int32_t *M, int32_t X, or_ext *e)
{
    int64_t s0 = 0;
    for (int k = 0; k < span; k++)
        s0 += M[T[t + k] * 4 + Qs[q + k]];

    int64_t sum = 0, best = 0, bestlen = 0, n = 0;
    while (t + span + n < tlen && q + span + n < qlen) {
        sum += M[T[t + span + n] * 4 + Qs[q + span + n]];
        n++;
        if (sum > best) {
            best = sum;
            bestlen = n;
        }
        if (best - sum > X)
            break;
    }
    int64_t rbest = best;
    e->rext = (int32_t)bestlen;
    e->rscored = (int32_t)n;

    sum = best = bestlen = n = 0;
    while (t - 1 - n >= 0 && q - 1 - n >= 0) {
        sum += M[T[t - 1 - n] * 4 + Qs[q - 1 - n]];
        n++;
        if (sum > best) {
            best = sum;
            bestlen = n;
        }
        if (best - sum > X)
            break;
    }
    e->lext = (int32_t)bestlen;
    e->lscored = (int32_t)n;
    e->score = s0 + rbest + best;
    e->t = (int32_t)t;
    e->q = (int32_t)q;
}

/* ------------------------------------------------------------- results */

typedef struct {
    or_hsp *hsp;
    int64_t n, cap;
    or_ext *ext; /* optional log of every extension, in processing order */
    int64_t next, extcap;
    int keep_log;
    or_stats st;
} or_result;

static int push_hsp(or_result *r, const or_hsp *h)
{
    if (r->n == r->cap) {
        int64_t nc = r->cap ? r->cap * 2 : 256;
        or_hsp *nv = (or_hsp *)realloc(r->hsp, (size_t)nc * sizeof(or_hsp));
        if (!nv)
            return OR_ENOMEM;
        r->hsp = nv;
        r->cap = nc;
    }
    r->hsp[r->n++] = *h;
    return OR_OK;
}

static int push_ext(or_result *r, const or_ext *e)
{
    if (r->next == r->extcap) {
        int64_t nc = r->extcap ? r->extcap * 2 : 1024;
        or_ext *nv = (or_ext *)realloc(r->ext, (size_t)nc * sizeof(or_ext));
        if (!nv)
            return OR_ENOMEM;
        r->ext = nv;
        r->extcap = nc;
    }
    r->ext[r->next++] = *e;
    return OR_OK;
}

static int cmp_hsp(const void *a, const void *b)
{
    const or_hsp *x = (const or_hsp *)a, *y = (const or_hsp *)b;
    if (x->strand != y->strand) return x->strand < y->strand ? -1 : 1;
    if (x->tpos != y->tpos) return x->tpos < y->tpos ? -1 : 1;
    if (x->qpos != y->qpos) return x->qpos < y->qpos ? -1 : 1;
    if (x->len != y->len) return x->len < y->len ? -1 : 1;
    if (x->score != y->score) return x->score < y->score ? -1 : 1;
    return 0;
}

/*
 * The serial walk over hits of one strand, already grouped by diagonal and
 * ordered by t (Algorithm 1 with X-drop as the extension, restricted to one
 * diagonal's masking state). With Ecarry == NULL every diagonal starts with
 * no masking state; otherwise diagonal d starts from Ecarry[d - dbase] and
 * leaves its final state there, so a diagonal's hits may be walked in several
 * calls as long as the calls come in increasing t.
 */
static int walk(const uint8_t *T, int64_t tlen, const uint8_t *Qs, int64_t qlen, int strand,
                const or_tq *v, int64_t nh, int64_t *Ecarry, int64_t dbase, const or_pattern *p,
                const int32_t *M, int32_t X, int32_t thresh, int flags, or_result *r)
{
    int64_t i = 0;
    while (i < nh) {
        int64_t d = v[i].t - v[i].q;
        int64_t E = Ecarry ? Ecarry[d - dbase] : INT64_MIN;
        for (; i < nh && v[i].t - v[i].q == d; i++) {
            int64_t t = v[i].t, q = v[i].q;
            r->st.hits++;
            if (t < E)
                continue; /* inside an HSP already extended on this diagonal */
            or_ext e;
            or_xdrop(T, tlen, Qs, qlen, t, q, p->span, M, X, &e);
            e.strand = strand;
            r->st.extended++;
            r->st.cells += p->span + e.lscored + e.rscored;
            int pass = e.score >= thresh;
            if (pass || !(flags & OR_SKIP_PASSING_ONLY))
                E = t + p->span + e.rext;
            if (r->keep_log && push_ext(r, &e))
                return OR_ENOMEM;
            if (pass) {
                or_hsp o;
                o.strand = strand;
                o.tpos = (int32_t)(t - e.lext);
                o.qpos = (int32_t)(q - e.lext);
                o.len = p->span + e.lext + e.rext;
                o.score = (int32_t)e.score;
                r->st.hsps++;
                if (push_hsp(r, &o))
                    return OR_ENOMEM;
            }
        }
        if (Ecarry)
            Ecarry[d - dbase] = E;
    }
    return OR_OK;
}

/*
 * Full filter stage for one target/query pair. strands: bit 0 = plus strand,
 * bit 1 = minus strand. Returns a result handle (NULL on error, with *err set).
 */
or_result *or_run(const uint8_t *T, int64_t tlen, const uint8_t *Q, int64_t qlen,
                  const char *pattern, int step, int transition, int strands, const int32_t *M,
                  int32_t X, int32_t thresh, int flags, int keep_log, int *err)
{
    or_pattern p;
    *err = OR_OK;
    if (or_parse_pattern(pattern, &p) || step < 1 || X < 0 || tlen < 0 || qlen < 0) {
        *err = OR_EINVAL;
        return NULL;
    }
    p.step = step;
    or_result *r = (or_result *)calloc(1, sizeof(or_result));
    if (!r) {
        *err = OR_ENOMEM;
        return NULL;
    }
    r->keep_log = keep_log;
    uint8_t *rc = NULL;
    for (int s = 0; s < 2; s++) {
        if (!(strands & (1 << s)))
            continue;
        const uint8_t *Qs = Q;
        if (s == 1) {
            rc = (uint8_t *)malloc((size_t)(qlen > 0 ? qlen : 1));
            if (!rc) {
                *err = OR_ENOMEM;
                break;
            }
            or_revcomp(Q, qlen, rc);
            Qs = rc;
        }
        tq_vec h;
        int e = enumerate_hits(T, tlen, Qs, qlen, &p, transition, &h);
        if (!e)
            e = walk(T, tlen, Qs, qlen, s, h.v, h.n, NULL, 0, &p, M, X, thresh, flags, r);
        free(h.v);
        if (e) {
            *err = e;
            break;
        }
    }
    free(rc);
    if (*err) {
        free(r->hsp);
        free(r->ext);
        free(r);
        return NULL;
    }
    qsort(r->hsp, (size_t)r->n, sizeof(or_hsp), cmp_hsp);
    return r;
}

/*
 * The same filter stage computed on several threads (OpenMP), for inputs
 * too large for the serial form. The arithmetic is the serial form's: the
 * same table, probes, walk and X-drop. Only the order of independent work
 * changes, which the method allows (diagonals are independent, and a
 * diagonal's hits are still walked in increasing t):
 *  - the query positions of a strand are taken in tiles of qtile positions
 *    (qtile <= 0: one tile), in increasing q;
 *  - a tile's hits are found on several threads (contiguous runs of query
 *    positions), split into blocks of whole diagonals, and each block is
 *    sorted by (diagonal, t) and walked on one thread;
 *  - each diagonal's masking state E lives in a per-strand array, so the
 *    hits of the next tile continue from the state the previous tile left.
 * Since t - q is fixed on a diagonal, increasing q is increasing t, and every
 * diagonal sees its hits in the order of the serial walk. No extension log.
 * nthreads <= 0: all threads OpenMP offers (1 without OpenMP).
 */
or_result *or_run_par(const uint8_t *T, int64_t tlen, const uint8_t *Q, int64_t qlen,
                      const char *pattern, int step, int transition, int strands,
                      const int32_t *M, int32_t X, int32_t thresh, int flags, int64_t qtile,
                      int nthreads, int *err)
{
    or_pattern p;
    *err = OR_OK;
    if (or_parse_pattern(pattern, &p) || step < 1 || X < 0 || tlen < 0 || qlen < 0) {
        *err = OR_EINVAL;
        return NULL;
    }
    p.step = step;
    if (nthreads <= 0) {
#ifdef _OPENMP
        nthreads = omp_get_max_threads();
#else
        nthreads = 1;
#endif
    }
    or_result *r = (or_result *)calloc(1, sizeof(or_result));
    or_result *part = (or_result *)calloc((size_t)nthreads, sizeof(or_result));
    uint8_t *rc = (uint8_t *)malloc((size_t)(qlen > 0 ? qlen : 1));
    or_entry *tab = NULL;
    int64_t nt = 0;
    if (!r || !part || !rc) {
        *err = OR_ENOMEM;
        goto done;
    }
    if (tlen < p.span || qlen < p.span)
        goto done;
    if (build_table(T, tlen, &p, nthreads, &tab, &nt)) {
        *err = OR_ENOMEM;
        goto done;
    }
    or_revcomp(Q, qlen, rc);
    const int64_t nq = qlen - p.span + 1;
    if (qtile <= 0 || qtile > nq)
        qtile = nq;
    const int64_t dbase = -(qlen - p.span);        /* smallest diagonal t - q */
    const int64_t ndiag = (tlen - p.span) - dbase + 1;
    const int64_t nblk = 64 * (int64_t)nthreads;   /* diagonal blocks per tile */
    const int64_t bw = (ndiag + nblk - 1) / nblk;  /* diagonals per block */
    for (int s = 0; s < 2 && !*err; s++) {
        if (!(strands & (1 << s)))
            continue;
        const uint8_t *Qs = s ? rc : Q;
        int64_t *Ecarry = (int64_t *)malloc((size_t)ndiag * sizeof(int64_t));
        if (!Ecarry) {
            *err = OR_ENOMEM;
            break;
        }
        for (int64_t d = 0; d < ndiag; d++)
            Ecarry[d] = INT64_MIN;
        for (int64_t q0 = 0; q0 < nq && !*err; q0 += qtile) {
            const int64_t q1 = q0 + qtile < nq ? q0 + qtile : nq;
            /* about four runs of query positions per thread, each probed by one task */
            const int64_t nrun = q1 - q0 < 4 * (int64_t)nthreads ? q1 - q0 : 4 * (int64_t)nthreads;
            const int64_t qrun = (q1 - q0 + nrun - 1) / nrun;
            tq_vec *runs = (tq_vec *)calloc((size_t)nrun, sizeof(tq_vec));
            int64_t *cnt = (int64_t *)calloc((size_t)(nrun * nblk + 1), sizeof(int64_t));
            if (!runs || !cnt) {
                free(runs);
                free(cnt);
                *err = OR_ENOMEM;
                break;
            }
            int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
            for (int64_t k = 0; k < nrun; k++) {
                const int64_t a = q0 + k * qrun, b = a + qrun < q1 ? a + qrun : q1;
                if (probe_range(tab, nt, Qs, qlen, a, b, &p, transition, &runs[k])) {
#pragma omp atomic write
                    fail = 1;
                }
                for (int64_t i = 0; i < runs[k].n; i++) {
                    const int64_t blk = (runs[k].v[i].t - runs[k].v[i].q - dbase) / bw;
                    cnt[blk * nrun + k + 1]++;
                }
            }
            /* block-major exclusive offsets: block blk, run k starts at cnt[blk * nrun + k] */
            for (int64_t i = 0; i < nrun * nblk; i++)
                cnt[i + 1] += cnt[i];
            or_tq *grouped = NULL;
            if (!fail && cnt[nrun * nblk] > 0) {
                grouped = (or_tq *)malloc((size_t)cnt[nrun * nblk] * sizeof(or_tq));
                if (!grouped)
                    fail = 1;
            }
            if (!fail && grouped) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
                for (int64_t k = 0; k < nrun; k++) {
                    for (int64_t i = 0; i < runs[k].n; i++) {
                        const int64_t blk = (runs[k].v[i].t - runs[k].v[i].q - dbase) / bw;
                        grouped[cnt[blk * nrun + k]++] = runs[k].v[i];
                    }
                }
                /* after the scatter, cnt[blk * nrun + nrun - 1] is the end of block blk */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
                for (int64_t blk = 0; blk < nblk; blk++) {
                    const int64_t a = blk ? cnt[blk * nrun - 1] : 0, b = cnt[blk * nrun + nrun - 1];
                    if (b <= a)
                        continue;
                    int tid = 0;
#ifdef _OPENMP
                    tid = omp_get_thread_num();
#endif
                    qsort(grouped + a, (size_t)(b - a), sizeof(or_tq), cmp_diag_t);
                    if (walk(T, tlen, Qs, qlen, s, grouped + a, b - a, Ecarry, dbase, &p, M, X,
                             thresh, flags, &part[tid])) {
#pragma omp atomic write
                        fail = 1;
                    }
                }
            }
            for (int64_t k = 0; k < nrun; k++)
                free(runs[k].v);
            free(runs);
            free(cnt);
            free(grouped);
            if (fail)
                *err = OR_ENOMEM;
        }
        free(Ecarry);
    }
    for (int i = 0; i < nthreads && !*err; i++) {
        for (int64_t j = 0; j < part[i].n && !*err; j++)
            if (push_hsp(r, &part[i].hsp[j]))
                *err = OR_ENOMEM;
        r->st.hits += part[i].st.hits;
        r->st.extended += part[i].st.extended;
        r->st.cells += part[i].st.cells;
        r->st.hsps += part[i].st.hsps;
    }
done:
    free(tab);
    free(rc);
    if (part)
        for (int i = 0; i < nthreads; i++)
            free(part[i].hsp);
    free(part);
    if (*err) {
        if (r)
            free(r->hsp);
        free(r);
        return NULL;
    }
    qsort(r->hsp, (size_t)r->n, sizeof(or_hsp), cmp_hsp);
    return r;
}

/*
 * The same walk restricted to one diagonal d = t - q of one strand (Qs given
 * directly), with hits found by testing every position of the diagonal with
 * the predicate. E0 is the skip state the diagonal starts with. Used for
 * sampled checks on inputs too large for or_run.
 */
or_result *or_run_diagonal(const uint8_t *T, int64_t tlen, const uint8_t *Qs, int64_t qlen,
                           int strand, int64_t d, int64_t E0, const char *pattern, int step,
                           int transition, const int32_t *M, int32_t X, int32_t thresh,
                           int flags, int keep_log, int *err)
{
    or_pattern p;
    *err = OR_OK;
    if (or_parse_pattern(pattern, &p) || step < 1 || X < 0) {
        *err = OR_EINVAL;
        return NULL;
    }
    or_result *r = (or_result *)calloc(1, sizeof(or_result));
    if (!r) {
        *err = OR_ENOMEM;
        return NULL;
    }
    r->keep_log = keep_log;
    int64_t E = E0;
    int64_t t0 = d > 0 ? d : 0;
    for (int64_t t = t0; t + p.span <= tlen && t - d + p.span <= qlen; t++) {
        int64_t q = t - d;
        if (t % step != 0 || !or_is_hit(T, Qs, t, q, &p, transition))
            continue;
        r->st.hits++;
        if (t < E)
            continue;
        or_ext e;
        or_xdrop(T, tlen, Qs, qlen, t, q, p.span, M, X, &e);
        e.strand = strand;
        r->st.extended++;
        r->st.cells += p.span + e.lscored + e.rscored;
        int pass = e.score >= thresh;
        if (pass || !(flags & OR_SKIP_PASSING_ONLY))
            E = t + p.span + e.rext;
        if (keep_log && push_ext(r, &e)) {
            *err = OR_ENOMEM;
            break;
        }
        if (pass) {
            or_hsp o = {strand, (int32_t)(t - e.lext), (int32_t)(q - e.lext),
                        p.span + e.lext + e.rext, (int32_t)e.score};
            r->st.hsps++;
            if (push_hsp(r, &o)) {
                *err = OR_ENOMEM;
                break;
            }
        }
    }
    if (*err) {
        free(r->hsp);
        free(r->ext);
        free(r);
        return NULL;
    }
    qsort(r->hsp, (size_t)r->n, sizeof(or_hsp), cmp_hsp);
    return r;
}

/* Seed hits of one strand, sorted by (diagonal, t): writes up to cap pairs. */
int64_t or_seed_hits(const uint8_t *T, int64_t tlen, const uint8_t *Qs, int64_t qlen,
                     const char *pattern, int step, int transition, int64_t *t_out,
                     int64_t *q_out, int64_t cap, int *err)
{
    or_pattern p;
    *err = OR_OK;
    if (or_parse_pattern(pattern, &p) || step < 1) {
        *err = OR_EINVAL;
        return -1;
    }
    p.step = step;
    tq_vec h;
    int e = enumerate_hits(T, tlen, Qs, qlen, &p, transition, &h);
    if (e) {
        *err = e;
        return -1;
    }
    for (int64_t i = 0; i < h.n && i < cap; i++) {
        t_out[i] = h.v[i].t;
        q_out[i] = h.v[i].q;
    }
    int64_t n = h.n;
    free(h.v);
    return n;
}

int64_t or_result_count(const or_result *r) { return r->n; }
int64_t or_result_ext_count(const or_result *r) { return r->next; }
void or_result_stats(const or_result *r, or_stats *st) { *st = r->st; }
void or_result_copy(const or_result *r, or_hsp *out)
{
    if (r->n)
        memcpy(out, r->hsp, (size_t)r->n * sizeof(or_hsp));
}
void or_result_copy_ext(const or_result *r, or_ext *out)
{
    if (r->next)
        memcpy(out, r->ext, (size_t)r->next * sizeof(or_ext));
}
void or_result_free(or_result *r)
{
    if (!r)
        return;
    free(r->hsp);
    free(r->ext);
    free(r);
}

/* ======================================================= gapped (Y-drop) stage
 *
 * The gapped extension that follows the filter (Algorithm 1: an anchor inside
 * an alignment already committed is skipped, the others are extended with
 * Y-drop and committed when they reach the threshold; Algorithm 3: the same
 * in speculative batches with a serial commit). The paper names Y-drop and
 * LASTZ's loop; the details below are this build's readings.
 *
 *  Scoring: substitutions M[t][q], affine gaps (a gap of L bases costs
 *  open + L * extend).
 *
 *  One half of an extension, from anchor (t0, q0) in direction dir: cell
 *  (i, j), 0 <= i <= TL, 0 <= j <= QL, has consumed i target and j query
 *  bases (forward: T[t0 .. t0+i), backward: T[t0-i .. t0)). H[0][0] = 0 and
 *    E[i][j] = max(E[i][j-1] - ext, H[i][j-1] - open - ext)   (gap in T)
 *    F[i][j] = max(F[i-1][j] - ext, H[i-1][j] - open - ext)   (gap in Q)
 *    H[i][j] = max(H[i-1][j-1] + M[T_i][Q_j], E[i][j], F[i][j])
 *  evaluated by anti-diagonals d = i + j. A cell is live when its H is at
 *  least best - Y, best being the maximum H of the anti-diagonals before d;
 *  a cell that is not live has H = E = F = -inf and feeds nothing. Anti-
 *  diagonal d computes every cell from the lowest to the highest i that has
 *  a live neighbour on d - 1 or a live diagonal predecessor on d - 2 (a
 *  contiguous range), at most `band` of them (from the lowest i on). A diagonal step skips an anti-diagonal, so the half stops
 *  only when two consecutive anti-diagonals hold no live cell. It returns
 *  best and the first cell (lowest d, then lowest i) where best was reached;
 *  cells = cells computed beyond the origin.
 *
 *  Anchor of an HSP: its midpoint (tpos + len/2, qpos + len/2). Alignment =
 *  backward half + forward half: score = sum of the two bests, box
 *  [t0 - bi_b, t0 + bi_f) x [q0 - bj_b, q0 + bj_f).
 *
 *  Order and containment: anchors in decreasing HSP score (then strand, tpos,
 *  qpos, len); an anchor (t, q) is contained when it lies in the box
 *  [tstart, tend) x [qstart, qend) of an alignment committed on its strand.
 *  Only alignments with score >= threshold are committed (Algorithm 1's
 *  CommitAlignment and UpdateMaskingLists).
 */

#define OR_YNEG (-(1 << 29))

typedef struct {
    int64_t best;
    int32_t bi, bj;
    int64_t cells;
} or_half;

typedef struct {
    int32_t strand, tstart, tend, qstart, qend, score;
} or_galign;

typedef struct {
    int64_t anchors;        /* anchors in the input */
    int64_t skipped;        /* contained when reached (never extended) */
    int64_t extended;       /* extensions whose result counts */
    int64_t cells;          /* DP cells of those extensions */
    int64_t shadow;         /* speculative extensions found contained at commit */
    int64_t shadow_cells;   /* their DP cells */
    int64_t committed;      /* alignments reported (score >= threshold) */
    int64_t batches;
} or_gstats;

static int32_t tbase(const uint8_t *S, int64_t p0, int dir, int64_t i)
{
    /* base consumed by step i (1-based) of a half from p0 in direction dir */
    return dir > 0 ? S[p0 + i - 1] : S[p0 - i];
}

void or_ydrop_half(const uint8_t *T, int64_t t0, int64_t TL, const uint8_t *Q, int64_t q0,
                   int64_t QL, int dir, const int32_t *M, int32_t gopen, int32_t gext,
                   int32_t Y, int band, or_half *out)
{
    int32_t *buf = (int32_t *)malloc((size_t)band * 7 * sizeof(int32_t));
    int32_t *H2 = buf, *H1 = buf + band, *E1 = buf + 2 * band, *F1 = buf + 3 * band;
    int32_t *H0 = buf + 4 * band, *E0 = buf + 5 * band, *F0 = buf + 6 * band;
    /* anti-diagonal 0: the origin */
    int64_t lo1 = 0, hi1 = 0, L1 = 0, R1 = 0;       /* computed range, live range of d - 1 */
    int64_t lo2 = 1, hi2 = 0, L2 = 1, R2 = 0;       /* d - 2: nothing yet */
    H1[0] = 0;
    E1[0] = F1[0] = OR_YNEG;
    int64_t best = 0;
    int32_t bi = 0, bj = 0;
    int64_t cells = 0;
    for (int64_t d = 1;; d++) {
        if (L1 > R1 && L2 > R2)
            break; /* two anti-diagonals without a live cell: nothing can follow */
        int64_t clo, chi;
        if (L1 <= R1 && L2 <= R2) {
            clo = L1 < L2 + 1 ? L1 : L2 + 1;
            chi = R1 + 1 > R2 + 1 ? R1 + 1 : R2 + 1;
        } else if (L1 <= R1) {
            clo = L1;
            chi = R1 + 1;
        } else {
            clo = L2 + 1;
            chi = R2 + 1;
        }
        if (clo < d - QL)
            clo = d - QL;
        if (clo < 0)
            clo = 0;
        if (chi > TL)
            chi = TL;
        if (chi > d)
            chi = d;
        if (chi > clo + band - 1)
            chi = clo + band - 1;
        int64_t L0 = 1, R0 = 0, dbest = OR_YNEG; /* live range of d (empty: L0 > R0) */
        int32_t dbi = 0;
        for (int64_t i = clo; i <= chi; i++) {
            int64_t j = d - i;
            int32_t dg = OR_YNEG, e = OR_YNEG, f = OR_YNEG;
            if (i >= 1 && j >= 1 && i - 1 >= lo2 && i - 1 <= hi2 && H2[i - 1 - lo2] > OR_YNEG)
                dg = H2[i - 1 - lo2] + M[tbase(T, t0, dir, i) * 4 + tbase(Q, q0, dir, j)];
            if (j >= 1 && i >= lo1 && i <= hi1 && H1[i - lo1] > OR_YNEG) {
                int32_t a = E1[i - lo1] - gext, b = H1[i - lo1] - gopen - gext;
                e = a > b ? a : b;
            }
            if (i >= 1 && i - 1 >= lo1 && i - 1 <= hi1 && H1[i - 1 - lo1] > OR_YNEG) {
                int32_t a = F1[i - 1 - lo1] - gext, b = H1[i - 1 - lo1] - gopen - gext;
                f = a > b ? a : b;
            }
            int32_t h = dg;
            if (e > h)
                h = e;
            if (f > h)
                h = f;
            if (h <= OR_YNEG || (int64_t)h < best - Y) {
                h = e = f = OR_YNEG;
            } else {
                if (L0 > R0)
                    L0 = i;
                R0 = i;
                if (h > dbest) {
                    dbest = h;
                    dbi = (int32_t)i;
                }
            }
            H0[i - clo] = h;
            E0[i - clo] = e;
            F0[i - clo] = f;
            cells++;
        }
        if (dbest > best) {
            best = dbest;
            bi = dbi;
            bj = (int32_t)(d - dbi);
        }
        /* rotate: d - 1 becomes d - 2, d becomes d - 1 */
        int32_t *t;
        t = H2; H2 = H1; H1 = H0; H0 = t;
        t = E1; E1 = E0; E0 = t;
        t = F1; F1 = F0; F0 = t;
        lo2 = lo1; hi2 = hi1; L2 = L1; R2 = R1;
        lo1 = clo; hi1 = chi; L1 = L0; R1 = R0;
        if (clo > chi) { /* no candidate at all: an empty anti-diagonal */
            lo1 = 1; hi1 = 0;
        }
    }
    free(buf);
    out->best = best;
    out->bi = bi;
    out->bj = bj;
    out->cells = cells;
}

/* Both halves from anchor (t0, q0) of Qs. */
static void ydrop_anchor(const uint8_t *T, int64_t tlen, const uint8_t *Qs, int64_t qlen,
                         int64_t t0, int64_t q0, const int32_t *M, int32_t gopen, int32_t gext,
                         int32_t Y, int band, int strand, or_galign *a, int64_t *cells)
{
    or_half f, b;
    or_ydrop_half(T, t0, tlen - t0, Qs, q0, qlen - q0, +1, M, gopen, gext, Y, band, &f);
    or_ydrop_half(T, t0, t0, Qs, q0, q0, -1, M, gopen, gext, Y, band, &b);
    a->strand = strand;
    a->tstart = (int32_t)(t0 - b.bi);
    a->tend = (int32_t)(t0 + f.bi);
    a->qstart = (int32_t)(q0 - b.bj);
    a->qend = (int32_t)(q0 + f.bj);
    a->score = (int32_t)(f.best + b.best);
    *cells = f.cells + b.cells;
}

typedef struct {
    or_hsp h;
    int64_t idx;
} or_anchor;

static int cmp_anchor(const void *x, const void *y)
{
    const or_hsp *a = &((const or_anchor *)x)->h, *b = &((const or_anchor *)y)->h;
    if (a->score != b->score) return a->score > b->score ? -1 : 1;
    if (a->strand != b->strand) return a->strand < b->strand ? -1 : 1;
    if (a->tpos != b->tpos) return a->tpos < b->tpos ? -1 : 1;
    if (a->qpos != b->qpos) return a->qpos < b->qpos ? -1 : 1;
    if (a->len != b->len) return a->len < b->len ? -1 : 1;
    return 0;
}

static int cmp_galign(const void *x, const void *y)
{
    const or_galign *a = (const or_galign *)x, *b = (const or_galign *)y;
    if (a->strand != b->strand) return a->strand < b->strand ? -1 : 1;
    if (a->tstart != b->tstart) return a->tstart < b->tstart ? -1 : 1;
    if (a->qstart != b->qstart) return a->qstart < b->qstart ? -1 : 1;
    if (a->tend != b->tend) return a->tend < b->tend ? -1 : 1;
    if (a->qend != b->qend) return a->qend < b->qend ? -1 : 1;
    if (a->score != b->score) return a->score < b->score ? -1 : 1;
    return 0;
}

/* Is (strand, t, q) inside the box of one of the n committed alignments? */
static int contained(const or_galign *c, int64_t n, int strand, int64_t t, int64_t q)
{
    for (int64_t k = 0; k < n; k++)
        if (c[k].strand == strand && c[k].tstart <= t && t < c[k].tend && c[k].qstart <= q &&
            q < c[k].qend)
            return 1;
    return 0;
}

/*
 * The gapped stage over the HSPs of a pair (strand 1 coordinates index the
 * reverse complement of Q). batch <= 0: Algorithm 1 (serial). batch K > 0:
 * Algorithm 3 (the next K anchors not contained in what is committed so far
 * are extended, then committed one by one in order unless an alignment
 * committed before them, in this batch or earlier, now contains them). Writes
 * at most cap alignments, sorted by (strand, tstart, qstart, tend, qend,
 * score); returns their number, or -1 on error.
 */
int64_t or_gapped(const uint8_t *T, int64_t tlen, const uint8_t *Q, int64_t qlen,
                  const or_hsp *hsps, int64_t nhsps, const int32_t *M, int32_t gopen,
                  int32_t gext, int32_t Y, int32_t thresh, int band, int64_t batch,
                  or_galign *out, int64_t cap, or_gstats *st)
{
    memset(st, 0, sizeof(*st));
    st->anchors = nhsps;
    if (band < 1 || gopen < 0 || gext < 0 || Y < 0)
        return -1;
    uint8_t *rc = (uint8_t *)malloc((size_t)(qlen > 0 ? qlen : 1));
    or_anchor *an = (or_anchor *)malloc((size_t)(nhsps > 0 ? nhsps : 1) * sizeof(or_anchor));
    or_galign *com = (or_galign *)malloc((size_t)(nhsps > 0 ? nhsps : 1) * sizeof(or_galign));
    or_galign *ext = (or_galign *)malloc((size_t)(nhsps > 0 ? nhsps : 1) * sizeof(or_galign));
    int64_t *ecells = (int64_t *)malloc((size_t)(nhsps > 0 ? nhsps : 1) * sizeof(int64_t));
    int64_t *pick = (int64_t *)malloc((size_t)(nhsps > 0 ? nhsps : 1) * sizeof(int64_t));
    if (!rc || !an || !com || !ext || !ecells || !pick) {
        free(rc); free(an); free(com); free(ext); free(ecells); free(pick);
        return -1;
    }
    or_revcomp(Q, qlen, rc);
    for (int64_t k = 0; k < nhsps; k++) {
        an[k].h = hsps[k];
        an[k].idx = k;
    }
    qsort(an, (size_t)nhsps, sizeof(or_anchor), cmp_anchor);
    int64_t ncom = 0, j = 0;
    while (j < nhsps) {
        /* phase 1: the next anchors not contained in what is committed */
        int64_t nb = 0;
        int64_t K = batch > 0 ? batch : 1;
        while (nb < K && j < nhsps) {
            const or_hsp *h = &an[j].h;
            int64_t ta = h->tpos + h->len / 2, qa = h->qpos + h->len / 2;
            if (contained(com, ncom, h->strand, ta, qa))
                st->skipped++;
            else
                pick[nb++] = j;
            j++;
        }
        if (nb == 0)
            break;
        st->batches++;
        /* phase 2: extend every picked anchor */
        for (int64_t b = 0; b < nb; b++) {
            const or_hsp *h = &an[pick[b]].h;
            int64_t ta = h->tpos + h->len / 2, qa = h->qpos + h->len / 2;
            const uint8_t *Qs = h->strand ? rc : Q;
            ydrop_anchor(T, tlen, Qs, qlen, ta, qa, M, gopen, gext, Y, band, h->strand, &ext[b],
                         &ecells[b]);
        }
        /* phase 3: commit in order */
        for (int64_t b = 0; b < nb; b++) {
            const or_hsp *h = &an[pick[b]].h;
            int64_t ta = h->tpos + h->len / 2, qa = h->qpos + h->len / 2;
            if (b > 0 && contained(com, ncom, h->strand, ta, qa)) {
                st->shadow++;
                st->shadow_cells += ecells[b];
                continue;
            }
            st->extended++;
            st->cells += ecells[b];
            if (ext[b].score >= thresh)
                com[ncom++] = ext[b];
        }
    }
    st->committed = ncom;
    qsort(com, (size_t)ncom, sizeof(or_galign), cmp_galign);
    for (int64_t k = 0; k < ncom && k < cap; k++)
        out[k] = com[k];
    free(rc); free(an); free(ext); free(ecells); free(pick);
    free(com);
    return ncom;
}
