/*
 * oracle/apriori.c -- TEST INFRASTRUCTURE ONLY (the CPU oracle).
 *
 * Nothing on the product path may link or call this file.  It is a plain,
 * slow, obviously correct level-wise Apriori that counts every candidate by
 * scanning the transactions themselves.  It shares no code, header, table or
 * helper with the GPU miner.
 *
 * What it computes (Section III of the paper):
 *   Eq. 1  M[i,j] = 1 iff item j is in transaction T_i (set membership, so a
 *          repeated item inside one transaction counts once);
 *   Eq. 2  S(X)   = number of transactions i with M[i,x] = 1 for every x in X
 *          (the pairwise AND generalised to any itemset, as the text after
 *          Eq. 2 extends it to higher orders);
 *   Eq. 3  X is frequent iff S(X) > theta.  The threshold is taken here as an
 *          absolute count; with strict == 0 the test is S(X) >= theta (the
 *          usual "minimum support" reading), with strict == 1 it is the
 *          paper's literal S(X) > theta.
 * The answer F = { X != {} : X frequent } is unique.  It is emitted in
 * canonical order: items ascending inside a set, sets ordered by size and
 * then lexicographically, supports as exact integers.
 *
 * Algorithm (textbook Apriori, Agrawal & Srikant 1994):
 *   1. sort and de-duplicate every transaction;
 *   2. L1 = frequent single items, by a scan;
 *   3. for k >= 2: C_k = join of two (k-1)-sets of L_{k-1} that share their
 *      first k-2 items; drop a candidate if any (k-1)-subset is not in
 *      L_{k-1}; count every candidate by walking each transaction through the
 *      sorted candidate list; L_k = frequent candidates;
 *   4. stop when L_k is empty (or k exceeds max_len when max_len > 0).
 * Counting is split over threads by transaction slices with private counters,
 * summed afterwards; integer sums make the thread count irrelevant to the
 * result.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2 };

/* OR_MUTANT selects a deliberately planted mistake, compiled only by the
 * tests that check that the pins catch it (0 = the oracle as written):
 *   1 threshold off by one, 2 duplicates not collapsed, 3 counting walk
 *   stops one item early, 4 join takes the wrong last item, 5 subset prune
 *   rejects frequent subsets. */
#ifndef OR_MUTANT
#define OR_MUTANT 0
#endif

typedef struct {
    uint64_t n_sets;
    uint64_t n_items_total;
    uint64_t *offsets;       /* [n_sets + 1] */
    uint32_t *items;         /* [n_items_total] */
    uint64_t *supports;      /* [n_sets] */
    uint64_t n_candidates;   /* candidates counted over all levels */
    int max_level;
} or_result;

/* ---- transactions: sorted, de-duplicated copy ------------------------- */

typedef struct {
    int64_t n;
    int64_t *ptr;   /* [n+1] */
    uint32_t *it;   /* sorted, distinct items per row */
} tdb;

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

static int tdb_make(tdb *t, const int64_t *indptr, const int32_t *indices,
                    int64_t n, int32_t m) {
    if (n < 0 || m < 0 || !indptr) return OR_EINVAL;
    if (indptr[0] != 0) return OR_EINVAL;
    for (int64_t i = 0; i < n; i++)
        if (indptr[i + 1] < indptr[i]) return OR_EINVAL;
    int64_t nnz = indptr[n];
    if (nnz > 0 && !indices) return OR_EINVAL;
    for (int64_t e = 0; e < nnz; e++)
        if (indices[e] < 0 || indices[e] >= m) return OR_EINVAL;
    t->n = n;
    t->ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    t->it = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!t->ptr || !t->it) return OR_ENOMEM;
    int64_t w = 0;
    t->ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t b = indptr[i], e = indptr[i + 1];
        uint32_t *row = t->it + w;
        for (int64_t k = b; k < e; k++) row[k - b] = (uint32_t)indices[k];
        int64_t len = e - b;
        qsort(row, (size_t)len, sizeof(uint32_t), cmp_u32);
        int64_t u = 0;
        for (int64_t k = 0; k < len; k++)
            if (u == 0 || row[k] != row[u - 1] || OR_MUTANT == 2) row[u++] = row[k];
        w += u;
        t->ptr[i + 1] = w;
    }
    return OR_OK;
}

static void tdb_free(tdb *t) {
    free(t->ptr);
    free(t->it);
}

static int is_frequent(uint64_t s, uint64_t thr, int strict) {
    if (OR_MUTANT == 1) return s > thr + (uint64_t)strict;
    return strict ? (s > thr) : (s >= thr);
}

/* ---- candidate counting: walk one transaction through the candidates -- */
/* Candidates of size k are stored flat (k items each), sorted
 * lexicographically.  Inside any range that shares the first d items, column
 * d is ascending, so the range with a given item at position d is found by
 * binary search. */

typedef struct {
    const uint32_t *cand; /* [nc * k] */
    uint64_t nc;
    int k;
} cset;

static uint64_t lower_col(const cset *c, uint64_t lo, uint64_t hi, int d, uint32_t x) {
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (c->cand[mid * (uint64_t)c->k + (uint64_t)d] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

static uint64_t upper_col(const cset *c, uint64_t lo, uint64_t hi, int d, uint32_t x) {
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (c->cand[mid * (uint64_t)c->k + (uint64_t)d] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* Every candidate in [lo,hi) matches the transaction on its first d items,
 * the last of them found at a position before `pos`. */
static void walk(const cset *c, const uint32_t *t, int64_t len, int64_t pos,
                 int d, uint64_t lo, uint64_t hi, uint32_t *counts) {
    int k = c->k;
    for (int64_t p = pos; p + (k - d) + (OR_MUTANT == 3) <= len && lo < hi; p++) {
        uint32_t x = t[p];
        uint64_t a = lower_col(c, lo, hi, d, x);
        if (a == hi) break; /* every remaining candidate has a larger item here */
        if (c->cand[a * (uint64_t)k + (uint64_t)d] != x) { lo = a; continue; }
        uint64_t b = upper_col(c, a, hi, d, x);
        if (d == k - 1) counts[a] += 1; /* candidates are distinct: b == a+1 */
        else walk(c, t, len, p + 1, d + 1, a, b, counts);
        lo = b;
    }
}

typedef struct {
    const tdb *db;
    const cset *c;
    int64_t r0, r1;
    uint32_t *counts;
} job;

static void *count_job(void *arg) {
    job *j = (job *)arg;
    for (int64_t i = j->r0; i < j->r1; i++) {
        const uint32_t *t = j->db->it + j->db->ptr[i];
        int64_t len = j->db->ptr[i + 1] - j->db->ptr[i];
        if (len >= j->c->k) walk(j->c, t, len, 0, 0, 0, j->c->nc, j->counts);
    }
    return NULL;
}

/* counts[i] = number of transactions containing candidate i (exact). */
static int count_candidates(const tdb *db, const cset *c, int nthreads, uint64_t *out) {
    if (nthreads < 1) nthreads = 1;
    if (c->nc == 0) return OR_OK;
    job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return OR_ENOMEM; }
    int rc = OR_OK;
    for (int t = 0; t < nthreads; t++) {
        jobs[t].db = db;
        jobs[t].c = c;
        jobs[t].r0 = db->n * t / nthreads;
        jobs[t].r1 = db->n * (t + 1) / nthreads;
        jobs[t].counts = (uint32_t *)calloc((size_t)c->nc, sizeof(uint32_t));
        if (!jobs[t].counts) rc = OR_ENOMEM;
    }
    if (rc == OR_OK) {
        for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, count_job, &jobs[t]);
        count_job(&jobs[0]);
        for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
        for (uint64_t i = 0; i < c->nc; i++) out[i] = 0;
        for (int t = 0; t < nthreads; t++)
            for (uint64_t i = 0; i < c->nc; i++) out[i] += jobs[t].counts[i];
    }
    for (int t = 0; t < nthreads; t++) free(jobs[t].counts);
    free(jobs);
    free(th);
    return rc;
}

/* ---- output accumulation ---------------------------------------------- */

typedef struct {
    uint64_t n_sets, n_items, cap_sets, cap_items;
    uint64_t *offsets, *supports;
    uint32_t *items;
} outbuf;

static int out_push(outbuf *o, const uint32_t *set, int k, uint64_t s) {
    if (o->n_sets + 2 > o->cap_sets) {
        uint64_t nc = o->cap_sets ? o->cap_sets * 2 : 1024;
        uint64_t *a = (uint64_t *)realloc(o->offsets, nc * sizeof(uint64_t));
        if (!a) return OR_ENOMEM;
        o->offsets = a;
        uint64_t *b = (uint64_t *)realloc(o->supports, nc * sizeof(uint64_t));
        if (!b) return OR_ENOMEM;
        o->supports = b;
        o->cap_sets = nc;
    }
    if (o->n_items + (uint64_t)k > o->cap_items) {
        uint64_t nc = o->cap_items ? o->cap_items * 2 : 4096;
        while (nc < o->n_items + (uint64_t)k) nc *= 2;
        uint32_t *a = (uint32_t *)realloc(o->items, nc * sizeof(uint32_t));
        if (!a) return OR_ENOMEM;
        o->items = a;
        o->cap_items = nc;
    }
    if (o->n_sets == 0) o->offsets[0] = 0;
    memcpy(o->items + o->n_items, set, (size_t)k * sizeof(uint32_t));
    o->n_items += (uint64_t)k;
    o->supports[o->n_sets] = s;
    o->n_sets += 1;
    o->offsets[o->n_sets] = o->n_items;
    return OR_OK;
}

/* is the (k-1)-set `s` one of the nl sorted sets in `lv`? */
static int in_level(const uint32_t *lv, uint64_t nl, int km1, const uint32_t *s) {
    uint64_t lo = 0, hi = nl;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        int cmp = 0;
        for (int q = 0; q < km1; q++) {
            uint32_t a = lv[mid * (uint64_t)km1 + (uint64_t)q], b = s[q];
            if (a != b) { cmp = a < b ? -1 : 1; break; }
        }
        if (cmp == 0) return OR_MUTANT != 5;
        if (cmp < 0) lo = mid + 1;
        else hi = mid;
    }
    return 0;
}

/* ---- public entry points ---------------------------------------------- */

int or_apriori(const int64_t *indptr, const int32_t *indices, int64_t n, int32_t m,
               uint64_t threshold, int strict, int nthreads, int max_len,
               or_result *res) {
    if (!res) return OR_EINVAL;
    memset(res, 0, sizeof(*res));
    tdb db;
    memset(&db, 0, sizeof(db));
    int rc = tdb_make(&db, indptr, indices, n, m);
    if (rc != OR_OK) { tdb_free(&db); return rc; }

    outbuf o;
    memset(&o, 0, sizeof(o));

    /* level 1: count each item by a scan of the transactions */
    uint64_t *c1 = (uint64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(uint64_t));
    if (!c1) { tdb_free(&db); return OR_ENOMEM; }
    for (int64_t e = 0; e < db.ptr[n]; e++) c1[db.it[e]] += 1;
    res->n_candidates += (uint64_t)m;
    uint32_t *lv = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    uint64_t nl = 0;
    for (int32_t j = 0; j < m; j++)
        if (is_frequent(c1[j], threshold, strict)) {
            lv[nl++] = (uint32_t)j;
            if ((rc = out_push(&o, (uint32_t *)&j, 1, c1[j])) != OR_OK) goto done;
        }
    free(c1);
    c1 = NULL;
    res->max_level = nl ? 1 : 0;

    for (int k = 2; nl > 0 && (max_len <= 0 || k <= max_len); k++) {
        int km1 = k - 1;
        /* join: sets i < j of L_{k-1} that agree on their first k-2 items */
        uint64_t cap = 1024, nc = 0;
        uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * cap * (uint64_t)k);
        uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k);
        uint32_t *sub = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k);
        if (!cand || !tmp || !sub) { free(cand); free(tmp); free(sub); rc = OR_ENOMEM; goto done; }
        uint64_t b0 = 0;
        while (b0 < nl) {
            uint64_t b1 = b0 + 1;
            while (b1 < nl && memcmp(lv + b1 * km1, lv + b0 * km1,
                                     sizeof(uint32_t) * (size_t)(km1 - 1)) == 0)
                b1++;
            for (uint64_t i = b0; i < b1; i++)
                for (uint64_t j = i + 1; j < b1; j++) {
                    memcpy(tmp, lv + i * km1, sizeof(uint32_t) * (size_t)km1);
                    tmp[km1] = lv[(OR_MUTANT == 4 ? i : j) * km1 + (uint64_t)(km1 - 1)];
                    /* prune: every (k-1)-subset must be frequent.  Dropping one
                     * of the last two items gives sets i and j themselves. */
                    int ok = 1;
                    for (int drop = 0; ok && drop < k - 2; drop++) {
                        int w = 0;
                        for (int q = 0; q < k; q++)
                            if (q != drop) sub[w++] = tmp[q];
                        ok = in_level(lv, nl, km1, sub);
                    }
                    if (!ok) continue;
                    if (nc == cap) {
                        cap *= 2;
                        uint32_t *g = (uint32_t *)realloc(cand, sizeof(uint32_t) * cap * (uint64_t)k);
                        if (!g) { free(cand); free(tmp); free(sub); rc = OR_ENOMEM; goto done; }
                        cand = g;
                    }
                    memcpy(cand + nc * (uint64_t)k, tmp, sizeof(uint32_t) * (size_t)k);
                    nc++;
                }
            b0 = b1;
        }
        free(tmp);
        free(sub);
        /* the join over a lexicographically sorted L_{k-1} emits candidates
         * in lexicographic order, which the counting walk relies on */
        cset cs = {cand, nc, k};
        uint64_t *cnt = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nc > 0 ? nc : 1));
        if (!cnt) { free(cand); rc = OR_ENOMEM; goto done; }
        rc = count_candidates(&db, &cs, nthreads, cnt);
        if (rc != OR_OK) { free(cand); free(cnt); goto done; }
        res->n_candidates += nc;
        uint64_t nn = 0;
        for (uint64_t i = 0; i < nc; i++)
            if (is_frequent(cnt[i], threshold, strict)) {
                memmove(cand + nn * (uint64_t)k, cand + i * (uint64_t)k, sizeof(uint32_t) * (size_t)k);
                if ((rc = out_push(&o, cand + nn * (uint64_t)k, k, cnt[i])) != OR_OK) {
                    free(cand); free(cnt); goto done;
                }
                nn++;
            }
        free(cnt);
        free(lv);
        lv = cand;
        nl = nn;
        if (nl) res->max_level = k;
    }

done:
    free(c1);
    free(lv);
    tdb_free(&db);
    if (rc != OR_OK) {
        free(o.offsets); free(o.items); free(o.supports);
        return rc;
    }
    if (o.n_sets == 0) {
        o.offsets = (uint64_t *)calloc(1, sizeof(uint64_t));
        if (!o.offsets) return OR_ENOMEM;
    }
    res->n_sets = o.n_sets;
    res->n_items_total = o.n_items;
    res->offsets = o.offsets;
    res->items = o.items;
    res->supports = o.supports;
    return OR_OK;
}

void or_free(or_result *r) {
    if (!r) return;
    free(r->offsets);
    free(r->items);
    free(r->supports);
    memset(r, 0, sizeof(*r));
}

/* ---- direct support of given itemsets, by a scan ---------------------- */
/* out[q] = S(X_q) for the itemsets X_q = items[qoff[q]:qoff[q+1]] (Eq. 2
 * generalised), counted over transactions with set semantics. */

typedef struct {
    const int64_t *indptr;
    const int32_t *indices;
    int64_t r0, r1;
    int32_t m;
    const uint64_t *qoff;
    const uint32_t *qitems;
    uint64_t nq;
    uint64_t *out;
    int rc;
} sjob;

static void *support_job(void *arg) {
    sjob *j = (sjob *)arg;
    uint8_t *here = (uint8_t *)calloc((size_t)(j->m > 0 ? j->m : 1), 1);
    if (!here) { j->rc = OR_ENOMEM; return NULL; }
    for (int64_t i = j->r0; i < j->r1; i++) {
        for (int64_t e = j->indptr[i]; e < j->indptr[i + 1]; e++) here[j->indices[e]] = 1;
        for (uint64_t q = 0; q < j->nq; q++) {
            int all = 1;
            for (uint64_t p = j->qoff[q]; p < j->qoff[q + 1]; p++)
                if (!here[j->qitems[p]]) { all = 0; break; }
            j->out[q] += (uint64_t)all;
        }
        for (int64_t e = j->indptr[i]; e < j->indptr[i + 1]; e++) here[j->indices[e]] = 0;
    }
    free(here);
    return NULL;
}

int or_support_many(const int64_t *indptr, const int32_t *indices, int64_t n, int32_t m,
                    const uint64_t *qoff, const uint32_t *qitems, uint64_t nq,
                    int nthreads, uint64_t *out) {
    if (n < 0 || m < 0 || !indptr || !qoff || !out) return OR_EINVAL;
    for (int64_t e = 0; e < indptr[n]; e++)
        if (indices[e] < 0 || indices[e] >= m) return OR_EINVAL;
    for (uint64_t p = 0; p < (nq ? qoff[nq] : 0); p++)
        if (qitems[p] >= (uint32_t)m) return OR_EINVAL;
    if (nthreads < 1) nthreads = 1;
    sjob *jobs = (sjob *)calloc((size_t)nthreads, sizeof(sjob));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return OR_ENOMEM; }
    for (int t = 0; t < nthreads; t++) {
        sjob s = {indptr, indices, n * t / nthreads, n * (t + 1) / nthreads, m,
                  qoff, qitems, nq, (uint64_t *)calloc((size_t)(nq ? nq : 1), sizeof(uint64_t)), OR_OK};
        jobs[t] = s;
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, support_job, &jobs[t]);
    support_job(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    int rc = OR_OK;
    for (uint64_t q = 0; q < nq; q++) out[q] = 0;
    for (int t = 0; t < nthreads; t++) {
        if (!jobs[t].out || jobs[t].rc != OR_OK) rc = OR_ENOMEM;
        else
            for (uint64_t q = 0; q < nq; q++) out[q] += jobs[t].out[q];
        free(jobs[t].out);
    }
    free(jobs);
    free(th);
    return rc;
}
