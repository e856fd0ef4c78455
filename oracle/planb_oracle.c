/*
 * CPU oracle for batched IPv6 longest-prefix-match (LPM).
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled into liboracle.so, which only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load. It shares no code, header or table with the
 * CUDA lookup library, and the lookup library never calls it.
 *
 * What it computes is the plain definition of LPM that the paper's method reaches exactly
 * (Section 1 and Section 3.1): the next hop of an address x is the next hop of the prefix (p, L) with
 * the largest L whose top L bits equal the top L bits of x; if no prefix matches, the default next hop
 * 0. A ::/0 entry in the table matches every address, so it supplies the default when present.
 * Host bits of a prefix beyond its length are ignored. When the same (prefix, length) occurs more than
 * once, the entry that comes last in the input wins.
 *
 *   O1  orc_brute_lookup   scan of every prefix per address (the definition written out)
 *   O2  orc_trie_*         binary trie: one node per bit, MSB first; a walk remembers the last next hop
 *   O3  orc_check_intervals
 *        checks a sorted elementary-interval array (start[], nh[]) against the prefix table: it must
 *        partition [0, 2^128) (Section 3.1, "Interval Partitioning": disjoint, contiguous), hold no
 *        more than 2N+1 intervals, have every prefix start and end as a boundary, and give every
 *        point of each interval that interval's LPM next hop (checked with O2 at both ends of every
 *        interval and on both sides of every prefix boundary; between two consecutive prefix
 *        boundaries the set of covering prefixes, and so the LPM, does not change).
 *
 * Addresses are (hi, lo) u64 pairs: hi is the first 8 bytes of the address in network order read as
 * a big-endian integer, lo the last 8 (Section 3.1: 2001:db8:: is hi = 0x20010db800000000, lo = 0).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static u128 mk(uint64_t hi, uint64_t lo) { return ((u128)hi << 64) | lo; }

/* top `len` bits of a 128-bit value set (len in 0..128) */
static void top_mask(int len, uint64_t *mhi, uint64_t *mlo) {
    if (len <= 0) { *mhi = 0; *mlo = 0; return; }
    if (len >= 128) { *mhi = ~0ULL; *mlo = ~0ULL; return; }
    if (len >= 64) {
        *mhi = ~0ULL;
        *mlo = (len == 64) ? 0 : (~0ULL << (128 - len));
    } else {
        *mhi = ~0ULL << (64 - len);
        *mlo = 0;
    }
}

/* ------------------------------------------------------------------------------ threads helper */

typedef void (*range_fn)(void *ctx, size_t begin, size_t end);
typedef struct { range_fn fn; void *ctx; size_t b, e; } slice_t;

static void *slice_main(void *p) {
    slice_t *s = (slice_t *)p;
    s->fn(s->ctx, s->b, s->e);
    return NULL;
}

/* run fn over [0, n) in `threads` contiguous slices; returns the number of threads used */
static int parallel_for(size_t n, int threads, range_fn fn, void *ctx) {
    if (threads < 1) threads = 1;
    if ((size_t)threads > n) threads = n ? (int)n : 1;
    if (threads == 1) { fn(ctx, 0, n); return 1; }
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * threads);
    slice_t *sl = (slice_t *)malloc(sizeof(slice_t) * threads);
    int started = 0;
    for (int t = 0; t < threads; t++) {
        sl[t].fn = fn; sl[t].ctx = ctx;
        sl[t].b = n * (size_t)t / threads;
        sl[t].e = n * (size_t)(t + 1) / threads;
        if (pthread_create(&tid[t], NULL, slice_main, &sl[t]) != 0) {
            fn(ctx, sl[t].b, sl[t].e);       /* could not start a thread: do the slice here */
            tid[t] = 0;
        } else {
            started++;
        }
    }
    for (int t = 0; t < threads; t++)
        if (tid[t]) pthread_join(tid[t], NULL);
    free(tid); free(sl);
    return started ? started : 1;
}

/* ---------------------------------------------------------------------------------- O1 brute force */

typedef struct {
    size_t np;
    const uint64_t *phi, *plo; const uint8_t *plen; const uint16_t *pnh;
    const uint64_t *xhi, *xlo; uint16_t *out;
} brute_ctx;

static void brute_range(void *c_, size_t b, size_t e) {
    brute_ctx *c = (brute_ctx *)c_;
    for (size_t i = b; i < e; i++) {
        uint64_t xh = c->xhi[i], xl = c->xlo[i];
        int best_len = -1;
        uint16_t best_nh = 0;
        for (size_t j = 0; j < c->np; j++) {
            uint64_t mh, ml;
            int L = c->plen[j];
            top_mask(L, &mh, &ml);
            if (((xh ^ c->phi[j]) & mh) == 0 && ((xl ^ c->plo[j]) & ml) == 0 && L >= best_len) {
                best_len = L;          /* ">=": a later duplicate of the same prefix wins */
                best_nh = c->pnh[j];
            }
        }
        c->out[i] = best_len >= 0 ? best_nh : 0;
    }
}

/* O1: returns threads used, or -1 if a length exceeds 128 */
int orc_brute_lookup(size_t np, const uint64_t *phi, const uint64_t *plo, const uint8_t *plen,
                     const uint16_t *pnh, size_t nk, const uint64_t *xhi, const uint64_t *xlo,
                     uint16_t *out, int threads) {
    for (size_t j = 0; j < np; j++)
        if (plen[j] > 128) return -1;
    brute_ctx c = {np, phi, plo, plen, pnh, xhi, xlo, out};
    return parallel_for(nk, threads, brute_range, &c);
}

/* ---------------------------------------------------------------------------------- O2 binary trie */

typedef struct { int32_t child[2]; int32_t nh; } tnode;   /* nh = -1: no prefix ends here */

typedef struct orc_trie {
    tnode *node;
    size_t used, cap;
} orc_trie;

static int bit_at(uint64_t hi, uint64_t lo, int t) {     /* t = 0 is the most significant bit */
    return t < 64 ? (int)((hi >> (63 - t)) & 1) : (int)((lo >> (127 - t)) & 1);
}

static int32_t trie_new_node(orc_trie *t) {
    if (t->used == t->cap) {
        size_t nc = t->cap ? t->cap * 2 : 1024;
        tnode *p = (tnode *)realloc(t->node, nc * sizeof(tnode));
        if (!p) return -1;
        t->node = p; t->cap = nc;
    }
    if (t->used >= 0x7fffffff) return -1;
    tnode *n = &t->node[t->used];
    n->child[0] = n->child[1] = -1;
    n->nh = -1;
    return (int32_t)t->used++;
}

void orc_trie_free(orc_trie *t) {
    if (!t) return;
    free(t->node);
    free(t);
}

/* O2 build: inserts the prefixes in input order (a later duplicate overwrites). NULL on failure. */
orc_trie *orc_trie_new(size_t np, const uint64_t *phi, const uint64_t *plo, const uint8_t *plen,
                       const uint16_t *pnh) {
    orc_trie *t = (orc_trie *)calloc(1, sizeof(orc_trie));
    if (!t) return NULL;
    if (trie_new_node(t) < 0) { orc_trie_free(t); return NULL; }
    for (size_t j = 0; j < np; j++) {
        if (plen[j] > 128) { orc_trie_free(t); return NULL; }
        int32_t cur = 0;
        for (int d = 0; d < plen[j]; d++) {
            int b = bit_at(phi[j], plo[j], d);
            int32_t nx = t->node[cur].child[b];
            if (nx < 0) {
                nx = trie_new_node(t);
                if (nx < 0) { orc_trie_free(t); return NULL; }
                t->node[cur].child[b] = nx;
            }
            cur = nx;
        }
        t->node[cur].nh = pnh[j];
    }
    return t;
}

size_t orc_trie_nodes(const orc_trie *t) { return t ? t->used : 0; }

static uint16_t trie_one(const orc_trie *t, uint64_t xh, uint64_t xl) {
    int32_t best = -1, cur = 0;
    for (int d = 0;; d++) {
        if (t->node[cur].nh >= 0) best = t->node[cur].nh;
        if (d == 128) break;
        int32_t nx = t->node[cur].child[bit_at(xh, xl, d)];
        if (nx < 0) break;
        cur = nx;
    }
    return best >= 0 ? (uint16_t)best : 0;
}

typedef struct { const orc_trie *t; const uint64_t *xhi, *xlo; uint16_t *out; } trie_ctx;

static void trie_range(void *c_, size_t b, size_t e) {
    trie_ctx *c = (trie_ctx *)c_;
    for (size_t i = b; i < e; i++) c->out[i] = trie_one(c->t, c->xhi[i], c->xlo[i]);
}

/* O2 lookup of nk addresses with `threads` threads; returns the threads used */
int orc_trie_lookup(const orc_trie *t, size_t nk, const uint64_t *xhi, const uint64_t *xlo,
                    uint16_t *out, int threads) {
    trie_ctx c = {t, xhi, xlo, out};
    return parallel_for(nk, threads, trie_range, &c);
}

/* ----------------------------------------------------------------------- O3 interval invariants */

static int cmp_u128(const void *a, const void *b) {
    u128 x = *(const u128 *)a, y = *(const u128 *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* index of the largest s[i] <= v (s sorted, s[0] == 0) */
static size_t pred_index(const u128 *s, size_t m, u128 v) {
    size_t lo = 0, hi = m;          /* answer in [lo, hi) */
    while (hi - lo > 1) {
        size_t mid = lo + (hi - lo) / 2;
        if (s[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

static int contains(const u128 *s, size_t m, u128 v) {
    size_t i = pred_index(s, m, v);
    return s[i] == v;
}

static int fail(char *msg, size_t ml, const char *what, size_t i) {
    if (msg && ml) snprintf(msg, ml, "%s (at %zu)", what, i);
    return 1;
}

/*
 * O3: checks (start[], nh[]) of m intervals against the prefix table.
 * merged = 0: boundaries must be exactly {0} and the prefix boundaries below 2^128 (Section 3.1);
 * merged = 1: neighbouring intervals with equal next hops may have been merged (the same-next-hop
 *             compression that Section 3 allows); neighbours must then differ.
 * Returns 0 when every invariant holds, else a non-zero code and a message.
 */
int orc_check_intervals(size_t np, const uint64_t *phi, const uint64_t *plo, const uint8_t *plen,
                        const uint16_t *pnh, size_t m, const uint64_t *shi, const uint64_t *slo,
                        const uint16_t *snh, int merged, char *msg, size_t msglen) {
    if (m == 0) return fail(msg, msglen, "no intervals", 0);
    orc_trie *t = orc_trie_new(np, phi, plo, plen, pnh);
    if (!t) return fail(msg, msglen, "oracle trie build failed", 0);
    int rc = 0;
    u128 *s = (u128 *)malloc(sizeof(u128) * m);
    u128 *bd = (u128 *)malloc(sizeof(u128) * (2 * np + 1));
    u128 *canon = (u128 *)malloc(sizeof(u128) * (np + 1) * 2);
    if (!s || !bd || !canon) { rc = fail(msg, msglen, "oracle out of memory", 0); goto out; }
    for (size_t i = 0; i < m; i++) s[i] = mk(shi[i], slo[i]);
    /* 1. partition: starts at 0, strictly increasing */
    if (s[0] != 0) { rc = fail(msg, msglen, "first interval does not start at 0", 0); goto out; }
    for (size_t i = 1; i < m; i++)
        if (!(s[i - 1] < s[i])) { rc = fail(msg, msglen, "starts not strictly increasing", i); goto out; }
    /* canonical prefixes: (masked prefix, length) pairs, distinct */
    size_t nc = 0;
    for (size_t j = 0; j < np; j++) {
        uint64_t mh, ml;
        top_mask(plen[j], &mh, &ml);
        canon[2 * nc] = mk(phi[j] & mh, plo[j] & ml);
        canon[2 * nc + 1] = plen[j];
        nc++;
    }
    size_t nb = 0;
    bd[nb++] = 0;
    for (size_t j = 0; j < nc; j++) {
        u128 p = canon[2 * j];
        int L = (int)canon[2 * j + 1];
        bd[nb++] = p;
        if (L > 0) {
            u128 width = (u128)1 << (128 - L);       /* L >= 1 so the shift is at most 127 */
            u128 e = p + width;                      /* wraps to 0 exactly when the end is 2^128 */
            if (e != 0) bd[nb++] = e;
        }
    }
    qsort(bd, nb, sizeof(u128), cmp_u128);
    size_t nu = 0;
    for (size_t i = 0; i < nb; i++)
        if (nu == 0 || bd[i] != bd[nu - 1]) bd[nu++] = bd[i];
    /* distinct prefixes N: bucket the canonical pairs by length, count distinct values per bucket */
    {
        u128 *key = (u128 *)malloc(sizeof(u128) * (nc ? nc : 1));
        if (!key) { rc = fail(msg, msglen, "oracle out of memory", 0); goto out; }
        size_t distinct = 0;
        for (int L = 0; L <= 128; L++) {
            size_t k = 0;
            for (size_t j = 0; j < nc; j++)
                if ((int)canon[2 * j + 1] == L) key[k++] = canon[2 * j];
            qsort(key, k, sizeof(u128), cmp_u128);
            for (size_t i = 0; i < k; i++)
                if (i == 0 || key[i] != key[i - 1]) distinct++;
        }
        free(key);
        if (m > 2 * distinct + 1) { rc = fail(msg, msglen, "more than 2N+1 intervals", m); goto out; }
    }
    /* 2. elementarity */
    for (size_t i = 0; i < nu; i++) {
        if (!contains(s, m, bd[i])) {
            if (!merged) { rc = fail(msg, msglen, "prefix boundary missing from the starts", i); goto out; }
        }
    }
    if (!merged) {
        for (size_t i = 0; i < m; i++)
            if (!contains(bd, nu, s[i])) { rc = fail(msg, msglen, "start is not a prefix boundary", i); goto out; }
    } else {
        for (size_t i = 1; i < m; i++)
            if (snh[i] == snh[i - 1]) { rc = fail(msg, msglen, "merged neighbours share a next hop", i); goto out; }
    }
    /* 3. every interval's next hop is the LPM at its first and last address */
    for (size_t i = 0; i < m; i++) {
        u128 a = s[i];
        u128 z = (i + 1 < m) ? s[i + 1] - 1 : ~(u128)0;
        if (trie_one(t, (uint64_t)(a >> 64), (uint64_t)a) != snh[i]) { rc = fail(msg, msglen, "next hop differs from LPM at interval start", i); goto out; }
        if (trie_one(t, (uint64_t)(z >> 64), (uint64_t)z) != snh[i]) { rc = fail(msg, msglen, "next hop differs from LPM at interval end", i); goto out; }
    }
    /* ... and on both sides of every prefix boundary (covers boundaries inside merged intervals) */
    for (size_t i = 0; i < nu; i++) {
        u128 b = bd[i];
        size_t k = pred_index(s, m, b);
        if (trie_one(t, (uint64_t)(b >> 64), (uint64_t)b) != snh[k]) { rc = fail(msg, msglen, "next hop differs from LPM at a prefix boundary", i); goto out; }
        if (b > 0) {
            u128 c = b - 1;
            k = pred_index(s, m, c);
            if (trie_one(t, (uint64_t)(c >> 64), (uint64_t)c) != snh[k]) { rc = fail(msg, msglen, "next hop differs from LPM below a prefix boundary", i); goto out; }
        }
    }
out:
    free(s); free(bd); free(canon);
    orc_trie_free(t);
    return rc;
}

/* version tag, so the Python side can tell a stale build */
int orc_version(void) { return 1; }
