/*
 * ETALE oracle: a plain, sequential CPU restatement of the index and its
 * update protocols, written from the paper.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package's smoke check and
 * the bench's CPU-baseline leg load this library.  The product path (the CUDA
 * library declared in include/etale.h) never calls it, and the two share no
 * source, header, table or helper.
 *
 * What each part restates:
 *   Definition 1 (Sec. 3.2)   state: reference word r(u) = <delta, d, s>,
 *                             slab map A(s) of (id, rho) entries, vectors x(u)
 *   Algorithm 1 (Sec. 3.3)    Publish: snapshot, AllocSlab, write, fence, CAS,
 *                             RetireSlab; the deletion flag is carried forward
 *   Sec. 3.3, pool paragraph  free stack popped and retired stack pushed inside
 *                             a launch; the host moves retired -> free between
 *                             launches (here: recycle() after every phase)
 *   Algorithm 2 (Sec. 3.4.1)  Insert: BeamSearch, RobustPrune, own publish,
 *                             reverse offers, refine pass
 *   Algorithm 3 (Sec. 3.4.2)  Delete: tombstone CAS, repair of live neighbours
 *   Algorithm 4 (Sec. 3.4.3)  Reclaim: compaction, then reclaim of tombstones
 *   Definition 2 (Sec. 4.1)   every phase below is one launch; a phase reads
 *                             the state left by the previous phase
 *
 * Where the paper is silent the code takes one reading, marked READING.  The
 * same readings are listed with reasons in the repository's design notes.
 *
 * Deterministic-round semantics (the oracle has no other mode): all inserts of
 * one sub-batch search the pre-insert graph; reverse offers are grouped by
 * target and applied in ascending source id; each target publishes once.
 *
 * Every mode, the refine pass in both readings included, is pinned by the
 * hand-derived cases and the other tests named in the design notes.
 *
 * Floating point: the canonical distance below fixes the order of every fp32
 * operation, so a GPU implementation of the same order reproduces each
 * distance bit for bit.  Build with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NIL 0xFFFFFFFFu

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ECAPACITY = 3 };
enum { ORC_L2 = 0, ORC_IP = 1 };

typedef struct {
    uint32_t dim, metric, degree;
    uint64_t capacity;
    uint32_t build_beam;
    float alpha;
    uint32_t max_hops;   /* 0: 4 * beam                                       */
    uint32_t max_cand;   /* 0: 2 * build_beam                                 */
    uint32_t refine;     /* 0: off, 1: two-hop refine, 2: two-hop, peers only */
    uint64_t max_batch;  /* 0: max(1, capacity / 100)                         */
    uint64_t pool_slabs; /* 0: 2 * capacity + 2 * (degree + 1) * max_batch    */
    uint32_t n_entry;    /* 0: 1024; size of the entry set E                  */
} orc_config;

typedef struct {
    uint64_t live, tombstones, reclaimed, next_id;
    uint64_t pool, free_slabs, retired_slabs, used_slabs;
    uint32_t n_entries;
    uint64_t n_dist, n_expand, n_publish, n_prune, n_search;
} orc_stats;

typedef struct { uint32_t id; float rho; } entry; /* one slab entry (a_i, rho_i) */

typedef struct {
    orc_config c;
    float alpha2;
    float *x;          /* C x m vectors                                     */
    uint64_t *ref;     /* C reference words                                 */
    entry *slab;       /* P x R entries                                     */
    uint32_t *fst;     /* free stack                                        */
    uint64_t nfree;
    uint32_t *rst;     /* retired stack                                     */
    uint64_t nret;
    uint64_t next_id, live;
    uint32_t *ent;     /* the entry set E, ascending ids                    */
    uint32_t n_ent;
    uint32_t *stamp;   /* visited marks, one per id, by search generation   */
    uint32_t gen;
    uint64_t n_dist, n_expand, n_publish, n_prune, n_search;
} orc;

static void recompute_entries(orc *o);

/* ---- reference word, Definition 1 --------------------------------------
 * READING: the paper fixes only that <delta, d, s> share one 64-bit word.
 * Layout: bit 63 = delta, bits 48..55 = d, bits 0..31 = s (NIL = none).     */
static uint64_t pack(uint32_t del, uint32_t d, uint32_t s) {
    return ((uint64_t)(del & 1u) << 63) | ((uint64_t)(d & 0xFFu) << 48) | (uint64_t)s;
}
static uint32_t ref_del(uint64_t r) { return (uint32_t)(r >> 63); }
static uint32_t ref_deg(uint64_t r) { return (uint32_t)(r >> 48) & 0xFFu; }
static uint32_t ref_slab(uint64_t r) { return (uint32_t)r; }

/* ---- canonical fp32 distance --------------------------------------------
 * READING: the paper writes ||x_v - x_w|| with no precision or order.  The
 * oracle stores the SQUARED L2 distance and compares it against alpha^2
 * times a squared distance, which orders exactly as the unsquared rule.
 * Inner product uses rho = 1 - <x, y>.
 * Order: element i belongs to partial j = (i mod 128) / 4; each partial is a
 * sequential fused multiply-add chain over its elements in ascending i,
 * starting from +0; the 32 partials are combined pairwise as q[j] = p[j] +
 * p[j + h] for h = 16, 8, 4, 2, 1.                                          */
float orc_dist(const float *a, const float *b, uint32_t m, uint32_t metric) {
    float p[32];
    for (uint32_t j = 0; j < 32; j++) {
        float acc = 0.0f;
        for (uint32_t base = 0; base < m; base += 128)
            for (uint32_t e = 0; e < 4; e++) {
                uint32_t i = base + 4 * j + e;
                if (i >= m) break;
                if (metric == ORC_L2) {
                    float t = a[i] - b[i];
                    acc = fmaf(t, t, acc);
                } else {
                    acc = fmaf(a[i], b[i], acc);
                }
            }
        p[j] = acc;
    }
    for (uint32_t h = 16; h >= 1; h >>= 1)
        for (uint32_t j = 0; j < h; j++) p[j] = p[j] + p[j + h];
    return metric == ORC_L2 ? p[0] : 1.0f - p[0];
}

/* fp64 distance for ground truth and error statements: plain sequential sum. */
double orc_dist64(const float *a, const float *b, uint32_t m, uint32_t metric) {
    double s = 0.0;
    for (uint32_t i = 0; i < m; i++) {
        if (metric == ORC_L2) {
            double t = (double)a[i] - (double)b[i];
            s += t * t;
        } else {
            s += (double)a[i] * (double)b[i];
        }
    }
    return metric == ORC_L2 ? s : 1.0 - s;
}

/* Total order on (rho, id): rho by its fp32 bit pattern mapped to an
 * unsigned order (negative values reversed), ties broken by the smaller id.
 * READING: the paper calls a slab an "ordered sequence" without the order. */
static uint64_t key_of(float rho, uint32_t id) {
    uint32_t u;
    memcpy(&u, &rho, 4);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((uint64_t)u << 32) | id;
}
static int cmp_entry(const void *pa, const void *pb) {
    const entry *a = pa, *b = pb;
    uint64_t ka = key_of(a->rho, a->id), kb = key_of(b->rho, b->id);
    return ka < kb ? -1 : ka > kb;
}

static const float *vec(const orc *o, uint32_t id) { return o->x + (uint64_t)id * o->c.dim; }
static float dist_ids(orc *o, uint32_t a, uint32_t b) {
    o->n_dist++;
    return orc_dist(vec(o, a), vec(o, b), o->c.dim, o->c.metric);
}
static int is_deleted(const orc *o, uint32_t id) { return (int)ref_del(o->ref[id]); }

/* N(u): the first d_u entries of A(s_u) (Definition 1).                     */
static uint32_t get_list(const orc *o, uint32_t u, entry *out) {
    uint64_t r = o->ref[u];
    uint32_t s = ref_slab(r), d = ref_deg(r);
    if (s == ORC_NIL) return 0;
    memcpy(out, o->slab + (uint64_t)s * o->c.degree, d * sizeof(entry));
    return d;
}

/* ---- Algorithm 1: Publish(u, N) -----------------------------------------
 * Sequentially every CAS succeeds on its first attempt.                     */
static int publish(orc *o, uint32_t u, const entry *N, uint32_t n) {
    uint64_t snap = o->ref[u];                         /* atomic snapshot  */
    if (o->nfree == 0) return ORC_ENOMEM;
    uint32_t s2 = o->fst[--o->nfree];                  /* AllocSlab        */
    memcpy(o->slab + (uint64_t)s2 * o->c.degree, N, n * sizeof(entry));
    /* Fence: a sequential program has nothing to order.                  */
    o->ref[u] = pack(ref_del(snap), n, s2);            /* CAS: wins        */
    if (ref_slab(snap) != ORC_NIL) o->rst[o->nret++] = ref_slab(snap); /* RetireSlab */
    o->n_publish++;
    return ORC_OK;
}

/* Host-side recycle at a launch boundary: retired stack -> free stack.      */
static void recycle(orc *o) {
    for (uint64_t i = 0; i < o->nret; i++) o->fst[o->nfree++] = o->rst[i];
    o->nret = 0;
}

/* ---- RobustPrune_alpha(C, R) for owner p (Sec. 3.4.1, after DiskANN) ----
 * c[i].rho must hold d(p, c[i].id).  The candidate list is consumed.
 * READING: p itself, tombstoned ids and repeated ids are dropped first
 * (dropping tombstones is the lazy cleanup of Sec. 3.4.2); the rest is sorted
 * by (rho, id); the head is kept and every later candidate p' with
 * alpha^2 * d(head, p') <= d(p, p') is discarded, until R are kept.         */
static uint32_t robust_prune(orc *o, uint32_t p, entry *c, uint32_t n, entry *out) {
    uint32_t k = 0;
    o->n_prune++;
    for (uint32_t i = 0; i < n; i++)
        if (c[i].id != p && !is_deleted(o, c[i].id)) c[k++] = c[i];
    qsort(c, k, sizeof(entry), cmp_entry);
    uint32_t u = 0;
    for (uint32_t i = 0; i < k; i++)
        if (u == 0 || c[i].id != c[u - 1].id) c[u++] = c[i];
    k = u;
    unsigned char *alive = malloc(k ? k : 1);
    memset(alive, 1, k ? k : 1);
    uint32_t nout = 0;
    for (uint32_t i = 0; i < k && nout < o->c.degree; i++) {
        if (!alive[i]) continue;
        out[nout++] = c[i];
        if (nout == o->c.degree) break;
        for (uint32_t j = i + 1; j < k; j++) {
            if (!alive[j]) continue;
            float dd = dist_ids(o, c[i].id, c[j].id);
            if (o->alpha2 * dd <= c[j].rho) alive[j] = 0;
        }
    }
    free(alive);
    return nout;
}

/* Stand-alone RobustPrune on explicit vectors, for pinning tests.
 * owner: m floats; cand: n x m; ids: n; out_ids: <= R.  No deletion flags. */
uint32_t orc_robust_prune_vectors(const float *owner, const float *cand, const uint32_t *ids,
                                  uint32_t n, uint32_t m, uint32_t metric, uint32_t R,
                                  float alpha, uint32_t *out_ids, float *out_rho) {
    float alpha2 = alpha * alpha;
    entry *c = malloc((n ? n : 1) * sizeof(entry));
    uint32_t *row = malloc((n ? n : 1) * sizeof(uint32_t));
    for (uint32_t i = 0; i < n; i++) {
        c[i].id = ids[i];
        c[i].rho = orc_dist(owner, cand + (uint64_t)i * m, m, metric);
    }
    qsort(c, n, sizeof(entry), cmp_entry);
    uint32_t k = 0;
    for (uint32_t i = 0; i < n; i++)
        if (k == 0 || c[i].id != c[k - 1].id) c[k++] = c[i];
    for (uint32_t i = 0; i < k; i++)
        for (uint32_t t = 0; t < n; t++)
            if (ids[t] == c[i].id) { row[i] = t; break; }
    unsigned char *alive = malloc(k ? k : 1);
    memset(alive, 1, k ? k : 1);
    uint32_t nout = 0;
    for (uint32_t i = 0; i < k && nout < R; i++) {
        if (!alive[i]) continue;
        out_ids[nout] = c[i].id;
        out_rho[nout++] = c[i].rho;
        if (nout == R) break;
        for (uint32_t j = i + 1; j < k; j++) {
            if (!alive[j]) continue;
            float dd = orc_dist(cand + (uint64_t)row[i] * m, cand + (uint64_t)row[j] * m, m, metric);
            if (alpha2 * dd <= c[j].rho) alive[j] = 0;
        }
    }
    free(alive); free(row); free(c);
    return nout;
}

/* ---- BeamSearch(q, L) (Sec. 3.4.1, Sec. 2.1) ----------------------------
 * READING (entry set, visited set, termination, tombstones):
 *  - the beam starts from the fixed entry set E: every member is evaluated
 *    and the L smallest (rho, id) are kept;
 *  - repeatedly expand the unexpanded beam entry with the smallest (rho, id):
 *    read its reference word (delta is sampled here), then for every id in
 *    its first d entries that was never evaluated, evaluate d(q, id) and keep
 *    the beam at the L smallest (rho, id);
 *  - stop when every beam entry is expanded or after max_hops expansions;
 *  - tombstones stay in the beam and are expanded (they relay, Definition 1);
 *    nodes whose reference names no slab are never expanded.
 * Output: the final beam in (rho, id) order with each entry's sampled delta,
 * and the expanded entries in expansion order.                              */
typedef struct { float rho; uint32_t id; uint32_t del; int expanded; } bentry;

/* Keep the beam at the L smallest (rho, id): insert in order, drop the tail. */
static uint32_t beam_offer(bentry *beam, uint32_t n, uint32_t L, float rho, uint32_t w) {
    uint64_t kw = key_of(rho, w);
    if (L == 0 || (n == L && kw >= key_of(beam[n - 1].rho, beam[n - 1].id))) return n;
    uint32_t pos = n < L ? n : L - 1;                /* slot freed at the tail */
    while (pos > 0 && key_of(beam[pos - 1].rho, beam[pos - 1].id) > kw) {
        beam[pos] = beam[pos - 1];
        pos--;
    }
    beam[pos].rho = rho; beam[pos].id = w; beam[pos].del = 0; beam[pos].expanded = 0;
    return n < L ? n + 1 : n;
}

static uint32_t beam_search(orc *o, const float *q, uint32_t L, uint32_t max_hops,
                            bentry *beam, bentry *exp_out, uint32_t *n_exp) {
    uint32_t n = 0, hops = 0;
    if (++o->gen == 0) { memset(o->stamp, 0, o->c.capacity * sizeof(uint32_t)); o->gen = 1; }
    o->n_search++;
    if (n_exp) *n_exp = 0;
    for (uint32_t t = 0; t < o->n_ent; t++) {         /* seed from E      */
        uint32_t e = o->ent[t];
        o->stamp[e] = o->gen;
        o->n_dist++;
        float rho = orc_dist(q, vec(o, e), o->c.dim, o->c.metric);
        n = beam_offer(beam, n, L, rho, e);
    }
    entry *nb = malloc(o->c.degree * sizeof(entry));
    for (;;) {
        uint32_t i = 0;
        while (i < n && beam[i].expanded) i++;
        if (i == n || hops == max_hops) break;
        beam[i].expanded = 1;
        hops++;
        o->n_expand++;
        uint64_t r = o->ref[beam[i].id];
        beam[i].del = ref_del(r);
        if (exp_out) exp_out[(*n_exp)++] = beam[i];
        uint32_t d = get_list(o, beam[i].id, nb);
        for (uint32_t j = 0; j < d; j++) {
            uint32_t w = nb[j].id;
            if (o->stamp[w] == o->gen) continue;
            o->stamp[w] = o->gen;
            o->n_dist++;
            float rho = orc_dist(q, vec(o, w), o->c.dim, o->c.metric);
            n = beam_offer(beam, n, L, rho, w);
        }
    }
    free(nb);
    /* entries never expanded sample delta now */
    for (uint32_t i = 0; i < n; i++)
        if (!beam[i].expanded) beam[i].del = ref_del(o->ref[beam[i].id]);
    return n;
}

/* ---- construction ----------------------------------------------------- */
orc *orc_create(const orc_config *cfg) {
    if (!cfg || cfg->dim == 0 || cfg->degree == 0 || cfg->degree > 255 || cfg->capacity == 0 ||
        cfg->capacity >= ORC_NIL || (cfg->metric != ORC_L2 && cfg->metric != ORC_IP))
        return NULL;
    orc *o = calloc(1, sizeof(orc));
    o->c = *cfg;
    if (o->c.build_beam == 0) o->c.build_beam = 64;
    if (o->c.alpha == 0.0f) o->c.alpha = 1.2f;
    if (o->c.max_cand == 0) o->c.max_cand = 2 * o->c.build_beam;
    if (o->c.max_batch == 0) o->c.max_batch = o->c.capacity / 100 ? o->c.capacity / 100 : 1;
    if (o->c.n_entry == 0) o->c.n_entry = 1024;
    if (o->c.pool_slabs == 0)
        o->c.pool_slabs = 2 * o->c.capacity + 2 * (uint64_t)(o->c.degree + 1) * o->c.max_batch;
    o->alpha2 = o->c.alpha * o->c.alpha;
    uint64_t C = o->c.capacity, P = o->c.pool_slabs;
    o->x = calloc(C * o->c.dim, sizeof(float));
    o->ref = malloc(C * sizeof(uint64_t));
    o->slab = calloc(P * o->c.degree, sizeof(entry));
    o->fst = malloc(P * sizeof(uint32_t));
    o->rst = malloc(P * sizeof(uint32_t));
    o->stamp = calloc(C, sizeof(uint32_t));
    o->ent = malloc(o->c.n_entry * sizeof(uint32_t));
    if (!o->x || !o->ref || !o->slab || !o->fst || !o->rst || !o->stamp || !o->ent) {
        free(o->x); free(o->ref); free(o->slab); free(o->fst); free(o->rst); free(o->stamp);
        free(o->ent);
        free(o);
        return NULL;
    }
    for (uint64_t i = 0; i < C; i++) o->ref[i] = pack(0, 0, ORC_NIL);
    for (uint64_t i = 0; i < P; i++) o->fst[i] = (uint32_t)(P - 1 - i);
    o->nfree = P;
    o->n_ent = 0;
    return o;
}

void orc_destroy(orc *o) {
    if (!o) return;
    free(o->x); free(o->ref); free(o->slab); free(o->fst); free(o->rst); free(o->stamp);
    free(o->ent);
    free(o);
}

static uint32_t hops_for(const orc *o, uint32_t L) { return o->c.max_hops ? o->c.max_hops : 4 * L; }

/* Offer (v, rho) to target w's evolving list (Algorithm 2, reverse edge).
 * READING: an id already in the list is a no-op.                          */
static uint32_t apply_offer(orc *o, uint32_t w, entry *list, uint32_t n, uint32_t v, float rho,
                            entry *scratch) {
    for (uint32_t i = 0; i < n; i++)
        if (list[i].id == v) return n;
    if (n < o->c.degree) {                       /* d_w < R: add the edge   */
        uint64_t kv = key_of(rho, v);
        uint32_t pos = n;
        while (pos > 0 && key_of(list[pos - 1].rho, list[pos - 1].id) > kv) {
            list[pos] = list[pos - 1];
            pos--;
        }
        list[pos].id = v; list[pos].rho = rho;
        return n + 1;
    }
    memcpy(scratch, list, n * sizeof(entry));    /* at capacity: re-prune   */
    scratch[n].id = v; scratch[n].rho = rho;
    return robust_prune(o, w, scratch, n + 1, list);
}

static int same_list(const entry *a, uint32_t na, const entry *b, uint32_t nb) {
    if (na != nb) return 0;
    for (uint32_t i = 0; i < na; i++)
        if (a[i].id != b[i].id || memcmp(&a[i].rho, &b[i].rho, 4) != 0) return 0;
    return 1;
}

typedef struct { uint32_t w, v; float rho; uint64_t seq; } offer;
static int cmp_offer(const void *pa, const void *pb) {
    const offer *a = pa, *b = pb;
    if (a->w != b->w) return a->w < b->w ? -1 : 1;
    return a->seq < b->seq ? -1 : a->seq > b->seq;
}

/* Reverse-offer phase: group offers by target, apply each group in
 * ascending source order against the target's current list, publish each
 * target once if its list changed.  Offers must arrive with seq ascending in
 * source id.                                                                */
static int offer_phase(orc *o, offer *of, uint64_t nof) {
    uint32_t R = o->c.degree;
    qsort(of, nof, sizeof(offer), cmp_offer);
    entry *list = malloc(R * sizeof(entry)), *orig = malloc(R * sizeof(entry));
    entry *scr = malloc((R + 1) * sizeof(entry));
    int st = ORC_OK;
    for (uint64_t i = 0; i < nof && st == ORC_OK;) {
        uint64_t j = i;
        uint32_t w = of[i].w;
        uint32_t n = get_list(o, w, list);
        uint32_t n0 = n;
        memcpy(orig, list, n * sizeof(entry));
        for (; j < nof && of[j].w == w; j++) n = apply_offer(o, w, list, n, of[j].v, of[j].rho, scr);
        if (!same_list(list, n, orig, n0)) st = publish(o, w, list, n);
        i = j;
    }
    free(list); free(orig); free(scr);
    recycle(o);
    return st;
}

/* One insert sub-batch: ids [first, first + b), vectors already stored.     */
static int insert_subbatch(orc *o, uint32_t first, uint32_t b) {
    uint32_t R = o->c.degree, L = o->c.build_beam, H = hops_for(o, L);
    uint32_t maxc = o->c.max_cand;
    int st = ORC_OK;
    /* Phase 1: every member searches the pre-insert graph (batch peers are
     * absent from one another's searches, Sec. 3.4.1).                     */
    entry **cand = malloc(b * sizeof(entry *));
    uint32_t *ncand = malloc(b * sizeof(uint32_t));
    bentry *beam = malloc((L + 1) * sizeof(bentry)), *ex = malloc((H + 1) * sizeof(bentry));
    for (uint32_t t = 0; t < b; t++) {
        uint32_t v = first + t, nex = 0;
        beam_search(o, vec(o, v), L, H, beam, ex, &nex);
        /* C = expanded set minus tombstones minus v, nearest max_cand first */
        entry *c = malloc((nex ? nex : 1) * sizeof(entry));
        uint32_t k = 0;
        for (uint32_t i = 0; i < nex; i++)
            if (!ex[i].del && ex[i].id != v) { c[k].id = ex[i].id; c[k].rho = ex[i].rho; k++; }
        qsort(c, k, sizeof(entry), cmp_entry);
        if (k > maxc) k = maxc;
        cand[t] = c; ncand[t] = k;
    }
    free(beam); free(ex);
    /* Phase 2: forward edges F_v = RobustPrune(C_v, R); Publish(v, F_v).   */
    entry **F = malloc(b * sizeof(entry *));
    uint32_t *nF = malloc(b * sizeof(uint32_t));
    for (uint32_t t = 0; t < b; t++) {
        F[t] = malloc(R * sizeof(entry));
        nF[t] = robust_prune(o, first + t, cand[t], ncand[t], F[t]);
        free(cand[t]);
        if (st == ORC_OK) st = publish(o, first + t, F[t], nF[t]);
    }
    free(cand); free(ncand);
    recycle(o);
    /* Phase 3: reverse offers (w <- v) for w in F_v.                        */
    offer *of = malloc(((uint64_t)b * R + 1) * sizeof(offer));
    uint64_t nof = 0;
    for (uint32_t t = 0; t < b; t++)
        for (uint32_t j = 0; j < nF[t]; j++) {
            of[nof].w = F[t][j].id; of[nof].v = first + t; of[nof].rho = F[t][j].rho;
            of[nof].seq = nof; nof++;
        }
    if (st == ORC_OK) st = offer_phase(o, of, nof);
    /* Phase 4 (READING of the refine pass): each member v re-selects its
     * edges from N(v) and the lists of its neighbours (two hops, live ids
     * only, v excluded, nearest max_cand kept) on the graph left by phase 3,
     * publishes if the list changed, and offers the edges it gained.  Mode 2
     * admits from the two-hop lists only members of the same sub-batch, the
     * nodes that phase 1 could not see.                                     */
    if (st == ORC_OK && o->c.refine) {
        entry **F2 = malloc(b * sizeof(entry *));
        uint32_t *nF2 = malloc(b * sizeof(uint32_t));
        entry *nv = malloc(R * sizeof(entry)), *nw = malloc(R * sizeof(entry));
        entry *c = malloc(((uint64_t)R + (uint64_t)R * R) * sizeof(entry));
        for (uint32_t t = 0; t < b; t++) {
            uint32_t v = first + t;
            if (++o->gen == 0) { memset(o->stamp, 0, o->c.capacity * sizeof(uint32_t)); o->gen = 1; }
            uint32_t k = 0, dv = get_list(o, v, nv);
            o->stamp[v] = o->gen;
            for (uint32_t i = 0; i < dv; i++) {
                o->stamp[nv[i].id] = o->gen;
                if (!is_deleted(o, nv[i].id)) c[k++] = nv[i];
            }
            for (uint32_t i = 0; i < dv; i++) {
                uint32_t dw = get_list(o, nv[i].id, nw);
                for (uint32_t j = 0; j < dw; j++) {
                    uint32_t y = nw[j].id;
                    if (o->stamp[y] == o->gen) continue;
                    if (o->c.refine == 2 && (y < first || y >= first + b)) continue;
                    o->stamp[y] = o->gen;
                    if (is_deleted(o, y)) continue;
                    c[k].id = y; c[k].rho = dist_ids(o, v, y); k++;
                }
            }
            qsort(c, k, sizeof(entry), cmp_entry);
            if (k > maxc) k = maxc;
            F2[t] = malloc(R * sizeof(entry));
            nF2[t] = robust_prune(o, v, c, k, F2[t]);
        }
        /* publish every changed list (all computed from the same snapshot) */
        nof = 0;
        offer *of2 = malloc(((uint64_t)b * R + 1) * sizeof(offer));
        for (uint32_t t = 0; t < b && st == ORC_OK; t++) {
            uint32_t v = first + t, dv = get_list(o, v, nv);
            if (!same_list(F2[t], nF2[t], nv, dv)) st = publish(o, v, F2[t], nF2[t]);
            for (uint32_t j = 0; j < nF2[t]; j++) {
                int had = 0;
                for (uint32_t i = 0; i < dv; i++) if (nv[i].id == F2[t][j].id) { had = 1; break; }
                if (!had) {
                    of2[nof].w = F2[t][j].id; of2[nof].v = v; of2[nof].rho = F2[t][j].rho;
                    of2[nof].seq = nof; nof++;
                }
            }
        }
        recycle(o);
        if (st == ORC_OK) st = offer_phase(o, of2, nof);
        for (uint32_t t = 0; t < b; t++) free(F2[t]);
        free(F2); free(nF2); free(nv); free(nw); free(c); free(of2);
    }
    for (uint32_t t = 0; t < b; t++) free(F[t]);
    free(F); free(nF); free(of);
    return st;
}

/* Insert n vectors.  Ids are fresh and ascending from next_id.
 * READING (initial build and batch size): the batch is split into
 * sub-batches of size min(remaining, max(1, live), max_batch), i.e. prefix
 * doubling from an empty index, capped; each sub-batch is one deterministic
 * round of Algorithm 2.                                                     */
int orc_insert(orc *o, const float *vecs, uint64_t n, uint32_t *out_ids) {
    if (o->next_id + n > o->c.capacity) return ORC_ECAPACITY;
    uint64_t done = 0;
    while (done < n) {
        uint64_t b = n - done, cap = o->live ? o->live : 1;
        if (b > cap) b = cap;
        if (b > o->c.max_batch) b = o->c.max_batch;
        uint32_t first = (uint32_t)o->next_id;
        memcpy(o->x + (uint64_t)first * o->c.dim, vecs + done * o->c.dim,
               b * o->c.dim * sizeof(float));
        o->next_id += b;
        int st = insert_subbatch(o, first, (uint32_t)b);
        if (st) return st;
        o->live += b;
        recompute_entries(o);
        for (uint64_t t = 0; t < b; t++) if (out_ids) out_ids[done + t] = first + (uint32_t)t;
        done += b;
    }
    return ORC_OK;
}

static int cmp_u32(const void *pa, const void *pb) {
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    return a < b ? -1 : a > b;
}

typedef struct { uint32_t a, u; uint32_t nk; uint64_t seq; entry *K; } repair;
static int cmp_repair(const void *pa, const void *pb) {
    const repair *x = pa, *y = pb;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    return x->seq < y->seq ? -1 : x->seq > y->seq;
}

/* ---- Algorithm 3: Delete with connectivity repair ------------------------
 * READING: ids never inserted, already tombstoned or repeated are no-ops.
 * All ids are tombstoned first; the repair then reads that snapshot.  For a
 * live a in B = N(u): K = RobustPrune_a(B \ {a}); N = RobustPrune_a((A(s_a)
 * \ {u}) u K).  When a neighbours several deleted u, the repairs are applied
 * in ascending u and a publishes once.  Returns the number tombstoned.     */
int orc_delete(orc *o, const uint32_t *ids, uint64_t n, uint64_t *n_tombstoned) {
    uint32_t R = o->c.degree;
    uint32_t *d = malloc((n ? n : 1) * sizeof(uint32_t));
    memcpy(d, ids, n * sizeof(uint32_t));
    qsort(d, n, sizeof(uint32_t), cmp_u32);
    uint64_t k = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint32_t u = d[i];
        if (i && u == d[i - 1]) continue;
        if (u >= o->next_id) continue;
        uint64_t r = o->ref[u];
        if (ref_del(r) || ref_slab(r) == ORC_NIL) continue;
        d[k++] = u;
    }
    /* Phase 1: tombstone CAS <0,d,s> -> <1,d,s>.                           */
    for (uint64_t i = 0; i < k; i++) {
        uint64_t r = o->ref[d[i]];
        o->ref[d[i]] = pack(1, ref_deg(r), ref_slab(r));
    }
    o->live -= k;
    if (n_tombstoned) *n_tombstoned = k;
    /* Phase 2: per (u, a) replacement sets K on the post-tombstone snapshot */
    repair *rp = malloc((k * R + 1) * sizeof(repair));
    uint64_t nrp = 0;
    entry *B = malloc(R * sizeof(entry)), *c = malloc(2 * (R + 1) * sizeof(entry));
    for (uint64_t i = 0; i < k; i++) {
        uint32_t u = d[i], nb = get_list(o, u, B);
        for (uint32_t j = 0; j < nb; j++) {
            uint32_t a = B[j].id;
            if (is_deleted(o, a)) continue;
            uint32_t nc = 0;
            for (uint32_t t = 0; t < nb; t++) {
                if (B[t].id == a) continue;
                c[nc].id = B[t].id; c[nc].rho = dist_ids(o, a, B[t].id); nc++;
            }
            rp[nrp].a = a; rp[nrp].u = u; rp[nrp].seq = nrp;
            rp[nrp].K = malloc(R * sizeof(entry));
            rp[nrp].nk = robust_prune(o, a, c, nc, rp[nrp].K);
            nrp++;
        }
    }
    /* Phase 3: fold per a in ascending u, publish once if changed.         */
    qsort(rp, nrp, sizeof(repair), cmp_repair);
    entry *list = malloc(R * sizeof(entry)), *orig = malloc(R * sizeof(entry));
    int st = ORC_OK;
    for (uint64_t i = 0; i < nrp;) {
        uint32_t a = rp[i].a, n0 = get_list(o, a, orig), nl = n0;
        memcpy(list, orig, n0 * sizeof(entry));
        uint64_t j = i;
        for (; j < nrp && rp[j].a == a; j++) {
            uint32_t nc = 0;
            for (uint32_t t = 0; t < nl; t++) if (list[t].id != rp[j].u) c[nc++] = list[t];
            for (uint32_t t = 0; t < rp[j].nk; t++) c[nc++] = rp[j].K[t];
            nl = robust_prune(o, a, c, nc, list);
        }
        if (st == ORC_OK && !same_list(list, nl, orig, n0)) st = publish(o, a, list, nl);
        i = j;
    }
    for (uint64_t i = 0; i < nrp; i++) free(rp[i].K);
    free(rp); free(B); free(c); free(list); free(orig); free(d);
    recycle(o);
    return st;
}

/* READING (entry set): the paper searches "from a fixed set of entry points"
 * without saying which.  E is a stride sample of the live set: with L live
 * ids in ascending order and S = min(n_entry, L), member j is the live id of
 * rank floor(j * L / S), j = 0..S-1.  E is recomputed after every insert
 * sub-batch and at the start of Reclaim, so it is live whenever phase 2
 * frees tombstone slabs.  A spread of entries keeps every region of the
 * data reachable even when the degree bound leaves no edges between
 * well-separated clusters.                                                 */
static void recompute_entries(orc *o) {
    uint64_t L = o->live, S = o->c.n_entry < L ? o->c.n_entry : L, rank = 0, j = 0;
    o->n_ent = 0;
    for (uint64_t id = 0; id < o->next_id && j < S; id++) {
        uint64_t r = o->ref[id];
        if (ref_del(r) || ref_slab(r) == ORC_NIL) continue;
        if (rank == (j * L) / S) { o->ent[o->n_ent++] = (uint32_t)id; j++; }
        rank++;
    }
}

/* ---- Algorithm 4: Reclaim -------------------------------------------------
 * READING: the entry set is recomputed first (it must be live before phase 2
 * frees tombstone slabs).                                                   */
int orc_reclaim(orc *o) {
    uint32_t R = o->c.degree;
    recompute_entries(o);
    entry *list = malloc(R * sizeof(entry)), *keep = malloc(R * sizeof(entry));
    int st = ORC_OK;
    /* Phase 1, compaction: every live node with a tombstoned neighbour is
     * republished with those entries dropped (order and rho kept).         */
    for (uint64_t u = 0; u < o->next_id && st == ORC_OK; u++) {
        uint64_t r = o->ref[u];
        if (ref_del(r) || ref_slab(r) == ORC_NIL) continue;
        uint32_t n = get_list(o, (uint32_t)u, list), nk = 0;
        for (uint32_t i = 0; i < n; i++) if (!is_deleted(o, list[i].id)) keep[nk++] = list[i];
        if (nk != n) st = publish(o, (uint32_t)u, keep, nk);
    }
    recycle(o);
    /* Phase 2, reclaim: CAS <1,d,s> -> <1,0,NIL>, retire s.                */
    for (uint64_t u = 0; u < o->next_id; u++) {
        uint64_t r = o->ref[u];
        if (!ref_del(r) || ref_slab(r) == ORC_NIL) continue;
        o->ref[u] = pack(1, 0, ORC_NIL);
        o->rst[o->nret++] = ref_slab(r);
    }
    recycle(o);
    free(list); free(keep);
    return st;
}

/* ---- query search (Sec. 3.4.2, Proposition 1) ---------------------------
 * The result is the first k beam entries whose sampled delta is 0, padded
 * with id NIL and rho +inf.  READING: the beam is max(beam, k).             */
int orc_search(orc *o, const float *q, uint64_t nq, uint32_t k, uint32_t beam_w,
               uint32_t *out_ids, float *out_rho) {
    uint32_t L = beam_w > k ? beam_w : k;
    bentry *beam = malloc((L + 1) * sizeof(bentry));
    for (uint64_t t = 0; t < nq; t++) {
        uint32_t n = beam_search(o, q + t * o->c.dim, L, hops_for(o, L), beam, NULL, NULL);
        uint32_t c = 0;
        for (uint32_t i = 0; i < n && c < k; i++)
            if (!beam[i].del) { out_ids[t * k + c] = beam[i].id; out_rho[t * k + c] = beam[i].rho; c++; }
        for (; c < k; c++) { out_ids[t * k + c] = ORC_NIL; out_rho[t * k + c] = INFINITY; }
    }
    free(beam);
    return ORC_OK;
}

/* Exact k nearest live nodes by fp64 distance, ties by id (Sec. 5.2,
 * Recall@10 against the current live set).                                 */
int orc_exact_knn(const orc *o, const float *q, uint64_t nq, uint32_t k, uint32_t *out_ids,
                  double *out_d) {
    for (uint64_t t = 0; t < nq; t++) {
        uint32_t *bi = out_ids + t * k;
        double *bd = out_d + t * k;
        uint32_t c = 0;
        for (uint64_t id = 0; id < o->next_id; id++) {
            uint64_t r = o->ref[id];
            if (ref_del(r) || ref_slab(r) == ORC_NIL) continue;
            double dd = orc_dist64(q + t * o->c.dim, o->x + id * o->c.dim, o->c.dim, o->c.metric);
            if (c == k && !(dd < bd[k - 1])) continue;
            uint32_t pos = c < k ? c : k - 1;
            while (pos > 0 && bd[pos - 1] > dd) { bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; pos--; }
            bd[pos] = dd; bi[pos] = (uint32_t)id;
            if (c < k) c++;
        }
        for (; c < k; c++) { bi[c] = ORC_NIL; bd[c] = INFINITY; }
    }
    return ORC_OK;
}

/* ---- introspection ------------------------------------------------------ */
int orc_node(const orc *o, uint32_t u, uint32_t *del, uint32_t *has_slab, uint32_t *ids, float *rho) {
    if (u >= o->c.capacity) return -1;
    uint64_t r = o->ref[u];
    *del = ref_del(r);
    *has_slab = ref_slab(r) != ORC_NIL;
    entry *l = malloc(o->c.degree * sizeof(entry));
    uint32_t n = get_list(o, u, l);
    for (uint32_t i = 0; i < n; i++) { ids[i] = l[i].id; rho[i] = l[i].rho; }
    free(l);
    return (int)n;
}

/* Whole logical graph: del/has_slab/deg per id, lists padded to R.          */
void orc_dump(const orc *o, uint8_t *del, uint8_t *has_slab, uint8_t *deg, uint32_t *ids, float *rho) {
    uint32_t R = o->c.degree;
    for (uint64_t u = 0; u < o->next_id; u++) {
        uint64_t r = o->ref[u];
        del[u] = (uint8_t)ref_del(r);
        has_slab[u] = ref_slab(r) != ORC_NIL;
        deg[u] = 0;
        for (uint32_t i = 0; i < R; i++) { ids[u * R + i] = ORC_NIL; rho[u * R + i] = 0.0f; }
        if (ref_slab(r) == ORC_NIL) continue;
        uint32_t d = ref_deg(r);
        deg[u] = (uint8_t)d;
        const entry *e = o->slab + (uint64_t)ref_slab(r) * R;
        for (uint32_t i = 0; i < d; i++) { ids[u * R + i] = e[i].id; rho[u * R + i] = e[i].rho; }
    }
}

/* ---- snapshot reader ------------------------------------------------------
 * Rebuilds the state of Definition 1 from a snapshot file (the format written
 * by the library's etale_save, read here by this file's own code).  cfg gives
 * the maintenance knobs; dim, metric and degree come from the file and
 * cfg->capacity (0: the saved capacity) must cover the saved next_id.  The
 * k-th id with a slab gets slab k; the free stack holds the remaining slabs.
 * The entry set is the saved one.  Used for timing on large graphs and for
 * round-trip tests; returns NULL on a malformed file.                       */
static int rd(FILE *f, void *p, size_t sz, size_t n) { return fread(p, sz, n, f) == n; }

orc *orc_load(const char *path, const orc_config *cfg) {
    FILE *f = fopen(path, "rb");
    if (!f) return NULL;
    char magic[8];
    uint32_t h[4], hb[2];
    uint64_t cap_n[2], cw[64];
    orc *o = NULL;
    uint8_t *fl = NULL, *dg = NULL;
    if (!rd(f, magic, 1, 8) || memcmp(magic, "ETALESN1", 8) != 0 || !rd(f, h, 4, 4) || h[0] != 1 ||
        !rd(f, cap_n, 8, 2) || !rd(f, hb, 4, 2) || hb[1] > 64 || !rd(f, cw, 8, hb[1]))
        goto bad;
    {
        orc_config c = *cfg;
        c.dim = h[1]; c.metric = h[2]; c.degree = h[3];
        if (c.capacity == 0) c.capacity = cap_n[0];
        uint64_t n = cap_n[1];
        uint32_t R = c.degree, ne = hb[0];
        if (n > c.capacity) goto bad;
        o = orc_create(&c);
        if (!o || ne > o->c.n_entry) goto bad;
        if (n && !rd(f, o->x, sizeof(float), n * c.dim)) goto bad;
        fl = malloc(n ? n : 1); dg = malloc(n ? n : 1);
        if (n && (!rd(f, fl, 1, n) || !rd(f, dg, 1, n))) goto bad;
        uint64_t k = 0, live = 0;
        for (uint64_t u = 0; u < n; u++) {
            uint32_t del = fl[u] & 1u, hs = (fl[u] >> 1) & 1u;
            if (dg[u] > R || (!hs && dg[u])) goto bad;
            if (!hs) { o->ref[u] = pack(del, 0, ORC_NIL); continue; }
            if (k >= o->c.pool_slabs) goto bad;
            entry *e = o->slab + k * R;
            for (uint32_t j = 0; j < dg[u]; j++) {
                if (!rd(f, &e[j].id, 4, 1) || !rd(f, &e[j].rho, 4, 1) || e[j].id >= n) goto bad;
            }
            o->ref[u] = pack(del, dg[u], (uint32_t)k);
            k++;
            live += !del;
        }
        /* free stack: every slab not taken above */
        o->nfree = 0;
        for (uint64_t i = o->c.pool_slabs; i-- > k;) o->fst[o->nfree++] = (uint32_t)i;
        if (ne && !rd(f, o->ent, 4, ne)) goto bad;
        for (uint32_t i = 0; i < ne; i++) if (o->ent[i] >= n) goto bad;
        o->n_ent = ne;
        o->next_id = n;
        o->live = live;
    }
    free(fl); free(dg);
    fclose(f);
    return o;
bad:
    free(fl); free(dg);
    orc_destroy(o);
    fclose(f);
    return NULL;
}

void orc_get_stats(const orc *o, orc_stats *s) {
    memset(s, 0, sizeof(*s));
    for (uint64_t u = 0; u < o->next_id; u++) {
        uint64_t r = o->ref[u];
        if (ref_slab(r) == ORC_NIL) { if (ref_del(r)) s->reclaimed++; continue; }
        if (ref_del(r)) s->tombstones++; else s->live++;
    }
    s->next_id = o->next_id;
    s->pool = o->c.pool_slabs;
    s->free_slabs = o->nfree;
    s->retired_slabs = o->nret;
    s->used_slabs = o->c.pool_slabs - o->nfree - o->nret;
    s->n_entries = o->n_ent;
    s->n_dist = o->n_dist; s->n_expand = o->n_expand; s->n_publish = o->n_publish;
    s->n_prune = o->n_prune; s->n_search = o->n_search;
}

void orc_effective_config(const orc *o, orc_config *c) { *c = o->c; }

uint32_t orc_entries(const orc *o, uint32_t *out) {
    memcpy(out, o->ent, o->n_ent * sizeof(uint32_t));
    return o->n_ent;
}
