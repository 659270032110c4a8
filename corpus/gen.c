/*
 * Seeded synthetic corpus generator.
 *
 * This module produces test and benchmark inputs only.  It holds none of the
 * counting method: it draws vocabulary ids from a Zipf law, writes the drawn
 * words (with random capitalisation) separated by non-letter bytes, and keeps
 * a tally of the ids it drew.  Because every separator it writes is a
 * non-letter byte and capitalisation never changes a word's lowercase form,
 * that tally is the exact word count of the text it wrote.
 *
 * Random numbers: splitmix64 (seeding) and xoshiro256** (streams), both as
 * published by S. Vigna (prng.di.unimi.it).  Zipf draws use Walker's alias
 * method (Vose's construction) over weights rank^-s.
 *
 * Documents are generated in fixed segments, each from its own stream, so the
 * output does not depend on the number of host threads used.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t seed;
    uint32_t vocab_size;
    uint32_t len_min, len_max;
    double len_a, len_b, len_jitter; /* target length at rank r: a + b*ln(r) + U(-j, j) */
    double len_tail, len_tail_mean;  /* ranks past 1000: with probability len_tail, add an exponential extra length */
    double zipf_s;
    double cap_prob;    /* token capitalised: first letter or all caps, 50/50 */
    double punct_prob;  /* separator group carries 1-2 punctuation bytes */
    double digit_prob;  /* separator group carries a run of 1-4 digits */
    double glue_prob;   /* separator group is digits only (no space), e.g. abc123def */
    double high_prob;   /* separator group carries a 2-byte UTF-8 letter (bytes >= 0x80) */
    uint32_t newline_min, newline_max; /* newline every U[min, max] tokens; 0 = never */
    uint32_t nclasses;
    uint32_t boost_per_class;
    uint32_t boost_rank_lo, boost_rank_hi;
    double boost_lo, boost_hi;
    /* document sizes */
    uint32_t ndocs;
    uint32_t size_mode; /* 0: words ~ U[a,b]; 1: bytes lognormal(median a, sigma c) clipped [b0,b1];
                           2: bytes fixed = a; 3: bytes log-uniform [a, b] */
    double size_a, size_b, size_c, clip_lo, clip_hi;
    uint32_t threads;
} gen_params;

/* ---------------- PRNG ---------------- */
static inline uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
typedef struct { uint64_t s[4]; } xo256;
static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t xo_next(xo256 *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl64(s[3], 45);
    return result;
}
static void xo_seed(xo256 *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (0xD1B54A32D192ED03ULL * (stream + 1));
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
static inline double xo_unit(xo256 *r) { return (double)(xo_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static inline uint32_t xo_below(xo256 *r, uint32_t n) { /* Lemire multiply-shift */
    return (uint32_t)(((xo_next(r) >> 32) * (uint64_t)n) >> 32);
}

/* ---------------- alias table ---------------- */
typedef struct { uint32_t n; uint32_t *thr; uint32_t *alias; } alias_t;

static int alias_build(alias_t *a, const double *w, uint32_t n) {
    a->n = n;
    a->thr = (uint32_t *)malloc(sizeof(uint32_t) * n);
    a->alias = (uint32_t *)malloc(sizeof(uint32_t) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    uint32_t *small = (uint32_t *)malloc(sizeof(uint32_t) * n), *large = (uint32_t *)malloc(sizeof(uint32_t) * n);
    if (!a->thr || !a->alias || !p || !small || !large) return -1;
    double tot = 0; for (uint32_t i = 0; i < n; i++) tot += w[i];
    uint32_t ns = 0, nl = 0;
    for (uint32_t i = 0; i < n; i++) { p[i] = w[i] * n / tot; if (p[i] < 1.0) small[ns++] = i; else large[nl++] = i; }
    while (ns && nl) {
        uint32_t s = small[--ns], l = large[--nl];
        a->alias[s] = l;
        a->thr[s] = p[s] >= 1.0 ? 0xFFFFFFFFu : (uint32_t)(p[s] * 4294967296.0);
        p[l] = (p[l] + p[s]) - 1.0;
        if (p[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl) { uint32_t l = large[--nl]; a->thr[l] = 0xFFFFFFFFu; a->alias[l] = l; }
    while (ns) { uint32_t s = small[--ns]; a->thr[s] = 0xFFFFFFFFu; a->alias[s] = s; }
    free(p); free(small); free(large);
    return 0;
}
static inline uint32_t alias_draw(const alias_t *a, xo256 *r) {
    uint64_t x = xo_next(r);
    uint32_t i = (uint32_t)(((x >> 32) * (uint64_t)a->n) >> 32);
    return ((uint32_t)x < a->thr[i] || a->thr[i] == 0xFFFFFFFFu) ? i : a->alias[i];
}

/* ---------------- generator state ---------------- */
typedef struct {
    uint32_t doc, seg;
    uint64_t target;    /* words (mode 0) or bytes */
    uint64_t out_off;   /* filled in later */
    uint64_t out_len;
} seg_t;

typedef struct {
    gen_params p;
    char *vbytes; uint64_t *voff; /* vocabulary, lowercase */
    alias_t *alias;              /* one per class (or one) */
    uint32_t nalias;
    uint32_t *doc_class;
    uint64_t *doc_target;        /* words or bytes */
    seg_t *segs; uint32_t nsegs;
    uint64_t bound;
    uint64_t *tally;             /* [nalias][vocab] -> filled per class, summed later */
    uint64_t total_bytes;
    uint64_t total_tokens;
    char err[160];
} gen_t;

#define SEG_BYTES (4u << 20)
#define SEG_WORDS (700000u)
#define MAX_SEP 16

static uint64_t word_hash(const char *s, uint32_t n) {
    uint64_t h = 1469598103934665603ULL;
    for (uint32_t i = 0; i < n; i++) { h ^= (uint8_t)s[i]; h *= 1099511628211ULL; }
    return h ? h : 1;
}

static int build_vocab(gen_t *g, xo256 *r) {
    const gen_params *p = &g->p;
    uint32_t V = p->vocab_size;
    uint64_t cap_slots = 1; while (cap_slots < 2ull * V + 16) cap_slots <<= 1;
    uint64_t *hs = (uint64_t *)calloc(cap_slots, sizeof(uint64_t));
    uint32_t *hi = (uint32_t *)calloc(cap_slots, sizeof(uint32_t));
    uint64_t per_len_cnt[64] = {0};
    g->voff = (uint64_t *)malloc(sizeof(uint64_t) * (V + 1));
    uint64_t vcap = (uint64_t)V * (p->len_max + 1) + 16;
    g->vbytes = (char *)malloc(vcap);
    if (!hs || !hi || !g->voff || !g->vbytes) return -1;
    uint64_t pos = 0;
    char buf[256];
    for (uint32_t r1 = 0; r1 < V; r1++) {
        double t = p->len_a + p->len_b * log((double)(r1 + 1)) + (xo_unit(r) * 2.0 - 1.0) * p->len_jitter;
        if (p->len_tail > 0 && r1 >= 1000 && xo_unit(r) < p->len_tail) t += -log(1.0 - xo_unit(r)) * p->len_tail_mean;
        int L = (int)floor(t + 0.5);
        if (L < (int)p->len_min) L = (int)p->len_min;
        if (L > (int)p->len_max) L = (int)p->len_max;
        /* keep each length at most half full so rejection sampling stays fast */
        for (;;) {
            double capL = pow(26.0, (double)L);
            if ((double)per_len_cnt[L] < capL * 0.5) break;
            if (L >= (int)p->len_max) { strcpy(g->err, "vocabulary does not fit the length range"); return -1; }
            L++;
        }
        for (;;) {
            for (int i = 0; i < L; i++) buf[i] = (char)('a' + xo_below(r, 26));
            uint64_t h = word_hash(buf, (uint32_t)L);
            uint64_t s = h & (cap_slots - 1);
            int dup = 0;
            while (hs[s]) {
                if (hs[s] == h) {
                    uint32_t j = hi[s];
                    uint64_t lj = g->voff[j + 1] - g->voff[j];
                    if (lj == (uint64_t)L && memcmp(g->vbytes + g->voff[j], buf, (size_t)L) == 0) { dup = 1; break; }
                }
                s = (s + 1) & (cap_slots - 1);
            }
            if (dup) continue;
            hs[s] = h; hi[s] = r1;
            break;
        }
        g->voff[r1] = pos;
        memcpy(g->vbytes + pos, buf, (size_t)L);
        pos += (uint64_t)L;
        g->voff[r1 + 1] = pos;
        per_len_cnt[L]++;
    }
    free(hs); free(hi);
    return 0;
}

static int build_alias(gen_t *g, xo256 *r) {
    const gen_params *p = &g->p;
    uint32_t V = p->vocab_size;
    double *w = (double *)malloc(sizeof(double) * V);
    if (!w) return -1;
    g->nalias = (p->nclasses > 1 && p->boost_per_class) ? p->nclasses : 1;
    g->alias = (alias_t *)calloc(g->nalias, sizeof(alias_t));
    /* boosted words: disjoint across classes, drawn from ranks [lo, hi) */
    uint32_t nb = p->boost_per_class * g->nalias;
    uint32_t *pick = NULL; double *fac = NULL;
    if (g->nalias > 1) {
        uint32_t lo = p->boost_rank_lo, hi = p->boost_rank_hi < V ? p->boost_rank_hi : V;
        if (hi <= lo || hi - lo < nb) { strcpy(g->err, "boost rank range too small"); return -1; }
        uint32_t span = hi - lo;
        uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * span);
        for (uint32_t i = 0; i < span; i++) perm[i] = lo + i;
        for (uint32_t i = 0; i < nb; i++) { /* partial Fisher-Yates */
            uint32_t j = i + xo_below(r, span - i);
            uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
        pick = perm;
        fac = (double *)malloc(sizeof(double) * nb);
        for (uint32_t i = 0; i < nb; i++) fac[i] = p->boost_lo + (p->boost_hi - p->boost_lo) * xo_unit(r);
    }
    for (uint32_t c = 0; c < g->nalias; c++) {
        for (uint32_t i = 0; i < V; i++) w[i] = pow((double)(i + 1), -p->zipf_s);
        if (pick) for (uint32_t k = 0; k < p->boost_per_class; k++) {
            uint32_t id = pick[c * p->boost_per_class + k];
            w[id] *= fac[c * p->boost_per_class + k];
        }
        if (alias_build(&g->alias[c], w, V)) return -1;
    }
    free(w); free(pick); free(fac);
    return 0;
}

static double normal(xo256 *r) { /* Box-Muller */
    double u1 = xo_unit(r), u2 = xo_unit(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static int plan_docs(gen_t *g, xo256 *r) {
    const gen_params *p = &g->p;
    uint32_t n = p->ndocs;
    g->doc_class = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    g->doc_target = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint64_t nseg = 0;
    for (uint32_t d = 0; d < n; d++) {
        g->doc_class[d] = p->nclasses > 1 ? d % p->nclasses : 0;
        uint64_t t;
        switch (p->size_mode) {
        case 0: t = (uint64_t)p->size_a + xo_below(r, (uint32_t)(p->size_b - p->size_a + 1)); break;
        case 1: {
            double v = exp(log(p->size_a) + p->size_c * normal(r));
            if (v < p->clip_lo) v = p->clip_lo;
            if (v > p->clip_hi) v = p->clip_hi;
            t = (uint64_t)v; break; }
        case 2: t = (uint64_t)p->size_a; break;
        case 3: t = (uint64_t)exp(log(p->size_a) + (log(p->size_b) - log(p->size_a)) * xo_unit(r)); break;
        default: strcpy(g->err, "bad size_mode"); return -1;
        }
        g->doc_target[d] = t;
        uint64_t unit = p->size_mode == 0 ? SEG_WORDS : SEG_BYTES;
        nseg += t / unit + 1;
    }
    g->segs = (seg_t *)calloc(nseg ? nseg : 1, sizeof(seg_t));
    uint32_t k = 0;
    uint64_t bound = 0;
    uint32_t maxword = p->len_max + MAX_SEP;
    for (uint32_t d = 0; d < n; d++) {
        uint64_t t = g->doc_target[d];
        uint64_t unit = p->size_mode == 0 ? SEG_WORDS : SEG_BYTES;
        uint32_t s = 0;
        do {
            uint64_t part = t > unit ? unit : t;
            g->segs[k].doc = d; g->segs[k].seg = s++; g->segs[k].target = part;
            bound += p->size_mode == 0 ? part * maxword : part;
            k++;
            t -= part;
        } while (t > 0);
    }
    g->nsegs = k;
    g->bound = bound;
    return 0;
}

/* one separator group after a token; returns bytes written */
static uint32_t write_sep(const gen_params *p, xo256 *r, char *o, int newline) {
    static const char P[] = ".,;:!?\"'()-";
    uint32_t n = 0;
    if (p->glue_prob > 0 && xo_unit(r) < p->glue_prob) {
        uint32_t nd = 1 + xo_below(r, 4);
        for (uint32_t i = 0; i < nd; i++) o[n++] = (char)('0' + xo_below(r, 10));
        return n;
    }
    if (p->punct_prob > 0 && xo_unit(r) < p->punct_prob) {
        uint32_t np = 1 + xo_below(r, 2);
        for (uint32_t i = 0; i < np; i++) o[n++] = P[xo_below(r, (uint32_t)(sizeof(P) - 1))];
    }
    if (p->high_prob > 0 && xo_unit(r) < p->high_prob) { o[n++] = (char)0xC3; o[n++] = (char)(0xA0 + xo_below(r, 0x1F)); }
    if (p->digit_prob > 0 && xo_unit(r) < p->digit_prob) {
        o[n++] = ' ';
        uint32_t nd = 1 + xo_below(r, 4);
        for (uint32_t i = 0; i < nd; i++) o[n++] = (char)('0' + xo_below(r, 10));
    }
    o[n++] = newline ? '\n' : ' ';
    return n;
}

typedef struct { gen_t *g; uint8_t *out; uint32_t first, step; uint64_t *tally; uint64_t tokens; } worker_t;

/* Generates segment k into out (at its planned offset in pass 2, or a scratch
 * area in pass 1 when out_base is NULL), returning bytes written. */
static uint64_t gen_segment(gen_t *g, uint32_t k, uint8_t *dst, uint64_t *tally, uint64_t *ntok) {
    const gen_params *p = &g->p;
    seg_t *sg = &g->segs[k];
    xo256 r; xo_seed(&r, p->seed, ((uint64_t)sg->doc << 20) ^ sg->seg ^ 0xC0FFEEull);
    const alias_t *a = &g->alias[g->nalias > 1 ? g->doc_class[sg->doc] : 0];
    uint64_t V = p->vocab_size;
    uint64_t *tl = tally + (g->nalias > 1 ? (uint64_t)g->doc_class[sg->doc] * V : 0);
    uint32_t nl_left = p->newline_max ? p->newline_min + xo_below(&r, p->newline_max - p->newline_min + 1) : 0;
    uint64_t pos = 0;
    char sep[MAX_SEP + 8];
    int bytes_mode = p->size_mode != 0;
    uint64_t t = 0;
    for (;;) {
        if (!bytes_mode && t >= sg->target) break;
        uint32_t id = alias_draw(a, &r);
        const char *w = g->vbytes + g->voff[id];
        uint32_t L = (uint32_t)(g->voff[id + 1] - g->voff[id]);
        int cap = 0;
        if (p->cap_prob > 0 && xo_unit(&r) < p->cap_prob) cap = 1 + (int)xo_below(&r, 2);
        int nl = 0;
        if (p->newline_max) { if (--nl_left == 0) { nl = 1; nl_left = p->newline_min + xo_below(&r, p->newline_max - p->newline_min + 1); } }
        uint32_t ns = write_sep(p, &r, sep, nl);
        if (bytes_mode && pos + L + ns > sg->target) break;
        for (uint32_t i = 0; i < L; i++) {
            char c = w[i];
            if (cap == 2 || (cap == 1 && i == 0)) c = (char)(c - 32);
            dst[pos + i] = (uint8_t)c;
        }
        pos += L;
        memcpy(dst + pos, sep, ns);
        pos += ns;
        tl[id]++;
        t++;
    }
    if (bytes_mode) { while (pos < sg->target) dst[pos++] = ' '; }
    *ntok += t;
    return pos;
}

static void *worker_pass(void *arg) {
    worker_t *w = (worker_t *)arg;
    gen_t *g = w->g;
    for (uint32_t k = w->first; k < g->nsegs; k += w->step) {
        seg_t *sg = &g->segs[k];
        uint64_t n = gen_segment(g, k, w->out + sg->out_off, w->tally, &w->tokens);
        sg->out_len = n;
    }
    return NULL;
}

/* ---------------- public API ---------------- */
void *gen_create(const gen_params *p, char *err, int errlen) {
    gen_t *g = (gen_t *)calloc(1, sizeof(gen_t));
    if (!g) return NULL;
    g->p = *p;
    if (p->vocab_size == 0 || p->len_min < 1 || p->len_max > 60 || p->len_min > p->len_max) {
        strncpy(err, "bad params", (size_t)errlen); free(g); return NULL;
    }
    xo256 r; xo_seed(&r, p->seed, 0);
    if (build_vocab(g, &r) || build_alias(g, &r) || plan_docs(g, &r)) {
        strncpy(err, g->err[0] ? g->err : "allocation failed", (size_t)errlen);
        return NULL;
    }
    return g;
}

uint64_t gen_bound_bytes(void *h) { return ((gen_t *)h)->bound; }
uint32_t gen_nsegs(void *h) { return ((gen_t *)h)->nsegs; }

/* Fills out (capacity >= gen_bound_bytes), doc_offsets[ndocs+1], doc_class[ndocs].
 * Word-count segments are generated into their bound-sized slots and then packed. */
int64_t gen_fill(void *h, uint8_t *out, uint64_t cap, uint64_t *doc_offsets, uint32_t *doc_class) {
    gen_t *g = (gen_t *)h;
    const gen_params *p = &g->p;
    if (cap < g->bound) return -1;
    uint64_t off = 0;
    uint32_t maxword = p->len_max + MAX_SEP;
    for (uint32_t k = 0; k < g->nsegs; k++) {
        g->segs[k].out_off = off;
        off += p->size_mode == 0 ? g->segs[k].target * maxword : g->segs[k].target;
    }
    uint32_t T = p->threads ? p->threads : 1;
    if (T > 256) T = 256;
    uint64_t V = p->vocab_size;
    uint64_t ntal = (uint64_t)g->nalias * V;
    worker_t ws[256];
    pthread_t th[256];
    for (uint32_t i = 0; i < T; i++) {
        ws[i].g = g; ws[i].out = out; ws[i].first = i; ws[i].step = T; ws[i].tokens = 0;
        ws[i].tally = (uint64_t *)calloc(ntal, sizeof(uint64_t));
        if (!ws[i].tally) return -2;
    }
    for (uint32_t i = 1; i < T; i++) pthread_create(&th[i], NULL, worker_pass, &ws[i]);
    worker_pass(&ws[0]);
    for (uint32_t i = 1; i < T; i++) pthread_join(th[i], NULL);
    free(g->tally);
    g->tally = (uint64_t *)calloc(ntal, sizeof(uint64_t));
    g->total_tokens = 0;
    for (uint32_t i = 0; i < T; i++) {
        for (uint64_t j = 0; j < ntal; j++) g->tally[j] += ws[i].tally[j];
        g->total_tokens += ws[i].tokens;
        free(ws[i].tally);
    }
    /* pack segments (memmove keeps order; offsets only shrink) */
    uint64_t w = 0;
    uint32_t d = 0;
    if (p->ndocs) doc_offsets[0] = 0;
    for (uint32_t k = 0; k < g->nsegs; k++) {
        seg_t *sg = &g->segs[k];
        while (d < sg->doc) { doc_offsets[++d] = w; }
        if (sg->out_off != w) memmove(out + w, out + sg->out_off, sg->out_len);
        w += sg->out_len;
    }
    while (d < p->ndocs) doc_offsets[++d] = w;
    for (uint32_t i = 0; i < p->ndocs; i++) doc_class[i] = g->doc_class[i];
    g->total_bytes = w;
    return (int64_t)w;
}

uint64_t gen_total_tokens(void *h) { return ((gen_t *)h)->total_tokens; }
uint32_t gen_ntally(void *h) { return ((gen_t *)h)->nalias; }

/* tally[c * vocab + id] = tokens of vocabulary word id written in class c (c = 0 when unclassed) */
void gen_tally(void *h, uint64_t *out) {
    gen_t *g = (gen_t *)h;
    memcpy(out, g->tally, sizeof(uint64_t) * g->nalias * g->p.vocab_size);
}
uint64_t gen_vocab_bytes(void *h) { gen_t *g = (gen_t *)h; return g->voff[g->p.vocab_size]; }
void gen_vocab(void *h, uint8_t *bytes, uint64_t *offs) {
    gen_t *g = (gen_t *)h;
    memcpy(bytes, g->vbytes, g->voff[g->p.vocab_size]);
    memcpy(offs, g->voff, sizeof(uint64_t) * (g->p.vocab_size + 1));
}
/* Expected word length under class-0 Zipf weights (for calibrating recipes). */
double gen_expected_len(void *h) {
    gen_t *g = (gen_t *)h;
    double tot = 0, acc = 0;
    for (uint32_t i = 0; i < g->p.vocab_size; i++) {
        double w = pow((double)(i + 1), -g->p.zipf_s);
        tot += w; acc += w * (double)(g->voff[i + 1] - g->voff[i]);
    }
    return acc / tot;
}
void gen_destroy(void *h) {
    gen_t *g = (gen_t *)h;
    if (!g) return;
    for (uint32_t c = 0; c < g->nalias; c++) { free(g->alias[c].thr); free(g->alias[c].alias); }
    free(g->alias); free(g->vbytes); free(g->voff); free(g->doc_class); free(g->doc_target);
    free(g->segs); free(g->tally); free(g);
}
