/*
 * CPU oracle for the biomass-logistics candidate search of M. G. Plessen,
 * "GPU-accelerated Logistics Optimisation for Biomass Production with Multiple
 * Simultaneous Harvesters Tours, Fields and Plants" (arXiv 1909.10286).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file. The product path (the CUDA
 * library) shares no code, header or table with it and must never call it.
 *
 * It is a plain, slow, FP64 restatement of the method:
 *   - plans are materialised as explicit lists (tour -> BPs, BP -> fields);
 *   - a move is applied by erasing and inserting list elements;
 *   - every quantity of the model is recomputed from scratch per plan;
 *   - discrete decisions that must be exact (the demand check of Eq. 2 and the
 *     ceiling of Eq. 4) are taken in exact integer arithmetic.
 * Each function names the passage of the paper it follows. Where the paper is
 * silent or ambiguous the reading taken is stated next to the code.
 *
 * Node numbering: node 0 = HQ, nodes 1..B = BPs, nodes B+1..B+F = fields.
 * BP b (0-based) is node 1+b, field f (0-based) is node 1+B+f.
 *
 * Decision margins: for the parity protocol every FP decision (arg-max/min
 * picks, acceptance and termination tests, the gate) records its relative gap
 * |a-b|/scale; the minimum over one candidate is its margin. Exact equality is
 * a structural tie (both sides resolve it with the same tie rule) and does not
 * lower the margin. or_score_plan_trace returns every counted gap with its
 * decision site, so tests can check each one against a hand derivation.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 Philox S-box with the     */
/* Weyl key schedule. Written from the published definition.                 */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform integer in [0, m): floor(r * m / 2^32), no rejection */
static uint32_t draw_below(uint32_t r, uint32_t m)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)m) >> 32);
}

/* exact 24-bit uniform in [0,1): (r >> 8) * 2^-24 */
static double unit24(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* Instance (Sec. 2.1, Table 1)                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t F, B, T, H, S;
    const float *xy;       /* (1+B+F) x 2 km */
    const float *dist;     /* optional (1+B+F)^2 km; NULL = straight lines (Sec. 3.1) */
    const float *area;     /* h_f, ha */
    const float *supply;   /* s_f, t (Eq. 3) */
    const float *demand;   /* d_b^min, t (Eq. 2) */
    const float *hu_rate;  /* ha/h per HU */
    float hu_speed;        /* km/h */
    const float *su_cap;   /* t per SU */
    const float *su_fill;  /* ha harvested while one SU fills */
    const float *su_speed; /* km/h per SU */
} or_instance_in;

typedef struct {
    double eps;            /* Eq. 5 */
    double p_swap;         /* probability of a swap move (0 = the paper's moves only) */
    uint64_t seed;
    uint32_t inst_idx;
    int32_t fix_field_bp;  /* Sec. 2.6: a removed field goes back into its own BP */
    int32_t fix_resources; /* Case 2: keep the initial HU/SU dealing, no local minimisation */
    int32_t gate;          /* 0 off, 1 discard Tmax > Tmax*, 2 discard Tmax >= Tmax* */
    int32_t k_moves;       /* Step 8 repeated: moves chained per candidate (0 or 1: one move) */
} or_params;

typedef struct {
    int F, B, T, H, S, N;
    double *D;             /* N x N */
    double *area, *supply, *demand, *hu_rate, hu_speed, *su_cap, *su_fill, *su_speed;
    int *hu_sorted;        /* HU ids by (rate ascending, id) */
    int *su_sorted;        /* SU ids by (fill area ascending, id) */
} or_ctx;

static const double *g_sort_key;
static int sort_by_key_then_id(const void *a, const void *b)
{
    int ia = *(const int *)a, ib = *(const int *)b;
    double ka = g_sort_key[ia], kb = g_sort_key[ib];
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return (ia > ib) - (ia < ib);
}

static void sorted_ids(const double *key, int n, int *out)
{
    for (int i = 0; i < n; ++i) out[i] = i;
    g_sort_key = key;
    qsort(out, (size_t)n, sizeof(int), sort_by_key_then_id);
    g_sort_key = NULL;
}

/* number of significant binary digits needed to hold every value of v[] on a
   common grid: used to check that FP64 sums of these FP32 inputs are exact */
static int exact_sum_bits(const double *v, int n)
{
    int emin = 100000, emax = -100000;
    for (int i = 0; i < n; ++i) {
        if (v[i] == 0.0) continue;
        int e; frexp(v[i], &e);
        if (e < emin) emin = e;
        if (e > emax) emax = e;
    }
    if (emin > emax) return 0;
    int lg = 0; while ((1 << lg) < n + 1) ++lg;
    return (emax - emin) + 24 + lg;
}

void or_free(or_ctx *c)
{
    if (!c) return;
    free(c->D); free(c->area); free(c->supply); free(c->demand); free(c->hu_rate);
    free(c->su_cap); free(c->su_fill); free(c->su_speed); free(c->hu_sorted); free(c->su_sorted);
    free(c);
}

or_ctx *or_new(const or_instance_in *in, char *err, int errlen)
{
    if (in->F < 1 || in->B < 1 || in->T < 1 || in->H < 1 || in->S < 1) {
        snprintf(err, (size_t)errlen, "sizes must be positive");
        return NULL;
    }
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->F = in->F; c->B = in->B; c->T = in->T; c->H = in->H; c->S = in->S;
    c->N = 1 + in->B + in->F;
    int N = c->N;
    c->D = (double *)malloc(sizeof(double) * (size_t)N * (size_t)N);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double d;
            if (in->dist) d = (double)in->dist[(size_t)i * N + j];
            else {
                /* straight-line edge cost (Sec. 3.1) */
                double dx = (double)in->xy[2 * i] - (double)in->xy[2 * j];
                double dy = (double)in->xy[2 * i + 1] - (double)in->xy[2 * j + 1];
                d = sqrt(dx * dx + dy * dy);
            }
            c->D[(size_t)i * N + j] = d;
        }
#define COPYD(dst, src, n) do { dst = (double *)malloc(sizeof(double) * (size_t)(n)); \
        for (int _i = 0; _i < (n); ++_i) dst[_i] = (double)(src)[_i]; } while (0)
    COPYD(c->area, in->area, c->F);
    COPYD(c->supply, in->supply, c->F);
    COPYD(c->demand, in->demand, c->B);
    COPYD(c->hu_rate, in->hu_rate, c->H);
    COPYD(c->su_cap, in->su_cap, c->S);
    COPYD(c->su_fill, in->su_fill, c->S);
    COPYD(c->su_speed, in->su_speed, c->S);
#undef COPYD
    c->hu_speed = (double)in->hu_speed;
    for (int f = 0; f < c->F; ++f)
        if (!(c->supply[f] > 0.0) || !(c->area[f] > 0.0)) { snprintf(err, (size_t)errlen, "field %d: area and supply must be > 0", f); or_free(c); return NULL; }
    for (int b = 0; b < c->B; ++b)
        if (!(c->demand[b] > 0.0)) { snprintf(err, (size_t)errlen, "BP %d: demand must be > 0", b); or_free(c); return NULL; }
    for (int h = 0; h < c->H; ++h)
        if (!(c->hu_rate[h] > 0.0)) { snprintf(err, (size_t)errlen, "HU rates must be > 0"); or_free(c); return NULL; }
    for (int s = 0; s < c->S; ++s)
        if (!(c->su_cap[s] > 0.0) || !(c->su_fill[s] > 0.0) || !(c->su_speed[s] > 0.0)) { snprintf(err, (size_t)errlen, "SU tables must be > 0"); or_free(c); return NULL; }
    if (c->H < c->T || c->S < c->T) { snprintf(err, (size_t)errlen, "need at least one HU and one SU per tour"); or_free(c); return NULL; }
    if (c->T > 64) { snprintf(err, (size_t)errlen, "at most 64 tours"); or_free(c); return NULL; }
    if (!(c->hu_speed > 0.0)) { snprintf(err, (size_t)errlen, "HU speed must be > 0"); or_free(c); return NULL; }
    /* the FP64 sums below (supplies, rates, capacities, fill areas) must be exact */
    if (exact_sum_bits(c->supply, c->F) > 52 || exact_sum_bits(c->hu_rate, c->H) > 52 ||
        exact_sum_bits(c->su_cap, c->S) > 52 || exact_sum_bits(c->su_fill, c->S) > 52) {
        snprintf(err, (size_t)errlen, "value range too wide for exact FP64 sums");
        or_free(c); return NULL;
    }
    c->hu_sorted = (int *)malloc(sizeof(int) * (size_t)c->H);
    c->su_sorted = (int *)malloc(sizeof(int) * (size_t)c->S);
    sorted_ids(c->hu_rate, c->H, c->hu_sorted);
    sorted_ids(c->su_fill, c->S, c->su_sorted);
    return c;
}

/* ------------------------------------------------------------------------ */
/* Plan x (Sec. 2.4): explicit lists                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int T, B, F;
    int *tlen;   /* T */
    int *tbp;    /* T x B: BP ids of tour g in visiting order */
    int *blen;   /* B */
    int *bfld;   /* B x F: field ids of BP b in harvest order */
} oplan;

static void plan_alloc(oplan *p, int T, int B, int F)
{
    p->T = T; p->B = B; p->F = F;
    p->tlen = (int *)calloc((size_t)T, sizeof(int));
    p->tbp = (int *)calloc((size_t)T * (size_t)B, sizeof(int));
    p->blen = (int *)calloc((size_t)B, sizeof(int));
    p->bfld = (int *)calloc((size_t)B * (size_t)F, sizeof(int));
}

static void plan_release(oplan *p)
{
    free(p->tlen); free(p->tbp); free(p->blen); free(p->bfld);
    memset(p, 0, sizeof(*p));
}

static void plan_copy(oplan *dst, const oplan *src)
{
    memcpy(dst->tlen, src->tlen, sizeof(int) * (size_t)src->T);
    memcpy(dst->tbp, src->tbp, sizeof(int) * (size_t)src->T * (size_t)src->B);
    memcpy(dst->blen, src->blen, sizeof(int) * (size_t)src->B);
    memcpy(dst->bfld, src->bfld, sizeof(int) * (size_t)src->B * (size_t)src->F);
}

/* encoding <-> lists. Encoding: bp_order[B] (BP ids, tours concatenated in
   tour order), tour_cnt[T], field_order[F] (grouped by BP id, each group in
   harvest order), bp_cnt[B]. */
static int plan_from_enc(oplan *p, const int16_t *bp_order, const int16_t *tour_cnt,
                         const int16_t *field_order, const int16_t *bp_cnt)
{
    int k = 0;
    for (int g = 0; g < p->T; ++g) {
        p->tlen[g] = tour_cnt[g];
        for (int j = 0; j < tour_cnt[g]; ++j) {
            if (k >= p->B) return -1;
            p->tbp[g * p->B + j] = bp_order[k++];
        }
    }
    if (k != p->B) return -1;
    k = 0;
    for (int b = 0; b < p->B; ++b) {
        p->blen[b] = bp_cnt[b];
        for (int j = 0; j < bp_cnt[b]; ++j) {
            if (k >= p->F) return -1;
            p->bfld[b * p->F + j] = field_order[k++];
        }
    }
    if (k != p->F) return -1;
    return 0;
}

static void plan_to_enc(const oplan *p, int16_t *bp_order, int16_t *tour_cnt,
                        int16_t *field_order, int16_t *bp_cnt)
{
    int k = 0;
    for (int g = 0; g < p->T; ++g) {
        tour_cnt[g] = (int16_t)p->tlen[g];
        for (int j = 0; j < p->tlen[g]; ++j) bp_order[k++] = (int16_t)p->tbp[g * p->B + j];
    }
    k = 0;
    for (int b = 0; b < p->B; ++b) {
        bp_cnt[b] = (int16_t)p->blen[b];
        for (int j = 0; j < p->blen[b]; ++j) field_order[k++] = (int16_t)p->bfld[b * p->F + j];
    }
}

/* every field and every BP exactly once (Sec. 2.4 decision variables) */
int or_validate_enc(int T, int B, int F, const int16_t *bp_order, const int16_t *tour_cnt,
                    const int16_t *field_order, const int16_t *bp_cnt)
{
    int sum = 0;
    for (int g = 0; g < T; ++g) { if (tour_cnt[g] < 0) return -1; sum += tour_cnt[g]; }
    if (sum != B) return -2;
    sum = 0;
    for (int b = 0; b < B; ++b) { if (bp_cnt[b] < 0) return -3; sum += bp_cnt[b]; }
    if (sum != F) return -4;
    int *seen = (int *)calloc((size_t)(B > F ? B : F), sizeof(int));
    for (int k = 0; k < B; ++k) {
        int b = bp_order[k];
        if (b < 0 || b >= B || seen[b]) { free(seen); return -5; }
        seen[b] = 1;
    }
    memset(seen, 0, sizeof(int) * (size_t)(B > F ? B : F));
    for (int k = 0; k < F; ++k) {
        int f = field_order[k];
        if (f < 0 || f >= F || seen[f]) { free(seen); return -6; }
        seen[f] = 1;
    }
    free(seen);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, Steps 1-3: the initial plan a human scheduler would draw     */
/* (Sec. 2.5).                                                               */
/* ------------------------------------------------------------------------ */
static void init_plan(const or_ctx *c, oplan *p)
{
    const int B = c->B, F = c->F, T = c->T, N = c->N;
    /* Step 1: nearest-neighbour chain HQ -> closest BP -> closest BP ...
       Reading: ties go to the lowest BP id; the chain is cut into contiguous
       pieces, tour g taking floor((g+1)B/T) - floor(gB/T) BPs. */
    int *chain = (int *)malloc(sizeof(int) * (size_t)B);
    int *used = (int *)calloc((size_t)(B > F ? B : F), sizeof(int));
    int cur = 0;
    for (int k = 0; k < B; ++k) {
        int best = -1;
        double bd = 0.0;
        for (int b = 0; b < B; ++b) {
            if (used[b]) continue;
            double d = c->D[(size_t)cur * N + 1 + b];
            if (best < 0 || d < bd) { best = b; bd = d; }
        }
        chain[k] = best; used[best] = 1; cur = 1 + best;
    }
    int k = 0;
    for (int g = 0; g < T; ++g) {
        int n = (int)(((long)(g + 1) * B) / T - ((long)g * B) / T);
        p->tlen[g] = n;
        for (int j = 0; j < n; ++j) p->tbp[g * B + j] = chain[k++];
    }
    /* Step 2: fields in id order go to the closest BP whose minimum demand is
       not yet met; once every BP is met, to the closest BP. Ties: lowest id. */
    double *acc = (double *)calloc((size_t)B, sizeof(double));
    int *bp_of = (int *)malloc(sizeof(int) * (size_t)F);
    for (int f = 0; f < F; ++f) {
        int any_open = 0;
        for (int b = 0; b < B; ++b) if (acc[b] < c->demand[b]) any_open = 1;
        int best = -1;
        double bd = 0.0;
        for (int b = 0; b < B; ++b) {
            if (any_open && !(acc[b] < c->demand[b])) continue;
            double d = c->D[(size_t)(1 + B + f) * N + 1 + b];
            if (best < 0 || d < bd) { best = b; bd = d; }
        }
        bp_of[f] = best;
        acc[best] += c->supply[f];
    }
    /* Step 3: per BP, nearest-neighbour chain starting from the HQ through the
       fields of that BP. Ties: lowest field id. */
    memset(used, 0, sizeof(int) * (size_t)(B > F ? B : F));
    for (int b = 0; b < B; ++b) {
        int n = 0;
        for (int f = 0; f < F; ++f) if (bp_of[f] == b) ++n;
        p->blen[b] = n;
        int at = 0;
        for (int j = 0; j < n; ++j) {
            int best = -1;
            double bd = 0.0;
            for (int f = 0; f < F; ++f) {
                if (bp_of[f] != b || used[f]) continue;
                double d = c->D[(size_t)at * N + 1 + B + f];
                if (best < 0 || d < bd) { best = f; bd = d; }
            }
            p->bfld[b * F + j] = best; used[best] = 1; at = 1 + B + best;
        }
    }
    free(chain); free(used); free(acc); free(bp_of);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, Step 8: one remove-and-reinsert move (Sec. 2.5).             */
/* Counter layout: key = (seed_lo, seed_hi), counter = (i, iter, inst, 0).   */
/* Reading: the vertex is uniform over all F+B vertices (fields first, so    */
/* fields are drawn F/(F+B) of the time); a field goes to a uniform BP       */
/* (its own BP when the field-to-BP assignment is fixed) and a BP to a       */
/* uniform tour (inactive tours included); the slot is uniform over the      */
/* len'+1 slots of the destination list after removal. With probability    */
/* p_swap the move is instead a swap of two same-type vertices.              */
/* Move record: {kind, vertex, a, b}: kind 0 field reinsert (a = BP,         */
/* b = slot), 1 BP reinsert (a = tour, b = slot), 2 field swap (a = field),  */
/* 3 BP swap (a = BP).                                                       */
/* Repeating Step 8 (Sec. 2.5 mentions doing it a second time): move j of a  */
/* candidate is drawn on the plan the first j moves made, from counter word  */
/* 3 = 0 for j = 0 and j + 1 after (word 3 = 1 is the eps rule's counter).   */
/* ------------------------------------------------------------------------ */
static uint32_t move_word3(int j) { return j == 0 ? 0u : (uint32_t)j + 1u; }

static void draw_move(const or_ctx *c, const or_params *prm, uint32_t iter, uint32_t i, int j,
                      const oplan *base, int16_t mv[4])
{
    uint32_t ctr[4] = {i, iter, prm->inst_idx, move_word3(j)};
    uint32_t key[2] = {(uint32_t)prm->seed, (uint32_t)(prm->seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    const int F = c->F, B = c->B, T = c->T;
    uint32_t v = draw_below(r[0], (uint32_t)(F + B));
    if (unit24(r[3]) < prm->p_swap) {
        if ((int)v < F) { mv[0] = 2; mv[1] = (int16_t)v; mv[2] = (int16_t)draw_below(r[1], (uint32_t)F); }
        else { mv[0] = 3; mv[1] = (int16_t)(v - F); mv[2] = (int16_t)draw_below(r[1], (uint32_t)B); }
        mv[3] = 0;
        return;
    }
    if ((int)v < F) {
        int f = (int)v, bs = -1;
        for (int b = 0; b < B && bs < 0; ++b)
            for (int j = 0; j < base->blen[b]; ++j) if (base->bfld[b * F + j] == f) { bs = b; break; }
        int bd = prm->fix_field_bp ? bs : (int)draw_below(r[1], (uint32_t)B);
        int len = base->blen[bd] - (bd == bs ? 1 : 0);
        mv[0] = 0; mv[1] = (int16_t)f; mv[2] = (int16_t)bd;
        mv[3] = (int16_t)draw_below(r[2], (uint32_t)(len + 1));
    } else {
        int b = (int)v - F, gs = -1;
        for (int g = 0; g < T && gs < 0; ++g)
            for (int j = 0; j < base->tlen[g]; ++j) if (base->tbp[g * B + j] == b) { gs = g; break; }
        int gd = (int)draw_below(r[1], (uint32_t)T);
        int len = base->tlen[gd] - (gd == gs ? 1 : 0);
        mv[0] = 1; mv[1] = (int16_t)b; mv[2] = (int16_t)gd;
        mv[3] = (int16_t)draw_below(r[2], (uint32_t)(len + 1));
    }
}

static void list_erase(int *a, int *len, int pos)
{
    for (int j = pos; j + 1 < *len; ++j) a[j] = a[j + 1];
    --*len;
}

static void list_insert(int *a, int *len, int pos, int val)
{
    for (int j = *len; j > pos; --j) a[j] = a[j - 1];
    a[pos] = val;
    ++*len;
}

/* apply a move to a copy of base: remove, then insert into the post-removal
   list (Step 8). A BP carries all its fields (their list is keyed by BP). */
static void apply_move(const oplan *base, const int16_t mv[4], oplan *out)
{
    plan_copy(out, base);
    const int B = base->B, F = base->F, T = base->T;
    if (mv[0] == 0) {
        int f = mv[1], bd = mv[2], pd = mv[3];
        for (int b = 0; b < B; ++b)
            for (int j = 0; j < out->blen[b]; ++j)
                if (out->bfld[b * F + j] == f) { list_erase(&out->bfld[b * F], &out->blen[b], j); goto field_removed; }
    field_removed:
        list_insert(&out->bfld[bd * F], &out->blen[bd], pd, f);
    } else if (mv[0] == 1) {
        int bp = mv[1], gd = mv[2], pd = mv[3];
        for (int g = 0; g < T; ++g)
            for (int j = 0; j < out->tlen[g]; ++j)
                if (out->tbp[g * B + j] == bp) { list_erase(&out->tbp[g * B], &out->tlen[g], j); goto bp_removed; }
    bp_removed:
        list_insert(&out->tbp[gd * B], &out->tlen[gd], pd, bp);
    } else if (mv[0] == 2) {
        int v = mv[1], w = mv[2];
        int *pv = NULL, *pw = NULL;
        for (int b = 0; b < B; ++b)
            for (int j = 0; j < out->blen[b]; ++j) {
                if (out->bfld[b * F + j] == v) pv = &out->bfld[b * F + j];
                if (out->bfld[b * F + j] == w) pw = &out->bfld[b * F + j];
            }
        *pv = w; *pw = v;
    } else if (mv[0] == 3) {
        int v = mv[1], w = mv[2];
        int *pv = NULL, *pw = NULL;
        for (int g = 0; g < T; ++g)
            for (int j = 0; j < out->tlen[g]; ++j) {
                if (out->tbp[g * B + j] == v) pv = &out->tbp[g * B + j];
                if (out->tbp[g * B + j] == w) pw = &out->tbp[g * B + j];
            }
        *pv = w; *pw = v;
    }
}

static int n_moves(const or_params *prm)
{
    if (prm->k_moves > 8) { fprintf(stderr, "oracle: at most 8 chained moves\n"); abort(); }
    return prm->k_moves > 1 ? prm->k_moves : 1;
}

/* Candidate i of iteration `iter`: Step 8 applied k times, move j drawn on the
   plan after the first j moves (a materialised list each time); mv receives
   the k move records (4 words each). `scratch` is a plan of the same sizes. */
static void make_candidate(const or_ctx *c, const or_params *prm, uint32_t iter, uint32_t i, const oplan *base,
                           oplan *out, oplan *scratch, int16_t *mv)
{
    plan_copy(out, base);
    for (int j = 0; j < n_moves(prm); ++j) {
        draw_move(c, prm, iter, i, j, out, mv + 4 * j);
        plan_copy(scratch, out);
        apply_move(scratch, mv + 4 * j, out);
    }
}

/* ------------------------------------------------------------------------ */
/* Exact arithmetic helpers                                                  */
/* ------------------------------------------------------------------------ */
/* sign of (a - k*b) for finite doubles a, b > 0 and integer k >= 0, exactly */
static int sign_a_minus_kb(double a, int64_t k, double b)
{
    int ea, eb;
    double fa = frexp(a, &ea), fb = frexp(b, &eb);
    __int128 L = (__int128)(int64_t)ldexp(fa, 53);
    __int128 R = (__int128)k * (__int128)(int64_t)ldexp(fb, 53);
    int sh = ea - eb;
    if (sh > 60 || sh < -60) { fprintf(stderr, "oracle: exponent gap too wide\n"); abort(); }
    if (sh >= 0) L <<= sh; else R <<= -sh;
    return (L > R) - (L < R);
}

/* Eq. 4: ceil(a / b) for a, b > 0, exact: the smallest k with k*b >= a */
static int64_t ceil_ratio(double a, double b)
{
    int64_t k = (int64_t)ceil(a / b);
    if (k < 0) k = 0;
    while (sign_a_minus_kb(a, k, b) > 0) ++k;
    while (k > 0 && sign_a_minus_kb(a, k - 1, b) <= 0) --k;
    return k;
}

/* Decision sites, for the trace of the gaps a score counts (the margin pins):
   the three picks of a local-minimisation round (Algorithm 2, Step 2), its
   acceptance test (Step 4), its termination test (Step 5), for the HU step
   and the SU step, and the completion-time gate (Sec. 2.5). */
enum {
    GAP_HU_MAX = 1, GAP_HU_MAX2 = 2, GAP_HU_MIN = 3, GAP_HU_ACCEPT = 4, GAP_HU_STOP = 5,
    GAP_SU_MAX = 6, GAP_SU_MAX2 = 7, GAP_SU_MIN = 8, GAP_SU_ACCEPT = 9, GAP_SU_STOP = 10,
    GAP_GATE = 11
};

typedef struct {
    int32_t site;
    int32_t pad;
    double a, b, scale;   /* the compared values and the scale of their relative gap */
} or_gap;

/* optional trace of the calling thread (single-plan scoring only) */
static __thread or_gap *g_trace;
static __thread int g_trace_n, g_trace_cap;

/* relative decision gap |a - b| / scale; exact equality is a structural tie
   and is neither counted nor traced */
static void note_gap(int site, double *margin, double a, double b, double scale)
{
    if (a == b || !isfinite(a) || !isfinite(b)) return;
    double s = scale;
    if (!(s > 0.0)) s = fmax(fabs(a), fabs(b));
    double m = fabs(a - b) / s;
    if (m < *margin) *margin = m;
    if (g_trace) {
        if (g_trace_n < g_trace_cap) {
            or_gap *r = &g_trace[g_trace_n];
            r->site = site; r->pad = 0; r->a = a; r->b = b; r->scale = s;
        }
        ++g_trace_n;
    }
}

/* ------------------------------------------------------------------------ */
/* Scoring one plan (Sec. 2.2 and the three evaluation steps of Sec. 2.5)    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int feasible;      /* Eq. 2 holds for every BP */
    double cost;       /* C (km); +inf when infeasible or discarded by the gate */
    double tmax;       /* max completion time over active tours (h); +inf when infeasible */
    double margin;     /* minimum relative decision gap (+inf if no FP decision) */
    double ops;        /* instrumented count of model operations */
} or_score;

typedef struct {
    int active[64];
    double LHU[64], LSU[64], A[64], Dbar[64];
} route_agg;

static void pick_max_max2_min(int site0, const double *val, const double *scale, const int *act, int na,
                              int *gmax, int *gmax2, int *gmin, double *margin, double *ops)
{
    /* Algorithm 2, Step 2: g_max = argmax, g_max,2nd = argmax over the rest,
       g_min = argmin over the rest without g_max,2nd. Ties: lowest tour id
       (act[] is in ascending tour order and only strictly better replaces).
       Reading for exactly two active tours: g_min is the other tour, which is
       also g_max,2nd. */
    int a = -1, a2 = -1, m = -1;
    for (int j = 0; j < na; ++j) { int g = act[j]; if (a < 0 || val[g] > val[a]) a = g; *ops += 1; }
    for (int j = 0; j < na; ++j) { int g = act[j]; if (g == a) continue; if (a2 < 0 || val[g] > val[a2]) a2 = g; *ops += 1; }
    if (na == 2) m = a2;
    else for (int j = 0; j < na; ++j) { int g = act[j]; if (g == a || g == a2) continue; if (m < 0 || val[g] < val[m]) m = g; *ops += 1; }
    /* margins of the three picks: the winner against every competitor */
    for (int j = 0; j < na; ++j) {
        int g = act[j];
        if (g != a) note_gap(site0, margin, val[a], val[g], fmax(scale[a], scale[g]));
        if (g != a && g != a2) note_gap(site0 + 1, margin, val[a2], val[g], fmax(scale[a2], scale[g]));
        if (na > 2 && g != a && g != a2 && g != m)
            note_gap(site0 + 2, margin, val[m], val[g], fmax(scale[m], scale[g]));
    }
    *gmax = a; *gmax2 = a2; *gmin = m;
}

/* HU completion time of tour g: road time plus harvest time (Sec. 2.5). The
   waiting time is not part of it (reading, checked against Table 3's ~360 h). */
static double t_compl(const or_ctx *c, const route_agg *ra, int g, double R)
{
    return ra->LHU[g] / c->hu_speed + ra->A[g] / R;
}

static double rate_sum(const or_ctx *c, const int *hu_tour, int g)
{
    double R = 0.0;
    for (int k = 0; k < c->H; ++k) { int h = c->hu_sorted[k]; if (hu_tour[h] == g) R += c->hu_rate[h]; }
    return R;
}

/* First evaluation step: assignment of HUs to tours (Sec. 2.5). Start from
   the average number per tour; repeatedly move one HU from g_min to g_max,
   trying HUs in rising working-rate order as Algorithm 2 does for SUs, until
   the maximum completion time stops falling.
   Reading of the start: HUs sorted by (rate, id) are dealt round robin over
   the active tours in tour order. Reading of the stop: each round accepts one
   move; if the new maximum is not below the old one the move is undone and
   the loop ends. At most H rounds; a tour keeps at least one HU. */
static void hu_assign(const or_ctx *c, const or_params *prm, const route_agg *ra, const int *act, int na,
                      int *hu_tour, double *R, double *Tc, double *margin, double *ops)
{
    for (int h = 0; h < c->H; ++h) hu_tour[h] = -1;
    for (int k = 0; k < c->H; ++k) hu_tour[c->hu_sorted[k]] = act[k % na];
    double scale[64];
    for (int j = 0; j < na; ++j) {
        int g = act[j];
        R[g] = rate_sum(c, hu_tour, g);
        Tc[g] = t_compl(c, ra, g, R[g]);
        scale[g] = Tc[g];
        *ops += 4;
    }
    if (prm->fix_resources) return;
    for (int round = 0; round < c->H; ++round) {
        if (na < 2) break;
        int gmax, gmax2, gmin;
        pick_max_max2_min(GAP_HU_MAX, Tc, scale, act, na, &gmax, &gmax2, &gmin, margin, ops);
        int cnt = 0, last = -1;
        for (int k = 0; k < c->H; ++k) if (hu_tour[c->hu_sorted[k]] == gmin) { ++cnt; last = k; }
        if (cnt <= 1) break;
        double old_max = Tc[gmax];
        int moved = -1;
        double newTmax = 0.0, newTmin = 0.0, newRmax = 0.0, newRmin = 0.0;
        for (int k = 0; k < c->H; ++k) {
            int h = c->hu_sorted[k];
            if (hu_tour[h] != gmin) continue;
            hu_tour[h] = gmax;
            double rmax = rate_sum(c, hu_tour, gmax), rmin = rate_sum(c, hu_tour, gmin);
            double tmx = t_compl(c, ra, gmax, rmax), tmn = t_compl(c, ra, gmin, rmin);
            double ref = (na == 2) ? tmn : Tc[gmax2];
            *ops += 8;
            int is_last = (k == last);
            if (!is_last) note_gap(GAP_HU_ACCEPT, margin, tmx, ref, fmax(tmx, ref));
            if (tmx < ref || is_last) {
                moved = h; newTmax = tmx; newTmin = tmn; newRmax = rmax; newRmin = rmin;
                break;
            }
            hu_tour[h] = gmin;
        }
        double saveTmax = Tc[gmax], saveTmin = Tc[gmin], saveRmax = R[gmax], saveRmin = R[gmin];
        Tc[gmax] = newTmax; Tc[gmin] = newTmin; R[gmax] = newRmax; R[gmin] = newRmin;
        scale[gmax] = newTmax; scale[gmin] = newTmin;
        double nm = -INFINITY;
        for (int j = 0; j < na; ++j) { if (Tc[act[j]] > nm) nm = Tc[act[j]]; *ops += 1; }
        note_gap(GAP_HU_STOP, margin, nm, old_max, fmax(nm, old_max));
        if (!(nm < old_max)) {
            hu_tour[moved] = gmin;
            Tc[gmax] = saveTmax; Tc[gmin] = saveTmin; R[gmax] = saveRmax; R[gmin] = saveRmin;
            scale[gmax] = saveTmax; scale[gmin] = saveTmin;
            break;
        }
    }
}

/* Eq. 6 and Algorithm 2, Step 1: average HU waiting time of tour g.
   Reading for per-unit SU classes: the critical SU s* is the SU of g with
   the largest fill area (ties: lowest id); its round trip uses its own speed;
   the other SUs of g fill while it drives, each taking a_s / R(g) hours.
   Because the subtracted term is the same for every field of g, the mean of
   per-BP means of Eq. 6 is 2*Dbar(g)/v_s* - (sum a_s - a_s*)/R(g). */
static double t_wait(const or_ctx *c, const route_agg *ra, const int *su_tour, int g, double R, double *scale)
{
    double sum_a = 0.0;
    int star = -1;
    for (int k = 0; k < c->S; ++k) {
        int s = c->su_sorted[k];
        if (su_tour[s] != g) continue;
        sum_a += c->su_fill[s];
        if (star < 0 || c->su_fill[s] > c->su_fill[star]) star = s;   /* first of the largest: lowest id */
    }
    double drive = 2.0 * ra->Dbar[g] / c->su_speed[star];
    double fill = (sum_a - c->su_fill[star]) / R;
    if (scale) *scale = fabs(drive) + fabs(fill);
    return drive - fill;
}

/* Second evaluation step: Algorithm 2, assignment of SUs to tours. Same
   skeleton and readings as the HU step; SUs of g_min are tried in rising
   fill-area order; at most S rounds; a tour keeps at least one SU. */
static void su_assign(const or_ctx *c, const or_params *prm, const route_agg *ra, const int *act, int na,
                      const double *R, int *su_tour, double *Tw, double *margin, double *ops)
{
    for (int s = 0; s < c->S; ++s) su_tour[s] = -1;
    for (int k = 0; k < c->S; ++k) su_tour[c->su_sorted[k]] = act[k % na];
    double scale[64];
    for (int j = 0; j < na; ++j) { int g = act[j]; Tw[g] = t_wait(c, ra, su_tour, g, R[g], &scale[g]); *ops += 6; }
    if (prm->fix_resources) return;
    for (int round = 0; round < c->S; ++round) {
        if (na < 2) break;
        int gmax, gmax2, gmin;
        pick_max_max2_min(GAP_SU_MAX, Tw, scale, act, na, &gmax, &gmax2, &gmin, margin, ops);
        int cnt = 0, last = -1;
        for (int k = 0; k < c->S; ++k) if (su_tour[c->su_sorted[k]] == gmin) { ++cnt; last = k; }
        if (cnt <= 1) break;
        double old_max = Tw[gmax];
        int moved = -1;
        double nmx = 0.0, nmn = 0.0, smx = 0.0, smn = 0.0;
        for (int k = 0; k < c->S; ++k) {
            int s = c->su_sorted[k];
            if (su_tour[s] != gmin) continue;
            su_tour[s] = gmax;
            double sc_mx, sc_mn;
            double tmx = t_wait(c, ra, su_tour, gmax, R[gmax], &sc_mx);
            double tmn = t_wait(c, ra, su_tour, gmin, R[gmin], &sc_mn);
            double ref = (na == 2) ? tmn : Tw[gmax2];
            double ref_scale = (na == 2) ? sc_mn : scale[gmax2];
            *ops += 12;
            int is_last = (k == last);
            if (!is_last) note_gap(GAP_SU_ACCEPT, margin, tmx, ref, fmax(sc_mx, ref_scale));
            if (tmx < ref || is_last) { moved = s; nmx = tmx; nmn = tmn; smx = sc_mx; smn = sc_mn; break; }
            su_tour[s] = gmin;
        }
        double svmx = Tw[gmax], svmn = Tw[gmin], sscmx = scale[gmax], sscmn = scale[gmin];
        Tw[gmax] = nmx; Tw[gmin] = nmn; scale[gmax] = smx; scale[gmin] = smn;
        double nm = -INFINITY, nm_scale = 0.0;
        for (int j = 0; j < na; ++j) { int g = act[j]; if (Tw[g] > nm) { nm = Tw[g]; nm_scale = scale[g]; } *ops += 1; }
        note_gap(GAP_SU_STOP, margin, nm, old_max, fmax(nm_scale, sscmx));
        if (!(nm < old_max)) {
            su_tour[moved] = gmin;
            Tw[gmax] = svmx; Tw[gmin] = svmn; scale[gmax] = sscmx; scale[gmin] = sscmn;
            break;
        }
    }
}

typedef struct {
    /* optional per-tour / per-unit outputs (may be NULL) */
    int32_t *n_hu, *n_su;          /* T */
    double *tcompl, *twait, *tcost; /* T */
    int32_t *hu_tour, *su_tour;    /* H, S: tour index or -1 */
} or_detail;

static void score_plan(const or_ctx *c, const or_params *prm, const oplan *p, double tmax_star,
                       int gate, or_score *res, or_detail *det)
{
    const int B = c->B, F = c->F, T = c->T, N = c->N;
    double ops = 0.0, margin = INFINITY;
    res->feasible = 0; res->cost = INFINITY; res->tmax = INFINITY; res->margin = INFINITY; res->ops = 0.0;
    if (T > 64) { fprintf(stderr, "oracle: T > 64\n"); abort(); }
    if (det) {
        for (int g = 0; g < T; ++g) {
            if (det->n_hu) det->n_hu[g] = 0;
            if (det->n_su) det->n_su[g] = 0;
            if (det->tcompl) det->tcompl[g] = 0.0;
            if (det->twait) det->twait[g] = 0.0;
            if (det->tcost) det->tcost[g] = 0.0;
        }
        if (det->hu_tour) for (int h = 0; h < c->H; ++h) det->hu_tour[h] = -1;
        if (det->su_tour) for (int s = 0; s < c->S; ++s) det->su_tour[s] = -1;
    }
    /* Eq. 2: every BP must be supplied its minimum demand; otherwise the
       candidate is discarded and its cost not evaluated (Sec. 2.5). The FP64
       sum of FP32 supplies is exact (checked in or_new). */
    for (int b = 0; b < B; ++b) {
        double s = 0.0;
        for (int j = 0; j < p->blen[b]; ++j) { s += c->supply[p->bfld[b * F + j]]; ops += 1; }
        ops += 1;
        if (!(s >= c->demand[b])) { res->ops = ops; return; }
    }
    res->feasible = 1;

    /* Route aggregates, traced as in Fig. 1 (Sec. 2.2):
       - HUs drive HQ -> fields of the tour in order (across its BPs) -> HQ;
         they never drive to BPs.
       - SUs leave the HQ for the first field of the first BP, move from each
         BP to the first field of the next BP, and return from the last BP to
         the HQ; between, they shuttle field <-> BP (counted in the cost).
       - A(g): harvested area; Dbar(g): mean over the tour's BPs of the mean
         field-to-BP distance (Algorithm 2, Step 1).
       BPs without fields would be skipped; with positive demands a feasible
       plan has none. */
    route_agg ra;
    int na = 0;
    for (int g = 0; g < T; ++g) {
        ra.LHU[g] = ra.LSU[g] = ra.A[g] = ra.Dbar[g] = 0.0;
        if (p->tlen[g] == 0) continue;
        ra.active[na++] = g;
        int prev_field_node = 0, prev_anchor = 0, nbp = 0;
        double dsum = 0.0;
        for (int j = 0; j < p->tlen[g]; ++j) {
            int b = p->tbp[g * B + j];
            if (p->blen[b] == 0) continue;
            double sb = 0.0;
            for (int k = 0; k < p->blen[b]; ++k) {
                int f = p->bfld[b * F + k];
                int fn = 1 + B + f;
                ra.LHU[g] += c->D[(size_t)prev_field_node * N + fn];
                if (k == 0) { ra.LSU[g] += c->D[(size_t)prev_anchor * N + fn]; ops += 2; }
                ra.A[g] += c->area[f];
                sb += c->D[(size_t)fn * N + 1 + b];
                prev_field_node = fn;
                ops += 5;
            }
            dsum += sb / (double)p->blen[b];
            ++nbp;
            prev_anchor = 1 + b;
            ops += 2;
        }
        ra.LHU[g] += c->D[(size_t)prev_field_node * N + 0];
        ra.LSU[g] += c->D[(size_t)prev_anchor * N + 0];
        ra.Dbar[g] = nbp ? dsum / (double)nbp : 0.0;
        ops += 5;
    }
    int act[64];
    for (int j = 0; j < na; ++j) act[j] = ra.active[j];

    int *hu_tour = (int *)malloc(sizeof(int) * (size_t)c->H);
    int *su_tour = (int *)malloc(sizeof(int) * (size_t)c->S);
    double R[64], Tc[64], Tw[64];
    hu_assign(c, prm, &ra, act, na, hu_tour, R, Tc, &margin, &ops);
    double tmax = -INFINITY;
    for (int j = 0; j < na; ++j) { if (Tc[act[j]] > tmax) tmax = Tc[act[j]]; ops += 1; }
    /* Model operations a result needs: Tmax depends on the HU assignment alone, so a
       candidate the gate discards is decided here (its C is +inf whatever follows); the
       rest is computed for every candidate all the same, only not counted for those. */
    const double ops_at_gate = ops;
    su_assign(c, prm, &ra, act, na, R, su_tour, Tw, &margin, &ops);

    /* Third step: the path-length cost (Sec. 2.2). N_HU(g) multiplies the HU
       route, N_SU(g) the SU repositioning route, and each field contributes
       2 * N_shuttle * d(f, b) for the back-and-forth shuttle drives (Eq. 4).
       Reading for mixed SU classes in one tour: N_shuttle = ceil(s_f / cbar)
       with cbar the mean capacity of the tour's SUs, i.e.
       ceil(s_f * N_SU(g) / sum of capacities), taken exactly. */
    double cost = 0.0;
    for (int j = 0; j < na; ++j) {
        int g = act[j];
        int nhu = 0, nsu = 0;
        double capsum = 0.0;
        for (int h = 0; h < c->H; ++h) if (hu_tour[h] == g) ++nhu;
        for (int k = 0; k < c->S; ++k) { int s = c->su_sorted[k]; if (su_tour[s] == g) { ++nsu; capsum += c->su_cap[s]; } }
        double shuttle = 0.0;
        for (int jj = 0; jj < p->tlen[g]; ++jj) {
            int b = p->tbp[g * B + jj];
            for (int k = 0; k < p->blen[b]; ++k) {
                int f = p->bfld[b * F + k];
                int64_t nf = ceil_ratio(c->supply[f] * (double)nsu, capsum);
                shuttle += 2.0 * (double)nf * c->D[(size_t)(1 + B + f) * N + 1 + b];
                ops += 5;
            }
        }
        double tc = (double)nhu * ra.LHU[g] + (double)nsu * ra.LSU[g] + shuttle;
        cost += tc;
        ops += 5;
        if (det) {
            if (det->n_hu) det->n_hu[g] = nhu;
            if (det->n_su) det->n_su[g] = nsu;
            if (det->tcompl) det->tcompl[g] = Tc[g];
            if (det->twait) det->twait[g] = Tw[g];
            if (det->tcost) det->tcost[g] = tc;
        }
    }
    if (det) {
        if (det->hu_tour) for (int h = 0; h < c->H; ++h) det->hu_tour[h] = hu_tour[h];
        if (det->su_tour) for (int s = 0; s < c->S; ++s) det->su_tour[s] = su_tour[s];
    }
    free(hu_tour); free(su_tour);

    /* Completion-time gate (Sec. 2.5). Reading: gate 1 discards candidates
       whose maximum completion time exceeds the best-so-far one; gate 2 is the
       literal "does not decrease" (>=). */
    res->tmax = tmax;
    if (gate) {
        note_gap(GAP_GATE, &margin, tmax, tmax_star, fmax(tmax, tmax_star));
        ops += 1;
        if ((gate == 1 && tmax > tmax_star) || (gate == 2 && tmax >= tmax_star)) {
            cost = INFINITY;
            ops = ops_at_gate + 1;
        }
    }
    res->cost = cost;
    res->margin = margin;
    res->ops = ops;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (ctypes)                                            */
/* ------------------------------------------------------------------------ */
void or_init_plan(const or_ctx *c, int16_t *bp_order, int16_t *tour_cnt, int16_t *field_order, int16_t *bp_cnt)
{
    oplan p;
    plan_alloc(&p, c->T, c->B, c->F);
    init_plan(c, &p);
    plan_to_enc(&p, bp_order, tour_cnt, field_order, bp_cnt);
    plan_release(&p);
}

int or_move(const or_ctx *c, const or_params *prm, uint32_t iter, uint32_t i,
            const int16_t *bp_order, const int16_t *tour_cnt, const int16_t *field_order, const int16_t *bp_cnt,
            int16_t mv[4])
{
    oplan p;
    plan_alloc(&p, c->T, c->B, c->F);
    if (plan_from_enc(&p, bp_order, tour_cnt, field_order, bp_cnt)) { plan_release(&p); return -1; }
    draw_move(c, prm, iter, i, 0, &p, mv);
    plan_release(&p);
    return 0;
}

/* Candidate i of iteration `iter` drawn from the plan given: its plan (encoding
   into o_*) and its k move records (mv, 4 k words). */
int or_candidate(const or_ctx *c, const or_params *prm, uint32_t iter, uint32_t i,
                 const int16_t *bp_order, const int16_t *tour_cnt, const int16_t *field_order, const int16_t *bp_cnt,
                 int16_t *mv, int16_t *o_bp_order, int16_t *o_tour_cnt, int16_t *o_field_order, int16_t *o_bp_cnt)
{
    oplan p, q, r;
    plan_alloc(&p, c->T, c->B, c->F); plan_alloc(&q, c->T, c->B, c->F); plan_alloc(&r, c->T, c->B, c->F);
    int rc = plan_from_enc(&p, bp_order, tour_cnt, field_order, bp_cnt);
    if (!rc) {
        make_candidate(c, prm, iter, i, &p, &q, &r, mv);
        plan_to_enc(&q, o_bp_order, o_tour_cnt, o_field_order, o_bp_cnt);
    }
    plan_release(&p); plan_release(&q); plan_release(&r);
    return rc ? -1 : 0;
}

int or_apply(const or_ctx *c, const int16_t *bp_order, const int16_t *tour_cnt, const int16_t *field_order,
             const int16_t *bp_cnt, const int16_t mv[4],
             int16_t *o_bp_order, int16_t *o_tour_cnt, int16_t *o_field_order, int16_t *o_bp_cnt)
{
    oplan p, q;
    plan_alloc(&p, c->T, c->B, c->F);
    plan_alloc(&q, c->T, c->B, c->F);
    if (plan_from_enc(&p, bp_order, tour_cnt, field_order, bp_cnt)) { plan_release(&p); plan_release(&q); return -1; }
    apply_move(&p, mv, &q);
    plan_to_enc(&q, o_bp_order, o_tour_cnt, o_field_order, o_bp_cnt);
    plan_release(&p); plan_release(&q);
    return 0;
}

int or_score_plan(const or_ctx *c, const or_params *prm, const int16_t *bp_order, const int16_t *tour_cnt,
                  const int16_t *field_order, const int16_t *bp_cnt, double tmax_star, int32_t gate,
                  or_score *res, int32_t *n_hu, int32_t *n_su, double *tcompl, double *twait, double *tcost,
                  int32_t *hu_tour, int32_t *su_tour)
{
    oplan p;
    plan_alloc(&p, c->T, c->B, c->F);
    if (plan_from_enc(&p, bp_order, tour_cnt, field_order, bp_cnt)) { plan_release(&p); return -1; }
    or_detail det = {n_hu, n_su, tcompl, twait, tcost, hu_tour, su_tour};
    score_plan(c, prm, &p, tmax_star, gate, res, &det);
    plan_release(&p);
    return 0;
}

/* or_score_plan with the trace of every decision gap the score counts, in the
   order taken (at most cap records; returns their number, or -1 for a bad
   plan). The margin is the smallest |a - b| / scale of the trace. */
int or_score_plan_trace(const or_ctx *c, const or_params *prm, const int16_t *bp_order, const int16_t *tour_cnt,
                        const int16_t *field_order, const int16_t *bp_cnt, double tmax_star, int32_t gate,
                        or_score *res, or_gap *trace, int32_t cap)
{
    oplan p;
    plan_alloc(&p, c->T, c->B, c->F);
    if (plan_from_enc(&p, bp_order, tour_cnt, field_order, bp_cnt)) { plan_release(&p); return -1; }
    g_trace = trace; g_trace_n = 0; g_trace_cap = cap;
    score_plan(c, prm, &p, tmax_star, gate, res, NULL);
    const int n = g_trace_n;
    g_trace = NULL; g_trace_n = 0; g_trace_cap = 0;
    plan_release(&p);
    return n;
}

/* Trace of the cost's edges for one plan (Fig. 1): kind 0 = HU drive,
   1 = empty-SU repositioning, 2 = loaded shuttle field->BP, 3 = empty shuttle
   BP->field. from/to are node ids. Returns the number of edges written. */
int or_trace_edges(const or_ctx *c, const int16_t *bp_order, const int16_t *tour_cnt,
                   const int16_t *field_order, const int16_t *bp_cnt,
                   int32_t *kind, int32_t *from, int32_t *to, int32_t *tour, int32_t cap)
{
    oplan p;
    plan_alloc(&p, c->T, c->B, c->F);
    if (plan_from_enc(&p, bp_order, tour_cnt, field_order, bp_cnt)) { plan_release(&p); return -1; }
    const int B = c->B, F = c->F;
    int n = 0;
#define EMIT(k, a, b_, g_) do { if (n < cap) { kind[n] = (k); from[n] = (a); to[n] = (b_); tour[n] = (g_); } ++n; } while (0)
    for (int g = 0; g < c->T; ++g) {
        if (p.tlen[g] == 0) continue;
        int prev_field_node = 0, prev_anchor = 0;
        for (int j = 0; j < p.tlen[g]; ++j) {
            int b = p.tbp[g * B + j];
            if (p.blen[b] == 0) continue;
            for (int k = 0; k < p.blen[b]; ++k) {
                int fn = 1 + B + p.bfld[b * F + k];
                EMIT(0, prev_field_node, fn, g);
                if (k == 0) EMIT(1, prev_anchor, fn, g);
                EMIT(2, fn, 1 + b, g);
                EMIT(3, 1 + b, fn, g);
                prev_field_node = fn;
            }
            prev_anchor = 1 + b;
        }
        EMIT(0, prev_field_node, 0, g);
        EMIT(1, prev_anchor, 0, g);
    }
#undef EMIT
    plan_release(&p);
    return n;
}

static void eps_select(const or_params *prm, uint32_t iter, int *use_best)
{
    /* Eq. 5: x = x* if u < eps else x_old; u from counter (0, iter, inst, 1) */
    uint32_t ctr[4] = {0u, iter, prm->inst_idx, 1u};
    uint32_t key[2] = {(uint32_t)prm->seed, (uint32_t)(prm->seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    *use_best = unit24(r[0]) < prm->eps;
}

int or_eps_select(const or_params *prm, uint32_t iter) { int u; eps_select(prm, iter, &u); return u; }

/* Score the n candidates of iteration `iter` drawn from `base`. Any output
   pointer may be NULL. moves: n x 4. */
int or_score_batch(const or_ctx *c, const or_params *prm, uint32_t iter,
                   const int16_t *bp_order, const int16_t *tour_cnt, const int16_t *field_order, const int16_t *bp_cnt,
                   double tmax_star, int32_t i0, int32_t n, int32_t nthreads,
                   double *cost, double *tmax, double *margin, int32_t *feasible, int16_t *moves,
                   int32_t *n_hu, int32_t *n_su, int32_t *hu_tour, int32_t *su_tour, double *ops_total)
{
    oplan base;
    plan_alloc(&base, c->T, c->B, c->F);
    if (plan_from_enc(&base, bp_order, tour_cnt, field_order, bp_cnt)) { plan_release(&base); return -1; }
    double ops_sum = 0.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(+ : ops_sum)
#endif
    {
        oplan cand, tmp;
        plan_alloc(&cand, c->T, c->B, c->F);
        plan_alloc(&tmp, c->T, c->B, c->F);
        const int km = n_moves(prm);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int32_t k = 0; k < n; ++k) {
            int16_t mv[4 * 8];
            make_candidate(c, prm, iter, (uint32_t)(i0 + k), &base, &cand, &tmp, mv);
            or_score r;
            or_detail det = {n_hu ? n_hu + (size_t)k * c->T : NULL, n_su ? n_su + (size_t)k * c->T : NULL,
                             NULL, NULL, NULL, hu_tour ? hu_tour + (size_t)k * c->H : NULL,
                             su_tour ? su_tour + (size_t)k * c->S : NULL};
            score_plan(c, prm, &cand, tmax_star, prm->gate, &r, &det);
            if (cost) cost[k] = r.cost;
            if (tmax) tmax[k] = r.tmax;
            if (margin) margin[k] = r.margin;
            if (feasible) feasible[k] = r.feasible;
            if (moves) memcpy(moves + (size_t)k * 4 * km, mv, sizeof(int16_t) * 4 * (size_t)km);
            ops_sum += r.ops;
        }
        plan_release(&cand);
        plan_release(&tmp);
    }
    if (ops_total) *ops_total = ops_sum;
    plan_release(&base);
    return 0;
}

/* Search state: the plans x_old and x* (encodings), C*, Tmax*, iteration. */
typedef struct {
    int16_t *xold_bp_order, *xold_tour_cnt, *xold_field_order, *xold_bp_cnt;
    int16_t *xbest_bp_order, *xbest_tour_cnt, *xbest_field_order, *xbest_bp_cnt;
    double cstar, tmaxstar;
    uint32_t iter;
} or_state;

/* Algorithm 1, Steps 5-16 (GPU version), n candidates per iteration.
   Per iteration outputs (each may be NULL): use_best, istar (the argmin),
   c_istar, cstar, tmaxstar, indicator (0 none, 1 improved by a field move,
   2 by a BP move), margin of the argmin candidate, relative gap to the
   second-best distinct cost. force_istar (may be NULL): when >= 0 at an
   iteration, the search continues from that index instead of the argmin
   (used to follow another run through near-ties); c_follow is the cost of
   the index actually followed. */
int or_search(const or_ctx *c, const or_params *prm, or_state *st, int32_t n_iters, int32_t n_cand,
              int32_t nthreads, int32_t *use_best_o, int32_t *istar_o, double *c_istar_o, double *cstar_o,
              double *tmaxstar_o, int32_t *indicator_o, double *margin_best_o, double *gap_o,
              const int32_t *force_istar, double *c_follow_o)
{
    const int T = c->T, B = c->B, F = c->F;
    oplan xold, xbest, base, cand;
    plan_alloc(&xold, T, B, F); plan_alloc(&xbest, T, B, F); plan_alloc(&base, T, B, F); plan_alloc(&cand, T, B, F);
    if (plan_from_enc(&xold, st->xold_bp_order, st->xold_tour_cnt, st->xold_field_order, st->xold_bp_cnt) ||
        plan_from_enc(&xbest, st->xbest_bp_order, st->xbest_tour_cnt, st->xbest_field_order, st->xbest_bp_cnt)) {
        plan_release(&xold); plan_release(&xbest); plan_release(&base); plan_release(&cand);
        return -1;
    }
    double *cost = (double *)malloc(sizeof(double) * (size_t)n_cand);
    double *tmx = (double *)malloc(sizeof(double) * (size_t)n_cand);
    double *mrg = (double *)malloc(sizeof(double) * (size_t)n_cand);
    int16_t *bo = (int16_t *)malloc(sizeof(int16_t) * (size_t)B), *tc = (int16_t *)malloc(sizeof(int16_t) * (size_t)T);
    int16_t *fo = (int16_t *)malloc(sizeof(int16_t) * (size_t)F), *bc = (int16_t *)malloc(sizeof(int16_t) * (size_t)B);
    for (int32_t it = 0; it < n_iters; ++it) {
        uint32_t iter = st->iter;
        int use_best;
        eps_select(prm, iter, &use_best);
        plan_copy(&base, use_best ? &xbest : &xold);
        plan_to_enc(&base, bo, tc, fo, bc);
        or_score_batch(c, prm, iter, bo, tc, fo, bc, st->tmaxstar, 0, n_cand, nthreads, cost, tmx, mrg,
                       NULL, NULL, NULL, NULL, NULL, NULL, NULL);
        /* Step 13: i* = argmin C_i, ties to the lowest index */
        int32_t istar = 0;
        for (int32_t k = 1; k < n_cand; ++k) if (cost[k] < cost[istar]) istar = k;
        double second = INFINITY;
        for (int32_t k = 0; k < n_cand; ++k) if (cost[k] != cost[istar] && cost[k] < second) second = cost[k];
        if (gap_o) gap_o[it] = (isfinite(cost[istar]) && isfinite(second)) ? (second - cost[istar]) / cost[istar] : INFINITY;
        if (istar_o) istar_o[it] = istar;
        if (c_istar_o) c_istar_o[it] = cost[istar];
        if (force_istar && force_istar[it] >= 0 && force_istar[it] < n_cand) istar = force_istar[it];
        if (c_follow_o) c_follow_o[it] = cost[istar];
        int ind = 0;
        int16_t mv[4 * 8];
        make_candidate(c, prm, iter, (uint32_t)istar, &base, &cand, &xold, mv);
        if (isfinite(cost[istar])) {
            /* Steps 13-16: rebuild x_{i*}; update x*, C*; x_old <- x_{i*} */
            plan_copy(&xold, &cand);
            if (cost[istar] < st->cstar) {
                plan_copy(&xbest, &cand);
                st->cstar = cost[istar];
                st->tmaxstar = tmx[istar];
                ind = (mv[0] == 0 || mv[0] == 2) ? 1 : 2;
            }
        } else {
            /* reading: no feasible candidate -> x_old <- base */
            plan_copy(&xold, &base);
        }
        if (use_best_o) use_best_o[it] = use_best;
        if (cstar_o) cstar_o[it] = st->cstar;
        if (tmaxstar_o) tmaxstar_o[it] = st->tmaxstar;
        if (indicator_o) indicator_o[it] = ind;
        if (margin_best_o) margin_best_o[it] = mrg[istar];
        st->iter = iter + 1;
    }
    plan_to_enc(&xold, st->xold_bp_order, st->xold_tour_cnt, st->xold_field_order, st->xold_bp_cnt);
    plan_to_enc(&xbest, st->xbest_bp_order, st->xbest_tour_cnt, st->xbest_field_order, st->xbest_bp_cnt);
    free(cost); free(tmx); free(mrg); free(bo); free(tc); free(fo); free(bc);
    plan_release(&xold); plan_release(&xbest); plan_release(&base); plan_release(&cand);
    return 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
