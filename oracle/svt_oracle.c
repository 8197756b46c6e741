/*
 * svt_oracle.c -- plain, serial CPU reference of the SVT linearised track fit.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  The product
 * (the CUDA library and its Python binding) never calls it, and it shares no
 * code, header or table with the product: every format constant below is
 * written out here again from the word-format definition.
 *
 * What it computes (the paper, Sec. 2 and Sec. 2.1):
 *   - three stages: unpack the input words, form every combination of one hit
 *     per layer inside each road, and fit each combination with the linear
 *     form p_i = f_i . x + q_i using integer multiply/add only;
 *   - three nested loops: events -> roads -> combinations.
 * Readings of what the paper leaves open (each one is a stated choice):
 *   - six coordinates per combination; x_l = 0 for a layer without hits;
 *   - acc_k = q_k * 2^qshift + sum_l F_kl * x_l, exact in int64;
 *     y_k = floor(acc_k / 2^oshift) (floor, i.e. toward minus infinity);
 *   - rows 0..2 are the track parameters (d0, phi, curvature), rows 3..5 are
 *     chi components; chi2 = sum_{k=3..5} clamp(y_k, -32767, 32767)^2;
 *   - a combination passes when chi2 <= chi2_cut; per road the passing
 *     combination with the smallest chi2 is kept, ties going to the smallest
 *     combination index;
 *   - combination index c is mixed radix over layers, layer 0 most
 *     significant and layer 5 fastest; hits keep their order of appearance;
 *   - a road with more than max_comb combinations evaluates only the first
 *     max_comb of them and is flagged OVERFLOW;
 *   - with xft_pairs set, layers 4 and 5 are the two coordinates (phi and
 *     curvature) of one track-trigger track: hit i of layer 4 goes with hit i
 *     of layer 5, a road must carry as many hits in layer 5 as in layer 4
 *     (rule V11), and the combinations run over layers 0..4 only, layer 5
 *     taking layer 4's hit index.
 * The input validation follows the word-format rules V1..V11 listed at
 * orc_validate() below.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KEY_OK UINT64_MAX

/* error codes (smaller code wins when two rules fire on one word) */
#define ORC_E_BAD_ARG 1u
#define ORC_E_BAD_TYPE 2u
#define ORC_E_BAD_RESERVED 3u
#define ORC_E_BAD_LAYER 4u
#define ORC_E_UNSORTED 5u
#define ORC_E_TOO_MANY_HITS 6u
#define ORC_E_BAD_SECTOR 7u
#define ORC_E_NROADS_MISMATCH 8u
#define ORC_E_BAD_CONFIG 10u
#define ORC_E_XFT_UNPAIRED 12u

/* output flags, stored in bits [31:24] of record word 0 */
#define ORC_F_PASS 1u
#define ORC_F_OVERFLOW 2u
#define ORC_F_BAD_PATTERN 4u
#define ORC_F_NO_HITS 8u

typedef struct {
    uint32_t oshift, qshift, chi2_cut, max_comb, min_layers, n_sectors, xft_pairs;
} orc_config;

/* ---- word fields ---- */
static uint32_t w_type(uint32_t w) { return w >> 30; }
static uint32_t ev_nroads(uint32_t w) { return w & 0xFFFu; }
static uint32_t rd_sector(uint32_t w) { return (w >> 21) & 0x1FFu; }
static uint32_t rd_id(uint32_t w) { return w & 0x1FFFFFu; }
static uint32_t hit_layer(uint32_t w) { return (w >> 27) & 7u; }
static uint32_t hit_reserved(uint32_t w) { return (w >> 15) & 0xFFFu; }
static uint32_t hit_coord(uint32_t w) { return w & 0x7FFFu; }

static uint64_t make_key(uint64_t word_index, uint32_t code) { return (word_index << 8) | code; }
static void note(uint64_t *key, uint64_t word_index, uint32_t code) {
    uint64_t k = make_key(word_index, code);
    if (k < *key) *key = k;
}

int orc_config_ok(const orc_config *cfg) {
    if (cfg->oshift < 9 || cfg->oshift > 31) return 0;
    if (cfg->qshift > 24) return 0;
    if (cfg->max_comb < 1) return 0;
    if (cfg->min_layers > 6) return 0;
    if (cfg->xft_pairs > 1) return 0;
    if (cfg->n_sectors < 1 || cfg->n_sectors > 512) return 0;
    return 1;
}

/*
 * Validation.  Returns the smallest key (word_index << 8 | code) over all
 * violations, or ORC_KEY_OK.  Offsets that are not 0 = off[0] < off[1] < ...
 * < off[E] = n_words give key (0, BAD_ARG).  For word i of event e
 * (start = off[e] <= i < off[e+1]), t = type(w[i]):
 *   V1  i == start and t != 3                                   BAD_TYPE
 *   V2  i != start and t == 3                                   BAD_TYPE
 *   V3  t == 1                                                  BAD_TYPE
 *   V4  t == 0, i > start and type(w[i-1]) == 3                 BAD_TYPE
 *   V5  t == 0 and reserved bits [26:15] != 0                   BAD_RESERVED
 *   V6  t == 0 and layer > 5                                    BAD_LAYER
 *   V7  t == 0, i > start, type(w[i-1]) == 0, layer(w[i-1]) > layer(w[i])
 *                                                               UNSORTED
 *   V8  t == 0 inside the run of hit words that follows a road header, and
 *       more than 16 words of the run up to i carry layer(w[i]) TOO_MANY_HITS
 *   V9  t == 2 and sector >= n_sectors                          BAD_SECTOR
 *   V10 i == start, t == 3 and n_roads(w) != number of type-2 words in the
 *       event                                                   NROADS_MISMATCH
 *   V11 (xft_pairs only) the hit run that follows a road header has a
 *       different number of layer-4 and layer-5 hits; reported at the run's
 *       last word (its last hit)                               XFT_UNPAIRED
 *       (A run of more than 96 hits always breaks V6, V7 or V8 at one of its
 *       words, so the smallest key never comes from V11 on such a run.)
 */
uint64_t orc_validate(const uint32_t *words, uint64_t n_words, const uint64_t *event_off,
                      uint64_t n_events, uint32_t n_sectors, uint32_t xft_pairs) {
    uint64_t key = ORC_KEY_OK;
    if (event_off[0] != 0 || event_off[n_events] != n_words) return make_key(0, ORC_E_BAD_ARG);
    for (uint64_t e = 0; e < n_events; ++e)
        if (event_off[e + 1] <= event_off[e]) return make_key(0, ORC_E_BAD_ARG);

    for (uint64_t e = 0; e < n_events; ++e) {
        uint64_t start = event_off[e], end = event_off[e + 1];
        uint64_t n_road_headers = 0;
        int in_road_run = 0;       /* inside the hit run that follows a road header */
        uint32_t run_count[8];
        memset(run_count, 0, sizeof run_count);
        for (uint64_t i = start; i <= end; ++i) {
            if (i == end) {        /* the end of the event closes the last run */
                if (in_road_run && xft_pairs && run_count[4] != run_count[5])
                    note(&key, i - 1, ORC_E_XFT_UNPAIRED);                          /* V11 */
                break;
            }
            uint32_t w = words[i], t = w_type(w);
            if (i == start && t != 3) note(&key, i, ORC_E_BAD_TYPE);            /* V1 */
            if (i != start && t == 3) note(&key, i, ORC_E_BAD_TYPE);            /* V2 */
            if (t == 1) note(&key, i, ORC_E_BAD_TYPE);                          /* V3 */
            if (t == 0) {
                uint32_t prev = (i > start) ? words[i - 1] : 0;
                if (i > start && w_type(prev) == 3) note(&key, i, ORC_E_BAD_TYPE);   /* V4 */
                if (hit_reserved(w) != 0) note(&key, i, ORC_E_BAD_RESERVED);         /* V5 */
                if (hit_layer(w) > 5) note(&key, i, ORC_E_BAD_LAYER);                /* V6 */
                if (i > start && w_type(prev) == 0 && hit_layer(prev) > hit_layer(w))
                    note(&key, i, ORC_E_UNSORTED);                                   /* V7 */
                if (in_road_run) {
                    run_count[hit_layer(w)] += 1;
                    if (run_count[hit_layer(w)] > 16) note(&key, i, ORC_E_TOO_MANY_HITS); /* V8 */
                }
            } else {
                if (in_road_run && xft_pairs && run_count[4] != run_count[5])
                    note(&key, i - 1, ORC_E_XFT_UNPAIRED);                          /* V11 */
                in_road_run = 0;
            }
            if (t == 2) {
                n_road_headers += 1;
                if (rd_sector(w) >= n_sectors) note(&key, i, ORC_E_BAD_SECTOR);    /* V9 */
                in_road_run = 1;
                memset(run_count, 0, sizeof run_count);
            }
        }
        if (w_type(words[start]) == 3 && ev_nroads(words[start]) != n_road_headers)
            note(&key, start, ORC_E_NROADS_MISMATCH);                               /* V10 */
    }
    return key;
}

/* floor(acc / 2^s), written as a division so it does not rely on how the
 * compiler shifts negative numbers */
static int64_t floor_div_pow2(int64_t acc, uint32_t s) {
    int64_t d = (int64_t)1 << s;
    int64_t qt = acc / d;
    if (acc % d != 0 && acc < 0) qt -= 1;
    return qt;
}

static int64_t clamp_chi(int64_t v) {
    if (v > 32767) return 32767;
    if (v < -32767) return -32767;
    return v;
}

/* One fit: F36 = the 6x6 rows F[k][l] of one (sector, mask), q6 = offsets. */
void orc_fit_one(const int16_t *F36, const int16_t *q6, const uint32_t *x6, uint32_t oshift,
                 uint32_t qshift, int64_t *y6, uint32_t *chi2) {
    uint64_t sum = 0;
    for (int k = 0; k < 6; ++k) {
        int64_t acc = (int64_t)q6[k] * ((int64_t)1 << qshift);
        for (int l = 0; l < 6; ++l) acc += (int64_t)F36[k * 6 + l] * (int64_t)x6[l];
        y6[k] = floor_div_pow2(acc, oshift);
    }
    for (int k = 3; k < 6; ++k) {
        int64_t c = clamp_chi(y6[k]);
        sum += (uint64_t)(c * c);
    }
    *chi2 = (uint32_t)sum;
}

/*
 * One road: n[l] hits per layer, coords[l*16 + i] = coordinate of hit i of
 * layer l.  Writes the 6-word output record.  When all_chi2 / all_y are given
 * they receive, for every evaluated combination c, its chi2 and its six y.
 * Returns the number of evaluated combinations.
 */
uint64_t orc_road(const uint32_t *n, const uint32_t *coords, uint32_t sector, uint32_t road_id,
                  const int16_t *F, const int16_t *q, const orc_config *cfg, uint32_t *rec,
                  uint32_t *all_chi2, int64_t *all_y) {
    uint32_t mask = 0, total_hits = 0, n_layers_hit = 0, flags = 0;
    for (int l = 0; l < 6; ++l) {
        total_hits += n[l];
        if (n[l] >= 1) { mask |= 1u << l; n_layers_hit += 1; }
    }
    if (total_hits == 0) flags |= ORC_F_NO_HITS;
    int have_best = 0;
    uint64_t best_c = 0;
    uint32_t best_chi2 = 0;
    int64_t best_y[3] = {0, 0, 0};
    uint64_t n_eval = 0;
    if (n_layers_hit < cfg->min_layers) {
        flags |= ORC_F_BAD_PATTERN;
    } else {
        /* with xft_pairs layer 5 is not a digit of its own (radix 1) */
        uint32_t radix[6];
        for (int l = 0; l < 6; ++l) radix[l] = (n[l] >= 1) ? n[l] : 1;
        if (cfg->xft_pairs) radix[5] = 1;
        uint64_t C = 1;
        for (int l = 0; l < 6; ++l) C *= radix[l];
        n_eval = C;
        if (C > cfg->max_comb) { flags |= ORC_F_OVERFLOW; n_eval = cfg->max_comb; }
        const int16_t *Fsm = F + ((uint64_t)sector * 64 + mask) * 36;
        const int16_t *qsm = q + ((uint64_t)sector * 64 + mask) * 6;
        for (uint64_t c = 0; c < n_eval; ++c) {
            uint32_t idx[6], x[6];
            uint64_t rem = c;
            for (int l = 5; l >= 0; --l) {
                idx[l] = (uint32_t)(rem % radix[l]);
                rem /= radix[l];
            }
            if (cfg->xft_pairs) idx[5] = idx[4];   /* the layer-4 hit's own partner */
            for (int l = 0; l < 6; ++l) x[l] = (n[l] >= 1) ? coords[l * 16 + idx[l]] : 0;
            int64_t y[6];
            uint32_t chi2;
            orc_fit_one(Fsm, qsm, x, cfg->oshift, cfg->qshift, y, &chi2);
            if (all_chi2) all_chi2[c] = chi2;
            if (all_y) for (int k = 0; k < 6; ++k) all_y[c * 6 + k] = y[k];
            if (chi2 <= cfg->chi2_cut && (!have_best || chi2 < best_chi2)) {
                have_best = 1;
                best_c = c;
                best_chi2 = chi2;
                for (int k = 0; k < 3; ++k) best_y[k] = y[k];
            }
        }
    }
    if (have_best) flags |= ORC_F_PASS;
    rec[0] = (road_id & 0x1FFFFFu) | (flags << 24);
    rec[1] = have_best ? (uint32_t)best_c : 0xFFFFFFFFu;
    rec[2] = have_best ? best_chi2 : 0;
    for (int k = 0; k < 3; ++k) rec[3 + k] = have_best ? (uint32_t)(int32_t)best_y[k] : 0;
    return n_eval;
}

/* Parse the road whose header is at word p (hits follow until a non-hit word
 * or the end of the event) into per-layer coordinate lists. */
static void parse_road(const uint32_t *words, uint64_t p, uint64_t end, uint32_t *n,
                       uint32_t *coords) {
    for (int l = 0; l < 6; ++l) n[l] = 0;
    for (uint64_t i = p + 1; i < end && w_type(words[i]) == 0; ++i) {
        uint32_t l = hit_layer(words[i]);
        if (l > 5 || n[l] >= 16) continue;  /* only reachable on unvalidated input */
        coords[l * 16 + n[l]] = hit_coord(words[i]);
        n[l] += 1;
    }
}

/* Events [e0, e1): the three nested loops.  Road r of the batch is written to
 * out[r*6 .. r*6+5], where road_base is the index of the first road of e0. */
static void run_events(const uint32_t *words, const uint64_t *event_off, uint64_t e0, uint64_t e1,
                       uint64_t road_base, const int16_t *F, const int16_t *q,
                       const orc_config *cfg, uint32_t *out) {
    uint64_t r = road_base;
    uint32_t n[6], coords[6 * 16];
    for (uint64_t e = e0; e < e1; ++e) {                                  /* loop 1: events */
        uint64_t start = event_off[e], end = event_off[e + 1];
        for (uint64_t p = start + 1; p < end; ++p) {                      /* loop 2: roads */
            if (w_type(words[p]) != 2) continue;
            parse_road(words, p, end, n, coords);
            orc_road(n, coords, rd_sector(words[p]), rd_id(words[p]), F, q, cfg, out + r * 6,
                     NULL, NULL);                                         /* loop 3 inside */
            r += 1;
        }
    }
}

/*
 * Whole batch.  Returns ORC_KEY_OK and writes *n_roads_out and out[R*6], or
 * returns the validation key (out untouched).  out_cap_roads bounds R.
 */
uint64_t orc_run(const uint32_t *words, uint64_t n_words, const uint64_t *event_off,
                 uint64_t n_events, const int16_t *F, const int16_t *q, const orc_config *cfg,
                 uint32_t *out, uint64_t out_cap_roads, uint64_t *n_roads_out) {
    if (!orc_config_ok(cfg)) return make_key(0, ORC_E_BAD_CONFIG);
    uint64_t key = orc_validate(words, n_words, event_off, n_events, cfg->n_sectors, cfg->xft_pairs);
    if (key != ORC_KEY_OK) return key;
    uint64_t R = 0;
    for (uint64_t e = 0; e < n_events; ++e) R += ev_nroads(words[event_off[e]]);
    *n_roads_out = R;
    if (R > out_cap_roads) return make_key(0, ORC_E_BAD_ARG);
    run_events(words, event_off, 0, n_events, 0, F, q, cfg, out);
    return ORC_KEY_OK;
}

/* Same result, one event per OpenMP thread (how the paper ran the loop over
 * events on the many-core coprocessor).  Used only to time the CPU baseline. */
uint64_t orc_run_omp(const uint32_t *words, uint64_t n_words, const uint64_t *event_off,
                     uint64_t n_events, const int16_t *F, const int16_t *q, const orc_config *cfg,
                     uint32_t *out, uint64_t out_cap_roads, uint64_t *n_roads_out) {
    if (!orc_config_ok(cfg)) return make_key(0, ORC_E_BAD_CONFIG);
    uint64_t key = orc_validate(words, n_words, event_off, n_events, cfg->n_sectors, cfg->xft_pairs);
    if (key != ORC_KEY_OK) return key;
    uint64_t *base = (uint64_t *)malloc((n_events + 1) * sizeof(uint64_t));
    if (!base) return make_key(0, ORC_E_BAD_ARG);
    base[0] = 0;
    for (uint64_t e = 0; e < n_events; ++e) base[e + 1] = base[e] + ev_nroads(words[event_off[e]]);
    *n_roads_out = base[n_events];
    if (base[n_events] > out_cap_roads) { free(base); return make_key(0, ORC_E_BAD_ARG); }
    long long ne = (long long)n_events;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long e = 0; e < ne; ++e)
        run_events(words, event_off, (uint64_t)e, (uint64_t)e + 1, base[e], F, q, cfg, out);
    free(base);
    return ORC_KEY_OK;
}

/* Records of selected roads only, given the word index of each road header
 * (hits follow it up to the next non-hit word, bounded by n_words).  Used to
 * check sampled roads of batches too large for a full oracle pass. */
void orc_run_roads(const uint32_t *words, uint64_t n_words, const uint64_t *road_pos,
                   uint64_t n_sel, const int16_t *F, const int16_t *q, const orc_config *cfg,
                   uint32_t *out) {
    uint32_t n[6], coords[6 * 16];
    for (uint64_t j = 0; j < n_sel; ++j) {
        uint64_t p = road_pos[j];
        parse_road(words, p, n_words, n, coords);
        orc_road(n, coords, rd_sector(words[p]), rd_id(words[p]), F, q, cfg, out + j * 6, NULL,
                 NULL);
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
