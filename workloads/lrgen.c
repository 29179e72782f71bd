/*
 * Seeded synthetic inputs for the longest-repeat query, and the untimed host
 * preparation of their suffix, rank and lcp arrays.
 *
 * This file holds no part of the longest-repeat method itself: it makes the
 * strings S and the arrays SA, Rank and LCP that the method takes as input
 * (the paper builds these on the host before any query, Section 4, and
 * excludes that time from its measurements, Section 5).  Both the CPU oracle
 * and the CUDA path are fed from here, and neither shares anything else.
 *
 * Conventions (0-based): sa[r] is the start of the r-th smallest suffix,
 * rank[sa[r]] = r, and lcp has n+1 entries with lcp[0] = lcp[n] = 0 and
 * lcp[r] = |lcp(S[sa[r-1]..], S[sa[r]..])| for 1 <= r < n (the paper's
 * LCP[1..n+1] shifted down by one, Section 3).
 *
 * Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), written here from
 * its published definition.  Everything is plain C99 + OpenMP, with no
 * architecture-specific code, so x86_64 and aarch64 produce identical bytes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* PRNG                                                                      */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t x; } rng_t;

static inline uint64_t rng_next(rng_t* r) {
    uint64_t z = (r->x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* uniform double in [0,1) from the top 53 bits */
static inline double rng_unif(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, m) (m > 0); the modulo bias is below 2^-40 for m < 2^24 */
static inline uint64_t rng_below(rng_t* r, uint64_t m) { return rng_next(r) % m; }
/* uniform integer in [lo, hi] */
static inline int64_t rng_range(rng_t* r, int64_t lo, int64_t hi) { return lo + (int64_t)rng_below(r, (uint64_t)(hi - lo + 1)); }

static rng_t rng_seed(uint64_t seed, uint64_t stream) {
    rng_t r; r.x = seed * 0xD1B54A32D192ED03ull + stream * 0x8CB92BA72F3D8DD7ull + 0x2545F4914F6CDD1Dull;
    rng_next(&r); rng_next(&r);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Generators                                                                */
/* ------------------------------------------------------------------------ */

static const char DNA[4] = {'A', 'C', 'G', 'T'};
static const char PROT[20] = {'A','C','D','E','F','G','H','I','K','L','M','N','P','Q','R','S','T','V','W','Y'};

/* i.i.d. uniform symbols from `alphabet` (sigma symbols). */
void gen_iid(uint8_t* out, int64_t n, const uint8_t* alphabet, int sigma, uint64_t seed) {
    rng_t r = rng_seed(seed, 1);
    for (int64_t i = 0; i < n; ++i) out[i] = alphabet[rng_below(&r, (uint64_t)sigma)];
}

/*
 * DNA-like text: an order-2 Markov background (16 contexts, each with four
 * transition probabilities drawn as seeded uniforms and normalised), then
 * planted repeats: copies of earlier segments of length uniform in
 * [seg_min, seg_max], each copy with its own point-mutation rate uniform in
 * [0, mut_max] (a mutated base becomes one of the three other bases), until
 * the copied lengths add up to `cover` * n.  Copies are written in order of
 * generation; a later copy may overwrite part of an earlier one.
 */
void gen_dna_planted(uint8_t* out, int64_t n, uint64_t seed,
                     int64_t seg_min, int64_t seg_max, double mut_max, double cover) {
    rng_t r = rng_seed(seed, 2);
    double cdf[16][4];
    for (int c = 0; c < 16; ++c) {
        double w[4], s = 0;
        for (int b = 0; b < 4; ++b) { w[b] = 0.05 + rng_unif(&r); s += w[b]; }
        double acc = 0;
        for (int b = 0; b < 4; ++b) { acc += w[b] / s; cdf[c][b] = acc; }
        cdf[c][3] = 1.0;
    }
    int p1 = 0, p2 = 0;
    for (int64_t i = 0; i < n; ++i) {
        int c = p2 * 4 + p1;
        double u = rng_unif(&r);
        int b = 0;
        while (b < 3 && u >= cdf[c][b]) ++b;
        out[i] = (uint8_t)DNA[b];
        p2 = p1; p1 = b;
    }
    if (n < 2 * seg_min) return;
    int64_t planted = 0, target = (int64_t)(cover * (double)n);
    rng_t rp = rng_seed(seed, 3);
    while (planted < target) {
        int64_t len = rng_range(&rp, seg_min, seg_max);
        if (len * 2 > n) len = n / 2;
        /* destination anywhere; source strictly before it and not overlapping */
        int64_t dst = rng_range(&rp, len, n - len);
        int64_t src = rng_range(&rp, 0, dst - len);
        double mu = rng_unif(&rp) * mut_max;
        for (int64_t t = 0; t < len; ++t) {
            uint8_t ch = out[src + t];
            if (rng_unif(&rp) < mu) {
                int cur = (ch == 'A') ? 0 : (ch == 'C') ? 1 : (ch == 'G') ? 2 : 3;
                cur = (cur + 1 + (int)rng_below(&rp, 3)) & 3;
                ch = (uint8_t)DNA[cur];
            }
            out[dst + t] = ch;
        }
        planted += len;
    }
}

/*
 * Protein-like text: i.i.d. uniform over the 20 amino-acid letters, then
 * tandem arrays (a random unit of length [unit_min, unit_max] repeated
 * [copies_min, copies_max] times back to back) written at random places
 * until they cover `tandem_frac` * n positions.
 */
void gen_protein_tandem(uint8_t* out, int64_t n, uint64_t seed, double tandem_frac,
                        int unit_min, int unit_max, int copies_min, int copies_max) {
    rng_t r = rng_seed(seed, 4);
    for (int64_t i = 0; i < n; ++i) out[i] = (uint8_t)PROT[rng_below(&r, 20)];
    int64_t covered = 0, target = (int64_t)(tandem_frac * (double)n);
    uint8_t unit[64];
    while (covered < target) {
        int u = (int)rng_range(&r, unit_min, unit_max);
        int c = (int)rng_range(&r, copies_min, copies_max);
        int64_t len = (int64_t)u * c;
        if (len >= n) { c = (int)(n / u); len = (int64_t)u * c; if (c < 1) break; }
        for (int t = 0; t < u; ++t) unit[t] = (uint8_t)PROT[rng_below(&r, 20)];
        int64_t at = rng_range(&r, 0, n - len);
        for (int64_t t = 0; t < len; ++t) out[at + t] = unit[t % u];
        covered += len;
    }
}

/*
 * English-like text over a 96-symbol alphabet (printable ASCII 32..126 plus
 * newline): a vocabulary of `vocab` words, each of length uniform in [2, 12]
 * over a-z; words are drawn with Zipf(s) probabilities over their rank and
 * separated by a space (probability 0.85), else by one of the 68 printable
 * symbols that are not a-z followed by a space, or by a newline (0.01).
 */
void gen_english(uint8_t* out, int64_t n, uint64_t seed, int vocab, double zipf_s) {
    rng_t r = rng_seed(seed, 5);
    int64_t* woff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(vocab + 1));
    uint8_t* wchars = (uint8_t*)malloc((size_t)vocab * 12);
    double* cdf = (double*)malloc(sizeof(double) * (size_t)vocab);
    woff[0] = 0;
    for (int w = 0; w < vocab; ++w) {
        int len = (int)rng_range(&r, 2, 12);
        for (int t = 0; t < len; ++t) wchars[woff[w] + t] = (uint8_t)('a' + rng_below(&r, 26));
        woff[w + 1] = woff[w] + len;
    }
    double acc = 0;
    for (int w = 0; w < vocab; ++w) { acc += pow((double)(w + 1), -zipf_s); cdf[w] = acc; }
    for (int w = 0; w < vocab; ++w) cdf[w] /= acc;
    cdf[vocab - 1] = 1.0;
    uint8_t punct[68];
    int np = 0;
    for (int ch = 33; ch <= 126; ++ch) if (ch < 'a' || ch > 'z') punct[np++] = (uint8_t)ch;
    int64_t i = 0;
    while (i < n) {
        double u = rng_unif(&r);
        int lo = 0, hi = vocab - 1;          /* first w with cdf[w] > u */
        while (lo < hi) { int mid = (lo + hi) / 2; if (cdf[mid] > u) hi = mid; else lo = mid + 1; }
        for (int64_t t = woff[lo]; t < woff[lo + 1] && i < n; ++t) out[i++] = wchars[t];
        double v = rng_unif(&r);
        if (v < 0.01) { if (i < n) out[i++] = '\n'; }
        else if (v < 0.01 + 0.85) { if (i < n) out[i++] = ' '; }
        else {
            if (i < n) out[i++] = punct[rng_below(&r, (uint64_t)np)];
            if (i < n) out[i++] = ' ';
        }
    }
    free(woff); free(wchars); free(cdf);
}

/* log-uniform and lognormal length draws for the batched and serving mixes */
void gen_lengths_loguniform(int64_t* out, int64_t count, int64_t lo, int64_t hi, uint64_t seed) {
    rng_t r = rng_seed(seed, 6);
    double a = log((double)lo), b = log((double)hi);
    for (int64_t j = 0; j < count; ++j) {
        int64_t v = (int64_t)floor(exp(a + (b - a) * rng_unif(&r)));
        out[j] = v < lo ? lo : (v > hi ? hi : v);
    }
}

void gen_lengths_lognormal(int64_t* out, int64_t count, double median, double sigma,
                           int64_t floor_len, int64_t cap, uint64_t seed) {
    rng_t r = rng_seed(seed, 7);
    for (int64_t j = 0; j < count; ++j) {
        /* Box-Muller from two uniforms */
        double u1 = rng_unif(&r), u2 = rng_unif(&r);
        if (u1 < 1e-300) u1 = 1e-300;
        double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
        int64_t v = (int64_t)floor(median * exp(sigma * z));
        out[j] = v < floor_len ? floor_len : (v > cap ? cap : v);
    }
}

/* uniform doubles for Poisson inter-arrival draws (host side turns them into exponentials) */
void gen_uniforms(double* out, int64_t count, uint64_t seed) {
    rng_t r = rng_seed(seed, 8);
    for (int64_t j = 0; j < count; ++j) out[j] = rng_unif(&r);
}

/* ------------------------------------------------------------------------ */
/* Sorting helpers for the suffix-array prep                                 */
/* ------------------------------------------------------------------------ */

/* LSD radix sort of (key, val) pairs by 64-bit key, 8-bit digits, parallel;
 * digits on which every key agrees are skipped.  Result in key/val. */
static void radix_sort_kv(uint64_t* key, int32_t* val, int64_t n, uint64_t* tk, int32_t* tv) {
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
    if (n < (1 << 16) || omp_in_parallel()) nt = 1;
#endif
    int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * 256 * (size_t)nt);
    uint64_t* sk = key; int32_t* sv = val; uint64_t* dk = tk; int32_t* dv = tv;
    for (int pass = 0; pass < 8; ++pass) {
        int shift = pass * 8;
        memset(hist, 0, sizeof(int64_t) * 256 * (size_t)nt);
#pragma omp parallel for schedule(static, 1) num_threads(nt)
        for (int t = 0; t < nt; ++t) {
            int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            int64_t* h = hist + 256 * t;
            for (int64_t i = lo; i < hi; ++i) h[(sk[i] >> shift) & 255]++;
        }
        int uniform = 0;
        for (int d = 0; d < 256; ++d) {
            int64_t tot = 0;
            for (int t = 0; t < nt; ++t) tot += hist[256 * t + d];
            if (tot == n) uniform = 1;
        }
        if (uniform) continue;
        int64_t run = 0;
        for (int d = 0; d < 256; ++d)
            for (int t = 0; t < nt; ++t) { int64_t c = hist[256 * t + d]; hist[256 * t + d] = run; run += c; }
#pragma omp parallel for schedule(static, 1) num_threads(nt)
        for (int t = 0; t < nt; ++t) {
            int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            int64_t* h = hist + 256 * t;
            for (int64_t i = lo; i < hi; ++i) {
                int64_t p = h[(sk[i] >> shift) & 255]++;
                dk[p] = sk[i]; dv[p] = sv[i];
            }
        }
        uint64_t* xk = sk; sk = dk; dk = xk;
        int32_t* xv = sv; sv = dv; dv = xv;
    }
    if (sk != key) { memcpy(key, sk, sizeof(uint64_t) * (size_t)n); memcpy(val, sv, sizeof(int32_t) * (size_t)n); }
    free(hist);
}

/* sequential sort of packed uint64 values (insertion sort for short runs,
 * LSD radix otherwise) */
static void sort_u64_seq(uint64_t* a, int64_t n, uint64_t* tmp) {
    if (n < 48) {
        for (int64_t i = 1; i < n; ++i) {
            uint64_t x = a[i]; int64_t j = i - 1;
            while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
            a[j + 1] = x;
        }
        return;
    }
    int64_t cnt[256];
    uint64_t* s = a; uint64_t* d = tmp;
    for (int pass = 0; pass < 8; ++pass) {
        int shift = pass * 8;
        memset(cnt, 0, sizeof(cnt));
        for (int64_t i = 0; i < n; ++i) cnt[(s[i] >> shift) & 255]++;
        int uniform = 0;
        for (int dgt = 0; dgt < 256; ++dgt) if (cnt[dgt] == n) uniform = 1;
        if (uniform) continue;
        int64_t run = 0;
        for (int dgt = 0; dgt < 256; ++dgt) { int64_t c = cnt[dgt]; cnt[dgt] = run; run += c; }
        for (int64_t i = 0; i < n; ++i) d[cnt[(s[i] >> shift) & 255]++] = s[i];
        uint64_t* x = s; s = d; d = x;
    }
    if (s != a) memcpy(a, s, sizeof(uint64_t) * (size_t)n);
}

/* ------------------------------------------------------------------------ */
/* Suffix array by prefix doubling                                           */
/* ------------------------------------------------------------------------ */

/*
 * Suffix array of s[0..n) by prefix doubling (Manber and Myers; refinement
 * of unsorted groups only, as in Larsson and Sadakane).  Suffixes are first
 * radix-sorted by their first K symbols packed into a 64-bit key (symbols
 * mapped to 1..sigma, 0 past the end of the string, so a shorter suffix sorts
 * first); then, with h the prefix length already sorted, every group of
 * suffixes that share an h-prefix is sorted by the group id of the suffix h
 * positions later and split, and h doubles, until every group is a singleton.
 * `rank` is scratch of n int32 and ends as the inverse of sa.
 * Returns 0, or -1 if n is out of range or memory runs out.
 */
int prep_sa(const uint8_t* s, int64_t n, int32_t* sa, int32_t* rank) {
    if (n <= 0 || n > 2147483646) return -1;
    if (n == 1) { sa[0] = 0; rank[0] = 0; return 0; }
    int code[256]; int sigma = 0;
    {
        int seen[256] = {0};
        for (int64_t i = 0; i < n; ++i) seen[s[i]] = 1;
        for (int c = 0; c < 256; ++c) code[c] = seen[c] ? ++sigma : 0;
    }
    int bits = 1;
    while ((1 << bits) < sigma + 1) ++bits;
    int K = 64 / bits;
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t* tk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    int32_t* tv = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!key || !tk || !tv) { free(key); free(tk); free(tv); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k = 0;
        for (int t = 0; t < K; ++t) {
            uint64_t c = (i + t < n) ? (uint64_t)code[s[i + t]] : 0;
            k = (k << bits) | c;
        }
        key[i] = k; sa[i] = (int32_t)i;
    }
    radix_sort_kv(key, sa, n, tk, tv);
    free(tv);
    /* group ids: the sorted index of the group's first member */
    int64_t ngroups_open = 0;
    int64_t* gstart = NULL; int64_t* gend = NULL; int64_t gcap = 0;
    {
        int64_t j = 0;
        while (j < n) {
            int64_t e = j + 1;
            while (e < n && key[e] == key[j]) ++e;
            for (int64_t t = j; t < e; ++t) rank[sa[t]] = (int32_t)j;
            if (e - j > 1) {
                if (ngroups_open == gcap) {
                    gcap = gcap ? gcap * 2 : 1024;
                    gstart = (int64_t*)realloc(gstart, sizeof(int64_t) * (size_t)gcap);
                    gend = (int64_t*)realloc(gend, sizeof(int64_t) * (size_t)gcap);
                }
                gstart[ngroups_open] = j; gend[ngroups_open] = e; ++ngroups_open;
            }
            j = e;
        }
    }
    /* key/tk are reused as packed (next-group-id + 1) << 32 | suffix */
    int64_t h = K;
    while (ngroups_open > 0) {
        /* phase A: every open group's keys from the current (h-) group ids */
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t g = 0; g < ngroups_open; ++g) {
            for (int64_t t = gstart[g]; t < gend[g]; ++t) {
                int64_t i = sa[t];
                uint64_t nxt = (i + h < n) ? (uint64_t)rank[i + h] + 1 : 0;
                key[t] = (nxt << 32) | (uint64_t)(uint32_t)i;
            }
        }
        /* phase B: sort each group and assign new group ids */
        int64_t* split_cnt = (int64_t*)calloc((size_t)ngroups_open, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t g = 0; g < ngroups_open; ++g) {
            int64_t a = gstart[g], b = gend[g];
            sort_u64_seq(key + a, b - a, tk + a);
            int64_t j = a, opened = 0;
            while (j < b) {
                int64_t e = j + 1;
                while (e < b && (key[e] >> 32) == (key[j] >> 32)) ++e;
                for (int64_t t = j; t < e; ++t) {
                    int32_t i = (int32_t)(uint32_t)(key[t] & 0xffffffffu);
                    sa[t] = i;
                    rank[i] = (int32_t)j;
                }
                if (e - j > 1) ++opened;
                j = e;
            }
            split_cnt[g] = opened;
        }
        int64_t nnew = 0;
        for (int64_t g = 0; g < ngroups_open; ++g) nnew += split_cnt[g];
        int64_t* ns = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnew ? nnew : 1));
        int64_t* ne = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnew ? nnew : 1));
        int64_t w = 0;
        for (int64_t g = 0; g < ngroups_open; ++g) {
            if (!split_cnt[g]) continue;
            int64_t a = gstart[g], b = gend[g], j = a;
            while (j < b) {
                int64_t e = j + 1;
                while (e < b && (key[e] >> 32) == (key[j] >> 32)) ++e;
                if (e - j > 1) { ns[w] = j; ne[w] = e; ++w; }
                j = e;
            }
        }
        free(split_cnt); free(gstart); free(gend);
        gstart = ns; gend = ne; ngroups_open = nnew;
        h *= 2;
    }
    free(gstart); free(gend); free(key); free(tk);
    /* group ids of singletons are their sorted indices, so rank is the inverse of sa */
    return 0;
}

/*
 * LCP array (n+1 entries, lcp[0] = lcp[n] = 0) from s, sa and rank by
 * Kasai et al.'s method (CPM 2001): walking the text left to right, the lcp
 * of suffix i with its predecessor in sa is at least the previous one minus 1.
 * The text is cut into chunks that run in parallel; each chunk starts its
 * running length at 0, which is only slower, not wrong.
 */
void prep_lcp(const uint8_t* s, int64_t n, const int32_t* sa, const int32_t* rank, int32_t* lcp) {
    lcp[0] = 0; lcp[n] = 0;
    int nchunks = 1;
#ifdef _OPENMP
    nchunks = omp_get_max_threads() * 8;
    if (n < (1 << 16)) nchunks = 1;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < nchunks; ++c) {
        int64_t lo = n * c / nchunks, hi = n * (c + 1) / nchunks;
        int64_t hh = 0;
        for (int64_t i = lo; i < hi; ++i) {
            int64_t r = rank[i];
            if (r == 0) { hh = 0; continue; }
            int64_t j = sa[r - 1];
            while (i + hh < n && j + hh < n && s[i + hh] == s[j + hh]) ++hh;
            lcp[r] = (int32_t)hh;
            if (hh > 0) --hh;
        }
    }
}

/* Suffix, rank and lcp arrays of s; rank must hold n entries, lcp n+1. */
int prep_all(const uint8_t* s, int64_t n, int32_t* sa, int32_t* rank, int32_t* lcp) {
    if (n == 0) { lcp[0] = 0; return 0; }   /* empty string: its lcp array is the one sentinel */
    int rc = prep_sa(s, n, sa, rank);
    if (rc) return rc;
    prep_lcp(s, n, sa, rank, lcp);
    return 0;
}

/*
 * Prep for many strings packed back to back: string j occupies
 * s[off[j] .. off[j+1]); its sa and rank (local, 0-based) go to the same
 * offsets and its lcp (n_j + 1 entries) to lcp[off[j] + j ..].  Strings run
 * in parallel, one thread each.
 */
int prep_many(const uint8_t* s, const int64_t* off, int64_t count, int32_t* sa, int32_t* rank, int32_t* lcp) {
    int err = 0;
    /* nested parallel regions inside run on one thread each */
#pragma omp parallel for schedule(dynamic, 1) reduction(|:err)
    for (int64_t j = 0; j < count; ++j) {
        int64_t a = off[j], nj = off[j + 1] - off[j];
        err |= prep_all(s + a, nj, sa + a, rank + a, lcp + a + j) ? 1 : 0;
    }
    return err ? -1 : 0;
}

int lrgen_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
