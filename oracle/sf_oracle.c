/*
 * sf_oracle.c -- plain, slow, sequential CPU oracle of the SF-sketch (SF_F form).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no source with the CUDA library.
 *
 * What it computes (Yang et al., "SF-sketch: A Two-stage Sketch for Data Streams"):
 *   - Slim-subsketch A: d arrays of w counters A_i[j]                    (Sec. 3.1, Table 1)
 *   - Fat-subsketch  B: d arrays of w buckets of z counters B_i[j][k];
 *     bucket chosen by h_i, counter inside the bucket by f_i;
 *     Slim and Fat share h_i                                             (Sec. 3.4, SF_4 structure;
 *                                                                         Sec. 3.5: SF_F = same structure)
 *   - insertion (SF_4 = SF_F insertion, Sec. 3.4 "Insertion"):
 *       B_i[h_i(e)][f_i(e)] += 1 for all i; Bmin = min over those d counters (after the increment);
 *       m = min_i A_i[h_i(e)]; if m < Bmin, every A_l[h_l(e)] equal to m is incremented by 1.
 *   - deletion (SF_F, Sec. 3.5 "Deletion"):
 *       B_i[h_i(e)][f_i(e)] -= 1; for each row i, if max_k B_i[h_i(e)][k] changed, then
 *       A_i[h_i(e)] is lowered to that maximum when it is larger; otherwise unchanged.
 *   - deletion, SF_4 variant (Sec. 3.4 "Deletion", kept for the ablation against SF_F):
 *       B_i[h_i(e)][f_i(e)] -= 1 for all i; then for each row i, A_i[h_i(e)] is decremented by 1
 *       when it is larger than the bucket sum sum_k B_i[h_i(e)][k].
 *   - query (Sec. 3.1 "Query"): min_i A_i[h_i(e)], Slim only.
 *
 * Indices are 0-based here (the paper is 1-based).  Counters are uint32 and wrap on
 * underflow, which only happens when a delete removes an occurrence that was never
 * inserted (the paper's proofs assume every delete removes an inserted occurrence).
 *
 * Two update semantics:
 *   SEQ      -- the paper's one-update-at-a-time rules above (literal delete rule, or the
 *               equivalent unconditional clamp, selectable).
 *   CHUNK(S) -- the batched schedule: the paper defines no batched update, so this one is a
 *               reading.  The call's stream is cut into chunks of S updates (the last may be
 *               short; a new call starts a new chunk).  With A0, B0 the state at chunk start:
 *                 1. B1 = B0 + sum of the chunk's +1/-1 updates (one counter per row each).
 *                 2. every distinct key e inserted at least once in the chunk gets
 *                    c_e = #inserts of e in the chunk, m_e = min_i A0_i[h_i(e)],
 *                    F_e = min_i B1_i[h_i(e)][f_i(e)], T_e = min(m_e + c_e, F_e).
 *                 3. every delete occurrence of e gets, per row i, M_i = max_k B1_i[h_i(e)][k].
 *                 4. the Slim ops are applied per counter in stream order:
 *                    an insert of e does A_i[h_i(e)] = max(A_i[h_i(e)], T_e),
 *                    a delete does A_i[h_i(e)] = min(A_i[h_i(e)], M_i).
 *               With S = 1 this reduces to SEQ (the raise max(A, min(m+1, F)) increments exactly
 *               the minimal rows when m < F; the clamp equals the literal delete rule because
 *               A_i[j] <= max_k B_i[j][k] always holds, Appendix I).
 *               SF_4 variant: step 3 takes the chunk-end bucket sum SUM_i = sum_k B1_i[h_i(e)][k]
 *               and step 4's delete does A_i[h_i(e)] -= 1 when A_i[h_i(e)] > SUM_i; with S = 1
 *               this is the SF_4 rule itself.
 *
 * Hash functions (the paper only asks for independent uniform h_i, f_i; this is a reading):
 *   row seeds s_0..s_{d-1} are the first d outputs of SplitMix64 started at the sketch seed
 *   (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014);
 *   mix64 is that generator's output finaliser.  Key words: x0 = bytes 0..7 little-endian
 *   (zero-padded for shorter keys), x1 = bytes 8..15 little-endian zero-padded (keys > 8 B).
 *   H_i = mix64(x0 ^ s_i) for keys <= 8 B, H_i = mix64(mix64(x0 ^ s_i) ^ x1) otherwise.
 *   h_i = (hi32(H_i) * w) >> 32,  f_i = (lo32(H_i) * z) >> 32
 *   (multiply-shift range reduction, Lemire, "Fast random integer generation in an interval",
 *   ACM TOMACS 2019).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OSF_GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

/* SplitMix64 output finaliser (Steele et al. 2014). */
uint64_t osf_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* One SplitMix64 step: advance the state by the golden gamma, return the mixed state. */
uint64_t osf_splitmix64_next(uint64_t *state)
{
    *state += OSF_GOLDEN_GAMMA;
    return osf_mix64(*state);
}

void osf_row_seeds(uint64_t seed, uint32_t d, uint64_t *out)
{
    uint64_t st = seed;
    for (uint32_t i = 0; i < d; i++)
        out[i] = osf_splitmix64_next(&st);
}

static uint64_t load_le(const uint8_t *p, uint32_t nbytes)
{
    uint64_t x = 0;
    for (uint32_t b = 0; b < nbytes; b++)
        x |= (uint64_t)p[b] << (8 * b);
    return x;
}

/* h and f of one key for one row (hash reading stated in the header). */
void osf_hash_row(const uint8_t *key, uint32_t key_bytes, uint64_t row_seed,
                  uint32_t w, uint32_t z, uint32_t *h, uint32_t *f)
{
    uint64_t x0 = load_le(key, key_bytes < 8 ? key_bytes : 8);
    uint64_t H = osf_mix64(x0 ^ row_seed);
    if (key_bytes > 8) {
        uint64_t x1 = load_le(key + 8, key_bytes - 8);
        H = osf_mix64(H ^ x1);
    }
    uint64_t hi = H >> 32, lo = H & 0xFFFFFFFFULL;
    *h = (uint32_t)((hi * (uint64_t)w) >> 32);
    *f = (uint32_t)((lo * (uint64_t)z) >> 32);
}

/* Index derivation for a batch of packed keys: h[t*d+i], f[t*d+i]. */
void osf_index_keys(const uint8_t *keys, uint32_t key_bytes, uint64_t n, uint64_t seed,
                    uint32_t d, uint32_t w, uint32_t z, uint32_t *h, uint32_t *f)
{
    uint64_t rs[64];
    osf_row_seeds(seed, d, rs);
    for (uint64_t t = 0; t < n; t++)
        for (uint32_t i = 0; i < d; i++)
            osf_hash_row(keys + t * key_bytes, key_bytes, rs[i], w, z,
                         &h[t * d + i], &f[t * d + i]);
}

static inline uint32_t *slim_at(uint32_t *A, uint32_t w, uint32_t i, uint32_t j)
{
    return &A[(uint64_t)i * w + j];
}

static inline uint32_t *fat_at(uint32_t *B, uint32_t w, uint32_t z, uint32_t i, uint32_t j, uint32_t k)
{
    return &B[((uint64_t)i * w + j) * z + k];
}

/* Sum of a bucket's z counters (64-bit: z counters of 32 bits each). */
static uint64_t bucket_sum(uint32_t *B, uint32_t w, uint32_t z, uint32_t i, uint32_t j)
{
    uint64_t s = 0;
    for (uint32_t k = 0; k < z; k++) s += *fat_at(B, w, z, i, j, k);
    return s;
}

static uint32_t bucket_max(uint32_t *B, uint32_t w, uint32_t z, uint32_t i, uint32_t j)
{
    uint32_t mx = 0;
    for (uint32_t k = 0; k < z; k++) {
        uint32_t v = *fat_at(B, w, z, i, j, k);
        if (v > mx) mx = v;
    }
    return mx;
}

/*
 * SEQ semantics, one update at a time, in stream order.
 * h, f: n*d indices; ops: +1 insert, -1 delete.
 * literal_delete == 1: the paper's SF_F delete rule with its "if the maximum changed" test;
 * literal_delete == 0: unconditional clamp A_i = min(A_i, max_k B_i[h][k]);
 * literal_delete == 2: the SF_4 delete rule (decrement by 1 above the bucket sum).
 */
void osf_seq_apply(uint32_t d, uint32_t w, uint32_t z, uint32_t *A, uint32_t *B,
                   const uint32_t *h, const uint32_t *f, const int8_t *ops, uint64_t n,
                   int literal_delete)
{
    for (uint64_t t = 0; t < n; t++) {
        const uint32_t *ht = h + t * d, *ft = f + t * d;
        if (ops[t] > 0) {
            /* Fat insertion, then Bmin over the d counters just incremented. */
            uint32_t Bmin = UINT32_MAX;
            for (uint32_t i = 0; i < d; i++) {
                uint32_t *c = fat_at(B, w, z, i, ht[i], ft[i]);
                *c += 1u;
            }
            for (uint32_t i = 0; i < d; i++) {
                uint32_t v = *fat_at(B, w, z, i, ht[i], ft[i]);
                if (v < Bmin) Bmin = v;
            }
            /* Slim: increment the smallest of the d hashed counters if below Bmin. */
            uint32_t m = UINT32_MAX;
            for (uint32_t i = 0; i < d; i++) {
                uint32_t v = *slim_at(A, w, i, ht[i]);
                if (v < m) m = v;
            }
            if (m < Bmin) {
                for (uint32_t i = 0; i < d; i++) {
                    uint32_t *a = slim_at(A, w, i, ht[i]);
                    if (*a == m) *a = m + 1u;
                }
            }
        } else if (ops[t] < 0 && literal_delete == 2) {
            for (uint32_t i = 0; i < d; i++)
                *fat_at(B, w, z, i, ht[i], ft[i]) -= 1u;
            for (uint32_t i = 0; i < d; i++) {
                uint32_t *a = slim_at(A, w, i, ht[i]);
                if ((uint64_t)*a > bucket_sum(B, w, z, i, ht[i])) *a -= 1u;
            }
        } else if (ops[t] < 0) {
            if (literal_delete) {
                for (uint32_t i = 0; i < d; i++) {
                    uint32_t before = bucket_max(B, w, z, i, ht[i]);
                    *fat_at(B, w, z, i, ht[i], ft[i]) -= 1u;
                    uint32_t after = bucket_max(B, w, z, i, ht[i]);
                    uint32_t *a = slim_at(A, w, i, ht[i]);
                    if (after != before && *a > after) *a = after;
                }
            } else {
                for (uint32_t i = 0; i < d; i++)
                    *fat_at(B, w, z, i, ht[i], ft[i]) -= 1u;
                for (uint32_t i = 0; i < d; i++) {
                    uint32_t mx = bucket_max(B, w, z, i, ht[i]);
                    uint32_t *a = slim_at(A, w, i, ht[i]);
                    if (*a > mx) *a = mx;
                }
            }
        }
    }
}

/* ---- CHUNK(S) ----------------------------------------------------------------- */

typedef struct {
    const uint8_t *ident;   /* key identity bytes of each update */
    uint32_t ident_bytes;
    uint64_t base;          /* first update of the chunk */
} sort_ctx;

static sort_ctx g_sort;     /* qsort has no context argument in C99 */

static int cmp_ident(const void *pa, const void *pb)
{
    uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
    int c = memcmp(g_sort.ident + (g_sort.base + a) * g_sort.ident_bytes,
                   g_sort.ident + (g_sort.base + b) * g_sort.ident_bytes, g_sort.ident_bytes);
    if (c) return c;
    return (a < b) ? -1 : (a > b);
}

/*
 * CHUNK(S) semantics (defined in the header comment).  ident: the key identity of every
 * update (the key bytes themselves, or a key id in explicit-index mode), used to find the
 * distinct keys of a chunk and their insert counts c_e.  delete_rule 0: SF_F (a delete
 * clamps to the chunk-end bucket maximum M_i); delete_rule 1: SF_4 (a delete decrements by 1
 * when above the chunk-end bucket sum, read as a 32-bit bound: a sum of 2^32 or more is never
 * exceeded).  Returns 0, or -1 on bad arguments or allocation failure.
 */
int osf_chunk_apply_rule(uint32_t d, uint32_t w, uint32_t z, uint32_t *A, uint32_t *B,
                         const uint32_t *h, const uint32_t *f, const int8_t *ops, uint64_t n,
                         uint64_t S, const uint8_t *ident, uint32_t ident_bytes, int delete_rule)
{
    if (S == 0 || d == 0 || w == 0 || z == 0) return -1;
    if (n == 0) return 0;
    uint64_t cmax = n < S ? n : S;
    uint64_t *order = (uint64_t *)malloc(cmax * sizeof(uint64_t));
    uint32_t *T = (uint32_t *)malloc(cmax * sizeof(uint32_t));       /* raise target per update */
    uint32_t *M = (uint32_t *)malloc(cmax * d * sizeof(uint32_t));   /* clamp bound per update, row */
    uint32_t *A0 = (uint32_t *)malloc((uint64_t)d * w * sizeof(uint32_t));
    if (!order || !T || !M || !A0) { free(order); free(T); free(M); free(A0); return -1; }

    for (uint64_t c0 = 0; c0 < n; c0 += S) {
        uint64_t len = (n - c0 < S) ? (n - c0) : S;

        /* 1. Fat: B1 = B0 + the chunk's updates. */
        memcpy(A0, A, (uint64_t)d * w * sizeof(uint32_t));
        for (uint64_t t = c0; t < c0 + len; t++)
            for (uint32_t i = 0; i < d; i++) {
                uint32_t *c = fat_at(B, w, z, i, h[t * d + i], f[t * d + i]);
                if (ops[t] > 0) *c += 1u;
                else if (ops[t] < 0) *c -= 1u;
            }

        /* 2. Distinct inserted keys: group the chunk by key identity. */
        for (uint64_t t = 0; t < len; t++) order[t] = t;
        g_sort.ident = ident; g_sort.ident_bytes = ident_bytes; g_sort.base = c0;
        qsort(order, len, sizeof(uint64_t), cmp_ident);
        uint64_t g0 = 0;
        while (g0 < len) {
            uint64_t g1 = g0 + 1;
            while (g1 < len &&
                   memcmp(ident + (c0 + order[g0]) * ident_bytes,
                          ident + (c0 + order[g1]) * ident_bytes, ident_bytes) == 0)
                g1++;
            uint64_t c_e = 0;
            for (uint64_t q = g0; q < g1; q++)
                if (ops[c0 + order[q]] > 0) c_e++;
            if (c_e > 0) {
                uint64_t t = c0 + order[g0];
                uint32_t m = UINT32_MAX, F = UINT32_MAX;
                for (uint32_t i = 0; i < d; i++) {
                    uint32_t a0 = *slim_at(A0, w, i, h[t * d + i]);
                    uint32_t b1 = *fat_at(B, w, z, i, h[t * d + i], f[t * d + i]);
                    if (a0 < m) m = a0;
                    if (b1 < F) F = b1;
                }
                uint64_t mc = (uint64_t)m + c_e;
                uint32_t Te = (mc < (uint64_t)F) ? (uint32_t)mc : F;
                for (uint64_t q = g0; q < g1; q++) T[order[q]] = Te;
            }
            g0 = g1;
        }

        /* 3. Bounds of the delete occurrences, from the chunk-end Fat. */
        for (uint64_t t = c0; t < c0 + len; t++)
            if (ops[t] < 0)
                for (uint32_t i = 0; i < d; i++)
                    M[(t - c0) * d + i] = bucket_max(B, w, z, i, h[t * d + i]);
        if (delete_rule == 1)
            for (uint64_t t = c0; t < c0 + len; t++)
                if (ops[t] < 0)
                    for (uint32_t i = 0; i < d; i++) {
                        uint64_t sb = bucket_sum(B, w, z, i, h[t * d + i]);
                        M[(t - c0) * d + i] = sb > UINT32_MAX ? UINT32_MAX : (uint32_t)sb;
                    }

        /* 4. Slim ops per counter in stream order. */
        for (uint64_t t = c0; t < c0 + len; t++) {
            for (uint32_t i = 0; i < d; i++) {
                uint32_t *a = slim_at(A, w, i, h[t * d + i]);
                if (ops[t] > 0) {
                    if (*a < T[t - c0]) *a = T[t - c0];
                } else if (ops[t] < 0) {
                    uint32_t mb = M[(t - c0) * d + i];
                    if (delete_rule == 1) {
                        if (*a > mb) *a -= 1u;
                    } else if (*a > mb) {
                        *a = mb;
                    }
                }
            }
        }
    }
    free(order); free(T); free(M); free(A0);
    return 0;
}

/* CHUNK(S) with the SF_F delete rule. */
int osf_chunk_apply(uint32_t d, uint32_t w, uint32_t z, uint32_t *A, uint32_t *B,
                    const uint32_t *h, const uint32_t *f, const int8_t *ops, uint64_t n,
                    uint64_t S, const uint8_t *ident, uint32_t ident_bytes)
{
    return osf_chunk_apply_rule(d, w, z, A, B, h, f, ops, n, S, ident, ident_bytes, 0);
}

/* Point query on a Slim-subsketch: out[t] = min_i A_i[h_i]. */
void osf_query_idx(uint32_t d, uint32_t w, const uint32_t *A, const uint32_t *h,
                   uint64_t n, uint32_t *out)
{
    for (uint64_t t = 0; t < n; t++) {
        uint32_t m = UINT32_MAX;
        for (uint32_t i = 0; i < d; i++) {
            uint32_t v = A[(uint64_t)i * w + h[t * d + i]];
            if (v < m) m = v;
        }
        out[t] = m;
    }
}
