/*
 * CPU FP64 oracle for embedding-based ad retrieval with an explicit
 * cross-feature (HitMatch) term.  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the benchmark's CPU-baseline leg call it; the library never
 * does.  It shares no code with the CUDA path.
 *
 * Everything is plain and slow on purpose.  Floating point is FP64; FP32
 * inputs are widened exactly.  Each function cites the passage it follows.
 *
 * Score of ad a for user u (Eq. 1 plus the HitMatch equation, Sec. 3.3):
 *     s(u, a) = <h_u, h_a> + sum_m w_m x_m L[a, m]
 * With synthetic cross features x = 1 and one feature per (pair (i, j),
 * user value u_i, ad value v), L[a, (i, j, u_i, v)] = [val_j(a) == v], so the
 * wide term is  sum_{(i, j) in P} w_ij(u_i, val_j(a)).
 *
 * Cross weights w_ij(u, v) come either from one dense table per pair
 * (row-major [u][v]) or from one shared table of 2^bits floats addressed by
 *     idx = splitmix64((p << 40) | (u << 20) | v) & (2^bits - 1),
 * where splitmix64(x) is the first output of Vigna's SplitMix64 generator
 * seeded with x (state += 0x9E3779B97F4A7C15, then the two xor-shift-multiply
 * rounds and a final xor-shift).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
/* An ad field without a value: the ad lacks that feature (its row of the
 * 0/1 matrix L has no non-zero in that field's key range). */
#define ORC_EMPTY 0xFFFFFFFFu

/* ------------------------------------------------------------------ */
/* Cross weights                                                       */
/* ------------------------------------------------------------------ */

uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct {
  uint32_t f_u, f_a;
  const uint32_t *vocab_u;  /* [F_u] */
  const uint32_t *vocab_a;  /* [F_a] */
  uint32_t n_pairs;
  const uint32_t *pairs;    /* [P][2] = (user field i, ad field j) */
  int hashed;               /* 0 = dense tables, 1 = hashed table */
  const float *w_table;
  const uint64_t *w_off;    /* [P] dense-table starts */
  uint32_t hash_bits;
} orc_cross;

/* w_ij(u, v) for cross pair p = (i, j). */
static double orc_weight(const orc_cross *c, uint32_t p, uint32_t u, uint32_t v) {
  if (c->hashed) {
    uint64_t x = ((uint64_t)p << 40) | ((uint64_t)u << 20) | (uint64_t)v;
    uint64_t idx = orc_splitmix64(x) & ((1ULL << c->hash_bits) - 1ULL);
    return (double)c->w_table[idx];
  }
  uint32_t j = c->pairs[2 * p + 1];
  return (double)c->w_table[c->w_off[p] + (uint64_t)u * c->vocab_a[j] + v];
}

/* ------------------------------------------------------------------ */
/* O1: brute force from raw per-ad values (the definition)             */
/* ------------------------------------------------------------------ */

/*
 * scores[a] = sum_t h_u[t] h_a[t] + sum_{(i,j) in P} w_ij(user[i], ad_vals[a][j])
 * cond[a]   = sum_t |h_u[t] h_a[t]| + sum_{(i,j) in P} |w_ij(...)|   (may be NULL)
 * Eq. 1 (Sec. 3.1), HitMatch equation (Sec. 3.3).
 */
int orc_scores_brute(uint32_t n_ads, uint32_t d, const float *h_u, const float *emb,
                     const orc_cross *c, const uint32_t *ad_vals, const uint32_t *user,
                     double *scores, double *cond) {
  for (uint32_t i = 0; i < c->f_u; i++)
    if (user[i] >= c->vocab_u[i]) return ORC_EINVAL;
  for (uint32_t a = 0; a < n_ads; a++) {
    double dot = 0.0, mag = 0.0;
    for (uint32_t t = 0; t < d; t++) {
      double prod = (double)h_u[t] * (double)emb[(uint64_t)a * d + t];
      dot += prod;
      mag += fabs(prod);
    }
    double wide = 0.0;
    for (uint32_t p = 0; p < c->n_pairs; p++) {
      uint32_t i = c->pairs[2 * p], j = c->pairs[2 * p + 1];
      uint32_t v = ad_vals[(uint64_t)a * c->f_a + j];
      if (v == ORC_EMPTY) continue;
      if (v >= c->vocab_a[j]) return ORC_EINVAL;
      double w = orc_weight(c, p, user[i], v);
      wide += w;
      mag += fabs(w);
    }
    scores[a] = dot + wide;
    if (cond) cond[a] = mag;
  }
  return ORC_OK;
}

/* user_ptr [F_u + 1] must start at 0 and not decrease; every value must lie
 * in its field's vocabulary. */
static int orc_check_seq(const orc_cross *c, const uint32_t *user_ptr,
                         const uint32_t *user_vals) {
  if (user_ptr[0] != 0) return ORC_EINVAL;
  for (uint32_t i = 0; i < c->f_u; i++) {
    if (user_ptr[i + 1] < user_ptr[i]) return ORC_EINVAL;
    for (uint32_t r = user_ptr[i]; r < user_ptr[i + 1]; r++)
      if (user_vals[r] >= c->vocab_u[i]) return ORC_EINVAL;
  }
  return ORC_OK;
}

/*
 * Multi-valued user fields (a user's history: field i holds the values
 * user_vals[user_ptr[i] .. user_ptr[i+1]), possibly none).  Each (user
 * value u, ad value v) of a cross pair (i, j) is one hit feature with x = 1
 * (HitMatch equation, Sec. 3.3), so
 *   scores[a] = sum_t h_u[t] h_a[t]
 *             + sum_{(i,j) in P} sum_{u in field i} w_ij(u, ad_vals[a][j]),
 * the pair's terms absent when ad field j is ORC_EMPTY.  With one value per
 * field this is orc_scores_brute, term for term in the same order.
 */
int orc_scores_brute_seq(uint32_t n_ads, uint32_t d, const float *h_u, const float *emb,
                         const orc_cross *c, const uint32_t *ad_vals, const uint32_t *user_ptr,
                         const uint32_t *user_vals, double *scores, double *cond) {
  if (orc_check_seq(c, user_ptr, user_vals) != ORC_OK) return ORC_EINVAL;
  for (uint32_t a = 0; a < n_ads; a++) {
    double dot = 0.0, mag = 0.0;
    for (uint32_t t = 0; t < d; t++) {
      double prod = (double)h_u[t] * (double)emb[(uint64_t)a * d + t];
      dot += prod;
      mag += fabs(prod);
    }
    double wide = 0.0;
    for (uint32_t p = 0; p < c->n_pairs; p++) {
      uint32_t i = c->pairs[2 * p], j = c->pairs[2 * p + 1];
      uint32_t v = ad_vals[(uint64_t)a * c->f_a + j];
      if (v == ORC_EMPTY) continue;
      if (v >= c->vocab_a[j]) return ORC_EINVAL;
      for (uint32_t r = user_ptr[i]; r < user_ptr[i + 1]; r++) {
        double w = orc_weight(c, p, user_vals[r], v);
        wide += w;
        mag += fabs(w);
      }
    }
    scores[a] = dot + wide;
    if (cond) cond[a] = mag;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Query expansion: the non-zero (k, w_hat) of a request               */
/* ------------------------------------------------------------------ */

/*
 * The query of Algorithm 2 is the set of non-zero feature values with their
 * weights, w_hat = w * x (Sec. 3.4, "sparse matrix multiplication L w~").
 * Cross features sharing an ad-field key k = key_off[j] + v fold into one
 * entry:  w_hat[k] = sum_{i : (i, j) in P} w_ij(user[i], v).
 * Output is dense over the key space: w_hat[k] for k < key_off[F_a]
 * (zero for ad fields that take part in no pair).
 */
int orc_expand(const orc_cross *c, const uint32_t *key_off, const uint32_t *user,
               double *w_hat) {
  uint32_t n_keys = key_off[c->f_a];
  for (uint32_t k = 0; k < n_keys; k++) w_hat[k] = 0.0;
  for (uint32_t i = 0; i < c->f_u; i++)
    if (user[i] >= c->vocab_u[i]) return ORC_EINVAL;
  for (uint32_t p = 0; p < c->n_pairs; p++) {
    uint32_t i = c->pairs[2 * p], j = c->pairs[2 * p + 1];
    for (uint32_t v = 0; v < c->vocab_a[j]; v++)
      w_hat[key_off[j] + v] += orc_weight(c, p, user[i], v);
  }
  return ORC_OK;
}

/*
 * The expansion for multi-valued user fields:
 *   w_hat[key_off[j] + v] = sum_{i : (i, j) in P} sum_{u in field i} w_ij(u, v).
 */
int orc_expand_seq(const orc_cross *c, const uint32_t *key_off, const uint32_t *user_ptr,
                   const uint32_t *user_vals, double *w_hat) {
  uint32_t n_keys = key_off[c->f_a];
  for (uint32_t k = 0; k < n_keys; k++) w_hat[k] = 0.0;
  if (orc_check_seq(c, user_ptr, user_vals) != ORC_OK) return ORC_EINVAL;
  for (uint32_t p = 0; p < c->n_pairs; p++) {
    uint32_t i = c->pairs[2 * p], j = c->pairs[2 * p + 1];
    for (uint32_t r = user_ptr[i]; r < user_ptr[i + 1]; r++)
      for (uint32_t v = 0; v < c->vocab_a[j]; v++)
        w_hat[key_off[j] + v] += orc_weight(c, p, user_vals[r], v);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* O2: inverted-list oracle from uncompressed postings                 */
/* ------------------------------------------------------------------ */

/*
 * scores[a] = <h_u, h_a> + sum over query entries (k, w) of w * L[a, k],
 * walking the uncompressed posting pairs (key, ad), which must be distinct
 * (each is one non-zero of the 0/1 matrix L; orc_unique_pairs collapses
 * repeats).  Duplicate query keys add (linearity).  This is the product L w~
 * of Sec. 3.4 evaluated key by key.
 */
int orc_scores_postings(uint32_t n_ads, uint32_t d, const float *h_u, const float *emb,
                        uint32_t n_keys, uint64_t nnz, const uint32_t *post_key,
                        const uint32_t *post_ad, uint32_t n_q, const uint32_t *q_key,
                        const double *q_w, double *scores) {
  double *w_of_key = (double *)calloc(n_keys ? n_keys : 1, sizeof(double));
  if (!w_of_key) return ORC_ENOMEM;
  for (uint32_t q = 0; q < n_q; q++) {
    if (q_key[q] >= n_keys) { free(w_of_key); return ORC_EINVAL; }
    w_of_key[q_key[q]] += q_w[q];
  }
  for (uint32_t a = 0; a < n_ads; a++) {
    double dot = 0.0;
    for (uint32_t t = 0; t < d; t++) dot += (double)h_u[t] * (double)emb[(uint64_t)a * d + t];
    scores[a] = dot;
  }
  for (uint64_t e = 0; e < nnz; e++) {
    if (post_key[e] >= n_keys || post_ad[e] >= n_ads) { free(w_of_key); return ORC_EINVAL; }
    scores[post_ad[e]] += w_of_key[post_key[e]];
  }
  free(w_of_key);
  return ORC_OK;
}

/*
 * L is a 0/1 matrix (Sec. 3.3): a (key, ad) pair listed more than once is
 * still one non-zero.  Writes the distinct pairs (sorted by key, then ad)
 * and returns their number.
 */
static int cmp_u64(const void *x, const void *y);
int64_t orc_unique_pairs(uint64_t nnz, const uint32_t *key, const uint32_t *ad,
                         uint32_t *out_key, uint32_t *out_ad) {
  uint64_t *kv = (uint64_t *)malloc((nnz ? nnz : 1) * sizeof(uint64_t));
  if (!kv) return ORC_ENOMEM;
  for (uint64_t e = 0; e < nnz; e++) kv[e] = ((uint64_t)key[e] << 32) | ad[e];
  qsort(kv, nnz, sizeof(uint64_t), cmp_u64);
  uint64_t m = 0;
  for (uint64_t e = 0; e < nnz; e++) {
    if (e > 0 && kv[e] == kv[e - 1]) continue;
    out_key[m] = (uint32_t)(kv[e] >> 32);
    out_ad[m] = (uint32_t)kv[e];
    m++;
  }
  free(kv);
  return (int64_t)m;
}

/* ------------------------------------------------------------------ */
/* O3: Algorithm 1 (indexing) and its decoder                          */
/* ------------------------------------------------------------------ */

static int cmp_u64(const void *x, const void *y) {
  uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* g = ceil(log2 n) for n >= 1 (Logarithmic Categorization, Sec. 3.4). */
static uint32_t ceil_log2(uint32_t n) {
  uint32_t g = 0;
  while ((1u << g) < n) g++;
  return g;
}

typedef struct {
  uint32_t n_keys;
  uint64_t n_blocks[9];
  uint32_t *keys[9];    /* [n_keys + 1] CSR row pointer per group */
  uint32_t *header[9];  /* [n_blocks[g]]: v >> 8 of the block's ads */
  uint8_t *values[9];   /* [n_blocks[g] << g]: v & 255, sorted, zero padded */
} orc_index;

/*
 * Algorithm 1.  Step 1 (Block Grouping): each pair (k, v) puts the low byte
 * l = v mod 2^8 into the set B[k, h], h = floor(v / 2^8).  Sets are kept as
 * sorted, duplicate-free runs: the pairs are sorted by (k, h, l) with a
 * library sort and repeated pairs dropped.  Step 2 (Group Partitioning): a
 * block of n ads goes to group g = ceil(log2 n) and is padded with 0 to 2^g
 * slots.  Step 3 (SoA storage): per group, header[g] and values[g] in (k, h)
 * order, and keys[g][k] = number of group-g blocks whose key is below k, so a
 * key's blocks are keys[g][k] .. keys[g][k + 1] - 1.
 *
 * Readings where the algorithm as printed is ambiguous: the low bytes of a
 * block are stored ascending and distinct, so slot 0 always holds a real ad
 * and a later zero byte is padding; keys[g] is a row pointer of n_keys + 1
 * entries (the printed loop appends k rather than an offset).
 */
int orc_build_index(uint32_t n_keys, uint32_t n_ads, uint64_t nnz, const uint32_t *post_key,
                    const uint32_t *post_ad, orc_index *out) {
  memset(out, 0, sizeof(*out));
  out->n_keys = n_keys;
  uint64_t *kv = (uint64_t *)malloc((nnz ? nnz : 1) * sizeof(uint64_t));
  if (!kv) return ORC_ENOMEM;
  for (uint64_t e = 0; e < nnz; e++) {
    if (post_key[e] >= n_keys || post_ad[e] >= n_ads) { free(kv); return ORC_EINVAL; }
    uint32_t v = post_ad[e];
    uint32_t h = v >> 8, l = v & 255u;
    kv[e] = ((uint64_t)post_key[e] << 32) | ((uint64_t)h << 8) | l;
  }
  /* Step 1: B[k, h] as sorted distinct runs. */
  qsort(kv, nnz, sizeof(uint64_t), cmp_u64);
  uint64_t m = 0;
  for (uint64_t e = 0; e < nnz; e++)
    if (m == 0 || kv[e] != kv[m - 1]) kv[m++] = kv[e];

  /* Step 2: size class of each block; count blocks per group. */
  for (int pass = 0; pass < 2; pass++) {
    uint64_t fill[9] = {0};
    if (pass == 1) {
      for (int g = 0; g < 9; g++) {
        out->keys[g] = (uint32_t *)calloc((size_t)n_keys + 1, sizeof(uint32_t));
        out->header[g] = (uint32_t *)malloc((out->n_blocks[g] ? out->n_blocks[g] : 1) * 4);
        out->values[g] = (uint8_t *)calloc((out->n_blocks[g] << g) ? (out->n_blocks[g] << g) : 1, 1);
        if (!out->keys[g] || !out->header[g] || !out->values[g]) { free(kv); return ORC_ENOMEM; }
      }
    }
    uint64_t e = 0;
    while (e < m) {
      uint64_t kh = kv[e] >> 8, end = e;
      while (end < m && (kv[end] >> 8) == kh) end++;
      uint32_t n = (uint32_t)(end - e);
      uint32_t g = ceil_log2(n);
      if (pass == 0) {
        out->n_blocks[g]++;
      } else {
        /* Step 3: append header and the padded low bytes, in (k, h) order. */
        uint64_t b = fill[g]++;
        uint32_t k = (uint32_t)(kh >> 24);
        out->header[g][b] = (uint32_t)(kh & 0xFFFFFFu);
        for (uint32_t s = 0; s < n; s++) out->values[g][(b << g) + s] = (uint8_t)(kv[e + s] & 255u);
        out->keys[g][k + 1]++;  /* count, prefix-summed below */
      }
      e = end;
    }
  }
  for (int g = 0; g < 9; g++)
    for (uint32_t k = 0; k < n_keys; k++) out->keys[g][k + 1] += out->keys[g][k];
  free(kv);
  return ORC_OK;
}

void orc_free_index(orc_index *ix) {
  for (int g = 0; g < 9; g++) {
    free(ix->keys[g]);
    free(ix->header[g]);
    free(ix->values[g]);
    ix->keys[g] = NULL; ix->header[g] = NULL; ix->values[g] = NULL;
  }
}

/*
 * Decoder (Algorithm 2's inner loop without the scatter): every real slot of
 * every block gives one (key, ad) pair, ad = h * 2^8 + l.  Slot s of a block
 * is real iff s == 0 or its byte is non-zero.  Writes at most cap pairs and
 * returns the number of pairs found (or a negative error).
 */
int64_t orc_decode_index(const uint32_t *const keys[9], const uint32_t *const header[9],
                         const uint8_t *const values[9], uint32_t n_keys, uint32_t *out_key,
                         uint32_t *out_ad, uint64_t cap) {
  uint64_t n = 0;
  for (int g = 0; g < 9; g++) {
    for (uint32_t k = 0; k < n_keys; k++) {
      for (uint32_t b = keys[g][k]; b < keys[g][k + 1]; b++) {
        uint32_t h = header[g][b];
        for (uint32_t s = 0; s < (1u << g); s++) {
          uint8_t l = values[g][((uint64_t)b << g) + s];
          if (s == 0 || l != 0) {
            if (n < cap) { out_key[n] = k; out_ad[n] = h * 256u + l; }
            n++;
          }
        }
      }
    }
  }
  return (int64_t)n;
}

/* ------------------------------------------------------------------ */
/* O4: top-K by full sort                                              */
/* ------------------------------------------------------------------ */

typedef struct { double s; uint32_t id; } orc_pair;

static int cmp_rank(const void *x, const void *y) {
  const orc_pair *a = (const orc_pair *)x, *b = (const orc_pair *)y;
  if (a->s > b->s) return -1;
  if (a->s < b->s) return 1;
  return a->id < b->id ? -1 : (a->id > b->id ? 1 : 0);
}

/*
 * The K ads with the largest score among those whose filter bit is set
 * (filter == NULL keeps all), ordered by score descending then id ascending.
 * Returns the number written (min(K, #eligible)).
 */
int64_t orc_topk(uint32_t n, const double *scores, const uint64_t *filter, uint32_t k,
                 uint32_t *out_ids, double *out_scores) {
  orc_pair *v = (orc_pair *)malloc((n ? n : 1) * sizeof(orc_pair));
  if (!v) return ORC_ENOMEM;
  uint32_t m = 0;
  for (uint32_t a = 0; a < n; a++) {
    if (filter && !((filter[a >> 6] >> (a & 63)) & 1ULL)) continue;
    v[m].s = scores[a];
    v[m].id = a;
    m++;
  }
  qsort(v, m, sizeof(orc_pair), cmp_rank);
  uint32_t r = m < k ? m : k;
  for (uint32_t i = 0; i < r; i++) { out_ids[i] = v[i].id; out_scores[i] = v[i].s; }
  free(v);
  return r;
}

/* ------------------------------------------------------------------ */
/* O5: BF16 and FP8-e4m3 quantisers, written from the format specs     */
/* ------------------------------------------------------------------ */

static float f32_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_from_f32(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* Value of a bfloat16 encoding: the top half of an IEEE binary32. */
float orc_bf16_value(uint16_t h) { return f32_from_bits((uint32_t)h << 16); }

/*
 * Round a binary32 to the nearest bfloat16, ties to the even encoding.
 * NaN stays NaN (quiet); values beyond the largest finite bfloat16 round to
 * infinity exactly as the round-to-nearest rule gives.
 */
uint16_t orc_bf16_rne(float x) {
  uint32_t b = bits_from_f32(x);
  if ((b & 0x7F800000u) == 0x7F800000u && (b & 0x007FFFFFu)) return (uint16_t)((b >> 16) | 0x40u);
  uint16_t lo = (uint16_t)(b >> 16);        /* truncation toward zero */
  uint16_t hi = (uint16_t)(lo + 1);         /* next encoding away from zero */
  double xv = (double)x;
  double dlo = fabs(xv - (double)orc_bf16_value(lo));
  double vhi = (double)orc_bf16_value(hi);
  double dhi = isinf(vhi) ? INFINITY : fabs(vhi - xv);
  if ((b & 0xFFFFu) == 0) return lo;
  if (isinf(vhi)) {
    /* Past the largest finite value: halfway point is 2^128 - 2^119 (Inf's
     * "virtual" neighbour); round-to-nearest sends ties and above to Inf. */
    double maxf = (double)orc_bf16_value(lo);
    double half = maxf + ldexp(1.0, 119);
    return fabs(xv) >= half ? hi : lo;
  }
  if (dlo < dhi) return lo;
  if (dhi < dlo) return hi;
  return (lo & 1u) ? hi : lo;
}

/*
 * Value of an FP8 E4M3 encoding (OCP 8-bit floating point, E4M3 variant):
 * sign bit, 4 exponent bits with bias 7, 3 mantissa bits.  Exponent field 0
 * is subnormal (2^-6 * m/8); S.1111.111 is NaN; there is no infinity; the
 * largest finite magnitude is 1.75 * 2^8 = 448.
 */
double orc_fp8_e4m3_value(uint8_t c) {
  int s = c >> 7, e = (c >> 3) & 15, m = c & 7;
  if (e == 15 && m == 7) return NAN;
  double mag = e == 0 ? ldexp((double)m / 8.0, -6) : ldexp(1.0 + (double)m / 8.0, e - 7);
  return s ? -mag : mag;
}

/*
 * Nearest E4M3 encoding to x, ties to the encoding with an even mantissa,
 * magnitudes above 448 saturate to +-448, NaN maps to 0x7F.  Found by search
 * over all finite encodings of x's sign.
 */
uint8_t orc_fp8_e4m3_rne_sat(float x) {
  if (isnan(x)) return 0x7F;
  int neg = signbit(x) ? 1 : 0;
  double ax = fabs((double)x);
  if (ax >= 448.0) return (uint8_t)((neg << 7) | 0x7E);
  int best = 0;
  double bestd = INFINITY;
  for (int c = 0; c < 0x7F; c++) {  /* positive finite encodings 0x00 .. 0x7E */
    double dv = fabs(orc_fp8_e4m3_value((uint8_t)c) - ax);
    if (dv < bestd || (dv == bestd && (c & 1) == 0)) { bestd = dv; best = c; }
  }
  return (uint8_t)((neg << 7) | best);
}

/*
 * Per-row FP8 quantisation of an [n][d] FP32 matrix: scale = max_t |x_t| / 448
 * (1 if the row is all zero), q_t = E4M3(x_t / scale).  The division and the
 * scale are binary32 operations, the precision the quantiser works in.
 */
void orc_quantize_fp8_rows(uint64_t n, uint32_t d, const float *x, uint8_t *q, float *scale) {
  for (uint64_t r = 0; r < n; r++) {
    float mx = 0.0f;
    for (uint32_t t = 0; t < d; t++) {
      float a = fabsf(x[r * d + t]);
      if (a > mx) mx = a;
    }
    volatile float sc = mx > 0.0f ? mx / 448.0f : 1.0f;
    scale[r] = sc;
    for (uint32_t t = 0; t < d; t++) {
      volatile float y = x[r * d + t] / sc;
      q[r * d + t] = orc_fp8_e4m3_rne_sat(y);
    }
  }
}

void orc_quantize_bf16(uint64_t n, const float *x, uint16_t *out) {
  for (uint64_t i = 0; i < n; i++) out[i] = orc_bf16_rne(x[i]);
}
