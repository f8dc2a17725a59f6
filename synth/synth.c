/*
 * Seeded synthetic inputs for RotorMap: reference genomes and planted reads.
 *
 * This module is shared by the FP64 oracle's tests and by the GPU path's
 * tests and benchmark. It holds none of the method's arithmetic (no s-mer
 * codes, no phases, no embeddings, no scores): it only draws DNA letters.
 *
 *   - synth_uniform_ref:  i.i.d. uniform A/C/G/T.
 *   - synth_markov_ref:   order-2 Markov chain at a target GC content with
 *                         CpG depletion, plus planted tandem repeats,
 *                         segmental duplicates and interspersed repeat
 *                         families (the human/maize-shaped genomes).
 *   - synth_reads:        reads sampled at uniform true positions, walked
 *                         along the reference with substitutions and
 *                         geometric-length insertions/deletions.
 *
 * Random numbers come from xoshiro256** seeded through splitmix64, so every
 * output is a pure function of its arguments and seed on any platform.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint64_t s[4];
} rng_t;

static uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static void rng_seed(rng_t* r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t* r) {
  uint64_t* s = r->s;
  const uint64_t result = rotl(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return result;
}

/* uniform double in [0, 1) */
static inline double rng_uniform(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, n) (Lemire's multiply-shift; n > 0) */
static inline uint64_t rng_below(rng_t* r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)rng_next(r) * (unsigned __int128)n) >> 64);
}

static double rng_normal(rng_t* r) {
  double u1 = rng_uniform(r), u2 = rng_uniform(r);
  if (u1 < 1e-300) u1 = 1e-300;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Gamma(a, 1) by Marsaglia and Tsang (a >= 1 branch; a < 1 boosted). */
static double rng_gamma(rng_t* r, double a) {
  if (a < 1.0) {
    double u = rng_uniform(r);
    if (u < 1e-300) u = 1e-300;
    return rng_gamma(r, a + 1.0) * pow(u, 1.0 / a);
  }
  const double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  for (;;) {
    double x = rng_normal(r), v = 1.0 + c * x;
    if (v <= 0) continue;
    v = v * v * v;
    double u = rng_uniform(r);
    if (u < 1.0 - 0.0331 * x * x * x * x) return d * v;
    if (log(u) < 0.5 * x * x + d * (1.0 - v + log(v))) return d * v;
  }
}

/* number of failures+1 before success: Geometric(p) on {1, 2, ...} */
static int rng_geometric(rng_t* r, double p) {
  int n = 1;
  while (rng_uniform(r) >= p && n < 1000) ++n;
  return n;
}

static const char kLetters[4] = {'A', 'C', 'G', 'T'};

static inline int letter_index(char c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return 0;
  }
}

/* a letter different from c, uniform among the other three */
static inline char substitute(rng_t* r, char c) {
  int i = letter_index(c);
  int j = (int)rng_below(r, 3);
  if (j >= i) ++j;
  return kLetters[j];
}

/* ------------------------------------------------------------------------ */

int64_t synth_uniform_ref(char* out, int64_t L, uint64_t seed) {
  rng_t r;
  rng_seed(&r, seed);
  int64_t i = 0;
  for (; i + 32 <= L; i += 32) {
    uint64_t x = rng_next(&r);
    for (int j = 0; j < 32; ++j) out[i + j] = kLetters[(x >> (2 * j)) & 3];
  }
  if (i < L) {
    uint64_t x = rng_next(&r);
    for (int j = 0; i < L; ++i, ++j) out[i] = kLetters[(x >> (2 * j)) & 3];
  }
  return L;
}

/* ------------------------------------------------------------------------ */
/* order-2 Markov chain                                                      */

typedef struct {
  double p[16][4]; /* P(next | prev2*4 + prev1) */
  double cdf[16][4];
} markov_t;

static void markov_build(markov_t* mk, double gc, rng_t* r) {
  const double base[4] = {(1 - gc) / 2, gc / 2, gc / 2, (1 - gc) / 2};
  const double alpha = 50.0;
  for (int ctx = 0; ctx < 16; ++ctx) {
    double s = 0;
    for (int b = 0; b < 4; ++b) {
      mk->p[ctx][b] = rng_gamma(r, alpha * base[b]) + 1e-9;
      s += mk->p[ctx][b];
    }
    for (int b = 0; b < 4; ++b) mk->p[ctx][b] /= s;
    /* CpG depletion: after a C, G is four times rarer */
    if ((ctx & 3) == 1) {
      mk->p[ctx][2] *= 0.25;
      double t = 0;
      for (int b = 0; b < 4; ++b) t += mk->p[ctx][b];
      for (int b = 0; b < 4; ++b) mk->p[ctx][b] /= t;
    }
  }
  /* rescale C/G mass until the stationary GC is within 0.5% of the target */
  for (int iter = 0; iter < 200; ++iter) {
    double pi[16], nxt[16];
    for (int i = 0; i < 16; ++i) pi[i] = 1.0 / 16;
    for (int it = 0; it < 500; ++it) {
      for (int i = 0; i < 16; ++i) nxt[i] = 0;
      for (int ctx = 0; ctx < 16; ++ctx)
        for (int b = 0; b < 4; ++b) nxt[((ctx & 3) << 2) | b] += pi[ctx] * mk->p[ctx][b];
      for (int i = 0; i < 16; ++i) pi[i] = nxt[i];
    }
    double cur = 0;
    for (int ctx = 0; ctx < 16; ++ctx)
      if ((ctx & 3) == 1 || (ctx & 3) == 2) cur += pi[ctx];
    if (fabs(cur - gc) < 0.002) break;
    double f = sqrt(gc / cur * (1 - cur) / (1 - gc));
    for (int ctx = 0; ctx < 16; ++ctx) {
      double t = 0;
      mk->p[ctx][1] *= f;
      mk->p[ctx][2] *= f;
      for (int b = 0; b < 4; ++b) t += mk->p[ctx][b];
      for (int b = 0; b < 4; ++b) mk->p[ctx][b] /= t;
    }
  }
  for (int ctx = 0; ctx < 16; ++ctx) {
    double c = 0;
    for (int b = 0; b < 4; ++b) {
      c += mk->p[ctx][b];
      mk->cdf[ctx][b] = c;
    }
    mk->cdf[ctx][3] = 1.0;
  }
}

static void markov_fill(const markov_t* mk, char* out, int64_t n, rng_t* r) {
  int ctx = (int)rng_below(r, 16);
  for (int64_t i = 0; i < n; ++i) {
    double u = rng_uniform(r);
    int b = 0;
    while (b < 3 && u >= mk->cdf[ctx][b]) ++b;
    out[i] = kLetters[b];
    ctx = ((ctx & 3) << 2) | b;
  }
}

/* copy src[0..len) to dst with substitution rate mu and small indels at
 * rate mu/10 (length-preserving: a deletion is padded by a duplicated base) */
static void mutated_copy(char* dst, const char* src, int64_t len, double mu, rng_t* r) {
  int64_t j = 0;
  for (int64_t i = 0; i < len && j < len; ++i) {
    double u = rng_uniform(r);
    if (u < mu) {
      dst[j++] = substitute(r, src[i]);
    } else if (u < mu * 1.05) {
      /* deletion of src[i] */
    } else if (u < mu * 1.10) {
      dst[j++] = kLetters[rng_below(r, 4)];
      if (j < len) dst[j++] = src[i];
    } else {
      dst[j++] = src[i];
    }
  }
  while (j < len) dst[j++] = kLetters[rng_below(r, 4)];
}

/*
 * Order-2 Markov genome with planted repeats. Fractions are of L and are
 * reached approximately (copies may overlap earlier ones).
 *   tandem_frac:       tandem arrays, unit 2-50 bp, array 100-2000 bp, 1% mutations
 *   segdup_frac:       segmental duplicates of 1-10 kbp at 95-99% identity
 *   interspersed_frac: copies of 500 repeat families (consensus 300 bp - 6 kbp)
 *                      at 70-99% identity
 */
int64_t synth_markov_ref(char* out, int64_t L, double gc, double tandem_frac, double segdup_frac,
                         double interspersed_frac, uint64_t seed) {
  rng_t r;
  rng_seed(&r, seed);
  markov_t mk;
  markov_build(&mk, gc, &r);
  markov_fill(&mk, out, L, &r);

  /* interspersed repeat families */
  if (interspersed_frac > 0 && L > 20000) {
    const int n_fam = 500;
    int64_t* fam_off = (int64_t*)malloc(sizeof(int64_t) * (n_fam + 1));
    int64_t total = 0;
    int lens[500];
    for (int f = 0; f < n_fam; ++f) {
      /* log-uniform consensus length in [300, 6000] */
      lens[f] = (int)(300.0 * exp(rng_uniform(&r) * log(20.0)));
      fam_off[f] = total;
      total += lens[f];
    }
    fam_off[n_fam] = total;
    char* cons = (char*)malloc((size_t)total);
    markov_fill(&mk, cons, total, &r);
    char* buf = (char*)malloc(6001);
    int64_t target = (int64_t)(interspersed_frac * (double)L), placed = 0;
    while (placed < target) {
      int f = (int)rng_below(&r, n_fam);
      int len = lens[f];
      if (len >= L) break;
      /* copies are often truncated fragments of the consensus */
      int frag = rng_uniform(&r) < 0.5 ? len : 100 + (int)rng_below(&r, (uint64_t)(len > 100 ? len - 99 : 1));
      if (frag > len) frag = len;
      int start = (int)rng_below(&r, (uint64_t)(len - frag + 1));
      double ident = 0.70 + 0.29 * rng_uniform(&r);
      mutated_copy(buf, cons + fam_off[f] + start, frag, 1.0 - ident, &r);
      int64_t pos = (int64_t)rng_below(&r, (uint64_t)(L - frag));
      memcpy(out + pos, buf, (size_t)frag);
      placed += frag;
    }
    free(buf);
    free(cons);
    free(fam_off);
  }

  /* segmental duplicates */
  if (segdup_frac > 0 && L > 30000) {
    int64_t target = (int64_t)(segdup_frac * (double)L), placed = 0;
    char* buf = (char*)malloc(10001);
    while (placed < target) {
      int len = 1000 + (int)rng_below(&r, 9001);
      int64_t src = (int64_t)rng_below(&r, (uint64_t)(L - len));
      int64_t dst = (int64_t)rng_below(&r, (uint64_t)(L - len));
      double ident = 0.95 + 0.04 * rng_uniform(&r);
      mutated_copy(buf, out + src, len, 1.0 - ident, &r);
      memcpy(out + dst, buf, (size_t)len);
      placed += len;
    }
    free(buf);
  }

  /* tandem repeats */
  if (tandem_frac > 0 && L > 4000) {
    int64_t target = (int64_t)(tandem_frac * (double)L), placed = 0;
    char unit[64];
    while (placed < target) {
      int ulen = 2 + (int)rng_below(&r, 49);
      int alen = 100 + (int)rng_below(&r, 1901);
      markov_fill(&mk, unit, ulen, &r);
      int64_t pos = (int64_t)rng_below(&r, (uint64_t)(L - alen));
      for (int i = 0; i < alen; ++i) {
        char c = unit[i % ulen];
        out[pos + i] = rng_uniform(&r) < 0.01 ? substitute(&r, c) : c;
      }
      placed += alen;
    }
  }
  return L;
}

/* ------------------------------------------------------------------------ */

/*
 * Planted reads. For read i a target length is fixed (len_mode 0: len_median
 * exactly; 1: lognormal with median len_median and log-sd len_sigma, clipped
 * to [len_min, len_max]); a true start p is drawn uniformly; the reference is
 * walked from p emitting bases until the read has its length:
 *   per reference base, with probability sub_rate emit a substitution;
 *   with probability indel_rate start an indel event, insertion or deletion
 *   with equal odds, of length Geometric(geom_p) on {1, 2, ...};
 *   otherwise copy the base.
 * Outputs: concatenated reads (out_seqs, capacity out_cap bytes), offsets
 * (n+1), true start, reference span consumed, total edit length, length.
 * Returns the number of bytes written, or -1 if out_cap is too small.
 */
int64_t synth_reads(const char* ref, int64_t L, int64_t n, int32_t len_mode, double len_median,
                    double len_sigma, int32_t len_min, int32_t len_max, double sub_rate, double indel_rate,
                    double geom_p, uint64_t seed, char* out_seqs, int64_t out_cap, int64_t* offsets,
                    int64_t* true_pos, int32_t* true_span, int32_t* n_edits, int32_t* lengths) {
  rng_t r;
  rng_seed(&r, seed);
  int64_t off = 0;
  offsets[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int len;
    if (len_mode == 0) {
      len = (int)len_median;
    } else {
      double x = len_median * exp(len_sigma * rng_normal(&r));
      if (x < len_min) x = len_min;
      if (x > len_max) x = len_max;
      len = (int)x;
    }
    if (off + len > out_cap) return -1;
    int64_t margin = (int64_t)len / 2 + 64;
    if (L <= (int64_t)len + margin) return -1;
    for (int attempt = 0;; ++attempt) {
      int64_t p = (int64_t)rng_below(&r, (uint64_t)(L - len - margin));
      int64_t q = p;
      int j = 0, edits = 0;
      char* o = out_seqs + off;
      while (j < len && q < L) {
        double u = rng_uniform(&r);
        if (u < sub_rate) {
          o[j++] = substitute(&r, ref[q++]);
          ++edits;
        } else if (u < sub_rate + indel_rate) {
          int el = rng_geometric(&r, geom_p);
          edits += el;
          if (rng_uniform(&r) < 0.5) {
            for (int e = 0; e < el && j < len; ++e) o[j++] = kLetters[rng_below(&r, 4)];
          } else {
            q += el;
          }
        } else {
          o[j++] = ref[q++];
        }
      }
      if (j == len) {
        true_pos[i] = p;
        true_span[i] = (int32_t)(q - p);
        n_edits[i] = edits;
        lengths[i] = len;
        break;
      }
      if (attempt > 1000) return -1;
    }
    off += len;
    offsets[i + 1] = off;
  }
  return off;
}
