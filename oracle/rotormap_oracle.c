/*
 * RotorMap FP64 CPU oracle — TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct implementation of what the GPU path
 * computes, written from the paper's definitions. It shares no code, header,
 * table or constant generator with the CUDA library, and the CUDA library
 * never calls it. Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Every floating-point quantity is FP64. Phases are reduced exactly in
 * integers before the trigonometric call: the factor f_k is held as a
 * fraction a_k/q, and the angle of location loc is 2*pi*((a_k*loc) mod qN)/(qN).
 *
 * Parity status of each function is stated at the function; all functions
 * here are pinned by tests/test_oracle_pins.py unless marked otherwise.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559

/* ---------------------------------------------------------------------- */
/* Letters and s-mers (§2.1)                                               */

/* A,C,G,T (either case) -> 0,1,2,3; anything else -> -1. */
int oracle_base(int c) {
  switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
  }
}

/* 2-bit packing: base i occupies bits 2*(i mod 16) of word i/16; unused high
 * bits of the last word are zero. Returns -1 on success, else the index of the
 * first letter outside {A,C,G,T}. */
int64_t oracle_pack_2bit(const uint8_t* seq, int64_t len, uint32_t* out) {
  int64_t n_words = (len + 15) / 16;
  for (int64_t w = 0; w < n_words; ++w) out[w] = 0;
  for (int64_t i = 0; i < len; ++i) {
    int b = oracle_base(seq[i]);
    if (b < 0) return i;
    out[i / 16] |= (uint32_t)b << (2 * (i % 16));
  }
  return -1;
}

/* s-mer code at location p: sum_{i<s} base(p+i) * 4^(s-1-i) (first letter most
 * significant). Caller guarantees valid letters. */
static uint32_t mer_code(const uint8_t* seq, int64_t p, int s) {
  uint32_t c = 0;
  for (int i = 0; i < s; ++i) c = c * 4u + (uint32_t)oracle_base(seq[p + i]);
  return c;
}

/* Default 4^s -> 4^t map of the compact version (§2.6). The paper leaves the
 * map to its external code; the reading taken here is the identity when s == t
 * and Knuth's multiplicative (Fibonacci) hash otherwise:
 *   bin = (code * 0x9E3779B97F4A7C15 mod 2^64) >> (64 - 2t). */
void oracle_default_bin_map(int s, int t, uint16_t* map) {
  uint64_t n = 1ull << (2 * s);
  for (uint64_t code = 0; code < n; ++code) {
    if (s == t) {
      map[code] = (uint16_t)code;
    } else {
      uint64_t h = code * 0x9E3779B97F4A7C15ull;
      map[code] = (uint16_t)(h >> (64 - 2 * t));
    }
  }
}

/* bins of every location 0..len-s; returns 0, or -1 on an invalid letter */
int oracle_mer_bins(const uint8_t* seq, int64_t len, int s, const uint16_t* map, int32_t* out) {
  for (int64_t i = 0; i < len; ++i)
    if (oracle_base(seq[i]) < 0) return -1;
  for (int64_t p = 0; p + s <= len; ++p) out[p] = map[mer_code(seq, p, s)];
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Multiplicity factors                                                     */

/* f_k as the exact fraction a/q (k = 1..m).
 *   variant 0, default (§2.2 Eq. mult-factor): f_k = k.
 *   variant 1, fine-tuned (§3.3 Eq. mult-factor-finetune):
 *       f_k = 2(k-1)/(m-1) + 1 = (2k + m - 3)/(m - 1); for m = 1 the formula
 *       divides by zero and f_1 = 1 is taken. */
void oracle_factor(int m, int variant, int k, int64_t* a, int64_t* q) {
  if (variant == 1 && m > 1) {
    *a = 2 * (int64_t)k + m - 3;
    *q = m - 1;
  } else {
    *a = k;
    *q = 1;
  }
}

/* e^{2 pi i f_k loc / N} with the exponent reduced exactly in integers */
static void unit_root(int64_t a, int64_t q, int64_t N, int64_t loc, double* re, double* im) {
  int64_t Q = q * N;
  int64_t r = (int64_t)(((__int128)a * (__int128)loc) % (__int128)Q);
  if (r < 0) r += Q;
  double ang = TWO_PI * (double)r / (double)Q;
  *re = cos(ang);
  *im = sin(ang);
}

/* ---------------------------------------------------------------------- */
/* Embedding by direct summation                                            */

/*
 * RoPE_{s,m(,t)} of a length-N string, unnormalised (§2.1 Eq. for c_mer, §2.2
 * Eq. mult-factor, §2.3 concatenation over k, §2.6 compact map, §3.3
 * fine-tuned factors):
 *     c_{k,b} = sum over loc in [0, N-s] with bin(mer(loc)) = b of
 *               exp(2 pi i f_k loc / N).
 * Output vector is band-major: index (k-1)*4^t + b, D = m*4^t complex entries.
 * Returns 0, or -1 on an invalid letter.
 */
int oracle_embed(const uint8_t* seq, int N, int s, int m, int t, int variant, const uint16_t* map, double* re,
                 double* im) {
  const int nb = 1 << (2 * t);
  const int D = m * nb;
  for (int i = 0; i < D; ++i) re[i] = im[i] = 0.0;
  for (int i = 0; i < N; ++i)
    if (oracle_base(seq[i]) < 0) return -1;
  for (int loc = 0; loc <= N - s; ++loc) {
    int b = map[mer_code(seq, loc, s)];
    for (int k = 1; k <= m; ++k) {
      int64_t a, q;
      oracle_factor(m, variant, k, &a, &q);
      double c, sn;
      unit_root(a, q, N, loc, &c, &sn);
      re[(k - 1) * nb + b] += c;
      im[(k - 1) * nb + b] += sn;
    }
  }
  return 0;
}

/*
 * The same vector in the matrix form of §2.10: sum over loc of
 *     D^loc (ones(m) (x) onehot(bin(mer(loc)))),
 * D = diag((w^{f_1},...,w^{f_m}) (x) ones(4^t)), w = exp(2 pi i / N).
 * D^loc is formed by repeated multiplication by D (loc matrix products of a
 * diagonal matrix, stored as its diagonal), an arithmetic path independent of
 * the reduced-angle evaluation in oracle_embed.
 */
int oracle_embed_matrix_form(const uint8_t* seq, int N, int s, int m, int t, int variant, const uint16_t* map,
                             double* re, double* im) {
  const int nb = 1 << (2 * t);
  const int D = m * nb;
  double* dr = (double*)malloc(sizeof(double) * D);
  double* di = (double*)malloc(sizeof(double) * D);
  double* pr = (double*)malloc(sizeof(double) * D);
  double* pi = (double*)malloc(sizeof(double) * D);
  double* v = (double*)malloc(sizeof(double) * D);
  for (int i = 0; i < N; ++i)
    if (oracle_base(seq[i]) < 0) {
      free(dr); free(di); free(pr); free(pi); free(v);
      return -1;
    }
  for (int k = 1; k <= m; ++k) {
    int64_t a, q;
    oracle_factor(m, variant, k, &a, &q);
    double ang = TWO_PI * (double)a / ((double)q * (double)N);
    for (int b = 0; b < nb; ++b) {
      dr[(k - 1) * nb + b] = cos(ang);
      di[(k - 1) * nb + b] = sin(ang);
    }
  }
  for (int i = 0; i < D; ++i) {
    re[i] = im[i] = 0.0;
    pr[i] = 1.0; /* D^0 = identity */
    pi[i] = 0.0;
  }
  for (int loc = 0; loc <= N - s; ++loc) {
    int b = map[mer_code(seq, loc, s)];
    /* v = ones(m) (x) onehot(b) */
    for (int i = 0; i < D; ++i) v[i] = 0.0;
    for (int k = 0; k < m; ++k) v[k * nb + b] = 1.0;
    /* acc += D^loc v  (diagonal matrix times vector) */
    for (int i = 0; i < D; ++i) {
      re[i] += pr[i] * v[i];
      im[i] += pi[i] * v[i];
    }
    /* D^{loc+1} = D^loc D */
    for (int i = 0; i < D; ++i) {
      double nr = pr[i] * dr[i] - pi[i] * di[i];
      double ni = pr[i] * di[i] + pi[i] * dr[i];
      pr[i] = nr;
      pi[i] = ni;
    }
  }
  free(dr); free(di); free(pr); free(pi); free(v);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Fidelity (§2.4: fid = |<RoPE(a)|RoPE(b)>|^2 of normalised encodings)     */

/* A vector whose squared norm is at most ZERO_NORM2 is the zero vector: §3.3
 * states that evenly spaced unit phases sum to zero; in floating point that
 * sum leaves rounding residue (about 1e-28 in FP64) instead of 0, while any
 * nonzero encoding has a squared norm of order N. */
#define ZERO_NORM2 1e-6

/* |<x|y>|^2 / (||x||^2 ||y||^2), <x|y> = sum conj(x) y. A zero vector gives 0. */
double oracle_fidelity(const double* xr, const double* xi, const double* yr, const double* yi, int D) {
  double ipr = 0, ipi = 0, nx = 0, ny = 0;
  for (int i = 0; i < D; ++i) {
    ipr += xr[i] * yr[i] + xi[i] * yi[i];
    ipi += xr[i] * yi[i] - xi[i] * yr[i];
    nx += xr[i] * xr[i] + xi[i] * xi[i];
    ny += yr[i] * yr[i] + yi[i] * yi[i];
  }
  if (nx <= ZERO_NORM2 || ny <= ZERO_NORM2) return 0.0;
  return (ipr * ipr + ipi * ipi) / (nx * ny);
}

/* Shift-invariant variant (§2.5): bands kept separate and normalised, the
 * score is the mean over k of the per-band fidelities. */
double oracle_fidelity_per_band(const double* xr, const double* xi, const double* yr, const double* yi, int m,
                                int band_dim) {
  double acc = 0;
  for (int k = 0; k < m; ++k)
    acc += oracle_fidelity(xr + k * band_dim, xi + k * band_dim, yr + k * band_dim, yi + k * band_dim, band_dim);
  return acc / m;
}

/* Hamming quantum fingerprint (§1): |Q(S)> = n^{-1/2} sum_i |i>|S_i>, built
 * explicitly as an (n*5)-dimensional real vector over the alphabet
 * {A, C, G, T, other}: any letter outside ACGT takes the fifth slot; returns
 * |<Q(S)|Q(T)>|^2. */
double oracle_hamming_fingerprint_fidelity(const uint8_t* S, const uint8_t* T, int n) {
  double* qs = (double*)calloc((size_t)n * 5, sizeof(double));
  double* qt = (double*)calloc((size_t)n * 5, sizeof(double));
  double norm = 1.0 / sqrt((double)n);
  for (int i = 0; i < n; ++i) {
    const int a = oracle_base(S[i]), b = oracle_base(T[i]);
    qs[i * 5 + (a < 0 ? 4 : a)] = norm;
    qt[i * 5 + (b < 0 ? 4 : b)] = norm;
  }
  double ip = 0;
  for (int i = 0; i < n * 5; ++i) ip += qs[i] * qt[i];
  free(qs);
  free(qt);
  return ip * ip;
}

/* ---------------------------------------------------------------------- */
/* Reference windows (§3.1: window of length N slides with a step)          */

/* number of windows of length N at the given stride: floor((L-N)/stride)+1 */
int64_t oracle_n_windows(int64_t L, int N, int stride) {
  if (L < N || N <= 0 || stride <= 0) return 0;
  return (L - N) / stride + 1;
}

/* Windows j = j0 .. j0+count-1 (start j*stride), each by direct summation;
 * output count x D complex, row-major. */
int oracle_windows_direct(const uint8_t* ref, int64_t L, int N, int stride, int64_t j0, int64_t count, int s, int m,
                          int t, int variant, const uint16_t* map, double* re, double* im) {
  const int D = m << (2 * t);
  for (int64_t j = 0; j < count; ++j) {
    int64_t w = (j0 + j) * stride;
    if (w + N > L) return -1;
    if (oracle_embed(ref + w, N, s, m, t, variant, map, re + j * D, im + j * D) != 0) return -1;
  }
  return 0;
}

/*
 * Windows w = w0 .. w0+count-1 at stride 1 by the slide-by-one relations of
 * §3.4: every c_mer is multiplied by w^{-f}, the s-mer leaving at the start
 * additionally loses w^{-f}, the s-mer entering at the end gains w^{f(N-s)}
 * (both when they coincide). The first window is a direct sum.
 */
int oracle_windows_recurrence(const uint8_t* ref, int64_t L, int N, int64_t w0, int64_t count, int s, int m, int t,
                              int variant, const uint16_t* map, double* re, double* im) {
  const int nb = 1 << (2 * t);
  const int D = m * nb;
  if (count <= 0) return 0;
  if (w0 + count - 1 + N > L) return -1;
  if (oracle_embed(ref + w0, N, s, m, t, variant, map, re, im) != 0) return -1;
  for (int64_t j = 1; j < count; ++j) {
    int64_t w = w0 + j - 1; /* slide from window w to w+1 */
    const double* cr = re + (j - 1) * D;
    const double* ci = im + (j - 1) * D;
    double* nr = re + j * D;
    double* ni = im + j * D;
    int b_old = map[mer_code(ref, w, s)];
    int b_new = map[mer_code(ref, w + N - s + 1, s)];
    for (int k = 1; k <= m; ++k) {
      int64_t a, q;
      oracle_factor(m, variant, k, &a, &q);
      double rr, ri, er, ei; /* w^{-f}, w^{f(N-s)} */
      unit_root(-a, q, N, 1, &rr, &ri);
      unit_root(a, q, N, N - s, &er, &ei);
      for (int b = 0; b < nb; ++b) {
        int i = (k - 1) * nb + b;
        double xr = cr[i], xi = ci[i];
        if (b == b_old) xr -= 1.0;
        double yr = xr * rr - xi * ri;
        double yi = xr * ri + xi * rr;
        if (b == b_new) {
          yr += er;
          yi += ei;
        }
        nr[i] = yr;
        ni[i] = yi;
      }
    }
  }
  return 0;
}

/*
 * Inner products ip(w) = <x | c(w)> for w = w0 .. w0+count-1 by the relation
 * of §3.4: ip_new = ip w^{-f} - conj(x_old) w^{-f} + conj(x_new) w^{f(N-s)},
 * applied per band k (so ip is held per band and summed). The first value is
 * a direct inner product. out_r/out_i: count values.
 */
int oracle_ip_recurrence(const uint8_t* ref, int64_t L, int N, int64_t w0, int64_t count, int s, int m, int t,
                         int variant, const uint16_t* map, const double* xr, const double* xi, double* out_r,
                         double* out_i) {
  const int nb = 1 << (2 * t);
  const int D = m * nb;
  if (count <= 0) return 0;
  if (w0 + count - 1 + N > L) return -1;
  double* cr = (double*)malloc(sizeof(double) * D);
  double* ci = (double*)malloc(sizeof(double) * D);
  double* ipr = (double*)malloc(sizeof(double) * m);
  double* ipi = (double*)malloc(sizeof(double) * m);
  if (oracle_embed(ref + w0, N, s, m, t, variant, map, cr, ci) != 0) {
    free(cr); free(ci); free(ipr); free(ipi);
    return -1;
  }
  for (int k = 0; k < m; ++k) {
    ipr[k] = ipi[k] = 0;
    for (int b = 0; b < nb; ++b) {
      int i = k * nb + b;
      ipr[k] += xr[i] * cr[i] + xi[i] * ci[i];
      ipi[k] += xr[i] * ci[i] - xi[i] * cr[i];
    }
  }
  for (int64_t j = 0; j < count; ++j) {
    if (j > 0) {
      int64_t w = w0 + j - 1;
      int b_old = map[mer_code(ref, w, s)];
      int b_new = map[mer_code(ref, w + N - s + 1, s)];
      for (int k = 1; k <= m; ++k) {
        int64_t a, q;
        oracle_factor(m, variant, k, &a, &q);
        double rr, ri, er, ei;
        unit_root(-a, q, N, 1, &rr, &ri);
        unit_root(a, q, N, N - s, &er, &ei);
        int io = (k - 1) * nb + b_old, in = (k - 1) * nb + b_new;
        /* conj(x_old) and conj(x_new) */
        double oxr = xr[io], oxi = -xi[io], nxr = xr[in], nxi = -xi[in];
        double pr = ipr[k - 1], pi = ipi[k - 1];
        double yr = pr * rr - pi * ri, yi = pr * ri + pi * rr;
        yr -= oxr * rr - oxi * ri;
        yi -= oxr * ri + oxi * rr;
        yr += nxr * er - nxi * ei;
        yi += nxr * ei + nxi * er;
        ipr[k - 1] = yr;
        ipi[k - 1] = yi;
      }
    }
    double sr = 0, si = 0;
    for (int k = 0; k < m; ++k) {
      sr += ipr[k];
      si += ipi[k];
    }
    out_r[j] = sr;
    out_i[j] = si;
  }
  free(cr); free(ci); free(ipr); free(ipi);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Exhaustive mapping (§3.1 linear scan; §3.5 top-1 generalised to top-k)   */

typedef struct {
  double score;
  int64_t w;
} cand_t;

/* order: score descending, then window start ascending */
static int cand_cmp(const void* pa, const void* pb) {
  const cand_t* a = (const cand_t*)pa;
  const cand_t* b = (const cand_t*)pb;
  if (a->score > b->score) return -1;
  if (a->score < b->score) return 1;
  if (a->w < b->w) return -1;
  if (a->w > b->w) return 1;
  return 0;
}

/*
 * For each read (its first N letters), the fidelity against every window
 * j in [j_begin, j_end) (start j*stride) is computed in FP64 from direct-sum
 * embeddings; the list is fully sorted by (score desc, start asc); with sep > 0
 * only the first (best) window of each bucket floor(start/sep) is kept; the
 * first k survivors are written (start, score), padded with (-1, -inf).
 * score_mode 0: concatenated fidelity; 1: per-band mean (§2.5).
 * Returns 0, -1 on invalid input, -2 if a read is shorter than N.
 */
int oracle_score_topk(const uint8_t* ref, int64_t L, const uint8_t* seqs, const int64_t* offsets, int64_t n_reads,
                      int N, int stride, int64_t j_begin, int64_t j_end, int s, int m, int t, int variant,
                      const uint16_t* map, int score_mode, int k, int sep, int n_threads, int64_t* out_w,
                      double* out_s) {
  const int nb = 1 << (2 * t);
  const int D = m * nb;
  int64_t W = oracle_n_windows(L, N, stride);
  if (j_begin < 0) j_begin = 0;
  if (j_end > W) j_end = W;
  int64_t n_win = j_end > j_begin ? j_end - j_begin : 0;
  for (int64_t r = 0; r < n_reads; ++r)
    if (offsets[r + 1] - offsets[r] < N) return -2;
  double* wr = (double*)malloc(sizeof(double) * (size_t)(n_win > 0 ? n_win : 1) * D);
  double* wi = (double*)malloc(sizeof(double) * (size_t)(n_win > 0 ? n_win : 1) * D);
  if (oracle_windows_direct(ref, L, N, stride, j_begin, n_win, s, m, t, variant, map, wr, wi) != 0) {
    free(wr); free(wi);
    return -1;
  }
  int bad = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t r = 0; r < n_reads; ++r) {
    double* xr = (double*)malloc(sizeof(double) * D);
    double* xi = (double*)malloc(sizeof(double) * D);
    cand_t* c = (cand_t*)malloc(sizeof(cand_t) * (size_t)(n_win > 0 ? n_win : 1));
    if (oracle_embed(seqs + offsets[r], N, s, m, t, variant, map, xr, xi) != 0) {
      bad = 1;
    } else {
      for (int64_t j = 0; j < n_win; ++j) {
        const double* yr = wr + j * D;
        const double* yi = wi + j * D;
        c[j].score = score_mode == 1 ? oracle_fidelity_per_band(xr, xi, yr, yi, m, nb)
                                     : oracle_fidelity(xr, xi, yr, yi, D);
        c[j].w = (j_begin + j) * stride;
      }
      qsort(c, (size_t)n_win, sizeof(cand_t), cand_cmp);
      int got = 0;
      for (int64_t j = 0; j < n_win && got < k; ++j) {
        if (sep > 0) {
          int64_t bucket = c[j].w / sep, dup = 0;
          for (int g = 0; g < got; ++g)
            if (out_w[r * k + g] / sep == bucket) dup = 1;
          if (dup) continue;
        }
        out_w[r * k + got] = c[j].w;
        out_s[r * k + got] = c[j].score;
        ++got;
      }
      for (; got < k; ++got) {
        out_w[r * k + got] = -1;
        out_s[r * k + got] = -INFINITY;
      }
    }
    free(xr);
    free(xi);
    free(c);
  }
  free(wr);
  free(wi);
  return bad ? -1 : 0;
}

/* Fidelity of given (read, window start) pairs, one by one (sampled parity at
 * sizes where the exhaustive scan is out of reach). */
int oracle_score_pairs(const uint8_t* ref, int64_t L, const uint8_t* seqs, const int64_t* offsets,
                       const int64_t* read_idx, const int64_t* win_start, int64_t n_pairs, int N, int s, int m, int t,
                       int variant, const uint16_t* map, int score_mode, int n_threads, double* out) {
  const int nb = 1 << (2 * t);
  const int D = m * nb;
  int bad = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int64_t i = 0; i < n_pairs; ++i) {
    /* dense vectors of any dimension (refinement encodings reach 4^8 bins) */
    double* buf = (double*)malloc(sizeof(double) * 4 * (size_t)D);
    int64_t r = read_idx[i], w = win_start[i];
    if (!buf) {
      bad = 1;
      out[i] = NAN;
      continue;
    }
    double *xr = buf, *xi = buf + D, *yr = buf + 2 * (size_t)D, *yi = buf + 3 * (size_t)D;
    if (w < 0 || w + N > L || offsets[r + 1] - offsets[r] < N ||
        oracle_embed(seqs + offsets[r], N, s, m, t, variant, map, xr, xi) != 0 ||
        oracle_embed(ref + w, N, s, m, t, variant, map, yr, yi) != 0) {
      bad = 1;
      out[i] = NAN;
      free(buf);
      continue;
    }
    out[i] = score_mode == 1 ? oracle_fidelity_per_band(xr, xi, yr, yi, m, nb) : oracle_fidelity(xr, xi, yr, yi, D);
    free(buf);
  }
  return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* Levenshtein distance (§1): minimal number of insertions, deletions and   */
/* substitutions, full O(n*m) dynamic programme with unit costs.            */

int oracle_levenshtein(const uint8_t* a, int na, const uint8_t* b, int nb) {
  int* prev = (int*)malloc(sizeof(int) * (nb + 1));
  int* cur = (int*)malloc(sizeof(int) * (nb + 1));
  for (int j = 0; j <= nb; ++j) prev[j] = j;
  for (int i = 1; i <= na; ++i) {
    cur[0] = i;
    for (int j = 1; j <= nb; ++j) {
      int sub = prev[j - 1] + (a[i - 1] != b[j - 1]);
      int del = prev[j] + 1;
      int ins = cur[j - 1] + 1;
      int v = sub < del ? sub : del;
      cur[j] = v < ins ? v : ins;
    }
    int* tmp = prev;
    prev = cur;
    cur = tmp;
  }
  int d = prev[nb];
  free(prev);
  free(cur);
  return d;
}

/* Levenshtein distance of many (read head, reference window) pairs. */
int oracle_levenshtein_pairs(const uint8_t* ref, int64_t L, const uint8_t* seqs, const int64_t* offsets,
                             const int64_t* read_idx, const int64_t* win_start, int64_t n_pairs, int N,
                             int n_threads, int32_t* out) {
  int bad = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
  for (int64_t i = 0; i < n_pairs; ++i) {
    int64_t r = read_idx[i], w = win_start[i];
    if (w < 0 || w + N > L || offsets[r + 1] - offsets[r] < N) {
      bad = 1;
      out[i] = -1;
      continue;
    }
    out[i] = oracle_levenshtein(seqs + offsets[r], N, ref + w, N);
  }
  return bad ? -1 : 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Candidate reranker network (the paper has none; this is the reference of  */
/* the library's learned reranker). Two layers, FP64:                        */
/*   pre = W1 x + b1   (W1: H x F, row-major),  h = GELU(pre),               */
/*   y   = w2 . h + b2,                                                       */
/* GELU(z) = z * Phi(z) = 0.5 z (1 + erf(z / sqrt 2)) (exact, not tanh).     */
/* Loss: mean over the batch of (y - t)^2.                                   */
/* Parity: the backward is pinned by finite differences of the forward, the */
/* forward by GELU's closed form; no passage of the paper pins either.      */

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / 1.4142135623730951)); }
static double gelu_grad(double z) {
  return 0.5 * (1.0 + erf(z / 1.4142135623730951)) + z * exp(-0.5 * z * z) / 2.5066282746310002;
}

/* y[b] for b < B; X is B x F row-major */
void oracle_mlp_forward(const double* W1, const double* b1, const double* w2, double b2, int F, int H,
                        const double* X, int64_t B, double* y) {
  for (int64_t b = 0; b < B; ++b) {
    double acc = b2;
    for (int j = 0; j < H; ++j) {
      double z = b1[j];
      for (int f = 0; f < F; ++f) z += W1[j * F + f] * X[b * F + f];
      acc += w2[j] * gelu(z);
    }
    y[b] = acc;
  }
}

/* loss and gradients of the mean squared error over the batch */
double oracle_mlp_grad(const double* W1, const double* b1, const double* w2, double b2, int F, int H,
                       const double* X, const double* t, int64_t B, double* gW1, double* gb1, double* gw2,
                       double* gb2) {
  double* z = (double*)malloc(sizeof(double) * H);
  for (int i = 0; i < H * F; ++i) gW1[i] = 0.0;
  for (int j = 0; j < H; ++j) gb1[j] = gw2[j] = 0.0;
  *gb2 = 0.0;
  double loss = 0.0;
  for (int64_t b = 0; b < B; ++b) {
    double y = b2;
    for (int j = 0; j < H; ++j) {
      z[j] = b1[j];
      for (int f = 0; f < F; ++f) z[j] += W1[j * F + f] * X[b * F + f];
      y += w2[j] * gelu(z[j]);
    }
    const double r = y - t[b];
    loss += r * r / (double)B;
    const double dy = 2.0 * r / (double)B;
    *gb2 += dy;
    for (int j = 0; j < H; ++j) {
      gw2[j] += dy * gelu(z[j]);
      const double dz = dy * w2[j] * gelu_grad(z[j]);
      gb1[j] += dz;
      for (int f = 0; f < F; ++f) gW1[j * F + f] += dz * X[b * F + f];
    }
  }
  free(z);
  return loss;
}

/* One AdamW step (Loshchilov & Hutter, decoupled weight decay) on n
 * parameters at step number `step` (1-based):
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p = p (1 - lr wd) - lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps) */
void oracle_adamw(double* p, const double* g, double* m, double* v, int64_t n, int64_t step, double lr, double beta1,
                  double beta2, double eps, double wd) {
  const double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    p[i] = p[i] * (1.0 - lr * wd) - lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

/* ---------------------------------------------------------------------- */
/* Threshold regime: per-fragment fidelity thresholds (§3.4: for a target  */
/* mutation rate, the expected fidelity of each reference fragment against */
/* mutated copies of itself, used as its cutting threshold) and the        */
/* multi-locus output of §3.5 (every window whose fidelity with the read    */
/* reaches its threshold).                                                  */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the i-th output (0-based)
 * of the generator started at state `seed`: the state advances by the
 * golden-ratio increment and each state is passed through the finaliser. */
static uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
uint64_t oracle_splitmix64(uint64_t seed, uint64_t i) { return sm64_mix(seed + (i + 1) * 0x9E3779B97F4A7C15ULL); }

static double sm64_unit(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

/* N letters of a mutated copy of ref read from `start`: each reference
 * letter in turn is mutated with probability err, the mutation being a
 * deletion, an insertion (a random letter before it) or a substitution (one
 * of the three other letters) with probability 1/3 each (the even split of
 * the paper's mutated companions, §2.4 scoring of correlations). Randomness:
 * the SplitMix64 stream keyed by key = oracle_splitmix64(seed, stream);
 * reference letter number d (from start) uses its draws 3d, 3d+1, 3d+2
 * (mutation?, which kind, which letter). Past the end of ref the walk reads
 * 'A'. Writes upper-case letters to out[0..N) and the numbers of reference
 * letters walked, deletions, insertions and substitutions to counts[0..3]. */
int oracle_mutate(const uint8_t* ref, int64_t L, int64_t start, int N, double err, uint64_t seed, uint64_t stream,
                  uint8_t* out, int64_t* counts) {
  static const char ACGT[4] = {'A', 'C', 'G', 'T'};
  const uint64_t key = oracle_splitmix64(seed, stream);
  int n = 0;
  int64_t d = 0, nd = 0, ni = 0, ns = 0;
  while (n < N) {
    const int64_t pos = start + d;
    int c = pos < L ? oracle_base(ref[pos]) : 0;
    if (c < 0) return -1;
    const double u0 = sm64_unit(oracle_splitmix64(key, 3 * (uint64_t)d));
    const double u1 = sm64_unit(oracle_splitmix64(key, 3 * (uint64_t)d + 1));
    const uint64_t z2 = oracle_splitmix64(key, 3 * (uint64_t)d + 2);
    ++d;
    if (u0 < err) {
      const int kind = (int)(u1 * 3.0);
      if (kind == 0) { /* deletion: the letter is skipped */
        ++nd;
        continue;
      }
      if (kind == 1) { /* insertion: a random letter, then the reference letter */
        ++ni;
        out[n++] = (uint8_t)ACGT[z2 >> 62];
        if (n < N) out[n++] = (uint8_t)ACGT[c];
        continue;
      }
      ++ns; /* substitution: one of the three other letters */
      c = (c + 1 + (int)(sm64_unit(z2) * 3.0)) & 3;
    }
    out[n++] = (uint8_t)ACGT[c];
  }
  if (counts) {
    counts[0] = d;
    counts[1] = nd;
    counts[2] = ni;
    counts[3] = ns;
  }
  return 0;
}

/* Per-fragment threshold of windows j0 .. j0+count-1 (start j*stride): the
 * mean over n_samples mutated copies (stream j*n_samples + t, t < n_samples)
 * of the fidelity between the window's encoding and the encoding of the
 * copy's N letters (concatenated or per-band score, §2.4/§2.5). */
int oracle_fragment_thresholds(const uint8_t* ref, int64_t L, int N, int stride, int64_t j0, int64_t count, int s,
                               int m, int t, int variant, const uint16_t* map, int score_mode, double err,
                               int n_samples, uint64_t seed, int n_threads, double* out) {
  const int nb = 1 << (2 * t);
  const int D = m * nb;
  int bad = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int64_t i = 0; i < count; ++i) {
    const int64_t j = j0 + i;
    const int64_t w = j * stride;
    double* buf = (double*)malloc(sizeof(double) * 4 * (size_t)D);
    uint8_t* copy = (uint8_t*)malloc((size_t)N);
    if (!buf || !copy || w < 0 || w + N > L) {
      bad = 1;
      out[i] = NAN;
      free(buf);
      free(copy);
      continue;
    }
    double *xr = buf, *xi = buf + D, *yr = buf + 2 * (size_t)D, *yi = buf + 3 * (size_t)D;
    double acc = 0.0;
    if (oracle_embed(ref + w, N, s, m, t, variant, map, yr, yi) != 0) bad = 1;
    for (int k = 0; k < n_samples && !bad; ++k) {
      if (oracle_mutate(ref, L, w, N, err, seed, (uint64_t)j * n_samples + k, copy, NULL) != 0 ||
          oracle_embed(copy, N, s, m, t, variant, map, xr, xi) != 0) {
        bad = 1;
        break;
      }
      acc += score_mode == 1 ? oracle_fidelity_per_band(xr, xi, yr, yi, m, nb) : oracle_fidelity(xr, xi, yr, yi, D);
    }
    out[i] = acc / n_samples;
    free(buf);
    free(copy);
  }
  return bad ? -1 : 0;
}

/* Every (read, window) pair with fidelity >= thr[j - jb] over windows
 * [jb, je), by exhaustive FP64 scoring (each window embedded once and scored
 * against every read), in (read, window) order. Writes at most cap pairs;
 * returns the number of pairs found (or -1). */
int64_t oracle_threshold_pairs(const uint8_t* ref, int64_t L, const uint8_t* seqs, const int64_t* offsets,
                               int64_t n_reads, int N, int stride, int64_t jb, int64_t je, int s, int m, int t,
                               int variant, const uint16_t* map, int score_mode, const double* thr, int64_t cap,
                               int64_t* out_read, int64_t* out_win, double* out_fid) {
  const int nb = 1 << (2 * t);
  const int D = m * nb;
  const int64_t nw = je - jb;
  double* x = (double*)malloc(sizeof(double) * 2 * (size_t)D * (size_t)(n_reads > 0 ? n_reads : 1));
  double* y = (double*)malloc(sizeof(double) * 2 * (size_t)D);
  uint8_t* hit = (uint8_t*)calloc((size_t)(n_reads > 0 ? n_reads : 1) * (size_t)(nw > 0 ? nw : 1), 1);
  double* fid = (double*)malloc(sizeof(double) * (size_t)(n_reads > 0 ? n_reads : 1) * (size_t)(nw > 0 ? nw : 1));
  int bad = !x || !y || !hit || !fid;
  for (int64_t r = 0; r < n_reads && !bad; ++r)
    if (offsets[r + 1] - offsets[r] < N ||
        oracle_embed(seqs + offsets[r], N, s, m, t, variant, map, x + 2 * (size_t)D * r, x + 2 * (size_t)D * r + D) != 0)
      bad = 1;
  for (int64_t j = jb; j < je && !bad; ++j) {
    if (j * stride + N > L || oracle_embed(ref + j * stride, N, s, m, t, variant, map, y, y + D) != 0) {
      bad = 1;
      break;
    }
    for (int64_t r = 0; r < n_reads; ++r) {
      const double* xr = x + 2 * (size_t)D * r;
      const double f = score_mode == 1 ? oracle_fidelity_per_band(xr, xr + D, y, y + D, m, nb)
                                       : oracle_fidelity(xr, xr + D, y, y + D, D);
      hit[r * nw + (j - jb)] = f >= thr[j - jb];
      fid[r * nw + (j - jb)] = f;
    }
  }
  int64_t found = 0;
  for (int64_t r = 0; r < n_reads && !bad; ++r)
    for (int64_t j = 0; j < nw; ++j)
      if (hit[r * nw + j]) {
        if (found < cap) {
          out_read[found] = r;
          out_win[found] = jb + j;
          out_fid[found] = fid[r * nw + j];
        }
        ++found;
      }
  free(x);
  free(y);
  free(hit);
  free(fid);
  return bad ? -1 : found;
}
