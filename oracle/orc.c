/*
 * orc.c -- CPU oracle (TEST INFRASTRUCTURE ONLY; see orc.h).
 *
 * Plain loops, one step of the format per function, FP64 wherever the format
 * leaves the precision open.  No blocking, no fusion, no SIMD intrinsics.
 */
#include "orc.h"

#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ CRC-32 */
/* IEEE 802.3 CRC-32, reflected polynomial 0xEDB88320, init and final xor
 * 0xFFFFFFFF, computed one bit at a time. */
uint32_t orc_crc32(const uint8_t* p, size_t n) {
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; i++) {
    c ^= p[i];
    for (int b = 0; b < 8; b++) c = (c & 1u) ? (c >> 1) ^ 0xEDB88320u : (c >> 1);
  }
  return c ^ 0xFFFFFFFFu;
}

/* ------------------------------------------------- integer lifting (mod 2^32) */
/* All transform arithmetic is on 32-bit two's complement words with
 * wraparound; the right shift is arithmetic (sign-extending).  Written on
 * uint32_t so that overflow is defined behaviour in C. */
static uint32_t asr1(uint32_t u) { return (u >> 1) | (u & 0x80000000u); }

void orc_fwd_lift4(int32_t v[4]) {
  uint32_t x0 = (uint32_t)v[0], x1 = (uint32_t)v[1], x2 = (uint32_t)v[2], x3 = (uint32_t)v[3];
  uint32_t d0 = x1 - x0;
  uint32_t s0 = x0 + asr1(d0);
  uint32_t d1 = x3 - x2;
  uint32_t s1 = x2 + asr1(d1);
  uint32_t d = s1 - s0;
  uint32_t s = s0 + asr1(d);
  uint32_t e = d1 - d0;
  v[0] = (int32_t)s;
  v[1] = (int32_t)d;
  v[2] = (int32_t)d0;
  v[3] = (int32_t)e;
}

void orc_inv_lift4(int32_t v[4]) {
  uint32_t s = (uint32_t)v[0], d = (uint32_t)v[1], d0 = (uint32_t)v[2], e = (uint32_t)v[3];
  uint32_t d1 = e + d0;
  uint32_t s0 = s - asr1(d);
  uint32_t s1 = d + s0;
  uint32_t x0 = s0 - asr1(d0);
  uint32_t x1 = d0 + x0;
  uint32_t x2 = s1 - asr1(d1);
  uint32_t x3 = d1 + x2;
  v[0] = (int32_t)x0;
  v[1] = (int32_t)x1;
  v[2] = (int32_t)x2;
  v[3] = (int32_t)x3;
}

/* Forward: every row (along the column index c), then every column (along r).
 * Afterwards b[4*i+j] holds coefficient (i, j): i from the column pass,
 * j from the row pass. */
void orc_fwd_xform(int32_t b[16]) {
  int32_t v[4];
  for (int r = 0; r < 4; r++) {
    for (int c = 0; c < 4; c++) v[c] = b[4 * r + c];
    orc_fwd_lift4(v);
    for (int c = 0; c < 4; c++) b[4 * r + c] = v[c];
  }
  for (int c = 0; c < 4; c++) {
    for (int r = 0; r < 4; r++) v[r] = b[4 * r + c];
    orc_fwd_lift4(v);
    for (int r = 0; r < 4; r++) b[4 * r + c] = v[r];
  }
}

/* Inverse: columns first, then rows (the exact reverse of the forward order). */
void orc_inv_xform(int32_t b[16]) {
  int32_t v[4];
  for (int c = 0; c < 4; c++) {
    for (int r = 0; r < 4; r++) v[r] = b[4 * r + c];
    orc_inv_lift4(v);
    for (int r = 0; r < 4; r++) b[4 * r + c] = v[r];
  }
  for (int r = 0; r < 4; r++) {
    for (int c = 0; c < 4; c++) v[c] = b[4 * r + c];
    orc_inv_lift4(v);
    for (int c = 0; c < 4; c++) b[4 * r + c] = v[c];
  }
}

/* ------------------------------------------------------------- negabinary */
/* Two's complement <-> base -2, valid for |c| < 2^30. */
uint32_t orc_int2nb(int32_t c) { return ((uint32_t)c + 0xAAAAAAAAu) ^ 0xAAAAAAAAu; }
int32_t orc_nb2int(uint32_t u) { return (int32_t)((u ^ 0xAAAAAAAAu) - 0xAAAAAAAAu); }

/* --------------------------------------------------------- sequency order */
/* Output slots of the lift carry the ranks (0, 1, 2, 2) for (s, d, d0, e).
 * Coefficients are sorted by (rank_i + rank_j, max(rank_i, rank_j), i, j). */
void orc_sequency(int perm[16]) {
  static const int rank[4] = {0, 1, 2, 2};
  int key[16][4];
  int idx[16];
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      int k = 4 * i + j;
      idx[k] = k;
      key[k][0] = rank[i] + rank[j];
      key[k][1] = rank[i] > rank[j] ? rank[i] : rank[j];
      key[k][2] = i;
      key[k][3] = j;
    }
  /* insertion sort on the 4-tuple key */
  for (int a = 1; a < 16; a++) {
    int t = idx[a];
    int b = a - 1;
    for (; b >= 0; b--) {
      int less = 0;
      for (int f = 0; f < 4; f++) {
        if (key[t][f] != key[idx[b]][f]) {
          less = key[t][f] < key[idx[b]][f];
          break;
        }
      }
      if (!less) break;
      idx[b + 1] = idx[b];
    }
    idx[b + 1] = t;
  }
  for (int k = 0; k < 16; k++) perm[k] = idx[k];
}

/* ------------------------------------------------------------ bit streams */
/* LSB-first within little-endian 64-bit words. */
static void put_bit(uint64_t* w, int64_t pos, unsigned bit) {
  if (bit) w[pos >> 6] |= (uint64_t)1 << (pos & 63);
}
static unsigned get_bit(const uint64_t* w, int64_t pos) { return (unsigned)((w[pos >> 6] >> (pos & 63)) & 1u); }

/* Embedded bit-plane coder with group tests.  For each plane k from 31 down
 * to 0, with n = length of the already-significant prefix:
 *   (a) the n prefix bits are sent verbatim;
 *   (b) while n < 16: one test bit says whether any of bits n..15 is set; if
 *       not, the plane ends; if so, bits n, n+1, ... are sent one at a time
 *       (n advancing after each) until a one has been sent; when bits n..14
 *       were all zero the one must be bit 15, which is then implied.
 * Every sent bit spends one unit of the budget; coding stops the moment the
 * budget is spent, even in the middle of a plane. */
int orc_encode_planes(const uint32_t u[16], int maxbits, uint64_t* words, int64_t pos) {
  int bits = maxbits;
  int n = 0;
  for (int k = 31; k >= 0 && bits > 0; k--) {
    for (int i = 0; i < n && bits > 0; i++) {
      put_bit(words, pos++, (u[i] >> k) & 1u);
      bits--;
    }
    while (n < 16 && bits > 0) {
      unsigned t = 0;
      for (int i = n; i < 16; i++) t |= (u[i] >> k) & 1u;
      put_bit(words, pos++, t);
      bits--;
      if (!t) break;
      for (;;) {
        if (n == 15) { /* bits n..14 were zero: bit 15 is the one, implied */
          n = 16;
          break;
        }
        if (bits == 0) break;
        unsigned b = (u[n] >> k) & 1u;
        put_bit(words, pos++, b);
        bits--;
        n++;
        if (b) break;
      }
    }
  }
  return maxbits - bits;
}

int orc_decode_planes(const uint64_t* words, int64_t pos, int maxbits, uint32_t u[16]) {
  int bits = maxbits;
  int n = 0;
  for (int i = 0; i < 16; i++) u[i] = 0;
  for (int k = 31; k >= 0 && bits > 0; k--) {
    for (int i = 0; i < n && bits > 0; i++) {
      u[i] |= (uint32_t)get_bit(words, pos++) << k;
      bits--;
    }
    while (n < 16 && bits > 0) {
      unsigned t = get_bit(words, pos++);
      bits--;
      if (!t) break;
      for (;;) {
        if (n == 15) {
          u[15] |= (uint32_t)1 << k;
          n = 16;
          break;
        }
        if (bits == 0) break;
        unsigned b = get_bit(words, pos++);
        bits--;
        if (b) {
          u[n] |= (uint32_t)1 << k;
          n++;
          break;
        }
        n++;
      }
    }
  }
  return maxbits - bits;
}

/* --------------------------------------------------------------- one block */
#define WZ1_PREC 26     /* fixed-point bits below the block exponent */
#define WZ1_EMIN (-100) /* blocks whose largest |a| < 2^-100 are coded as zero */

int orc_wz1_encode_block(const float a[16], int rate, uint64_t* words) {
  int nwords = rate / 4;
  for (int w = 0; w < nwords; w++) words[w] = 0;
  /* block exponent: the largest e with |a| < 2^e over nonzero entries */
  int emax = WZ1_EMIN - 1000;
  for (int i = 0; i < 16; i++) {
    if (!isfinite(a[i])) return ORC_ENONFINITE;
    if (fabs((double)a[i]) >= ldexp(1.0, 127)) return ORC_ERANGE;
    if (a[i] != 0.0f) {
      int e;
      frexp((double)a[i], &e);
      if (e > emax) emax = e;
    }
  }
  if (emax <= WZ1_EMIN) return ORC_OK; /* zero block: flag 0, all bits zero */
  /* block-floating-point: q = trunc(a * 2^(26 - emax)), exact scaling in double */
  int32_t q[16];
  for (int i = 0; i < 16; i++) q[i] = (int32_t)trunc(ldexp((double)a[i], WZ1_PREC - emax));
  orc_fwd_xform(q);
  int perm[16];
  orc_sequency(perm);
  uint32_t u[16];
  for (int k = 0; k < 16; k++) u[k] = orc_int2nb(q[perm[k]]);
  /* header: nonzero flag, then emax + 127 in 8 bits */
  put_bit(words, 0, 1);
  unsigned eb = (unsigned)(emax + 127);
  for (int b = 0; b < 8; b++) put_bit(words, 1 + b, (eb >> b) & 1u);
  orc_encode_planes(u, 16 * rate - 9, words, 9);
  return ORC_OK;
}

void orc_wz1_decode_block(const uint64_t* words, int rate, int32_t q[16], int* emax, int* nonzero) {
  for (int i = 0; i < 16; i++) q[i] = 0;
  *nonzero = (int)get_bit(words, 0);
  *emax = 0;
  if (!*nonzero) return;
  unsigned eb = 0;
  for (int b = 0; b < 8; b++) eb |= get_bit(words, 1 + b) << b;
  *emax = (int)eb - 127;
  uint32_t u[16];
  orc_decode_planes(words, 9, 16 * rate - 9, u);
  int perm[16];
  orc_sequency(perm);
  for (int k = 0; k < 16; k++) q[perm[k]] = orc_nb2int(u[k]);
  orc_inv_xform(q);
}

double orc_wz1_value(int32_t q, int emax, int nonzero) {
  if (!nonzero) return 0.0;
  float f = (float)q; /* int -> float, round to nearest even */
  return ldexp((double)f, emax - WZ1_PREC);
}

/* ------------------------------------------------------ WZ2 (fixed widths) */
#define WZ2_PREC 24
#define WZ2_KMAX 27

static const int64_t F4[4][4] = {{1, 1, 1, 1}, {-2, -2, 2, 2}, {-4, 4, 0, 0}, {4, -4, -4, 4}};
static const int64_t G2[4][4] = {{2, -1, -1, 0}, {2, -1, 1, 0}, {2, 1, -1, -1}, {2, 1, 1, 1}};

int orc_wz2_width(int rate) { return (16 * rate - 13) / 16; }

static void put_bits(uint64_t* w, int64_t pos, uint64_t v, int n) {
  for (int b = 0; b < n; b++) put_bit(w, pos + b, (unsigned)((v >> b) & 1u));
}
static uint64_t get_bits(const uint64_t* w, int64_t pos, int n) {
  uint64_t v = 0;
  for (int b = 0; b < n; b++) v |= (uint64_t)get_bit(w, pos + b) << b;
  return v;
}

/* C = L B L^T for 4x4 integer matrices (plain triple loops). */
static void sandwich(const int64_t L[4][4], const int64_t B[16], int64_t C[16]) {
  int64_t T[16];
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      int64_t t = 0;
      for (int k = 0; k < 4; k++) t += L[i][k] * B[4 * k + j];
      T[4 * i + j] = t;
    }
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      int64_t t = 0;
      for (int k = 0; k < 4; k++) t += T[4 * i + k] * L[j][k];
      C[4 * i + j] = t;
    }
}

int orc_wz2_encode_block(const float a[16], int rate, int lift, uint64_t* words) {
  int nwords = rate / 4;
  for (int w = 0; w < nwords; w++) words[w] = 0;
  int emax = WZ1_EMIN - 1000;
  for (int i = 0; i < 16; i++) {
    if (!isfinite(a[i])) return ORC_ENONFINITE;
    if (fabs((double)a[i]) >= ldexp(1.0, 127)) return ORC_ERANGE;
    if (a[i] != 0.0f) {
      int e;
      frexp((double)a[i], &e);
      if (e > emax) emax = e;
    }
  }
  if (emax <= WZ1_EMIN) return ORC_OK; /* zero block: all bits zero */
  int64_t q[16], c[16], seq[16];
  for (int i = 0; i < 16; i++) q[i] = (int64_t)trunc(ldexp((double)a[i], WZ2_PREC - emax));
  if (lift)
    sandwich(F4, q, c);
  else
    for (int i = 0; i < 16; i++) c[i] = q[i];
  int perm[16];
  orc_sequency(perm);
  for (int k = 0; k < 16; k++) seq[k] = lift ? c[perm[k]] : c[k];
  const int W = orc_wz2_width(rate);
  const double lo = -ldexp(1.0, W - 1), hi = ldexp(1.0, W - 1) - 1.0;
  int K = 0;
  double v[16];
  for (K = 0; K <= WZ2_KMAX; K++) {
    int fits = 1;
    for (int k = 0; k < 16; k++) {
      v[k] = nearbyint(ldexp((double)seq[k], -K)); /* round half to even */
      if (v[k] < lo || v[k] > hi) fits = 0;
    }
    if (fits) break;
  }
  put_bits(words, 0, (uint64_t)(emax + 127), 8);
  put_bits(words, 8, (uint64_t)K, 5);
  for (int k = 0; k < 16; k++) put_bits(words, 13 + (int64_t)W * k, (uint64_t)(int64_t)(v[k] - lo), W);
  return ORC_OK;
}

void orc_wz2_decode_block(const uint64_t* words, int rate, int lift, double out[16]) {
  int E = (int)get_bits(words, 0, 8);
  for (int i = 0; i < 16; i++) out[i] = 0.0;
  if (E == 0) return;
  int emax = E - 127;
  int K = (int)get_bits(words, 8, 5);
  const int W = orc_wz2_width(rate);
  int64_t v[16], V[16], T[16];
  for (int k = 0; k < 16; k++) v[k] = (int64_t)get_bits(words, 13 + (int64_t)W * k, W) - ((int64_t)1 << (W - 1));
  int perm[16];
  orc_sequency(perm);
  for (int k = 0; k < 16; k++) V[lift ? perm[k] : k] = v[k];
  if (lift) {
    sandwich(G2, V, T);
    for (int i = 0; i < 16; i++) out[i] = ldexp((double)T[i], K + emax - 30);
  } else {
    for (int i = 0; i < 16; i++) out[i] = ldexp((double)V[i], K + emax - WZ2_PREC);
  }
}

/* ---------------------------------------------------- WZ3 (fixed accuracy) */
#define WZ3_WMAX 31 /* widest field: 13 + 16*31 bits fill one 64-byte block */
/* The decoded block of WZ2's layout for coefficients v (sequency order with
 * the lift), shift K and exponent emax: the same formulas as
 * orc_wz2_decode_block, written once more here for a given v. */
static void wz3_values(const int64_t v[16], int K, int emax, int lift, double out[16]) {
  int64_t V[16], T[16];
  int perm[16];
  orc_sequency(perm);
  for (int k = 0; k < 16; k++) V[lift ? perm[k] : k] = v[k];
  if (lift) {
    sandwich(G2, V, T);
    for (int i = 0; i < 16; i++) out[i] = ldexp((double)T[i], K + emax - 30);
  } else {
    for (int i = 0; i < 16; i++) out[i] = ldexp((double)V[i], K + emax - WZ2_PREC);
  }
}

int orc_wz3_block(const float a[16], double tol, int lift, int* emax_out, int* K_out, int64_t v[16],
                  int* need_w) {
  for (int k = 0; k < 16; k++) v[k] = 0;
  *emax_out = 0;
  *K_out = 0;
  *need_w = 0;
  if (!(tol >= 0.0)) return ORC_EINVAL;
  int emax = WZ1_EMIN - 1000;
  for (int i = 0; i < 16; i++) {
    if (!isfinite(a[i])) return ORC_ENONFINITE;
    if (fabs((double)a[i]) >= ldexp(1.0, 127)) return ORC_ERANGE;
    if (a[i] != 0.0f) {
      int e;
      frexp((double)a[i], &e);
      if (e > emax) emax = e;
    }
  }
  if (emax <= WZ1_EMIN) return ORC_OK; /* zero block */
  int64_t q[16], c[16], seq[16];
  for (int i = 0; i < 16; i++) q[i] = (int64_t)trunc(ldexp((double)a[i], WZ2_PREC - emax));
  if (lift)
    sandwich(F4, q, c);
  else
    for (int i = 0; i < 16; i++) c[i] = q[i];
  int perm[16];
  orc_sequency(perm);
  for (int k = 0; k < 16; k++) seq[k] = lift ? c[perm[k]] : c[k];
  /* The floor: the smallest shift whose fields fit the widest field the
   * layout has (WZ3_WMAX bits, one 64-byte block).  With the lift the
   * coefficients reach 2^32 in magnitude, so K = 0 does not always fit. */
  int Kfloor;
  for (Kfloor = 0; Kfloor < WZ2_KMAX; Kfloor++) {
    int fits = 1;
    for (int k = 0; k < 16; k++) {
      const double t = nearbyint(ldexp((double)seq[k], -Kfloor));
      if (t < -ldexp(1.0, WZ3_WMAX - 1) || t > ldexp(1.0, WZ3_WMAX - 1) - 1.0) fits = 0;
    }
    if (fits) break;
  }
  /* the largest shift down to the floor whose decoded block stays within tol
   * of a (else the floor, the finest quantisation the layout holds) */
  int K;
  for (K = WZ2_KMAX; K >= Kfloor; K--) {
    int64_t t[16];
    double d[16], err = 0.0;
    for (int k = 0; k < 16; k++) t[k] = (int64_t)nearbyint(ldexp((double)seq[k], -K));
    wz3_values(t, K, emax, lift, d);
    for (int i = 0; i < 16; i++) err = fmax(err, fabs((double)a[i] - d[i]));
    if (err <= tol || K == Kfloor) {
      for (int k = 0; k < 16; k++) v[k] = t[k];
      break;
    }
  }
  int W = 1;
  for (int k = 0; k < 16; k++)
    while (v[k] < -((int64_t)1 << (W - 1)) || v[k] > ((int64_t)1 << (W - 1)) - 1) W++;
  *emax_out = emax;
  *K_out = K;
  *need_w = W;
  return ORC_OK;
}

int orc_wz3_block_bytes(int W) { return 8 * ((13 + 16 * W + 63) / 64); }

int orc_wz3_encode_run(const float* blocks, int nb, double tol, int lift, uint64_t* words, int* w_run) {
  if (nb < 1 || nb > 32) return ORC_EINVAL;
  int emax[32], K[32], need[32];
  int64_t v[32][16];
  int W = 0;
  for (int b = 0; b < nb; b++) {
    int e = orc_wz3_block(blocks + 16 * b, tol, lift, &emax[b], &K[b], v[b], &need[b]);
    if (e != ORC_OK) return e;
    if (need[b] > W) W = need[b];
  }
  const int nw = orc_wz3_block_bytes(W) / 8;
  for (int i = 0; i < nb * nw; i++) words[i] = 0;
  for (int b = 0; b < nb; b++) {
    uint64_t* w = words + (int64_t)b * nw;
    if (need[b] == 0) continue; /* zero block: all bits zero */
    put_bits(w, 0, (uint64_t)(emax[b] + 127), 8);
    put_bits(w, 8, (uint64_t)K[b], 5);
    for (int k = 0; k < 16; k++)
      put_bits(w, 13 + (int64_t)W * k, (uint64_t)(v[b][k] + ((int64_t)1 << (W - 1))), W);
  }
  *w_run = W;
  return ORC_OK;
}

void orc_wz3_decode_block(const uint64_t* words, int W, int lift, double out[16]) {
  for (int i = 0; i < 16; i++) out[i] = 0.0;
  const int E = (int)get_bits(words, 0, 8);
  if (E == 0 || W < 1) return;
  const int K = (int)get_bits(words, 8, 5);
  int64_t v[16];
  for (int k = 0; k < 16; k++) v[k] = (int64_t)get_bits(words, 13 + (int64_t)W * k, W) - ((int64_t)1 << (W - 1));
  wz3_values(v, K, E - 127, lift, out);
}

/* --------------------------------------------------------- scaled formats */
/* Per 128x128 tile b: amax = max |a| (FP64); s = RN_fp32(amax / FMTMAX),
 * s = 1 when amax = 0; q = RN_fmt(a / s) with the quotient in FP64 and
 * saturation to +-FMTMAX; decoded value s * q (exact in FP64).  FP32 is
 * stored unscaled: s = 1 and q = RN_fp32(a). */
#define SC_TILE 128

typedef struct {
  int mant;      /* stored fraction bits */
  int emin;      /* exponent of the smallest normal */
  int ebits;     /* exponent field width */
  int bias;
  double fmtmax; /* the value that the tile amax is scaled to */
  double satmax; /* saturation bound for q */
  int bytes;
  int unscaled;  /* 1: every tile scale is 1 */
} fmtdesc;

static int fmt_desc(int fmt, fmtdesc* d) {
  switch (fmt) {
    case ORC_FMT_BF16: *d = (fmtdesc){7, -126, 8, 127, 1.0, 1.0, 2, 0}; return 1;
    case ORC_FMT_FP16: *d = (fmtdesc){10, -14, 5, 15, 32768.0, 32768.0, 2, 0}; return 1;
    case ORC_FMT_FP8E4M3: *d = (fmtdesc){3, -6, 4, 7, 448.0, 448.0, 1, 0}; return 1;
    case ORC_FMT_FP32: /* largest finite FP32: (2 - 2^-23) 2^127 */
      *d = (fmtdesc){23, -126, 8, 127, 1.0, ldexp(2.0 - ldexp(1.0, -23), 127), 4, 1};
      return 1;
    default: return 0;
  }
}

double orc_fmt_max(int fmt) {
  fmtdesc d;
  return fmt_desc(fmt, &d) ? d.fmtmax : 0.0;
}

double orc_round_fmt(int fmt, double v, uint32_t* bits) {
  fmtdesc d;
  if (!fmt_desc(fmt, &d)) return 0.0;
  int sign = signbit(v) ? 1 : 0;
  double a = fabs(v);
  double r = 0.0;
  if (a != 0.0) {
    int e;
    frexp(a, &e);         /* a in [2^(e-1), 2^e) */
    int ex = e - 1;       /* a = 1.f * 2^ex */
    if (ex < d.emin) ex = d.emin;
    double quantum = ldexp(1.0, ex - d.mant);
    r = nearbyint(a / quantum) * quantum; /* ties to even (default rounding mode) */
  }
  if (r > d.satmax) r = d.satmax;
  /* encode the bit pattern */
  uint32_t pat = 0;
  if (r != 0.0) {
    int e;
    double m = frexp(r, &e); /* r = m * 2^e, m in [0.5, 1) */
    int ex = e - 1;
    if (ex < d.emin) { /* subnormal */
      uint32_t frac = (uint32_t)ldexp(r, d.mant - d.emin);
      pat = frac;
    } else {
      uint32_t frac = (uint32_t)(ldexp(m, d.mant + 1) - ldexp(1.0, d.mant));
      pat = ((uint32_t)(ex + d.bias) << d.mant) | frac;
    }
  }
  pat |= (uint32_t)sign << (d.mant + d.ebits);
  if (bits) *bits = pat;
  return sign ? -r : r;
}

double orc_fmt_decode(int fmt, uint32_t bits) {
  fmtdesc d;
  if (!fmt_desc(fmt, &d)) return 0.0;
  int sign = (bits >> (d.mant + d.ebits)) & 1;
  uint32_t ef = (bits >> d.mant) & ((1u << d.ebits) - 1);
  uint32_t frac = bits & ((1u << d.mant) - 1);
  double v;
  if (ef == 0)
    v = ldexp((double)frac, d.emin - d.mant);
  else
    v = ldexp((double)((1u << d.mant) | frac), (int)ef - d.bias - d.mant);
  return sign ? -v : v;
}

/* ------------------------------------------------------------------- blobs */
int orc_rate_ok(int rate) { return rate >= 4 && rate <= 64 && rate % 4 == 0; }
static int wz2_rate_ok(int rate) { return rate >= 8 && rate <= 24 && rate % 4 == 0; }
static int is_wz2(int fmt) { return fmt == ORC_FMT_FIXED_LIFT || fmt == ORC_FMT_FIXED_BFP; }

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

static int64_t scaled_ld(int64_t N) { return cdiv(N, 16) * 16; }

static size_t stream_bytes(int fmt, int rate, int64_t M, int64_t N) {
  if (fmt == ORC_FMT_ZFP || is_wz2(fmt)) return (size_t)(cdiv(M, 4) * cdiv(N, 4)) * (size_t)(2 * rate);
  fmtdesc d;
  if (!fmt_desc(fmt, &d)) return 0;
  size_t payload = (size_t)M * (size_t)scaled_ld(N) * (size_t)d.bytes;
  size_t scales = (size_t)(cdiv(M, SC_TILE) * cdiv(N, SC_TILE)) * 4;
  return payload + scales;
}

size_t orc_blob_size(int fmt, int rate, int64_t M, int64_t N) {
  if (M <= 0 || N <= 0) return 0;
  if (fmt == ORC_FMT_ZFP && !orc_rate_ok(rate)) return 0;
  if (is_wz2(fmt) && !wz2_rate_ok(rate)) return 0;
  size_t s = stream_bytes(fmt, rate, M, N);
  return s ? ORC_HEADER_BYTES + s : 0;
}

static void wr32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void wr64(uint8_t* p, uint64_t v) {
  for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static uint32_t rd32(const uint8_t* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
static uint64_t rd64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

static void write_header(uint8_t* blob, int fmt, int rate, int64_t M, int64_t N, size_t sbytes) {
  memset(blob, 0, ORC_HEADER_BYTES);
  blob[0] = 'W';
  blob[1] = 'Z';
  blob[2] = '1';
  blob[3] = 0;
  wr32(blob + 4, 1);
  wr32(blob + 8, (uint32_t)fmt);
  wr32(blob + 12, (uint32_t)rate);
  wr64(blob + 16, (uint64_t)M);
  wr64(blob + 24, (uint64_t)N);
  wr64(blob + 32, (uint64_t)sbytes);
  wr32(blob + 40, orc_crc32(blob + ORC_HEADER_BYTES, sbytes));
  wr32(blob + 44, orc_crc32(blob, 44));
}

static int encode_zfp(int fmt, int rate, const double* A, int64_t M, int64_t N, int64_t lda, uint8_t* stream) {
  int64_t BM = cdiv(M, 4), BN = cdiv(N, 4);
  int nwords = rate / 4;
  int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t I = 0; I < BM; I++) {
    uint64_t w[16];
    for (int64_t J = 0; J < BN; J++) {
      float a[16];
      /* edge blocks replicate the last valid row, then the last valid column */
      for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
          int64_t gi = 4 * I + r, gj = 4 * J + c;
          if (gi > M - 1) gi = M - 1;
          if (gj > N - 1) gj = N - 1;
          a[4 * r + c] = (float)A[gi * lda + gj]; /* FP64 -> FP32, round to nearest even */
        }
      int e = fmt == ORC_FMT_ZFP ? orc_wz1_encode_block(a, rate, w)
                                 : orc_wz2_encode_block(a, rate, fmt == ORC_FMT_FIXED_LIFT, w);
      if (e != ORC_OK) {
#pragma omp critical
        err = e;
      }
      uint8_t* dst = stream + (size_t)(I * BN + J) * (size_t)(8 * nwords);
      for (int k = 0; k < nwords; k++) wr64(dst + 8 * k, w[k]);
    }
  }
  return err;
}

static int encode_scaled(int fmt, const double* A, int64_t M, int64_t N, int64_t lda, uint8_t* stream) {
  fmtdesc d;
  fmt_desc(fmt, &d);
  int64_t ld = scaled_ld(N);
  int64_t TM = cdiv(M, SC_TILE), TN = cdiv(N, SC_TILE);
  uint8_t* scales = stream + (size_t)M * (size_t)ld * (size_t)d.bytes;
  int err = ORC_OK;
  for (int64_t i = 0; i < M; i++)
    for (int64_t j = 0; j < N; j++) {
      double v = A[i * lda + j];
      if (!isfinite(v)) return ORC_ENONFINITE;
      if (fabs(v) >= ldexp(1.0, 127)) err = ORC_ERANGE;
    }
  if (err) return err;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ti = 0; ti < TM; ti++) {
    for (int64_t tj = 0; tj < TN; tj++) {
      double amax = 0.0;
      for (int64_t i = ti * SC_TILE; i < M && i < (ti + 1) * SC_TILE; i++)
        for (int64_t j = tj * SC_TILE; j < N && j < (tj + 1) * SC_TILE; j++) {
          double a = fabs(A[i * lda + j]);
          if (a > amax) amax = a;
        }
      float s = amax == 0.0 || d.unscaled ? 1.0f : (float)(amax / d.fmtmax);
      if (s == 0.0f) s = 1.0f; /* amax so small that the scale underflows */
      union {
        float f;
        uint32_t u;
      } su;
      su.f = s;
      wr32(scales + 4 * (size_t)(ti * TN + tj), su.u);
      for (int64_t i = ti * SC_TILE; i < M && i < (ti + 1) * SC_TILE; i++)
        for (int64_t j = tj * SC_TILE; j < N && j < (tj + 1) * SC_TILE; j++) {
          uint32_t bits;
          orc_round_fmt(fmt, A[i * lda + j] / (double)s, &bits);
          uint8_t* p = stream + ((size_t)i * (size_t)ld + (size_t)j) * (size_t)d.bytes;
          for (int b = 0; b < d.bytes; b++) p[b] = (uint8_t)(bits >> (8 * b));
        }
    }
  }
  return ORC_OK;
}

int orc_encode(int fmt, int rate, const double* A, int64_t M, int64_t N, int64_t lda, uint8_t* blob, size_t cap) {
  size_t need = orc_blob_size(fmt, rate, M, N);
  if (!need || cap < need || lda < N) return ORC_EINVAL;
  size_t sbytes = need - ORC_HEADER_BYTES;
  uint8_t* stream = blob + ORC_HEADER_BYTES;
  memset(stream, 0, sbytes);
  int err;
  if (fmt == ORC_FMT_ZFP || is_wz2(fmt))
    err = encode_zfp(fmt, rate, A, M, N, lda, stream);
  else {
    fmtdesc d;
    if (!fmt_desc(fmt, &d)) return ORC_EINVAL;
    rate = 8 * d.bytes;
    err = encode_scaled(fmt, A, M, N, lda, stream);
  }
  if (err) return err;
  write_header(blob, fmt, rate, M, N, sbytes);
  return ORC_OK;
}

static int parse_impl(const uint8_t* blob, size_t len, int* fmt, int* rate, int64_t* M, int64_t* N, int check_stream) {
  if (len < ORC_HEADER_BYTES) return ORC_EFORMAT;
  if (blob[0] != 'W' || blob[1] != 'Z' || blob[2] != '1' || blob[3] != 0) return ORC_EFORMAT;
  if (rd32(blob + 4) != 1) return ORC_EFORMAT;
  if (rd32(blob + 44) != orc_crc32(blob, 44)) return ORC_EFORMAT;
  int f = (int)rd32(blob + 8), r = (int)rd32(blob + 12);
  int64_t m = (int64_t)rd64(blob + 16), n = (int64_t)rd64(blob + 24);
  uint64_t sb = rd64(blob + 32);
  size_t need = orc_blob_size(f, r, m, n);
  if (!need || need != ORC_HEADER_BYTES + sb || len < need) return ORC_EFORMAT;
  if (check_stream && rd32(blob + 40) != orc_crc32(blob + ORC_HEADER_BYTES, (size_t)sb)) return ORC_EFORMAT;
  *fmt = f;
  *rate = r;
  *M = m;
  *N = n;
  return ORC_OK;
}

int orc_parse(const uint8_t* blob, size_t len, int* fmt, int* rate, int64_t* M, int64_t* N) {
  return parse_impl(blob, len, fmt, rate, M, N, 1);
}

/* Decoding a band checks the header and its CRC; the whole-stream CRC is
 * orc_parse's job (it would dominate the time of a small band). */
int orc_decode_rows(const uint8_t* blob, size_t len, int64_t row0, int64_t nrows, double* out, int64_t ldo) {
  int fmt, rate;
  int64_t M, N;
  int e = parse_impl(blob, len, &fmt, &rate, &M, &N, 0);
  if (e) return e;
  if (row0 < 0 || nrows < 0 || row0 + nrows > M || ldo < N) return ORC_EINVAL;
  const uint8_t* stream = blob + ORC_HEADER_BYTES;
  if (fmt == ORC_FMT_ZFP || is_wz2(fmt)) {
    if (row0 % 4) return ORC_EINVAL;
    int64_t BN = cdiv(N, 4);
    int nwords = rate / 4;
    int64_t I0 = row0 / 4, I1 = cdiv(row0 + nrows, 4);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t I = I0; I < I1; I++) {
      uint64_t w[16];
      for (int64_t J = 0; J < BN; J++) {
        const uint8_t* src = stream + (size_t)(I * BN + J) * (size_t)(8 * nwords);
        for (int k = 0; k < nwords; k++) w[k] = rd64(src + 8 * k);
        double v[16];
        if (fmt == ORC_FMT_ZFP) {
          int32_t q[16];
          int emax, nz;
          orc_wz1_decode_block(w, rate, q, &emax, &nz);
          for (int i = 0; i < 16; i++) v[i] = orc_wz1_value(q[i], emax, nz);
        } else {
          orc_wz2_decode_block(w, rate, fmt == ORC_FMT_FIXED_LIFT, v);
        }
        for (int r = 0; r < 4; r++)
          for (int c = 0; c < 4; c++) {
            int64_t gi = 4 * I + r, gj = 4 * J + c;
            if (gi >= row0 + nrows || gj >= N) continue;
            out[(gi - row0) * ldo + gj] = v[4 * r + c];
          }
      }
    }
    return ORC_OK;
  }
  fmtdesc d;
  fmt_desc(fmt, &d);
  int64_t ld = scaled_ld(N);
  int64_t TN = cdiv(N, SC_TILE);
  const uint8_t* scales = stream + (size_t)M * (size_t)ld * (size_t)d.bytes;
#pragma omp parallel for schedule(static)
  for (int64_t i = row0; i < row0 + nrows; i++)
    for (int64_t j = 0; j < N; j++) {
      union {
        float f;
        uint32_t u;
      } su;
      su.u = rd32(scales + 4 * (size_t)((i / SC_TILE) * TN + j / SC_TILE));
      const uint8_t* p = stream + ((size_t)i * (size_t)ld + (size_t)j) * (size_t)d.bytes;
      uint32_t bits = 0;
      for (int b = 0; b < d.bytes; b++) bits |= (uint32_t)p[b] << (8 * b);
      out[(i - row0) * ldo + j] = (double)su.f * orc_fmt_decode(fmt, bits);
    }
  return ORC_OK;
}

/* -------------------------------------------------------------------- GEMV */
void orc_gemv64(const double* A, int64_t M, int64_t N, int64_t lda, const double* X, int R, int64_t ldx,
                double* Y, int64_t ldy) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; i++)
    for (int r = 0; r < R; r++) {
      double sum = 0.0;
      for (int64_t j = 0; j < N; j++) sum += A[i * lda + j] * X[(size_t)r * ldx + j];
      Y[(size_t)r * ldy + i] = sum;
    }
}

void orc_gemv_mp(const double* A, int64_t M, int64_t N, int64_t lda, const double* x, float* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; i++) {
    double sum = 0.0;
    for (int64_t j = 0; j < N; j++) {
      float product = (float)A[i * lda + j] * (float)x[j];
      sum += (double)product;
    }
    y[i] = (float)sum;
  }
}

void orc_state_update(double* s, int64_t M, const double* Y, int R, int64_t ldy, double decay) {
  for (int r = 0; r < R; r++)
    for (int64_t i = 0; i < M; i++) s[i] = decay * s[i] + Y[(size_t)r * ldy + i];
}

/* ---------------------------------------------------- WZ3 matrix layout */
/* Stream: [tol: f64] [index: one u64 per run, band-major; bits 0..55 the
 * byte offset of the run within the block area, bits 56..63 its width W]
 * [block area: the runs one after another].  A run is up to 32 consecutive
 * blocks of one band (the last run of a band may be shorter); its nb blocks
 * of nw = bytes(W) / 8 words are stored word-interleaved: word k of block b
 * at byte 8 (k nb + b) of the run (the same bytes as nb blocks side by side,
 * in the order in which nb readers each taking one block load them
 * together).  Edge blocks replicate the last valid row, then column, as
 * WZ1/WZ2. */
static int64_t wz3_runs_per_band(int64_t N) { return cdiv(cdiv(N, 4), 32); }

size_t orc_wz3_max_blob_size(int64_t M, int64_t N) {
  if (M <= 0 || N <= 0) return 0;
  const int64_t BM = cdiv(M, 4), BN = cdiv(N, 4);
  return ORC_HEADER_BYTES + 8 + 8 * (size_t)(BM * wz3_runs_per_band(N)) +
         (size_t)(BM * BN) * (size_t)orc_wz3_block_bytes(31);
}

int orc_wz3_encode_matrix(const double* A, int64_t M, int64_t N, int64_t lda, double tol, uint8_t* blob, size_t cap,
                          size_t* len) {
  if (M <= 0 || N <= 0 || lda < N || !(tol >= 0.0) || cap < orc_wz3_max_blob_size(M, N)) return ORC_EINVAL;
  const int64_t BM = cdiv(M, 4), BN = cdiv(N, 4), RB = wz3_runs_per_band(N);
  uint8_t* stream = blob + ORC_HEADER_BYTES;
  uint8_t* index = stream + 8;
  uint8_t* area = index + 8 * (size_t)(BM * RB);
  union {
    double d;
    uint64_t u;
  } t;
  t.d = tol;
  wr64(stream, t.u);
  uint64_t off = 0;
  float blocks[32 * 16];
  uint64_t words[32 * 9];
  for (int64_t I = 0; I < BM; I++)
    for (int64_t r = 0; r < RB; r++) {
      const int64_t J0 = 32 * r, nb = (BN - J0) < 32 ? (BN - J0) : 32;
      for (int64_t b = 0; b < nb; b++)
        for (int rr = 0; rr < 4; rr++)
          for (int c = 0; c < 4; c++) {
            int64_t gi = 4 * I + rr, gj = 4 * (J0 + b) + c;
            if (gi > M - 1) gi = M - 1;
            if (gj > N - 1) gj = N - 1;
            blocks[16 * b + 4 * rr + c] = (float)A[gi * lda + gj];
          }
      int W;
      int e = orc_wz3_encode_run(blocks, (int)nb, tol, 1, words, &W);
      if (e != ORC_OK) return e;
      wr64(index + 8 * (size_t)(I * RB + r), off | ((uint64_t)W << 56));
      const int nw = orc_wz3_block_bytes(W) / 8;
      for (int64_t b = 0; b < nb; b++) /* block b's words: words[b nw + k] */
        for (int k = 0; k < nw; k++) wr64(area + off + 8 * (uint64_t)(k * nb + b), words[b * nw + k]);
      off += (uint64_t)(nb * nw * 8);
    }
  const size_t sbytes = 8 + 8 * (size_t)(BM * RB) + (size_t)off;
  write_header(blob, ORC_FMT_FIXED_ACC, 0, M, N, sbytes);
  *len = ORC_HEADER_BYTES + sbytes;
  return ORC_OK;
}

int orc_wz3_decode_matrix(const uint8_t* blob, size_t len, double* out, int64_t ldo, double* tol) {
  if (len < ORC_HEADER_BYTES || blob[0] != 'W' || blob[1] != 'Z' || blob[2] != '1' || blob[3] != 0 ||
      rd32(blob + 4) != 1 || rd32(blob + 44) != orc_crc32(blob, 44) || rd32(blob + 8) != ORC_FMT_FIXED_ACC)
    return ORC_EFORMAT;
  const int64_t M = (int64_t)rd64(blob + 16), N = (int64_t)rd64(blob + 24);
  const uint64_t sb = rd64(blob + 32);
  if (M <= 0 || N <= 0 || ldo < N || len < ORC_HEADER_BYTES + sb) return ORC_EFORMAT;
  const uint8_t* stream = blob + ORC_HEADER_BYTES;
  if (rd32(blob + 40) != orc_crc32(stream, (size_t)sb)) return ORC_EFORMAT;
  const int64_t BM = cdiv(M, 4), BN = cdiv(N, 4), RB = wz3_runs_per_band(N);
  if (sb < 8 + 8 * (uint64_t)(BM * RB)) return ORC_EFORMAT;
  union {
    double d;
    uint64_t u;
  } t;
  t.u = rd64(stream);
  if (tol) *tol = t.d;
  const uint8_t* index = stream + 8;
  const uint8_t* area = index + 8 * (size_t)(BM * RB);
  const uint64_t area_bytes = sb - 8 - 8 * (uint64_t)(BM * RB);
  for (int64_t I = 0; I < BM; I++)
    for (int64_t r = 0; r < RB; r++) {
      const uint64_t ent = rd64(index + 8 * (size_t)(I * RB + r));
      const uint64_t off = ent & ((1ull << 56) - 1);
      const int W = (int)(ent >> 56);
      const int64_t J0 = 32 * r, nb = (BN - J0) < 32 ? (BN - J0) : 32;
      const int bb = orc_wz3_block_bytes(W);
      if (W > 31 || off + (uint64_t)(nb * bb) > area_bytes) return ORC_EFORMAT;
      for (int64_t b = 0; b < nb; b++) {
        uint64_t w[9];
        for (int k = 0; k < bb / 8; k++) w[k] = rd64(area + off + 8 * (uint64_t)(k * nb + b));
        double v[16];
        orc_wz3_decode_block(w, W, 1, v);
        for (int rr = 0; rr < 4; rr++)
          for (int c = 0; c < 4; c++) {
            const int64_t gi = 4 * I + rr, gj = 4 * (J0 + b) + c;
            if (gi < M && gj < N) out[gi * ldo + gj] = v[4 * rr + c];
          }
      }
    }
  return ORC_OK;
}
