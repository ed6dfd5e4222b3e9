// whff_encode.cpp -- host side of the library: blob container, CRC-32 and the
// offline encoders (Sec. 4.3: "compression can be done offline ... the
// encoding part is completely out of the time budget").
//
// WZ1 is this project's reading of zfp's fixed-rate mode (Sec. 4.3, Table 2):
// per 4x4 block, an FP32 block-floating-point quantiser with 26 fraction bits
// below the block exponent, a reversible integer lift (rows, then columns),
// sequency ordering, negabinary words and an embedded bit-plane coder with
// group tests that stops exactly at 16*rate bits.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "whff.h"
#include "whff_blob.h"

namespace whff {
void set_error(const std::string& msg);  // whff_runtime.cu

// ------------------------------------------------------------------ container
int elem_bytes(int fmt) {
  switch (fmt) {
    case WHFF_FMT_BF16:
    case WHFF_FMT_FP16:
      return 2;
    case WHFF_FMT_FP8E4M3:
      return 1;
    case WHFF_FMT_FP32:
      return 4;
    default:
      return 0;
  }
}

bool rate_valid(int rate) { return rate >= 4 && rate <= 64 && (rate & 3) == 0; }
bool wz2_rate_valid(int rate) { return rate >= 8 && rate <= 24 && (rate & 3) == 0; }
bool is_blocked(int fmt) { return fmt == WHFF_FMT_ZFP || fmt == WHFF_FMT_FIXED_LIFT || fmt == WHFF_FMT_FIXED_BFP; }

uint64_t stream_size(int fmt, int rate, int64_t M, int64_t N) {
  if (!shape_ok(M, N)) return 0;
  if (is_blocked(fmt)) {
    if (fmt == WHFF_FMT_ZFP ? !rate_valid(rate) : !wz2_rate_valid(rate)) return 0;
    return (uint64_t)ceil_div(M, 4) * (uint64_t)ceil_div(N, 4) * (uint64_t)(2 * rate);
  }
  int eb = elem_bytes(fmt);
  if (!eb) return 0;
  return (uint64_t)M * (uint64_t)scaled_ld(N) * (uint64_t)eb +
         (uint64_t)ceil_div(M, kScaleTile) * (uint64_t)ceil_div(N, kScaleTile) * 4u;
}

// Slicing-by-8 CRC-32 (IEEE, reflected 0xEDB88320).
namespace {
struct CrcTables {
  uint32_t t[8][256];
  CrcTables() {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
      t[0][i] = c;
    }
    for (uint32_t i = 0; i < 256; ++i)
      for (int s = 1; s < 8; ++s) t[s][i] = (t[s - 1][i] >> 8) ^ t[0][t[s - 1][i] & 0xFF];
  }
};
const CrcTables& crc_tables() {
  static const CrcTables tabs;
  return tabs;
}
inline void st32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = uint8_t(v >> (8 * i));
}
inline void st64(uint8_t* p, uint64_t v) {
  for (int i = 0; i < 8; ++i) p[i] = uint8_t(v >> (8 * i));
}
inline uint32_t ld32(const uint8_t* p) {
  uint32_t v = 0;
  for (int i = 3; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}
inline uint64_t ld64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}
}  // namespace

uint32_t crc32_update(uint32_t crc, const uint8_t* p, size_t n) {
  const auto& T = crc_tables().t;
  uint32_t c = ~crc;
  while (n >= 8) {
    uint32_t lo = ld32(p) ^ c, hi = ld32(p + 4);
    c = T[7][lo & 0xFF] ^ T[6][(lo >> 8) & 0xFF] ^ T[5][(lo >> 16) & 0xFF] ^ T[4][lo >> 24] ^ T[3][hi & 0xFF] ^
        T[2][(hi >> 8) & 0xFF] ^ T[1][(hi >> 16) & 0xFF] ^ T[0][hi >> 24];
    p += 8;
    n -= 8;
  }
  while (n--) c = (c >> 8) ^ T[0][(c ^ *p++) & 0xFF];
  return ~c;
}

void write_header(uint8_t* blob, int fmt, int rate, int64_t M, int64_t N, uint64_t sbytes, uint32_t crc_stream) {
  std::memset(blob, 0, kHeaderBytes);
  std::memcpy(blob, "WZ1\0", 4);
  st32(blob + 4, 1);
  st32(blob + 8, (uint32_t)fmt);
  st32(blob + 12, (uint32_t)rate);
  st64(blob + 16, (uint64_t)M);
  st64(blob + 24, (uint64_t)N);
  st64(blob + 32, sbytes);
  st32(blob + 40, crc_stream);
  st32(blob + 44, crc32(blob, 44));
}

int read_header(const uint8_t* blob, size_t len, BlobInfo* info, bool check_stream) {
  if (!blob || len < (size_t)kHeaderBytes) return WHFF_EFORMAT;
  if (std::memcmp(blob, "WZ1\0", 4) != 0 || ld32(blob + 4) != 1) return WHFF_EFORMAT;
  if (ld32(blob + 44) != crc32(blob, 44)) return WHFF_EFORMAT;
  BlobInfo b;
  b.fmt = (int)ld32(blob + 8);
  b.rate = (int)ld32(blob + 12);
  b.M = (int64_t)ld64(blob + 16);
  b.N = (int64_t)ld64(blob + 24);
  b.stream_bytes = ld64(blob + 32);
  b.crc_stream = ld32(blob + 40);
  b.crc_header = ld32(blob + 44);
  if (!shape_ok(b.M, b.N)) return WHFF_EFORMAT;
  uint64_t want = stream_size(b.fmt, b.rate, b.M, b.N);
  if (b.fmt == WHFF_FMT_FIXED_ACC && b.rate == 0) {  // variable length, within its bounds
    const int64_t BM = ceil_div(b.M, 4), BN = ceil_div(b.N, 4), RB = ceil_div(BN, 32);
    const uint64_t lo = 8 + 8 * (uint64_t)(BM * RB) + 8 * (uint64_t)(BM * BN);
    const uint64_t hi = 8 + 8 * (uint64_t)(BM * RB) + 64 * (uint64_t)(BM * BN);
    if (b.stream_bytes < lo || b.stream_bytes > hi) return WHFF_EFORMAT;
    want = b.stream_bytes;
  }
  if (!want || want != b.stream_bytes || len < kHeaderBytes + want) return WHFF_EFORMAT;
  if (!is_blocked(b.fmt) && b.fmt != WHFF_FMT_FIXED_ACC && b.rate != 8 * elem_bytes(b.fmt)) return WHFF_EFORMAT;
  if (check_stream && crc32(blob + kHeaderBytes, want) != b.crc_stream) return WHFF_EFORMAT;
  *info = b;
  return WHFF_OK;
}

// ------------------------------------------------------------------ WZ1 coder
namespace {

// Sequency order of the 16 lift coefficients: slot ranks (0, 1, 2, 2) for
// (s, d, d0, e); sort key (rank_i + rank_j, max rank, i, j).  kSeq[k] is the
// row-major index 4*i + j of the k-th coefficient.
struct SeqTable {
  int idx[16];
  SeqTable() {
    const int rank[4] = {0, 1, 2, 2};
    std::vector<int> v(16);
    for (int k = 0; k < 16; ++k) v[k] = k;
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
      int ia = a >> 2, ja = a & 3, ib = b >> 2, jb = b & 3;
      int sa = rank[ia] + rank[ja], sb = rank[ib] + rank[jb];
      if (sa != sb) return sa < sb;
      int ma = std::max(rank[ia], rank[ja]), mb = std::max(rank[ib], rank[jb]);
      if (ma != mb) return ma < mb;
      if (ia != ib) return ia < ib;
      return ja < jb;
    });
    for (int k = 0; k < 16; ++k) idx[k] = v[k];
  }
};
const SeqTable& seq_table() {
  static const SeqTable t;
  return t;
}

// Forward reversible lift of (a, b, c, d) -> (s, dd, d0, e), two's complement mod 2^32.
inline void lift_fwd(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  auto half = [](uint32_t v) { return (uint32_t)((int32_t)v >> 1); };
  uint32_t lo_diff = b - a;
  uint32_t lo_mean = a + half(lo_diff);
  uint32_t hi_diff = d - c;
  uint32_t hi_mean = c + half(hi_diff);
  uint32_t mean_diff = hi_mean - lo_mean;
  a = lo_mean + half(mean_diff);  // s
  b = mean_diff;                  // d
  d = hi_diff - lo_diff;          // e
  c = lo_diff;                    // d0
}

// LSB-first writer into a zeroed word array, one block at a time.
struct BitSink {
  uint64_t* w;
  int pos = 0;
  void put(uint64_t v, int n) {  // the low n (<= 32) bits of v
    if (n <= 0) return;
    v &= (n == 64) ? ~0ull : ((1ull << n) - 1);
    int s = pos & 63;
    w[pos >> 6] |= v << s;
    if (s + n > 64) w[(pos >> 6) + 1] |= v >> (64 - s);
    pos += n;
  }
};

// FP32 exponent e with 2^(e-1) <= |f| < 2^e (f != 0), from the bit pattern.
inline int f32_exponent(uint32_t bits) {
  uint32_t E = (bits >> 23) & 0xFF;
  if (E) return (int)E - 126;
  uint32_t m = bits & 0x7FFFFF;
  return (32 - __builtin_clz(m)) - 149;
}

// trunc(f * 2^(prec - emax)) from the FP32 bit pattern, by shifting the significand.
inline int32_t f32_to_fixed(uint32_t bits, int emax, int prec = kWz1Prec) {
  uint32_t E = (bits >> 23) & 0xFF;
  uint32_t m = bits & 0x7FFFFF;
  int sh;  // f = sig * 2^(sh0), q = sig * 2^(sh0 + 26 - emax)
  uint32_t sig;
  if (E) {
    sig = m | 0x800000u;
    sh = (int)E - 150 + prec - emax;
  } else {
    sig = m;
    sh = -149 + prec - emax;
  }
  uint32_t mag = sh >= 0 ? (sig << sh) : (sh <= -32 ? 0u : (sig >> -sh));
  return (bits >> 31) ? -(int32_t)mag : (int32_t)mag;
}

int encode_block(const float* vals, int rate, uint64_t* out) {
  const int nw = rate / 4;
  std::memset(out, 0, sizeof(uint64_t) * nw);
  uint32_t bits[16];
  int emax = INT32_MIN;
  for (int i = 0; i < 16; ++i) {
    std::memcpy(&bits[i], &vals[i], 4);
    uint32_t E = (bits[i] >> 23) & 0xFF;
    if (E == 0xFF) return WHFF_ENONFINITE;
    if (E >= 254) return WHFF_ERANGE;  // |f| >= 2^127
    if (bits[i] & 0x7FFFFFFFu) emax = std::max(emax, f32_exponent(bits[i]));
  }
  if (emax <= kWz1Emin) return WHFF_OK;  // zero block
  uint32_t c[16];
  for (int i = 0; i < 16; ++i) c[i] = (uint32_t)f32_to_fixed(bits[i], emax);
  for (int r = 0; r < 4; ++r) lift_fwd(c[4 * r], c[4 * r + 1], c[4 * r + 2], c[4 * r + 3]);
  for (int j = 0; j < 4; ++j) lift_fwd(c[j], c[4 + j], c[8 + j], c[12 + j]);
  const int* seq = seq_table().idx;
  uint32_t u[16];
  for (int k = 0; k < 16; ++k) u[k] = (c[seq[k]] + 0xAAAAAAAAu) ^ 0xAAAAAAAAu;  // negabinary

  BitSink bs{out};
  bs.put(1, 1);
  bs.put((uint64_t)(emax + 127), 8);
  int budget = 16 * rate - 9;
  int n = 0;
  for (int k = 31; k >= 0 && budget > 0; --k) {
    uint32_t plane = 0;
    for (int i = 0; i < 16; ++i) plane |= ((u[i] >> k) & 1u) << i;
    int m = std::min(n, budget);
    bs.put(plane, m);
    budget -= m;
    uint32_t rest = plane >> n;  // bit 0 <-> coefficient n
    while (n < 16 && budget > 0) {
      if (!rest) {  // group test: nothing left in this plane
        bs.put(0, 1);
        --budget;
        break;
      }
      bs.put(1, 1);
      --budget;
      int z = __builtin_ctz(rest);
      int run = 15 - n;  // positions n..14 are sent, 15 is implied
      if (z >= run) {
        int e = std::min(run, budget);
        bs.put(0, e);
        budget -= e;
        n = 16;  // (if the budget ran out the coder stops anyway)
        break;
      }
      int e = std::min(z + 1, budget);
      bs.put(1ull << z, e);
      budget -= e;
      if (e < z + 1) break;
      n += z + 1;
      rest >>= z + 1;
    }
  }
  return WHFF_OK;
}

// ------------------------------------------------ WZ2 fixed-allocation coder
constexpr int kWz2Prec = 24;
constexpr int kWz2Kmax = 27;

inline int wz2_width(int rate) { return (16 * rate - 13) / 16; }

// (4F) applied to one 4-vector: (x0+x1+x2+x3, 2(x2+x3-x0-x1), 4(x1-x0), 4((x3-x2)-(x1-x0)))
inline void lin_fwd4(int64_t& a, int64_t& b, int64_t& c, int64_t& d) {
  const int64_t lo = a + b, hi = c + d, dl = b - a, dh = d - c;
  a = lo + hi;
  b = 2 * (hi - lo);
  c = 4 * dl;
  d = 4 * (dh - dl);
}

// c / 2^K rounded half to even, in integers (c exact, K >= 0).
inline int64_t shift_round_even(int64_t c, int K) {
  if (K == 0) return c;
  const int64_t fl = c >> K;  // floor
  const int64_t rem = c - fl * ((int64_t)1 << K);
  const int64_t half = (int64_t)1 << (K - 1);
  return (rem > half || (rem == half && (fl & 1))) ? fl + 1 : fl;
}

int encode_block_wz2(const float* vals, int rate, bool lift, uint64_t* out) {
  const int nw = rate / 4;
  std::memset(out, 0, sizeof(uint64_t) * nw);
  uint32_t bits[16];
  int emax = INT32_MIN;
  for (int i = 0; i < 16; ++i) {
    std::memcpy(&bits[i], &vals[i], 4);
    uint32_t E = (bits[i] >> 23) & 0xFF;
    if (E == 0xFF) return WHFF_ENONFINITE;
    if (E >= 254) return WHFF_ERANGE;
    if (bits[i] & 0x7FFFFFFFu) emax = std::max(emax, f32_exponent(bits[i]));
  }
  if (emax <= kWz1Emin) return WHFF_OK;
  int64_t c[16];
  for (int i = 0; i < 16; ++i) c[i] = f32_to_fixed(bits[i], emax, kWz2Prec);
  if (lift) {
    for (int r = 0; r < 4; ++r) lin_fwd4(c[4 * r], c[4 * r + 1], c[4 * r + 2], c[4 * r + 3]);
    for (int j = 0; j < 4; ++j) lin_fwd4(c[j], c[4 + j], c[8 + j], c[12 + j]);
  }
  const int* seq = seq_table().idx;
  int64_t ord[16];
  for (int k = 0; k < 16; ++k) ord[k] = lift ? c[seq[k]] : c[k];
  const int W = wz2_width(rate);
  const int64_t lo = -((int64_t)1 << (W - 1)), hi = ((int64_t)1 << (W - 1)) - 1;
  // The smallest K that fits is at least bitlen(max |c|) - W: below it the
  // largest coefficient rounds to a magnitude >= 2^W.  Start the search there.
  uint64_t mag = 0;
  for (int k = 0; k < 16; ++k) mag = std::max(mag, (uint64_t)(ord[k] < 0 ? -ord[k] : ord[k]));
  int blen = 0;
  while (blen < 64 && (mag >> blen) != 0) ++blen;
  int K = std::min(std::max(0, blen - W), kWz2Kmax);
  int64_t v[16];
  for (;; ++K) {
    bool fits = true;
    for (int k = 0; k < 16; ++k) {
      v[k] = shift_round_even(ord[k], K);
      fits &= v[k] >= lo && v[k] <= hi;
    }
    if (fits || K == kWz2Kmax) break;
  }
  BitSink bs{out};
  bs.put((uint64_t)(emax + 127), 8);
  bs.put((uint64_t)K, 5);
  for (int k = 0; k < 16; ++k) bs.put((uint64_t)(v[k] - lo), W);
  return WHFF_OK;
}

// ------------------------------------------------------- WZ3 (fixed accuracy)
// WZ2's block (emax, shift K, 16 offset-binary fields of the lifted, sequency
// ordered coefficients) with, per block, the largest K in 0..27 whose decoded
// block is within tol of the FP32 input (max absolute error) -- never below the
// smallest K whose fields fit 31 bits -- and one field width per run of up to
// 32 blocks of a band, the widest its blocks need.
constexpr int kWz3Wmax = 31;

inline int wz3_block_bytes(int W) { return 8 * ((13 + 16 * W + 63) / 64); }

// (2G) applied to one 4-vector (s, d, d0, e): the exact inverse of lin_fwd4 up
// to the factor 8 that the decoded value's exponent absorbs.
inline void lin_inv4(int64_t& a, int64_t& b, int64_t& c, int64_t& d) {
  const int64_t s2 = 2 * a, x = b, y = c, z = d;
  a = s2 - x - y;
  b = s2 - x + y;
  c = s2 + x - y - z;
  d = s2 + x + y + z;
}

struct Wz3Block {
  int emax = 0, K = 0, need = 0;  // need 0: a zero block
  int64_t v[16] = {};             // sequency order
};

// One block of 16 FP32 values (row-major 4x4) at tolerance tol.
int wz3_block(const float* vals, double tol, Wz3Block* out) {
  *out = Wz3Block();
  uint32_t bits[16];
  int emax = INT32_MIN;
  for (int i = 0; i < 16; ++i) {
    std::memcpy(&bits[i], &vals[i], 4);
    const uint32_t E = (bits[i] >> 23) & 0xFF;
    if (E == 0xFF) return WHFF_ENONFINITE;
    if (E >= 254) return WHFF_ERANGE;
    if (bits[i] & 0x7FFFFFFFu) emax = std::max(emax, f32_exponent(bits[i]));
  }
  if (emax <= kWz1Emin) return WHFF_OK;
  int64_t c[16];
  for (int i = 0; i < 16; ++i) c[i] = f32_to_fixed(bits[i], emax, kWz2Prec);
  for (int r = 0; r < 4; ++r) lin_fwd4(c[4 * r], c[4 * r + 1], c[4 * r + 2], c[4 * r + 3]);
  for (int j = 0; j < 4; ++j) lin_fwd4(c[j], c[4 + j], c[8 + j], c[12 + j]);
  const int* seq = seq_table().idx;
  int64_t ord[16];
  for (int k = 0; k < 16; ++k) ord[k] = c[seq[k]];
  const int64_t lim_lo = -((int64_t)1 << (kWz3Wmax - 1)), lim_hi = ((int64_t)1 << (kWz3Wmax - 1)) - 1;
  int Kf = 0;
  for (; Kf < kWz2Kmax; ++Kf) {
    bool fits = true;
    for (int k = 0; k < 16 && fits; ++k) {
      const int64_t t = shift_round_even(ord[k], Kf);
      fits = t >= lim_lo && t <= lim_hi;
    }
    if (fits) break;
  }
  // A cheap necessary condition first.  The decoded block minus the FP32 input
  // is D u - t, with u = 2^(emax-30), t the truncation remainder of the block
  // floating point, D = (2G) (V 2^K - C) (2G)^T.  The column sums of 2G are
  // (8, 0, 0, 0), so the mean of D over the block is 4 E00, E00 the DC
  // coefficient's rounding error.  The largest error is at least the absolute
  // mean, |mean(t) - 4 E00 u|: a shift for which that exceeds tol (with a
  // margin far above the rounding of this sum) cannot be the answer.
  double tsum = 0.0, tabs = 0.0;
  const double grid = std::ldexp(1.0, emax - kWz2Prec);  // the block floating point's step
  for (int i = 0; i < 16; ++i) {
    const double a = (double)vals[i];
    const double t = a - std::trunc(a / grid) * grid;  // exact: a and its truncation share the grid
    tsum += t;
    tabs += std::fabs(t);
  }
  const double u = std::ldexp(1.0, emax - 30), tmean = tsum / 16.0;
  const int64_t c00 = ord[0];  // sequency slot 0: the DC coefficient
  int64_t v[16];
  int K = kWz2Kmax;
  for (;; --K) {
    if (K != Kf) {
      const int64_t e00 = shift_round_even(c00, K) * ((int64_t)1 << K) - c00;
      const double m = 4.0 * (double)e00 * u;
      const double lb = std::fabs(tmean - m) - 1e-12 * (tabs + std::fabs(m));
      if (lb > tol) continue;
    }
    for (int k = 0; k < 16; ++k) v[k] = shift_round_even(ord[k], K);
    int64_t T[16];
    for (int k = 0; k < 16; ++k) T[seq[k]] = v[k];
    for (int j = 0; j < 4; ++j) lin_inv4(T[j], T[4 + j], T[8 + j], T[12 + j]);
    for (int r = 0; r < 4; ++r) lin_inv4(T[4 * r], T[4 * r + 1], T[4 * r + 2], T[4 * r + 3]);
    // |T| < 2^40 and 2^(K+emax-30) is a normal double: the product is exact, as ldexp
    const double scale = std::ldexp(1.0, K + emax - 30);
    bool within = true;
    for (int i = 0; i < 16 && within; ++i) within = std::fabs((double)vals[i] - (double)T[i] * scale) <= tol;
    if (within || K == Kf) break;
  }
  int W = 1;
  for (int k = 0; k < 16; ++k)
    while (v[k] < -((int64_t)1 << (W - 1)) || v[k] > ((int64_t)1 << (W - 1)) - 1) ++W;
  out->emax = emax;
  out->K = K;
  out->need = W;
  for (int k = 0; k < 16; ++k) out->v[k] = v[k];
  return WHFF_OK;
}

// Block (emax, K, v) written with field width W (nothing for a zero block).
void wz3_put(const Wz3Block& b, int W, uint64_t* out) {
  const int nw = wz3_block_bytes(W) / 8;
  std::memset(out, 0, sizeof(uint64_t) * nw);
  if (b.need == 0) return;
  BitSink bs{out};
  bs.put((uint64_t)(b.emax + 127), 8);
  bs.put((uint64_t)b.K, 5);
  for (int k = 0; k < 16; ++k) bs.put((uint64_t)(b.v[k] + ((int64_t)1 << (W - 1))), W);
}

// --------------------------------------------------------- scaled formats
struct FmtSpec {
  int mant, emin, bias, ebits;
  double fmtmax;  // the value a tile's amax is scaled to; 0: no scaling (scale 1)
};
bool fmt_spec(int fmt, FmtSpec* s) {
  switch (fmt) {
    case WHFF_FMT_BF16: *s = {7, -126, 127, 8, 1.0}; return true;
    case WHFF_FMT_FP16: *s = {10, -14, 15, 5, 32768.0}; return true;
    case WHFF_FMT_FP8E4M3: *s = {3, -6, 7, 4, 448.0}; return true;
    case WHFF_FMT_FP32: *s = {23, -126, 127, 8, 0.0}; return true;
    default: return false;
  }
}

// Round a finite double to the format (ties to even, saturating at fmtmax) and
// return the bit pattern, working on the double's integer significand.
uint32_t round_to_format(double v, const FmtSpec& f) {
  uint64_t db;
  std::memcpy(&db, &v, 8);
  uint32_t sign = (uint32_t)(db >> 63);
  uint32_t sign_bit = sign << (f.mant + f.ebits);
  int E = (int)((db >> 52) & 0x7FF);
  uint64_t frac = db & ((1ull << 52) - 1);
  // saturation pattern (the format's largest finite value when it is unscaled)
  const double fmtmax = f.fmtmax > 0.0 ? f.fmtmax : std::ldexp(2.0 - std::ldexp(1.0, -f.mant), (1 << f.ebits) - 2 - f.bias);
  int sat_e;
  double sat_m = std::frexp(fmtmax, &sat_e);  // fmtmax = sat_m * 2^sat_e
  uint32_t sat_pat = ((uint32_t)(sat_e - 1 + f.bias) << f.mant) |
                     (uint32_t)(std::ldexp(sat_m, f.mant + 1) - std::ldexp(1.0, f.mant));
  if (E == 0) return sign_bit;  // zero or FP64 subnormal: far below every format's quantum
  uint64_t sig = frac | (1ull << 52);
  int ex = std::max(E - 1023, f.emin);           // exponent of the quantum's binade
  int sh = 52 + ex - f.mant - (E - 1023);        // sig >> sh = value / quantum
  uint64_t q;
  if (sh >= 64) {
    q = 0;
  } else {
    q = sig >> sh;
    uint64_t rem = sig & ((1ull << sh) - 1);
    uint64_t half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
  }
  if (q == 0) return sign_bit;
  if (q >> (f.mant + 1)) {  // rounding carried into the next binade
    q >>= 1;
    ++ex;
  }
  // compare against fmtmax: value = q * 2^(ex - mant)
  if (std::ldexp((double)q, ex - f.mant) > fmtmax) return sign_bit | sat_pat;
  if (q < (1ull << f.mant)) return sign_bit | (uint32_t)q;  // subnormal of the format
  return sign_bit | ((uint32_t)(ex + f.bias) << f.mant) | (uint32_t)(q - (1ull << f.mant));
}

// -------------------------------------------------------------- band encoder
template <class F>
void parallel_for(int64_t n, int nthreads, F&& fn) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  nthreads = (int)std::min<int64_t>(nthreads, std::max<int64_t>(1, n));
  if (nthreads == 1) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&] {
      for (int64_t i; (i = next.fetch_add(1)) < n;) fn(i);
    });
  for (auto& th : pool) th.join();
}

int encode_band_zfp(uint8_t* stream, const BlobInfo& b, const double* band, int64_t row0, int64_t nrows,
                    int64_t lda, int nthreads) {
  const int64_t BN = ceil_div(b.N, 4);
  const int nw = b.rate / 4;
  const int64_t I0 = row0 / 4, I1 = ceil_div(row0 + nrows, 4);
  std::atomic<int> err{WHFF_OK};
  parallel_for(I1 - I0, nthreads, [&](int64_t ii) {
    const int64_t I = I0 + ii;
    float vals[16];
    uint64_t w[16];
    for (int64_t J = 0; J < BN; ++J) {
      for (int r = 0; r < 4; ++r) {
        int64_t gi = std::min(4 * I + r, b.M - 1);
        if (gi >= row0 + nrows) gi = row0 + nrows - 1;  // only the matrix's last band is ragged
        const double* row = band + (gi - row0) * lda;
        for (int c = 0; c < 4; ++c) vals[4 * r + c] = (float)row[std::min(4 * J + c, b.N - 1)];
      }
      int e = b.fmt == WHFF_FMT_ZFP ? encode_block(vals, b.rate, w)
                                    : encode_block_wz2(vals, b.rate, b.fmt == WHFF_FMT_FIXED_LIFT, w);
      if (e != WHFF_OK) err.store(e);
      uint8_t* dst = stream + (uint64_t)(I * BN + J) * (uint64_t)(8 * nw);
      for (int k = 0; k < nw; ++k) st64(dst + 8 * k, w[k]);
    }
  });
  return err.load();
}

int encode_band_scaled(uint8_t* stream, const BlobInfo& b, const double* band, int64_t row0, int64_t nrows,
                       int64_t lda, int nthreads) {
  FmtSpec f;
  fmt_spec(b.fmt, &f);
  const int eb = elem_bytes(b.fmt);
  const int64_t ld = scaled_ld(b.N), TN = ceil_div(b.N, kScaleTile);
  uint8_t* scales = stream + (uint64_t)b.M * (uint64_t)ld * (uint64_t)eb;
  const int64_t T0 = row0 / kScaleTile, T1 = ceil_div(row0 + nrows, kScaleTile);
  std::atomic<int> err{WHFF_OK};
  parallel_for((T1 - T0) * TN, nthreads, [&](int64_t t) {
    const int64_t ti = T0 + t / TN, tj = t % TN;
    const int64_t i0 = ti * kScaleTile, i1 = std::min(b.M, i0 + kScaleTile);
    const int64_t j0 = tj * kScaleTile, j1 = std::min(b.N, j0 + kScaleTile);
    double amax = 0.0;
    for (int64_t i = i0; i < i1; ++i)
      for (int64_t j = j0; j < j1; ++j) {
        double a = band[(i - row0) * lda + j];
        if (!std::isfinite(a)) {
          err.store(WHFF_ENONFINITE);
          return;
        }
        if (std::fabs(a) >= 0x1p127) {
          err.store(WHFF_ERANGE);
          return;
        }
        amax = std::max(amax, std::fabs(a));
      }
    float s = amax == 0.0 || f.fmtmax == 0.0 ? 1.0f : (float)(amax / f.fmtmax);
    if (s == 0.0f) s = 1.0f;
    uint32_t sb;
    std::memcpy(&sb, &s, 4);
    st32(scales + 4 * (uint64_t)(ti * TN + tj), sb);
    for (int64_t i = i0; i < i1; ++i)
      for (int64_t j = j0; j < j1; ++j) {
        uint32_t pat = round_to_format(band[(i - row0) * lda + j] / (double)s, f);
        uint8_t* p = stream + ((uint64_t)i * (uint64_t)ld + (uint64_t)j) * (uint64_t)eb;
        for (int k = 0; k < eb; ++k) p[k] = uint8_t(pat >> (8 * k));
      }
  });
  return err.load();
}

}  // namespace
}  // namespace whff

using namespace whff;

extern "C" size_t whff_compressed_size(int fmt, int rate, int64_t M, int64_t N) {
  if (!is_blocked(fmt)) rate = 8 * elem_bytes(fmt);
  uint64_t s = stream_size(fmt, rate, M, N);
  return s ? (size_t)(kHeaderBytes + s) : 0;
}

extern "C" int whff_blob_init(void* blob, size_t cap, int fmt, int rate, int64_t M, int64_t N) {
  if (!is_blocked(fmt)) rate = 8 * elem_bytes(fmt);
  uint64_t s = stream_size(fmt, rate, M, N);
  if (!blob || !s || cap < kHeaderBytes + s) {
    set_error("whff_blob_init: invalid format, rate, shape or capacity");
    return WHFF_EINVAL;
  }
  std::memset(blob, 0, kHeaderBytes + s);
  write_header((uint8_t*)blob, fmt, rate, M, N, s, 0);
  return WHFF_OK;
}

static int parse_unsealed(const void* blob, size_t cap, BlobInfo* b) {
  // header CRC is valid from init on; the stream CRC is only valid after sealing
  return read_header((const uint8_t*)blob, cap, b, false);
}

extern "C" int whff_compress_band(void* blob, size_t cap, const double* band, int64_t row0, int64_t nrows,
                                  int64_t lda, int nthreads) {
  BlobInfo b;
  if (parse_unsealed(blob, cap, &b) != WHFF_OK) {
    set_error("whff_compress_band: blob not initialised");
    return WHFF_EFORMAT;
  }
  const int align = is_blocked(b.fmt) ? 4 : kScaleTile;
  if (!band || row0 < 0 || nrows <= 0 || nrows > b.M - row0 || lda < b.N || row0 % align ||
      (nrows % align && nrows != b.M - row0)) {
    set_error("whff_compress_band: band must start on a block/tile row and cover whole blocks");
    return WHFF_EINVAL;
  }
  uint8_t* stream = (uint8_t*)blob + kHeaderBytes;
  int e = is_blocked(b.fmt) ? encode_band_zfp(stream, b, band, row0, nrows, lda, nthreads)
                                : encode_band_scaled(stream, b, band, row0, nrows, lda, nthreads);
  if (e != WHFF_OK) set_error(e == WHFF_ERANGE ? "whff_compress: |a| >= 2^127" : "whff_compress: non-finite value");
  return e;
}

extern "C" int whff_blob_seal(void* blob, size_t cap) {
  BlobInfo b;
  if (parse_unsealed(blob, cap, &b) != WHFF_OK) {
    set_error("whff_blob_seal: blob not initialised");
    return WHFF_EFORMAT;
  }
  uint8_t* p = (uint8_t*)blob;
  write_header(p, b.fmt, b.rate, b.M, b.N, b.stream_bytes, crc32(p + kHeaderBytes, b.stream_bytes));
  return WHFF_OK;
}

// ------------------------------------------------------ fixed accuracy (WZ3)
namespace {

int64_t wz3_runs_per_band(int64_t N) { return ceil_div(ceil_div(N, 4), 32); }

// The 16 FP32 values of block (I, J), edge rows and columns replicated.
}  // namespace

extern "C" size_t whff_accuracy_max_size(int64_t M, int64_t N) {
  if (!shape_ok(M, N)) return 0;
  const int64_t BM = ceil_div(M, 4), BN = ceil_div(N, 4);
  return (size_t)kHeaderBytes + 8 + 8 * (size_t)(BM * wz3_runs_per_band(N)) +
         (size_t)(BM * BN) * (size_t)wz3_block_bytes(kWz3Wmax);
}

namespace {
// A fixed-accuracy blob under construction keeps two counters in the header's
// reserved bytes (zero once sealed): the next row a band must start at, and
// the bytes of block area written so far.
constexpr int kAccNextRow = 48, kAccArea = 56;

// Block (I, J) of a band holding matrix rows [row0, row0 + rows): rows past M
// repeat row M-1, columns past N column N-1 (the matrix's edge rule).
void gather_band_block(const double* band, int64_t row0, int64_t M, int64_t N, int64_t ld, int64_t I, int64_t J,
                       float* vals) {
  for (int r = 0; r < 4; ++r) {
    const int64_t gi = std::min(4 * I + r, M - 1) - row0;
    for (int c = 0; c < 4; ++c) vals[4 * r + c] = (float)band[gi * ld + std::min(4 * J + c, N - 1)];
  }
}
}  // namespace

extern "C" int whff_accuracy_begin(void* out, size_t out_cap, int64_t M, int64_t N, double tol) {
  if (!out || !shape_ok(M, N) || !(tol >= 0.0)) {
    set_error("whff_accuracy_begin: null output, empty or oversized shape, or tol < 0");
    return WHFF_EINVAL;
  }
  const int64_t BM = ceil_div(M, 4), RB = wz3_runs_per_band(N);
  const size_t head = (size_t)kHeaderBytes + 8 + 8 * (size_t)(BM * RB);
  if (out_cap < head) {
    set_error("whff_accuracy_begin: capacity below header, tolerance and run index");
    return WHFF_EINVAL;
  }
  uint8_t* blob = static_cast<uint8_t*>(out);
  std::memset(blob, 0, head);
  write_header(blob, WHFF_FMT_FIXED_ACC, 0, M, N, 0, 0);  // sizes and CRCs are final after the seal
  uint64_t tol_bits;
  std::memcpy(&tol_bits, &tol, 8);
  st64(blob + kHeaderBytes, tol_bits);
  st64(blob + kAccNextRow, 0);
  st64(blob + kAccArea, 0);
  return WHFF_OK;
}

extern "C" int whff_compress_accuracy_band(void* out, size_t out_cap, const double* band, int64_t row0, int64_t rows,
                                           int64_t ld, int nthreads) {
  uint8_t* blob = static_cast<uint8_t*>(out);
  if (!out || !band || out_cap < (size_t)kHeaderBytes + 8) {
    set_error("whff_compress_accuracy_band: null argument");
    return WHFF_EINVAL;
  }
  const int64_t M = (int64_t)ld64(blob + 16), N = (int64_t)ld64(blob + 24);
  const int64_t next = (int64_t)ld64(blob + kAccNextRow);
  if ((int)ld32(blob + 8) != WHFF_FMT_FIXED_ACC || !shape_ok(M, N) || ld < N || row0 != next || rows <= 0 ||
      rows > M - row0 || (rows % 4 != 0 && rows != M - row0)) {
    set_error("whff_compress_accuracy_band: not a blob begun by whff_accuracy_begin, ld < N, or the band does not "
              "start at the next row / is not a multiple of 4 rows before the last");
    return WHFF_EINVAL;
  }
  double tol;
  const uint64_t tol_bits = ld64(blob + kHeaderBytes);
  std::memcpy(&tol, &tol_bits, 8);
  const int64_t BM = ceil_div(M, 4), BN = ceil_div(N, 4), RB = wz3_runs_per_band(N);
  const int64_t I0 = row0 / 4, nI = ceil_div(rows, 4);
  // One pass over the band's block rows: each row's blocks are coded once, its
  // runs' widths taken from them and its runs written, word-interleaved, into a
  // buffer of the row's own; the rows are then placed after the area written so
  // far, in band-major order.
  std::vector<uint8_t> width((size_t)(nI * RB));
  std::vector<std::vector<uint8_t>> rowbuf((size_t)nI);
  std::atomic<int> err{WHFF_OK};
  parallel_for(nI, nthreads, [&](int64_t i) {
    float vals[16];
    std::vector<Wz3Block> blk((size_t)BN);
    for (int64_t J = 0; J < BN; ++J) {
      gather_band_block(band, row0, M, N, ld, I0 + i, J, vals);
      const int e = wz3_block(vals, tol, &blk[(size_t)J]);
      if (e != WHFF_OK) {
        err.store(e);
        return;
      }
    }
    size_t bytes = 0;
    for (int64_t r = 0; r < RB; ++r) {
      int W = 0;
      const int64_t nb = std::min(BN, 32 * r + 32) - 32 * r;
      for (int64_t J = 32 * r; J < 32 * r + nb; ++J) W = std::max(W, blk[(size_t)J].need);
      width[(size_t)(i * RB + r)] = (uint8_t)W;
      bytes += (size_t)nb * (size_t)wz3_block_bytes(W);
    }
    std::vector<uint8_t>& out_row = rowbuf[(size_t)i];
    out_row.assign(bytes, 0);
    uint64_t w[8];
    size_t at = 0;
    for (int64_t r = 0; r < RB; ++r) {
      const int W = width[(size_t)(i * RB + r)];
      const int nw = wz3_block_bytes(W) / 8;
      const int64_t nb = std::min(BN, 32 * r + 32) - 32 * r;
      for (int64_t J = 32 * r; J < 32 * r + nb; ++J) {
        wz3_put(blk[(size_t)J], W, w);
        // word-interleaved run: word k of block j at byte 8 (k nb + j)
        for (int k = 0; k < nw; ++k) st64(out_row.data() + at + 8 * (k * nb + (J - 32 * r)), w[k]);
      }
      at += (size_t)nb * (size_t)(8 * nw);
    }
  });
  if (err.load() != WHFF_OK) {
    set_error(err.load() == WHFF_ERANGE ? "whff_compress_accuracy: |a| >= 2^127"
                                        : "whff_compress_accuracy: non-finite value");
    return err.load();
  }
  // offsets of the runs, after the area written so far
  std::vector<uint64_t> off((size_t)(nI * RB));
  uint64_t area = ld64(blob + kAccArea);
  if (area > (uint64_t)whff_accuracy_max_size(M, N)) {
    set_error("whff_compress_accuracy_band: the blob's area counter exceeds its capacity (damaged header)");
    return WHFF_EINVAL;
  }
  for (int64_t i = 0; i < nI; ++i)
    for (int64_t r = 0; r < RB; ++r) {
      off[(size_t)(i * RB + r)] = area;
      area += (uint64_t)(std::min(BN, 32 * r + 32) - 32 * r) * (uint64_t)wz3_block_bytes(width[(size_t)(i * RB + r)]);
    }
  uint8_t* stream = blob + kHeaderBytes;
  uint8_t* index = stream + 8;
  uint8_t* blocks = index + 8 * (size_t)(BM * RB);
  if ((size_t)(blocks - blob) + area > out_cap) {
    set_error("whff_compress_accuracy_band: capacity exceeded (whff_accuracy_max_size bounds the whole blob)");
    return WHFF_EINVAL;
  }
  for (int64_t k = 0; k < nI * RB; ++k)
    st64(index + 8 * ((I0 * RB) + k), off[(size_t)k] | ((uint64_t)width[(size_t)k] << 56));
  parallel_for(nI, nthreads, [&](int64_t i) {
    const std::vector<uint8_t>& row = rowbuf[(size_t)i];
    if (!row.empty()) std::memcpy(blocks + off[(size_t)(i * RB)], row.data(), row.size());
  });
  st64(blob + kAccNextRow, (uint64_t)(row0 + rows));
  st64(blob + kAccArea, area);
  return WHFF_OK;
}

extern "C" int whff_accuracy_seal(void* out, size_t out_cap, size_t* out_len) {
  uint8_t* blob = static_cast<uint8_t*>(out);
  if (!out || out_cap < (size_t)kHeaderBytes + 8 || (int)ld32(blob + 8) != WHFF_FMT_FIXED_ACC) {
    set_error("whff_accuracy_seal: not a blob begun by whff_accuracy_begin");
    return WHFF_EINVAL;
  }
  const int64_t M = (int64_t)ld64(blob + 16), N = (int64_t)ld64(blob + 24);
  if (!shape_ok(M, N) || (int64_t)ld64(blob + kAccNextRow) != M) {
    set_error("whff_accuracy_seal: rows still missing (the bands must cover rows 0..M-1 in order)");
    return WHFF_EINVAL;
  }
  const int64_t BM = ceil_div(M, 4), RB = wz3_runs_per_band(N);
  const uint64_t area = ld64(blob + kAccArea);
  const uint64_t sbytes = 8 + 8 * (uint64_t)(BM * RB) + area;
  if (area > (uint64_t)whff_accuracy_max_size(M, N) || sbytes > out_cap - (size_t)kHeaderBytes) {
    set_error("whff_accuracy_seal: the blob's area counter exceeds its capacity (damaged header)");
    return WHFF_EINVAL;
  }
  write_header(blob, WHFF_FMT_FIXED_ACC, 0, M, N, sbytes, crc32(blob + kHeaderBytes, sbytes));  // clears 48..63
  if (out_len) *out_len = (size_t)(kHeaderBytes + sbytes);
  return WHFF_OK;
}

extern "C" int whff_compress_accuracy(const double* A, int64_t M, int64_t N, int64_t lda, double tol, void* out,
                                      size_t out_cap, size_t* out_len, int nthreads) {
  if (!A || !out || !shape_ok(M, N) || lda < N || !(tol >= 0.0) || out_cap < whff_accuracy_max_size(M, N)) {
    set_error("whff_compress_accuracy: null argument, empty or oversized shape, lda < N, tol < 0 or capacity "
              "below whff_accuracy_max_size");
    return WHFF_EINVAL;
  }
  int e = whff_accuracy_begin(out, out_cap, M, N, tol);
  if (!e) e = whff_compress_accuracy_band(out, out_cap, A, 0, M, lda, nthreads);
  if (!e) e = whff_accuracy_seal(out, out_cap, out_len);
  return e;
}

extern "C" int whff_compress(const double* A, int64_t M, int64_t N, int64_t lda, int fmt, int rate, void* out,
                             size_t out_cap, size_t* out_len, int nthreads) {
  if (!A || lda < N) {
    set_error("whff_compress: null matrix or lda < N");
    return WHFF_EINVAL;
  }
  int e = whff_blob_init(out, out_cap, fmt, rate, M, N);
  if (e) return e;
  e = whff_compress_band(out, out_cap, A, 0, M, lda, nthreads);
  if (e) return e;
  e = whff_blob_seal(out, out_cap);
  if (e) return e;
  if (out_len) *out_len = whff_compressed_size(fmt, rate, M, N);
  return WHFF_OK;
}
