// whff_blob.h -- blob container layout shared by the host encoder and the
// device runtime of the library (not by the CPU oracle, which has its own).
//
// 64-byte little-endian header, then the stream:
//   0 "WZ1\0" | 4 version u32 | 8 fmt u32 | 12 rate u32 | 16 M i64 | 24 N i64 |
//   32 stream bytes u64 | 40 CRC-32 of the stream u32 | 44 CRC-32 of bytes 0..43 u32 |
//   48..63 zero.
// WZ1 stream: block (I, J) of the ceil(M/4) x ceil(N/4) block grid at byte
// (I*ceil(N/4) + J) * 2*rate, i.e. row-major block order, so a band of block
// rows is one contiguous byte range.
// Scaled stream: payload M x ld elements (ld = roundup(N, 16)), row-major,
// then FP32 scales, ceil(M/128) x ceil(N/128), row-major (all 1 for FP32).
#pragma once
#include <cstddef>
#include <cstdint>

namespace whff {

constexpr int kHeaderBytes = 64;
constexpr int kScaleTile = 128;
constexpr int kWz1Prec = 26;    // fixed-point bits below the block exponent
constexpr int kWz1Emin = -100;  // blocks with max |a| < 2^-100 are zero blocks

struct BlobInfo {
  int fmt = 0;
  int rate = 0;
  int64_t M = 0, N = 0;
  uint64_t stream_bytes = 0;
  uint32_t crc_stream = 0, crc_header = 0;
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t scaled_ld(int64_t N) { return ceil_div(N, 16) * 16; }

int elem_bytes(int fmt);  // 2, 2, 1, 4 for BF16, FP16, FP8, FP32; 0 otherwise
// values per 16-byte chunk of a scaled format's row
inline int scaled_vec(int fmt) { return 16 / (fmt == 4 ? 1 : fmt == 7 ? 4 : 2); }
bool rate_valid(int rate);       // WZ1: 4..64, multiple of 4
bool wz2_rate_valid(int rate);   // WZ2: 8..24, multiple of 4
bool is_blocked(int fmt);        // fixed-size 4x4-block formats (WZ1, WZ2)
inline bool is_wz3(int fmt) { return fmt == 8; }  // fixed accuracy: 4x4 blocks of variable size, indexed runs
// row alignment of a row view: a 4-row band (block formats) or a 128-row scale tile
inline int row_align(int fmt) { return (is_blocked(fmt) || is_wz3(fmt)) ? 4 : kScaleTile; }
// Shapes the container takes: 1..2^48 rows and columns and at most 2^56 4x4
// blocks, so that every byte count derived from a shape (a stream, an index,
// a workspace) fits in 63 bits.  A header outside these bounds is refused
// before any size is computed from it.
constexpr int64_t kMaxDim = int64_t(1) << 48;
constexpr uint64_t kMaxBlocks = uint64_t(1) << 56;
inline bool shape_ok(int64_t M, int64_t N) {
  if (M <= 0 || N <= 0 || M > kMaxDim || N > kMaxDim) return false;
  return (uint64_t)ceil_div(M, 4) <= kMaxBlocks / (uint64_t)ceil_div(N, 4);
}
uint64_t stream_size(int fmt, int rate, int64_t M, int64_t N);  // 0 if invalid
uint32_t crc32_update(uint32_t crc, const uint8_t* p, size_t n);  // crc = 0 to start
inline uint32_t crc32(const uint8_t* p, size_t n) { return crc32_update(0, p, n); }
void write_header(uint8_t* blob, int fmt, int rate, int64_t M, int64_t N, uint64_t sbytes, uint32_t crc_stream);
// Parses and checks magic, version, sizes and the header CRC; with
// check_stream also the stream CRC.  Returns a WHFF_* code.
int read_header(const uint8_t* blob, size_t len, BlobInfo* info, bool check_stream);

}  // namespace whff
