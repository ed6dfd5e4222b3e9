/*
 * orc.h -- the CPU oracle for the compressed control-step GEMV.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * statement of what the library computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library never
 * links, includes or calls anything here, and nothing here calls the library.
 *
 * Everything is plain C99 with FP64 arithmetic wherever the format does not
 * fix a narrower precision.  OpenMP (when compiled in) is used only on the
 * outermost row / block-row loop, so every result is independent of the
 * thread count.
 *
 * What it follows (paper: "GPU Acceleration of Real-Time Control Loops"):
 *   - Sec. 4.3: A is stored in zfp's fixed-rate mode, i.e. every block of
 *     values costs exactly the same number of bits (rate = bits per value);
 *     the paper sweeps rate 8 (Table 2) and names zfp as the codec.  The
 *     paper gives no block shape, transform or coder, so the "WZ1" layout
 *     below is this project's reading of a zfp-style fixed-rate coder:
 *     4x4 blocks, block-floating-point with a shared exponent, a reversible
 *     integer lifting transform, sequency ordering, negabinary, and an
 *     embedded bit-plane coder with group tests truncated to the budget.
 *   - Sec. 4.4, dot-product equation: r_i = sum_j A(i,j) b_j, the GEMV.
 *   - Sec. 4.4, sequential mixed-precision listing: FP32 products summed
 *     into an FP64 accumulator, result stored as FP32 (orc_gemv_mp).
 *   - Sec. 2.1, thermal update T_{k+1} = A T_k + B u_k: the carried state
 *     s <- decay*s + y is its stand-in (orc_state_update).
 */
#ifndef WHFF_ORACLE_H
#define WHFF_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Blob container (shared by every format). 64-byte little-endian header:
 *   0  char[4]  magic "WZ1\0"
 *   4  u32      version (1)
 *   8  u32      fmt: 1 = zfp-style fixed rate, 2 = BF16, 3 = FP16, 4 = FP8 E4M3
 *   12 u32      rate: bits per value (fmt 1), element bits otherwise
 *   16 i64      M (rows)
 *   24 i64      N (columns)
 *   32 u64      stream bytes (everything after the header)
 *   40 u32      CRC-32 (IEEE, reflected 0xEDB88320) of the stream
 *   44 u32      CRC-32 of header bytes 0..43
 *   48 u8[16]   zero
 * followed by the stream at byte 64. */
#define ORC_HEADER_BYTES 64
#define ORC_FMT_ZFP 1
#define ORC_FMT_BF16 2
#define ORC_FMT_FP16 3
#define ORC_FMT_FP8E4M3 4
#define ORC_FMT_FIXED_LIFT 5 /* WZ2: fixed-width fields of the linear lift's coefficients */
#define ORC_FMT_FIXED_BFP 6  /* WZ2 without transform: fixed-width block floating point */
#define ORC_FMT_FP32 7       /* A rounded to FP32, every tile scale 1 (the uncompressed comparison) */
#define ORC_FMT_FIXED_ACC 8  /* WZ3: fixed accuracy, variable-length runs (oracle only so far) */

/* Error codes (same meaning as the library's, separate definitions). */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ERANGE -2
#define ORC_ENONFINITE -3
#define ORC_EFORMAT -5

uint32_t orc_crc32(const uint8_t* p, size_t n);

/* ---- WZ1 building blocks (exposed so the tests can pin each step) ---- */
/* forward lift of one 4-vector, in place: (x0,x1,x2,x3) -> (s,d,d0,e); mod 2^32 */
void orc_fwd_lift4(int32_t v[4]);
/* inverse lift, in place: (s,d,d0,e) -> (x0,x1,x2,x3); mod 2^32 */
void orc_inv_lift4(int32_t v[4]);
/* 2-D transforms on a row-major 4x4 block (forward: rows then columns) */
void orc_fwd_xform(int32_t b[16]);
void orc_inv_xform(int32_t b[16]);
uint32_t orc_int2nb(int32_t c);
int32_t orc_nb2int(uint32_t u);
/* perm[k] = row-major index 4*i+j of the k-th coefficient in sequency order */
void orc_sequency(int perm[16]);
/* embedded plane coder on 16 negabinary words; writes exactly maxbits bits
 * starting at bit `pos` of the LSB-first word array; returns bits actually
 * emitted (<= maxbits; the caller's buffer is pre-zeroed) */
int orc_encode_planes(const uint32_t u[16], int maxbits, uint64_t* words, int64_t pos);
/* inverse: reads at most maxbits bits; untransmitted bits are zero */
int orc_decode_planes(const uint64_t* words, int64_t pos, int maxbits, uint32_t u[16]);

/* One 4x4 block, float input (already FP32).  `words` must hold 16*rate bits
 * (rate/4 words) and is fully written.  Returns ORC_OK or ORC_ERANGE/ENONFINITE. */
int orc_wz1_encode_block(const float a[16], int rate, uint64_t* words);
/* Decode one block: q (row-major, after the inverse transform), emax, nonzero flag. */
void orc_wz1_decode_block(const uint64_t* words, int rate, int32_t q[16], int* emax, int* nonzero);
/* The decoded value of one element: (double)(float)q * 2^(emax-26); 0 for a zero block. */
double orc_wz1_value(int32_t q, int emax, int nonzero);

/* ---- WZ2: fixed-allocation variant (rates 8..24, multiple of 4) ----
 * Same 4x4 blocks, FP32 rounding and block exponent as WZ1, 24 fraction bits
 * (q = trunc(a * 2^(24-emax))).  lift = 1: C = (4F) Q (4F)^T with the lift in
 * exact linear form, 4F rows (1,1,1,1), (-2,-2,2,2), (-4,4,0,0), (4,-4,-4,4),
 * coefficients in sequency order; lift = 0: C = Q in row-major order.  One
 * shift K per block (the smallest in 0..27 with every round-half-even
 * C/2^K inside W-bit two's complement), W = floor((16*rate - 13)/16).
 * Header: 8 bits emax+127 (0 = zero block), 5 bits K; then 16 offset-binary
 * fields v + 2^(W-1), W bits each, LSB-first from bit 13; the rest zero.
 * Decoded value (exact in FP64): lift: (2G) V (2G)^T * 2^(K+emax-30) with 2G
 * rows (2,-1,-1,0), (2,-1,1,0), (2,1,-1,-1), (2,1,1,1) = 8 (4F)^-1;
 * no lift: V * 2^(K+emax-24). */
int orc_wz2_width(int rate);
int orc_wz2_encode_block(const float a[16], int rate, int lift, uint64_t* words);
void orc_wz2_decode_block(const uint64_t* words, int rate, int lift, double out[16]);

/* ---- WZ3: fixed accuracy (planned device format; oracle and pins only) ----
 * zfp's fixed-accuracy mode (Sec. 4.3 names zfp; its modes other than fixed
 * rate are the paper's outlook) read GPU-first: WZ2's blocks, exponent,
 * transform and bit layout, but per block the LARGEST shift K in 0..27 whose
 * decoded block stays within tol of the FP32 input (max absolute error; when
 * none does, the floor: the smallest K whose fields fit 31 bits -- the lifted
 * coefficients reach 2^32, so K = 0 can need 34 -- and the block's error is
 * then above tol), and per run of up to
 * 32 blocks of a band ONE field width: the largest width the run's blocks
 * need (a block needs the smallest W >= 1 holding its round-half-even
 * C/2^K in W-bit two's complement, W <= 31; 0 for a zero block).  Every block of a run
 * takes 8 * ceil((13 + 16 W) / 64) bytes: header 8 bits emax+127 (0 = zero
 * block), 5 bits K, then 16 offset-binary W-bit fields from bit 13, the rest
 * zero -- exactly WZ2's layout with W chosen per run. */
int orc_wz3_block(const float a[16], double tol, int lift, int* emax, int* K, int64_t v[16], int* need_w);
int orc_wz3_block_bytes(int W);
/* Encode nb (1..32) blocks (nb x 16 floats, row-major 4x4 each) as one run;
 * words receives nb * block_bytes(W)/8 words; *w_run = W. */
int orc_wz3_encode_run(const float* blocks, int nb, double tol, int lift, uint64_t* words, int* w_run);
void orc_wz3_decode_block(const uint64_t* words, int W, int lift, double out[16]);
/* Whole matrix, with the lift (fmt ORC_FMT_FIXED_ACC): the usual 64-byte header
 * (rate 0, M, N, stream bytes, both CRCs), then the stream: the tolerance
 * (f64), one u64 per run in band-major order (bits 0..55: byte offset of the
 * run's first block in the block area; bits 56..63: W), then the runs' blocks.
 * blob must hold orc_wz3_max_blob_size bytes; *len receives the bytes used. */
size_t orc_wz3_max_blob_size(int64_t M, int64_t N);
int orc_wz3_encode_matrix(const double* A, int64_t M, int64_t N, int64_t lda, double tol, uint8_t* blob, size_t cap,
                          size_t* len);
int orc_wz3_decode_matrix(const uint8_t* blob, size_t len, double* out, int64_t ldo, double* tol);

/* ---- whole matrices ---- */
int orc_rate_ok(int rate);
size_t orc_blob_size(int fmt, int rate, int64_t M, int64_t N);
/* A: FP64 row-major M x N with leading dimension lda.  blob must hold orc_blob_size bytes. */
int orc_encode(int fmt, int rate, const double* A, int64_t M, int64_t N, int64_t lda, uint8_t* blob, size_t cap);
/* Parse and validate a blob header (magic, version, sizes, both CRCs). */
int orc_parse(const uint8_t* blob, size_t len, int* fmt, int* rate, int64_t* M, int64_t* N);
/* Decode rows [row0, row0+nrows) to FP64 (row-major, ldo); row0 % 4 == 0 for fmt 1. */
int orc_decode_rows(const uint8_t* blob, size_t len, int64_t row0, int64_t nrows, double* out, int64_t ldo);

/* ---- scaled formats (precision layer) ---- */
/* round an FP64 value to the given format, ties to even, saturating to +-fmtmax;
 * returns the rounded value as a double and its bit pattern in *bits */
double orc_round_fmt(int fmt, double v, uint32_t* bits);
double orc_fmt_max(int fmt);        /* FMTMAX used to size the per-tile scale */
double orc_fmt_decode(int fmt, uint32_t bits);

/* ---- GEMV ---- */
/* Y[:,r] = Ahat * X[:,r], FP64, sequential j order (dot-product equation). X: N x R column-major. */
void orc_gemv64(const double* A, int64_t M, int64_t N, int64_t lda, const double* X, int R, int64_t ldx,
                double* Y, int64_t ldy);
/* The paper's mixed-precision rule: float product, double sum, float result. */
void orc_gemv_mp(const double* A, int64_t M, int64_t N, int64_t lda, const double* x, float* y);
/* Carried state: for r = 0..R-1 in order, s <- decay*s + Y[:,r]. */
void orc_state_update(double* s, int64_t M, const double* Y, int R, int64_t ldy, double decay);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
