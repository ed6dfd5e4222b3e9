/*
 * whff.h -- C ABI of the compressed-matrix control-step library (sm_103a).
 *
 * The library computes the deformation / thermal control step of the paper
 * "GPU Acceleration of Real-Time Control Loops" (Sec. 2.1, deformation
 * equation Delta_d = C_d * S_{k+1}; Sec. 4.4, dot-product equation
 * r_i = sum_j A(i,j) b_j) on a matrix A that stays resident in GPU memory in a
 * compressed form (Sec. 4.3: zfp fixed-rate mode, "every value costs BPV
 * bits"), decoded on the fly inside the GEMV kernel and never written back.
 *
 * Conventions for every call:
 *   - Return value: WHFF_OK (0) or a negative WHFF_E* code; the thread-local
 *     message of the last failure is whff_last_error().
 *   - "stream" is a cudaStream_t passed as void* (0 = the legacy default
 *     stream).  Device calls are asynchronous on that stream; errors found on
 *     the device are recorded in the handle's status word and returned by
 *     whff_sync_status().
 *   - Device pointers are plain CUDA device addresses owned by the caller;
 *     the library never frees them.  Host pointers are plain host memory.
 *   - No call falls back to the CPU: without a usable sm_103a device the
 *     device calls fail with WHFF_ECUDA.
 *
 * Matrix layout on input: A is FP64, row-major, M x N, leading dimension lda
 * (>= N).  Vectors: x is FP32 N x R column-major (leading dimension ldx >= N),
 * y is FP64 M x R column-major (ldy >= M), the state s is FP64 of length M.
 */
#ifndef WHFF_H
#define WHFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Storage formats.
 *  WHFF_FMT_ZFP: zfp-style fixed rate (Sec. 4.3; Table 2 sweeps rate 8).  The
 *    matrix is cut into 4x4 blocks (edge blocks replicate the last valid row,
 *    then column); each block costs exactly 16*rate bits: a nonzero flag, an
 *    8-bit biased block exponent, and the embedded bit-plane code (group
 *    tests, sequency order, negabinary) of the reversible integer lift of its
 *    26-bit fixed-point values, cut at the budget.  rate: 4..64, multiple of 4.
 *  WHFF_FMT_BF16 / FP16 / FP8E4M3: element-wise storage with one FP32 scale
 *    per 128x128 tile, scale = amax / FMTMAX (FMTMAX 1, 32768, 448); rate is
 *    ignored on input.
 */
#define WHFF_FMT_ZFP 1
#define WHFF_FMT_BF16 2
#define WHFF_FMT_FP16 3
#define WHFF_FMT_FP8E4M3 4
/*  WHFF_FMT_FIXED_LIFT / WHFF_FMT_FIXED_BFP ("WZ2"): the GPU-friendly
 *    fixed-allocation variant that Sec. 5.2 and Sec. 6 call for.  Same 4x4
 *    blocks, FP32 rounding and block exponent; 24 fraction bits; FIXED_LIFT
 *    takes the lift in exact linear form (coefficients C = (4F) Q (4F)^T in
 *    sequency order), FIXED_BFP no transform.  Each block stores emax+127
 *    (8 bits, 0 = zero block), one shift K (5 bits, the smallest in 0..27 that
 *    fits) and 16 offset-binary fields of W = floor((16*rate-13)/16) bits of
 *    round-half-even(C / 2^K).  rate: 8..24, multiple of 4. */
#define WHFF_FMT_FIXED_LIFT 5
#define WHFF_FMT_FIXED_BFP 6
/*  WHFF_FMT_FP32: the matrix uncompressed, A rounded to FP32 (scales all 1),
 *    for the like-for-like comparison of Sec. 5.1: the step then follows the
 *    paper's mixed precision (Sec. 4.4) -- every product a*x rounded to FP32,
 *    the products summed without further rounding error (compensated FP32
 *    sums, FP64 across lanes) -- up to the order of the additions. */
#define WHFF_FMT_FP32 7
/*  WHFF_FMT_FIXED_ACC ("WZ3"): zfp's fixed-accuracy mode (Sec. 4.3 names zfp;
 *    Table 2 reports its modes) read GPU-first.  WZ2's blocks, lifted
 *    coefficients and bit layout, but each block takes the largest shift K in
 *    0..27 whose decoded block stays within an absolute tolerance tol of the
 *    FP32 input (max error; when none does, the smallest K whose fields fit 31
 *    bits), and every run of up to 32 blocks of a band one field width W, the
 *    widest its blocks need; a block takes 8*ceil((13 + 16 W)/64) bytes.  Blob:
 *    the 64-byte header (rate 0, variable stream length), then the tolerance
 *    (f64), one u64 per run in band-major order (bits 0-55: byte offset of the
 *    run in the block area; bits 56-63: W), then the runs back to back, each
 *    word-interleaved (64-bit word k of its block b at byte 8 (k nb + b) of
 *    the run, nb its block count) so that a warp loads a run coalesced.
 *    Written by whff_compress_accuracy; decoded value (2G) V (2G)^T *
 *    2^(K+emax-30), exact in FP64. */
#define WHFF_FMT_FIXED_ACC 8

#define WHFF_OK 0
#define WHFF_EINVAL -1     /* bad argument (null, size, leading dimension, rate) */
#define WHFF_ERANGE -2     /* |a| >= 2^127 after rounding to FP32 */
#define WHFF_ENONFINITE -3 /* NaN or infinity in A */
#define WHFF_ENOMEM -4     /* device allocation failed */
#define WHFF_EFORMAT -5    /* blob header, size or CRC mismatch */
#define WHFF_ECUDA -6      /* a CUDA runtime call failed */
#define WHFF_ETIMEOUT -7   /* a bounded device-side wait gave up */
#define WHFF_EBUSY -8      /* admission refused (serving layer) */

#define WHFF_BLOB_HEADER_BYTES 64

typedef struct whff_handle whff_handle;

/* ------------------------------------------------------------------ host side */

/* Shapes: every call takes 1 <= M, N <= 2^48 with at most 2^56 4x4 blocks
 * (ceil(M/4) * ceil(N/4)), so that every derived byte count fits in 63 bits;
 * a larger shape is WHFF_EINVAL on input and WHFF_EFORMAT in a blob header. */

/* Bytes of the blob (64-byte header + stream) for a format, rate and shape;
 * 0 if the combination is invalid.  WZ1 (fmt 1): 64 + ceil(M/4)*ceil(N/4)*2*rate.
 * Scaled formats: 64 + M*roundup(N,16)*elem_bytes + ceil(M/128)*ceil(N/128)*4
 * (elem_bytes 2, 2, 1, 4 for BF16, FP16, FP8 E4M3, FP32). */
size_t whff_compressed_size(int fmt, int rate, int64_t M, int64_t N);

/* Compress all of A (offline encoding, Sec. 4.3: "compression can be done
 * offline") into out[0..out_cap).  On success *out_len = the blob size.
 * Uses all host threads (nthreads <= 0) or the given number; the result is
 * byte-identical for every thread count.  Errors: WHFF_EINVAL, WHFF_ERANGE,
 * WHFF_ENONFINITE. */
int whff_compress(const double* A, int64_t M, int64_t N, int64_t lda, int fmt, int rate, void* out, size_t out_cap,
                  size_t* out_len, int nthreads);

/* Fixed-accuracy encoding (WHFF_FMT_FIXED_ACC) of all of A at absolute
 * tolerance tol >= 0: every decoded entry within tol of A rounded to FP32,
 * except in blocks where 31-bit fields cannot reach it (near-full-scale blocks
 * at tiny tolerances: those take the finest quantisation that fits).  out must
 * hold whff_accuracy_max_size(M, N) bytes; *out_len = the blob's bytes.  All
 * host threads (nthreads <= 0) or the given number; the bytes do not depend on
 * the thread count.  Errors: WHFF_EINVAL, WHFF_ERANGE, WHFF_ENONFINITE. */
size_t whff_accuracy_max_size(int64_t M, int64_t N);
int whff_compress_accuracy(const double* A, int64_t M, int64_t N, int64_t lda, double tol, void* out, size_t out_cap,
                           size_t* out_len, int nthreads);

/* Band interface for matrices too large to hold in FP64 at once.
 * whff_blob_init writes the header fields of an empty blob; whff_compress_band
 * encodes rows [row0, row0+nrows) given as a band (row-major, lda) -- row0 and
 * nrows must be multiples of 4 (block formats: WZ1, WZ2) or 128 (scaled
 * formats) except for the last band; whff_blob_seal computes both CRCs once
 * every band is in.  Errors: WHFF_EINVAL (format, shape, capacity, band
 * bounds), WHFF_EFORMAT (a blob whff_blob_init did not write), WHFF_ERANGE,
 * WHFF_ENONFINITE. */
int whff_blob_init(void* blob, size_t cap, int fmt, int rate, int64_t M, int64_t N);
int whff_compress_band(void* blob, size_t cap, const double* band, int64_t row0, int64_t nrows, int64_t lda,
                       int nthreads);
int whff_blob_seal(void* blob, size_t cap);

/* The band interface of the fixed-accuracy format (WHFF_FMT_FIXED_ACC), whose
 * run offsets follow the bands in order: whff_accuracy_begin writes the header,
 * the tolerance and an empty run index (cap >= 64 + 8 + 8 * ceil(M/4) *
 * ceil(ceil(N/4)/32) bytes); whff_compress_accuracy_band appends rows [row0,
 * row0+nrows) given as a band (row-major, lda >= N), row0 the next row not yet
 * encoded and nrows a multiple of 4 except for the last band (WHFF_EINVAL
 * otherwise, or when cap cannot hold the band's runs; whff_accuracy_max_size
 * bounds the whole blob); whff_accuracy_seal checks that every row is in,
 * writes the stream size and both CRCs and returns the blob length.  Until
 * sealed the blob is refused by whff_create.  The result equals
 * whff_compress_accuracy's byte for byte, whatever the band split. */
int whff_accuracy_begin(void* blob, size_t cap, int64_t M, int64_t N, double tol);
int whff_compress_accuracy_band(void* blob, size_t cap, const double* band, int64_t row0, int64_t nrows, int64_t lda,
                                int nthreads);
int whff_accuracy_seal(void* blob, size_t cap, size_t* len);

/* --------------------------------------------------------------- device side */

/* Make A resident: validate the blob (magic, version, sizes, CRCs), copy its
 * stream once to device memory on the current device, allocate the split-K
 * workspace for up to max_rhs right-hand sides (0 -> 32) and pick the launch
 * shape.  The handle owns every device allocation it makes; the host blob may
 * be freed afterwards.  The calls that launch work on a handle (steps, graphs,
 * decompress, tune, batches) refuse with WHFF_EINVAL while a device other
 * than the one current at its creation is current.  Errors: WHFF_EFORMAT,
 * WHFF_ENOMEM, WHFF_ECUDA. */
int whff_create(const void* blob, size_t len, int max_rhs, void* stream, whff_handle** h);

/* As whff_create, with flags.  WHFF_CREATE_HOST_RESIDENT keeps the compressed
 * stream in pinned, mapped host memory instead of HBM: the fused kernels read
 * the blocks over the CPU-GPU link (NVLink-C2C on a GB300 superchip) every
 * step, as the paper's system moves each step's matrix over the host link
 * (Sec. 4.2; Sec. 5.2 measures the transfer share).  Compression then divides
 * the bytes that cross the link.  Same results bit for bit as a resident
 * handle; whff_info's device_bytes leaves the stream out.  Errors: as
 * whff_create, WHFF_EINVAL for an unknown flag. */
#define WHFF_CREATE_HOST_RESIDENT 1u
int whff_create_ex(const void* blob, size_t len, int max_rhs, unsigned flags, void* stream, whff_handle** h);

/* Shape and footprint of a resident matrix (device_bytes = all device memory held). */
int whff_info(const whff_handle* h, int* fmt, int* rate, int64_t* M, int64_t* N, size_t* device_bytes);

/* Launch plan of a resident matrix: *ksplit = column splits per 4-row band
 * (1 for matrices with enough rows to fill the GPU), *launches = kernel
 * launches of one CUDA-core whff_step pass: the fused kernel, the epilogue of
 * shared bands or split-K if any, and for FIXED_LIFT and FIXED_ACC the (2G)^T x transform of
 * x that the fused kernel reads. */
int whff_plan(const whff_handle* h, int* ksplit, int* launches);

/* One control step (Sec. 2.1 / Sec. 4.4): y[:,r] = Ahat * x[:,r] for r < R,
 * taken in passes: with a WZ2, BF16, FP16 or FP8 matrix whose handle allows
 * max_rhs >= 2, passes of crossover..32 columns (default crossover 4, see
 * whff_set_crossover) run on the tensor cores (tcgen05: the stored values
 * split exactly into 1-3 BF16 pieces -- WZ2 by field width, FP16 into two,
 * BF16 and FP8 into one -- and x, transformed for FIXED_LIFT, into three;
 * FP16 in device memory instead keeps its values and takes x, scaled per
 * column by a power of two, in three FP16 pieces; the
 * piece products above 2^-24 accumulate in FP32 TMEM, drained every 128
 * columns of K into compensated sums, the scaled formats' tile scale applied
 * at the drain); otherwise passes of 8, 4, 2, 1 columns run on the CUDA cores.
 * Ahat = the decoded matrix (exactly whff_decompress's output).  Products and
 * per-lane sums in FP32 (compensated), cross-warp and cross-CTA sums and y in
 * FP64.  If state != NULL, afterwards for r = 0..R-1 in order:
 * state <- decay*state + y[:,r] (FP64).  x, y, state: device pointers.
 * Deterministic for a fixed (handle, R).  Errors: WHFF_EINVAL (R > max_rhs,
 * bad ld), WHFF_ECUDA. */
int whff_step(whff_handle* h, const float* x, int R, int64_t ldx, double* y, int64_t ldy, double* state,
              double decay, void* stream);

/* The step on a slit (Sec. 2.1, divide and conquer: the deformation of the
 * slit under scan needs only C_slit, a block of rows of the resident C_field;
 * Fig. whff_algo fetches it from C_field every millisecond):
 * y[:,r] = Ahat[row0:row0+nrows, :] * x[:,r] for r < R.  Block formats need
 * row0 % 4 == 0, scaled formats row0 % 128 == 0; the slit's rows are one
 * contiguous range of the resident stream, so nothing is copied.  y is
 * nrows x R (ldy >= nrows) and state, if not NULL, has nrows entries (the
 * slit's own state); both are device pointers.  Same passes, engines and
 * accuracy as whff_step; the launch plan is the slit's own (its roundings
 * can differ from the same rows of a whole-matrix step within the bar).
 * Capturable in a graph.  Errors: WHFF_EINVAL (rows outside the matrix,
 * misaligned row0, R > max_rhs, bad ld), WHFF_ECUDA. */
int whff_step_rows(whff_handle* h, int64_t row0, int64_t nrows, const float* x, int R, int64_t ldx, double* y,
                   int64_t ldy, double* state, double decay, void* stream);

/* Time slicing: with rows > 0, whff_step (and every graph captured from it
 * afterwards) runs each pass as consecutive slits of `rows` rows (the last
 * one shorter), each its own launch sequence, so that kernels on other,
 * higher-priority streams are scheduled between slits instead of waiting for
 * the persistent grid of a whole pass.  The results are the slits' (within
 * the bar of a whole-matrix step).  rows = 0 (default) turns it off; rows is
 * a multiple of 4 (block formats) or 128 (scaled formats), else WHFF_EINVAL. */
int whff_get_slice_rows(const whff_handle* h, int64_t* rows);
int whff_set_slice_rows(whff_handle* h, int64_t rows);

/* The same step on HOST buffers: copies x (N x R, ldx) host->device, runs
 * whff_step into handle-owned device buffers, copies y (M x R, ldy) back, all
 * asynchronously on the stream (pinned host memory makes the copies truly
 * asynchronous).  state is a DEVICE pointer or NULL.  The caller synchronizes
 * the stream before reading y.  Errors: as whff_step. */
int whff_step_host(whff_handle* h, const float* x_host, int R, int64_t ldx, double* y_host, int64_t ldy,
                   double* state, double decay, void* stream);

/* ----------------------------------------------------- graph-captured steps */
/* A control step captured once as a CUDA graph and replayed every period
 * (the firm real-time loop of Sec. 1: one GEMV per millisecond, corrections
 * within 50 ms).  whff_graph_create captures whff_step on fixed device
 * buffers (x, y, state as in whff_step; the caller rewrites x between
 * replays).  whff_graph_create_host captures, in order, the copy of x_host
 * (N x R, ldx, pinned host memory) to a graph-owned device buffer, the step,
 * and the copy of y back to y_host (M x R, ldy, pinned); state is a device
 * pointer or NULL.  The stream is used only to capture (a temporary stream is
 * used when it is 0); whff_graph_launch replays on any stream.  The graph owns
 * its device buffers; the handle must outlive it.  Errors: WHFF_EINVAL,
 * WHFF_ENOMEM, WHFF_ECUDA. */
typedef struct whff_graph whff_graph;
int whff_graph_create(whff_handle* h, const float* x, int R, int64_t ldx, double* y, int64_t ldy, double* state,
                      double decay, void* stream, whff_graph** g);
int whff_graph_create_host(whff_handle* h, const float* x_host, int R, int64_t ldx, double* y_host, int64_t ldy,
                           double* state, double decay, void* stream, whff_graph** g);
int whff_graph_launch(whff_graph* g, void* stream);
void whff_graph_destroy(whff_graph* g);

/* A slit step captured once and moved from slit to slit (Sec. 2.1, divide and
 * conquer; Fig. whff_algo fetches a new C_slit from C_field every
 * millisecond): the graph of whff_step_rows(h, row0, nrows, ...) whose slit
 * offset is a parameter of the instantiated graph.  y (ldy >= M) and state
 * (M entries, or NULL) are FIELD-sized device buffers: a replay writes
 * y[row0 .. row0+nrows-1, r] and updates state[row0 .. row0+nrows-1]; x (N x R,
 * ldx) is read in place, so the caller rewrites it between replays.
 * whff_graph_set_rows moves the slit to row0 and, with h != NULL, onto another
 * resident matrix of the same format, rate, shape and max_rhs (e.g. the next
 * field of a whff_fields pipeline): the slit step is captured again on the
 * host (no GPU work) and the kernel arguments of the instantiated graph are
 * updated in place (cudaGraphExecUpdate) -- the slit height fixes the launch
 * plan, so every offset has the same nodes.  Replays already enqueued keep
 * the slit they were launched with; the update applies to later launches.
 * Same results bit for bit as whff_step_rows on that slit.
 * Errors: WHFF_EINVAL (rows outside the matrix, row0 not a multiple of 4 for
 * block formats or 128 for scaled ones, R > max_rhs, a mismatching handle, the
 * handle's launch shape or crossover changed since the capture), WHFF_ECUDA. */
int whff_graph_create_rows(whff_handle* h, int64_t row0, int64_t nrows, const float* x, int R, int64_t ldx,
                           double* y, int64_t ldy, double* state, double decay, void* stream, whff_graph** g);
int whff_graph_set_rows(whff_graph* g, whff_handle* h, int64_t row0);

/* ------------------------------------------------------------ field pipeline */
/* Compressed fields streamed over the host link (Sec. 4.2-4.3: the scanner
 * fetches one C_field per exposure field from host memory and the slits of
 * that field from it; compression divides the bytes on the link, Fig.
 * compression_cost, and the pipeline period and latency of Table comp_metrics
 * follow).  nbuf resident slots (2 = double buffering), each a handle of its
 * own (device copy of the stream, workspaces, launch plan) for one format,
 * rate and shape.  whff_fields_load(slot, blob, copy_stream) copies a blob's
 * stream (header + stream in host memory; pinned memory makes the copy
 * asynchronous) into the slot on copy_stream, after the work released from
 * that slot has finished; only the header is checked (its CRC, format, rate
 * and shape) unless the pipeline was created with WHFF_FIELDS_VERIFY_CRC,
 * which also checks the stream's CRC on the host before the copy.
 * whff_fields_acquire(slot, compute_stream) makes compute_stream wait for the
 * slot's last load and returns its handle, for whff_step / whff_step_rows /
 * graphs (whff_graph_set_rows moves a slit graph onto it).
 * whff_fields_release(slot, compute_stream) marks the slot free once the work
 * enqueued on compute_stream so far has run; the next load of the slot waits
 * for it.  The host blob must stay valid until its copy has run.  The handles
 * belong to the pipeline (do not destroy them).  Errors: WHFF_EINVAL (slot,
 * shape or format mismatch), WHFF_EFORMAT (header or CRC), WHFF_ENOMEM,
 * WHFF_ECUDA. */
#define WHFF_FIELDS_VERIFY_CRC 1u
typedef struct whff_fields whff_fields;
int whff_fields_create(int fmt, int rate, int64_t M, int64_t N, int nbuf, int max_rhs, unsigned flags, void* stream,
                       whff_fields** f);
int whff_fields_load(whff_fields* f, int slot, const void* blob, size_t len, void* copy_stream);
int whff_fields_acquire(whff_fields* f, int slot, void* compute_stream, whff_handle** h);
int whff_fields_release(whff_fields* f, int slot, void* compute_stream);
void whff_fields_destroy(whff_fields* f);

/* ------------------------------------------------------- tuning and batches */
/* Launch shape of the fixed-allocation (WZ2) kernels: blocks kept in flight
 * per lane (2, 4 or 8), resident CTAs per SM of the persistent grid, and the
 * fold flags: WHFF_FOLD_FP32_PAIRS folds a band's 32 lane sums as FP32
 * (hi, lo) pairs with TwoSum, widened once, instead of widening to FP64 and
 * adding in FP64 (cheaper on GB300's small FP64 pipe; pays on short bands);
 * WHFF_FOLD_LANE_GROUPS lets four 8-lane groups of a warp take four bands at
 * once (short bands: tall matrices), with unroll 2 only.  Defaults: FP32
 * pairs below 4096 blocks per band, lane groups below 256.  Unroll does not
 * change the arithmetic; CTAs per SM (the warp ranges) and the fold flags
 * change its rounding within the bar.
 * whff_tune times every candidate on the resident matrix (iters steps each,
 * R = 1, CUDA events on the stream) and keeps the fastest; *best_ms (optional)
 * receives its step time.  With tensor-core passes available it then sets
 * the engine crossover: the fewest columns (2..8) for which one tensor-core
 * pass is no slower than the CUDA-core passes, else 9.  whff_get_config / whff_set_config read and apply a
 * shape (e.g. from a cache keyed by format, rate, shape and SM count).  WZ2
 * handles only (WHFF_EINVAL otherwise).  Handles of the scaled formats (BF16,
 * FP16, FP8, FP32) take the same fold defaults, counting 16-byte column chunks
 * per band instead of blocks, and are not tunable. */
#define WHFF_FOLD_FP32_PAIRS 1
#define WHFF_FOLD_LANE_GROUPS 2
/* Launch flag (same word as the folds): one-right-hand-side passes stream each
 * warp's block range through a shared-memory ring filled by 1-D bulk copies
 * (cp.async.bulk on mbarriers) instead of keeping `unroll` blocks in flight
 * in registers -- more bytes in flight per SM for the short blocks of low
 * rates.  Same results bit for bit as the register-fed kernel; not with lane
 * groups, and device-resident streams only (host-resident handles ignore it).
 * whff_tune includes it among its candidates. */
#define WHFF_CONFIG_BULK 4
int whff_tune(whff_handle* h, int iters, void* stream, double* best_ms);
int whff_get_config(const whff_handle* h, int* unroll, int* ctas_per_sm, int* fold);
int whff_set_config(whff_handle* h, int unroll, int ctas_per_sm, int fold);

/* Crossover of the two engines (Sec. 4.4's GEMV with many right-hand sides is
 * a GEMM): passes of at least min_rhs columns run on the tensor cores, smaller
 * ones on the CUDA cores.  Default 4 (from 4 columns on, one tensor-core
 * pass is at least as fast as the CUDA cores on GB300; whff_tune measures it
 * per matrix); 33 = CUDA cores only.  Tensor-core
 * passes need a WZ2, BF16, FP16 or FP8 handle created with max_rhs >= 2 (WHFF_EINVAL otherwise,
 * unless min_rhs = 33); whff_get_crossover reports 33 for handles without
 * them.  Both engines meet the same accuracy bar; their roundings differ. */
int whff_get_crossover(const whff_handle* h, int* min_rhs);
int whff_set_crossover(whff_handle* h, int min_rhs);

/* Many resident matrices in one step (uneven sizes, R[i] right-hand sides
 * each, 1 <= R[i] <= the max_rhs of handle i, else WHFF_EINVAL): one persistent launch per right-hand-side class (8, 4, 2, 1) whose
 * warps split the concatenated block order of all matrices into equal
 * ranges; R[i] is taken in column groups of 8, then one group of 4, 2, 1;
 * a matrix with R[i] at or above its handle's crossover (tensor-core passes
 * available, see whff_set_crossover) is instead stepped by its own
 * tensor-core passes (see whff_step).
 * All matrices must be WZ2 of one format and rate, or all of one scaled
 * format (BF16, FP16, FP8, FP32: units are then the 16-byte column chunks of
 * a band, and a matrix at or above its crossover is stepped by its own
 * tensor-core passes within the batch step).  whff_batch_step: x[i]
 * (N_i x R[i], ldx[i]), y[i] (M_i x R[i], ldy[i]), state[i] (M_i, may be NULL,
 * or state itself NULL) are device pointers; each state is updated for
 * r = 0..R[i]-1 in order after all of its matrix's columns are computed.
 * The device work tables of a batch are rewritten by every step: issue the
 * steps of one batch on one stream (they are ordered there). */
typedef struct whff_batch whff_batch;
int whff_batch_create(whff_handle* const* hs, const int* R, int count, whff_batch** b);
int whff_batch_step(whff_batch* b, const float* const* x, const int64_t* ldx, double* const* y, const int64_t* ldy,
                    double* const* state, double decay, void* stream);
void whff_batch_destroy(whff_batch* b);

/* ------------------------------------------------------------- serving layer */
/* A request server over resident models (Sec. 1: a firm real-time loop that
 * tolerates a missed deadline).  Requests that arrive while a model's
 * previous pass is on the GPU are queued and folded into its next pass as
 * extra right-hand sides (continuous batching, batch buckets 1, 2, 4, ...,
 * max_batch), each bucket a captured CUDA graph (H2D x, step, D2H y); the
 * columns of a pass are applied in arrival order, so the carried state and
 * every y are the same as for one-at-a-time service (bit for bit when both
 * passes run on the same engine; within the accuracy bar when a wide pass
 * runs on the tensor cores).  Different models run concurrently on nstreams
 * streams.  A model whose pass streams more than 512 MB is captured as
 * consecutive row slits of at most that size (whff_set_slice_rows), so the
 * kernels of smaller, higher-priority models get SMs between slits instead of
 * waiting for a whole pass.  Models are admitted while the sum of
 * their device footprints (matrix, workspace, state, staging) stays within
 * hbm_budget bytes; otherwise whff_server_add_model returns WHFF_EBUSY.  The
 * server does not own the handles (destroy it before them). */
typedef struct whff_server whff_server;
int whff_server_create(size_t hbm_budget, int max_batch, int nstreams, whff_server** s);
int whff_server_add_model(whff_server* s, whff_handle* h, double decay, int* model_id);
/* As whff_server_add_model; with WHFF_SERVER_WAIT a model that does not fit
 * the budget (or arrives while earlier models wait) is registered as waiting
 * (returns WHFF_OK with its id) instead of refused, and is admitted -- state,
 * staging and graphs allocated and captured -- as soon as removals free
 * enough memory, in registration order (first come, first served).
 * whff_server_model_state: 1 admitted, 2 waiting, 0 removed.
 * whff_server_remove_model waits for the model's stream, frees its state,
 * staging and graphs (not its handle, which the caller owns), returns its
 * footprint to the budget and admits waiting models that now fit.  Requests
 * for a model that is not admitted are refused by whff_server_run (status 3). */
#define WHFF_SERVER_WAIT 1u
int whff_server_add_model_ex(whff_server* s, whff_handle* h, double decay, unsigned flags, int* model_id);
int whff_server_model_state(const whff_server* s, int model_id, int* state);
int whff_server_remove_model(whff_server* s, int model_id);
int whff_server_reset_state(whff_server* s, int model_id);
int whff_server_read_state(whff_server* s, int model_id, double* host_out);
/* Replay a trace in real time: request i for model[i] arrives arrival_s[i]
 * seconds after the start (non-decreasing) with x[i] (N floats, host).
 * Dispatch is earliest-deadline-first; each model runs on its own stream,
 * smaller models at higher stream priority.  With drop_after_s > 0 the server
 * is firm real-time (Sec. 1: a late correction is useless): a request still
 * queued drop_after_s after arrival is discarded.  On return latency_s[i] =
 * completion - arrival as seen by the host (for a dropped request its age
 * when discarded), batch[i] = requests in its pass (0 if dropped), status[i]
 * (optional) = 0 in time, 1 late, 2 dropped, 3 refused (model not admitted),
 * and y[i] (if y and y[i] are not
 * NULL) holds its M doubles.  WHFF_ETIMEOUT if the run exceeds max_wait_s. */
int whff_server_run(whff_server* s, int n, const int* model, const double* arrival_s, const float* const* x,
                    double* const* y, double* latency_s, int* batch, int* status, double drop_after_s,
                    double max_wait_s);
void whff_server_destroy(whff_server* s);

/* Decode the whole matrix to FP64 row-major (ldo >= N) on the device,
 * bit-identical to the format's definition (WZ1: (double)(float)q * 2^(emax-26);
 * scaled: scale * q).  Sec. 5.2 measures this as decompression throughput. */
int whff_decompress(whff_handle* h, double* out, int64_t ldo, void* stream);

/* Read and clear the handle's device status word (synchronizes the stream). */
int whff_sync_status(whff_handle* h, void* stream);

/* Failure detection of the tensor-core passes: every device-side wait of
 * their kernels (an MMA group's commit, a bulk copy's arrival) is bounded; a
 * wait that runs out records WHFF_ETIMEOUT in the status word, the CTA stops
 * at its next barrier, waits once more -- with the full limit -- for its MMAs
 * and copy in flight, frees its tensor memory and returns, so the context
 * stays usable.  whff_set_wait_limit sets the polls of the in-loop waits of
 * this handle's passes (default about 2^22, about a second; polls < 0 restores
 * it; 0 makes every in-loop wait give up at once).  Lowering it is for tests of
 * failure detection; the y of a pass that timed out is not valid.  Errors:
 * WHFF_EINVAL. */
int whff_set_wait_limit(whff_handle* h, int64_t polls);

/* Free every device allocation of the handle (stream-ordered on its stream). */
void whff_destroy(whff_handle* h);

/* A step that allocates nothing (the paper has no counterpart: this serves
 * callers that cannot call cudaMalloc -- fixed-memory real-time controllers,
 * code inside a private memory pool, loops that must not allocate).  The
 * caller passes the WZ1 stream (the blob minus its 64-byte header, in row-major
 * block order, in caller-owned device memory, 16-byte aligned; 8 for rate 12),
 * its rate (8, 12 or 16) and shape, and x, y, state as in whff_step; R must be
 * 1, 2, 4 or 8.  Split-K partials go to a file-scope device array of
 * WHFF_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * exit; a call whose partials would not fit returns WHFF_EINVAL.  The first
 * call on each device looks up the array's device address (make it before any
 * stream capture); the address is kept for the life of the process, so after
 * cudaDeviceReset (a new primary context) this entry point must not be used
 * again in that process.  All calls share the array: calls that overlap on
 * the GPU race and must be serialised by the caller.  The stream's length is
 * not passed: stream_dev must hold ceil(M/4)*ceil(N/4)*2*rate bytes, else the
 * kernel reads past it.  Calls no cudaMalloc/cudaFree. */
#define WHFF_NOALLOC_SCRATCH_BYTES (4u << 20)
int whff_step_noalloc(const void* stream_dev, int rate, int64_t M, int64_t N, const float* x, int R, int64_t ldx,
                      double* y, int64_t ldy, double* state, double decay, void* stream);

/* Measurement: read a device buffer once at full bandwidth (16-byte streaming
 * loads, a persistent grid, four loads in flight per thread) and XOR all its
 * 32-bit words into *d_xor (device memory; XOR-ed into, so zero it first).
 * This is the achievable-read roofline the fused kernels stream against: a
 * read-only stream is not a copy, and can exceed the copy bandwidth.
 * buf must be 16-byte aligned and bytes a multiple of 16 (WHFF_EINVAL
 * otherwise).  Asynchronous on `stream`. */
int whff_read_probe(const void* buf, size_t bytes, uint32_t* d_xor, void* stream);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* whff_last_error(void);

/* Library version string, e.g. "whff 0.1 sm_103a". */
const char* whff_version(void);

#ifdef __cplusplus
}
#endif
#endif
