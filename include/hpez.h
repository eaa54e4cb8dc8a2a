/*
 * hpez.h -- C-ABI of libhpez.so: the HPEZ interpolation predict-and-quantize
 * path (arXiv 2311.12133) as hand-written sm_103a CUDA kernels.
 *
 * Conventions for every entry point:
 *  - Plain pointers and sizes only.  "d_" pointers are CUDA device pointers,
 *    "h_" pointers are host pointers.  `stream` is a cudaStream_t passed as
 *    void* (NULL = the legacy default stream).
 *  - The caller owns every input and output buffer; the context owns the
 *    device scratch it allocates (grown on demand, freed by hpez_destroy).
 *  - Return value: HPEZ_OK (0) or a negative HPEZ_ERR_* code; nothing is
 *    written to an output on error except where stated.  Errors that the
 *    kernels detect (non-finite input, corrupt stream, capacity) are read
 *    back at the end of the call, which synchronizes `stream` once.
 *  - A context is not thread-safe; use one per host thread.
 *  - Output streams must start at a 16-byte aligned device address
 *    (cudaMalloc gives 256).
 *
 * Field layout: float32, row-major, dims[0] slowest, 1 <= ndim <= 3,
 * every dim >= 1, total points < 2^32.
 */
#ifndef HPEZ_H
#define HPEZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HPEZ_API __attribute__((visibility("default")))
#else
#define HPEZ_API
#endif

#define HPEZ_MAX_LEVELS 16
#define HPEZ_HEADER_BYTES 512

/* error codes */
#define HPEZ_OK 0
#define HPEZ_ERR_INVALID_ARG (-1)    /* bad ndim/dims/eb/config/pointer */
#define HPEZ_ERR_NONFINITE_INPUT (-2)/* NaN/Inf with a relative bound */
#define HPEZ_ERR_OUT_TOO_SMALL (-3)  /* output capacity too small */
#define HPEZ_ERR_CORRUPT_STREAM (-4) /* stream fails validation */
#define HPEZ_ERR_NO_MEMORY (-5)      /* device allocation failed */
#define HPEZ_ERR_CUDA (-7)           /* a CUDA runtime call failed */
#define HPEZ_ERR_UNSUPPORTED (-8)    /* valid but not implemented */
#define HPEZ_ERR_TIMEOUT (-9)        /* a bounded device wait gave up */
#define HPEZ_ERR_TOO_LARGE (-10)     /* beyond hpez_decompress_noalloc's limit */

/* error-bound modes: Sec. 3.1 Eq. 1 (absolute e) and Sec. 7.1.3
 * (value-range relative eps, e = eps * (max - min)) */
#define HPEZ_EB_ABS 0
#define HPEZ_EB_REL 1

/* interpolators, Sec. 5.2: Eq. 2 linear, Eq. 4 not-a-knot cubic, Eq. 6
 * natural cubic (same-level forms Eq. 10 / Eq. 11, Sec. 5.4.2) */
#define HPEZ_LINEAR 0
#define HPEZ_CUBIC_NAK 1
#define HPEZ_CUBIC_NAT 2
/* the natural cubic spline through every known point of a pass line, solved
 * per line (a whole-line form beside the paper's local Eq. 6; opt in, for
 * the 1D-style paradigm without same-level halves or a block map) */
#define HPEZ_SPLINE_GLOBAL 3
/* paradigms, Sec. 5.3: 1D-style passes or multi-dimensional (Eq. 8) */
#define HPEZ_PARADIGM_1D 0
#define HPEZ_PARADIGM_MD 1

/* Predictor configuration theta (Sec. 6.2-6.6).  Per-level arrays are
 * indexed by l-1, l = 1 the finest level (stride 1). */
typedef struct {
  int32_t anchor_stride; /* A, power of two in [2, 32768] (Sec. 5.1) */
  int32_t frozen_dim;    /* -1, or a dim never interpolated (Sec. 6.3) */
  int32_t chunk_syms;    /* Huffman chunk of 32 lanes, 2^k in [256, 32768] */
  int32_t blockwise;     /* 1: per-block interpolator map (Sec. 6.6) */
  int32_t block_size;    /* block side of the map (Sec. 6.6 default 32) */
  int32_t predictor;     /* 0 interpolation; 1, 2: the Lorenzo predictor of
                            that order (Sec. 6.5) on blocks of side
                            anchor_stride, not with blockwise.  A block's
                            columns must fit one CTA: A <= 32 in 3D, <= 1024
                            in 2D, else hpez_compress returns UNSUPPORTED;
                            hpez_decompress_noalloc takes interpolation
                            streams only (UNSUPPORTED) */
  double alpha, beta;    /* Eq. 15 level bounds, both >= 1 */
  double md_inv_var[3];  /* 1/sigma_d^2 for the Eq. 14 weights, > 0 */
  uint8_t interp[HPEZ_MAX_LEVELS];     /* HPEZ_LINEAR / _CUBIC_NAK / _NAT /
                                          _SPLINE_GLOBAL */
  uint8_t paradigm[HPEZ_MAX_LEVELS];   /* HPEZ_PARADIGM_* */
  uint8_t same_level[HPEZ_MAX_LEVELS]; /* Sec. 5.4.2, cubic only */
  uint8_t order[HPEZ_MAX_LEVELS][3];   /* 1D-style dim order (interp dims) */
  const uint8_t* h_blockmap; /* host; per block: bits 0-1 interp, bit 2
                                same-level; row-major over ceil(n/bs) */
} hpez_config;

typedef struct hpez_ctx hpez_ctx;

/* Create a context on CUDA device `device` (made current for the call).
 * *out receives the handle.  Errors: INVALID_ARG, CUDA. */
HPEZ_API int hpez_create(hpez_ctx** out, int device);

/* Free the context and its device scratch.  NULL is accepted. */
HPEZ_API int hpez_destroy(hpez_ctx* ctx);

/* Default theta for ndim: A = 128/64/32 for 1D/2D/3D, not-a-knot cubic
 * (Eq. 4) at every level, 1D-style order 0..ndim-1, alpha = beta = 1,
 * chunk 16384, no freezing, no block map. */
HPEZ_API int hpez_default_config(int ndim, hpez_config* out);

/* Upper bound of the compressed size in bytes for a field of these dims. */
HPEZ_API int hpez_compress_bound(int ndim, const uint64_t* dims, uint64_t* out_bytes);

/* Compress (Sec. 4 Steps 2-4): anchors, level-wise interpolation
 * prediction, linear quantization with outlier escape, Huffman coding.
 *   d_in      device, N float32 (not modified)
 *   eb_mode   HPEZ_EB_ABS (eb = e) or HPEZ_EB_REL (eb = eps)
 *   cfg       host pointer, NULL = hpez_default_config(ndim)
 *   d_out     device, out_cap bytes, 16-byte aligned
 *   h_out_size host, receives the stream size
 * Errors: INVALID_ARG, NONFINITE_INPUT (REL mode only), OUT_TOO_SMALL,
 * NO_MEMORY, CUDA.  Synchronizes `stream` once at the end. */
HPEZ_API int hpez_compress(hpez_ctx* ctx, const float* d_in, int ndim,
                  const uint64_t* dims, int eb_mode, double eb,
                  const hpez_config* cfg, void* d_out, uint64_t out_cap,
                  uint64_t* h_out_size, void* stream);

/* Decompress a stream made by hpez_compress (the mirror of the level
 * sweep: x' = prediction + 2 e_l q, or the stored outlier).
 *   d_in      device, in_size bytes, 16-byte aligned
 *   d_out     device, out_cap_elems float32 (>= N)
 * Reads the 512-byte header to the host first (one synchronization).
 * Errors: CORRUPT_STREAM, OUT_TOO_SMALL, INVALID_ARG, NO_MEMORY, CUDA. */
HPEZ_API int hpez_decompress(hpez_ctx* ctx, const void* d_in, uint64_t in_size,
                    float* d_out, uint64_t out_cap_elems, void* stream);

/* The same compress and decompress, enqueued on `stream` with no host
 * synchronization (the launch sequences of hpez_compress / hpez_decompress,
 * so the streams and fields are the same byte for byte).  The outcome is
 * written on the device by the last kernel:
 *   d_size    device u64: the stream size (0 on error)
 *   d_status  device int32: 0 or a negative HPEZ_ERR_* (NONFINITE_INPUT,
 *             OUT_TOO_SMALL, CORRUPT_STREAM, TIMEOUT)
 *   h_header  host copy of the stream's first 512 bytes (decompress): the
 *             launches are planned from it, so it must be the header of the
 *             stream at d_in when the work runs
 * The returned code covers only what the host checks before enqueueing
 * (arguments, the header, capacities), as in the synchronous calls.  A call
 * on a field larger than the context's scratch grows it first (cudaMalloc
 * after a device synchronization); a call that needs no growth makes no
 * allocation and no host read, so it can be captured in a CUDA graph
 * (the capture replays the same pointers, sizes, bound and header).
 * Refused (UNSUPPORTED): a config with a block map (compress reads the map
 * from host memory) and a stream that went through the lossless stage
 * (undoing it sizes a buffer on the host).  Block maps inside a stream are
 * read on the device. */
HPEZ_API int hpez_compress_async(hpez_ctx* ctx, const float* d_in, int ndim,
                                 const uint64_t* dims, int eb_mode, double eb,
                                 const hpez_config* cfg, void* d_out, uint64_t out_cap,
                                 uint64_t* d_size, int32_t* d_status, void* stream);
HPEZ_API int hpez_decompress_async(hpez_ctx* ctx, const void* d_in, uint64_t in_size,
                                   const void* h_header, float* d_out,
                                   uint64_t out_cap_elems, int32_t* d_status, void* stream);

/* Decompression that allocates nothing -- no counterpart in the paper; it
 * exists for callers that may not allocate memory: code running under a
 * memory manager that owns the device heap, or a pre-sized loop that must
 * not call cudaMalloc/cudaFree (or an allocating library) once running.
 * Same result as hpez_decompress, needs no context.
 *   d_in   device, in_size bytes, 16-byte aligned; d_out device, >= N floats
 *   stream cudaStream_t as void*; uses the current CUDA device
 * Scratch is one file-scope device array of HPEZ_NOALLOC_SCRATCH_BYTES
 * (16 MiB), held by every GPU that loads the library until the process
 * exits.  Fields of more than HPEZ_NOALLOC_MAX_POINTS points (2^21) are
 * refused with HPEZ_ERR_TOO_LARGE.  The first call on a device looks the
 * array's device address up (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialized by the caller.  Synchronizes `stream`.
 * Errors: as hpez_decompress, plus HPEZ_ERR_TOO_LARGE, and
 * HPEZ_ERR_UNSUPPORTED for a Lorenzo-predictor stream, a stream with a
 * global natural-spline level (interp HPEZ_SPLINE_GLOBAL) or a stream that
 * went through the lossless stage (hpez_lossless_encode). */
#define HPEZ_NOALLOC_MAX_POINTS 2097152u
#define HPEZ_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
HPEZ_API int hpez_decompress_noalloc(const void* d_in, uint64_t in_size,
                                     float* d_out, uint64_t out_cap_elems,
                                     void* stream);

/* Host-buffer forms of the two calls above: copy h_in to the device, run
 * the call, copy the result back (all on `stream`, synchronous). */
HPEZ_API int hpez_compress_host(hpez_ctx* ctx, const float* h_in, int ndim,
                       const uint64_t* dims, int eb_mode, double eb,
                       const hpez_config* cfg, void* h_out, uint64_t out_cap,
                       uint64_t* h_out_size, void* stream);
HPEZ_API int hpez_decompress_host(hpez_ctx* ctx, const void* h_in, uint64_t in_size,
                         float* h_out, uint64_t out_cap_elems, void* stream);

/* Parse a host copy of the header (>= 512 bytes): ndim, dims[3] and the
 * absolute error bound in use.  Errors: CORRUPT_STREAM, INVALID_ARG. */
HPEZ_API int hpez_inspect(const void* h_header, uint64_t n, int* ndim, uint64_t* dims,
                 double* abs_eb);

/* Static text for an error code. */
HPEZ_API const char* hpez_strerror(int code);

/* ---- batched form (no counterpart in the paper: a GPU execution form of
 * the same method) ----
 * Many fields compressed (or streams decompressed) together.  Each field
 * runs exactly the single-field operations, so its stream is byte-identical
 * to hpez_compress's.  The operations are grouped into ticks: the ops
 * before the sweep by position, then level by level from the coarsest
 * (level l of every field in the same tick, fields with fewer levels
 * joining at theirs), then the ops after the sweep by position.  A tick
 * launches one kernel per operation kind over the concatenated work of its
 * fields; a level's launch is persistent (at most the CTAs resident on the
 * GPU, each walking tiles of several fields).  The kernel family and tile
 * shape of each level come from the context's schedule table (below) when
 * it holds the level's key, else from fixed rules.  Creation plans every
 * field, allocates one workspace and uploads every tick's job tables; a run
 * is kernel launches only. */
typedef struct {
  const float* d_in;     /* device, N float32, row-major */
  int32_t ndim;
  int32_t eb_mode;       /* HPEZ_EB_ABS / HPEZ_EB_REL */
  uint64_t dims[3];
  double eb;
  const hpez_config* cfg; /* host, NULL = default; read at creation */
  void* d_out;           /* device, out_cap bytes, 16-byte aligned */
  uint64_t out_cap;
} hpez_field_desc;

typedef struct {
  const void* d_in;      /* device stream, 16-byte aligned */
  uint64_t in_size;
  const void* h_header;  /* host copy of the stream's first 512 bytes */
  float* d_out;          /* device, >= N floats, 4-byte aligned */
  uint64_t out_cap_elems;
} hpez_stream_desc;

typedef struct hpez_batch hpez_batch;

/* Plan n fields (streams) into one batch.  The device pointers are bound
 * to the batch: every run reads and writes the same buffers.  Errors:
 * INVALID_ARG / CORRUPT_STREAM / OUT_TOO_SMALL for the first bad entry,
 * UNSUPPORTED (a global natural-spline level, or a Lorenzo-predictor
 * geometry the Lorenzo kernel does not take), NO_MEMORY, CUDA.  A
 * Lorenzo-predictor field (Sec. 6.5) runs its pass in the finest level's
 * tick.  Synchronizes the device once (the uploads). */
HPEZ_API int hpez_batch_create_compress(hpez_ctx* ctx, int n,
                                        const hpez_field_desc* fields,
                                        hpez_batch** out);
HPEZ_API int hpez_batch_create_decompress(hpez_ctx* ctx, int n,
                                          const hpez_stream_desc* streams,
                                          hpez_batch** out);
/* Enqueue one run on `stream` (asynchronous, launches only). */
HPEZ_API int hpez_batch_run(hpez_batch* b, void* stream);
/* The same run through a CUDA graph: the first call captures the launch
 * sequence on `stream` (which must not be the legacy default stream),
 * later calls replay it. */
HPEZ_API int hpez_batch_run_graph(hpez_batch* b, void* stream);
/* After a run: per-field stream sizes (compress; 0 for decompress) and
 * status (0 or a negative HPEZ_ERR_*), copied to host arrays of n entries
 * (either may be NULL).  Synchronizes `stream`. */
HPEZ_API int hpez_batch_results(hpez_batch* b, void* stream, uint64_t* h_sizes,
                                int32_t* h_status);
/* Kernel launches and ticks of one run. */
HPEZ_API int hpez_batch_launch_count(hpez_batch* b, uint64_t* launches,
                                     uint64_t* ticks);
/* Frees the batch's device memory.  Batches and servers belong to the
 * context they were made on: destroy them before that context. */
HPEZ_API int hpez_batch_destroy(hpez_batch* b);

/* ---- level schedules of the batched and served forms (no counterpart in
 * the paper: how the GPU runs a level, never what it computes) ----
 * A schedule table maps a level key -- the field's shape class, the level's
 * stride s = 2^(l-1), its interpolator, paradigm and direction -- to a
 * kernel family and tile shape.  hpez_tuning_search finds the entries by
 * timing every candidate schedule on the GPU (an offline search); the table
 * is saved to and loaded from a text file.  A schedule changes speed only:
 * streams and fields are byte-identical under any table.  A table entry
 * that a field's level cannot run (shape, alignment, shared memory) falls
 * back to the fixed rules. */
typedef struct {
  int32_t ndim;      /* 1..3 */
  int32_t cls[3];    /* floor(2 log2 n) (half-octave class) of each slot
                        of the field seen as 3D, slowest first (0 for the
                        leading slots of 1D and 2D fields) */
  int32_t stride;    /* s = 2^(l-1) */
  int32_t interp;    /* HPEZ_LINEAR..HPEZ_CUBIC_NAT, or 3: a block map or
                        same-level halves (the per-point interpolator) */
  int32_t paradigm;  /* HPEZ_PARADIGM_1D / HPEZ_PARADIGM_MD */
  int32_t decomp;    /* 0 compress, 1 decompress */
} hpez_level_key;

#define HPEZ_FAM_LEVEL3D 1  /* 3D level, rows along dim 1 per tile: tile[1] */
#define HPEZ_FAM_MD3W 2     /* finest 3D multi-dimensional level as warp
                               strips, `chunks` chunks of planes per field
                               (0: as many as fill the GPU alone) */
#define HPEZ_FAM_MD3 3      /* 3D multi-dimensional level, even then odd
                               planes, tile[1] rows per tile */
#define HPEZ_FAM_FUSED 4    /* fused tile of extents tile[0..2] */
#define HPEZ_FAM_PASS 5     /* upsample + one launch per pass */

typedef struct {
  int32_t family;    /* HPEZ_FAM_* */
  int32_t tile[3];   /* as the family says; 0 = the fixed rule's value */
  int32_t chunks;
  float time_us;     /* the search's time for this level (informational) */
} hpez_level_sched;

typedef struct hpez_tuning hpez_tuning;

/* A table of level schedules (host memory; no GPU needed). */
HPEZ_API int hpez_tuning_create(hpez_tuning** out);
HPEZ_API int hpez_tuning_destroy(hpez_tuning* t);
/* Insert or replace one entry.  INVALID_ARG for an out-of-range key or
 * family. */
HPEZ_API int hpez_tuning_set(hpez_tuning* t, const hpez_level_key* key,
                             const hpez_level_sched* sched);
/* *found = 1 and *sched filled when the key is in the table, else 0. */
HPEZ_API int hpez_tuning_get(const hpez_tuning* t, const hpez_level_key* key,
                             hpez_level_sched* sched, int* found);
HPEZ_API int hpez_tuning_count(const hpez_tuning* t, uint64_t* n);
/* Text file, one entry per line: ndim cls0 cls1 cls2 stride interp
 * paradigm decomp family tile0 tile1 tile2 chunks time_us ('#' starts a
 * comment line).  Load merges into the table.  Errors: INVALID_ARG (no
 * file, or a malformed line, with the table unchanged). */
HPEZ_API int hpez_tuning_save(const hpez_tuning* t, const char* path);
HPEZ_API int hpez_tuning_load(hpez_tuning* t, const char* path);
/* The key of level l (1 = finest) of a field of these dims and config
 * (NULL = default) in direction decomp.  INVALID_ARG for bad dims, config
 * or level. */
HPEZ_API int hpez_level_key_of(int ndim, const uint64_t* dims, const hpez_config* cfg,
                               int level, int decomp, hpez_level_key* out);
/* The context copies the table (NULL: back to the fixed rules); batches
 * and server requests planned afterwards use it. */
HPEZ_API int hpez_use_tuning(hpez_ctx* ctx, const hpez_tuning* t);
/* The offline search for one field class: `copies` copies of the device
 * field (0: enough to hold about 2^25 points) are compressed, and their
 * streams decompressed, as one batch under each candidate schedule (every
 * family the field's levels can run, with tile shapes or chunk counts from
 * a fixed list); each level's ticks are timed with CUDA events over `reps`
 * runs (median) after a warm-up run, and the fastest candidate of each
 * level and direction goes into t.  Synchronizes; allocates the batches'
 * buffers.  Errors as hpez_batch_create_compress. */
HPEZ_API int hpez_tuning_search(hpez_ctx* ctx, hpez_tuning* t, const float* d_x, int ndim,
                                const uint64_t* dims, int eb_mode, double eb,
                                const hpez_config* cfg, int copies, int reps, void* stream);

/* ---- served form (no counterpart in the paper) ----
 * A request loop with continuous batching.  Requests carry HOST buffers.
 * Each step: finished requests copy their result to the host and free their
 * memory; queued requests are admitted (FIFO) while a slot is free and their
 * device memory (input + output + workspace) fits the budget, their input
 * is copied to the device; then one tick advances every admitted request by
 * one operation (as in the batched form), so a request admitted now runs
 * alongside requests that are levels or stages ahead.  Results equal the
 * single-call results. */
#define HPEZ_REQ_COMPRESS 0
#define HPEZ_REQ_DECOMPRESS 1
typedef struct {
  int32_t op;             /* HPEZ_REQ_* */
  int32_t ndim;           /* compress */
  uint64_t dims[3];       /* compress */
  int32_t eb_mode;        /* compress */
  int32_t reserved;
  double eb;              /* compress */
  const hpez_config* cfg; /* compress, NULL = default; copied at submit */
  const void* h_in;       /* host: the field (compress) or stream (decompress);
                             must stay valid until the request completes */
  uint64_t in_bytes;      /* decompress: stream size */
  void* h_out;            /* host: stream (compress) or field (decompress) */
  uint64_t out_cap;       /* bytes of h_out */
} hpez_request;

typedef struct hpez_server hpez_server;

/* budget_bytes of device memory is allocated at creation; max_slots bounds
 * the requests in flight.  Errors: INVALID_ARG, NO_MEMORY, CUDA. */
HPEZ_API int hpez_server_create(hpez_ctx* ctx, uint64_t budget_bytes,
                                int max_slots, void* stream,
                                hpez_server** out);
/* Queue a request; *id identifies it in hpez_server_poll.  Errors:
 * INVALID_ARG / CORRUPT_STREAM (checked now), TOO_LARGE (it can never fit
 * the budget), UNSUPPORTED (as hpez_batch_create_compress). */
HPEZ_API int hpez_server_submit(hpez_server* s, const hpez_request* req,
                                uint64_t* id);
/* One step: retire, admit, one tick.  Never waits for the GPU except to
 * reuse a job-table buffer (at most 8 ticks in flight). */
HPEZ_API int hpez_server_step(hpez_server* s);
/* Completed requests since the last poll (up to cap): id, status, result
 * bytes, latency from submit to completion in seconds. */
HPEZ_API int hpez_server_poll(hpez_server* s, int cap, uint64_t* ids,
                              int32_t* status, uint64_t* sizes,
                              double* latency_s, int* n);
HPEZ_API int hpez_server_stats(hpez_server* s, int* active, int* queued,
                               uint64_t* used_bytes, uint64_t* ticks,
                               uint64_t* launches);
HPEZ_API int hpez_server_destroy(hpez_server* s);

/* ---- auto-tuning (Sec. 6) ----
 * The tuner picks theta for one field from compression tests on samples:
 *   Sec. 6.1  statistics on a uniform lattice (stride t, the smallest with
 *             t^ndim * sample_rate >= 1) of points whose +-3 neighbours
 *             exist on every dim: per dim, the squared error of linear and
 *             of not-a-knot cubic interpolation of the original values, as
 *             fixed-point sums of floor(min(|err|/e, 2^16)^2 * 256).  They
 *             give the Eq. 14 inverse variances count*256/max(sum, 1) and
 *             the most non-smooth dim (largest cubic sum, first on ties).
 *   Sec. 6.2  per level, coarsest first, every candidate (linear, then
 *             not-a-knot, then natural cubic; for each the 1D-style orders
 *             of the interpolation dims in lexicographic order and then the
 *             multi-dimensional paradigm; cubic ones without and with
 *             same-level interpolation) is tested on the sample blocks
 *             (A+1 points per side on a lattice of blocks, about block_rate
 *             of the volume); the smallest sum of floor(min(|err|/e_l, 2^24)
 *             * 256) over the level's points wins, the first on ties.
 *   Sec. 6.4  (alpha, beta) from {(1,1)} + {1.25,1.5,1.75,2} x {2,4,8,16}:
 *             the smallest estimate of Huffman bits of the sample codes
 *             + 32 per escape + 32 per anchor.
 *   Sec. 6.3  the same tuning with the most non-smooth dim frozen; kept
 *             if its estimate is smaller.
 *   Sec. 6.5  order-1 and order-2 Lorenzo tests on the same blocks (zero
 *             padding, global bound), bits * lorenzo_coef compared with the
 *             interpolation estimate; when the smaller is strictly below,
 *             theta selects the Lorenzo predictor of that order
 *             (predictor 1 or 2, order 1 on a tie) and no block map is
 *             tuned.
 *   Sec. 6.6  per block of block_size^ndim, a centred sub-block of side
 *             max(5, round(block_size * sub_frac^(1/ndim))), anchor stride
 *             the largest power of two <= max(2, side-1); candidates
 *             linear, not-a-knot, not-a-knot + same-level, natural,
 *             natural + same-level, one for all levels; the smallest
 *             summed level score wins -> block map codes 0,1,5,2,6.
 * All scores are integers, so the choices do not depend on the order of
 * the reductions. */
typedef struct {
  double sample_rate;   /* Sec. 6.1 lattice density, default 0.002 */
  double block_rate;    /* Sec. 6.2 sampled volume fraction, default 0.01 */
  double sub_frac;      /* Sec. 6.6 sub-block volume fraction, default 0.04 */
  double lorenzo_coef;  /* Sec. 6.5 multiplier of the Lorenzo bits, 1.0 */
  int32_t block_size;   /* Sec. 6.6 block side, default 32 */
  int32_t tune_levels, tune_eb, tune_freeze, tune_lorenzo, tune_blockwise;
  int32_t allow_natural, allow_same_level;  /* candidate sets */
  int32_t anchor_stride; /* 0: the default for ndim */
} hpez_tune_params;

typedef struct {
  uint64_t stats_count, mse_lin[3], mse_cub[3]; /* Sec. 6.1 fixed-point sums */
  int32_t nonsmooth_dim, froze, lorenzo_better;
  uint32_t n_sample_blocks;
  uint64_t bits[2];          /* sample estimate without / with freezing */
  uint64_t lorenzo_bits[2];  /* order 1, order 2 */
  uint8_t level_choice[2][HPEZ_MAX_LEVELS]; /* candidate index per level */
  uint64_t level_score[2][HPEZ_MAX_LEVELS]; /* its score */
} hpez_tune_report;

HPEZ_API int hpez_default_tune_params(hpez_tune_params* out);
/* Entries of the block map for these dims: prod ceil(dims[d]/block_size). */
HPEZ_API uint64_t hpez_blockmap_size(int ndim, const uint64_t* dims, int block_size);

/* Tune theta for the field d_in (device, N float32, row-major).
 *   tp          host, NULL = hpez_default_tune_params
 *   h_cfg       host, receives theta (ready for hpez_compress)
 *   h_blockmap  host, >= hpez_blockmap_size entries when tune_blockwise;
 *               h_cfg->h_blockmap points at it when the map is produced
 *   h_report    host, optional, the intermediate results
 * A constant field (relative mode) yields the default theta.  The sample
 * blocks must fit in shared memory: (A+1)^k * (other extents) * 4 bytes
 * <= 200 KiB, else UNSUPPORTED.  Errors: INVALID_ARG, NONFINITE_INPUT
 * (relative mode), OUT_TOO_SMALL (block map), UNSUPPORTED, NO_MEMORY,
 * CUDA.  Synchronizes `stream` several times (not graph-capturable). */
/* Compress with full auto-tuning (the paper's compression: Sec. 6 tuning,
 * then Sec. 4-5 with the tuned theta): hpez_tune (tp NULL = defaults) then
 * hpez_compress.  Arguments and errors as in those two calls; h_report is
 * optional. */
HPEZ_API int hpez_compress_auto(hpez_ctx* ctx, const float* d_in, int ndim,
                                const uint64_t* dims, int eb_mode, double eb,
                                const hpez_tune_params* tp, void* d_out,
                                uint64_t out_cap, uint64_t* h_out_size,
                                hpez_tune_report* h_report, void* stream);
/* The same from host memory: the field is copied to the device, tuned and
 * compressed, and the stream copied back.  Synchronizes `stream`. */
HPEZ_API int hpez_compress_auto_host(hpez_ctx* ctx, const float* h_in, int ndim,
                                     const uint64_t* dims, int eb_mode, double eb,
                                     const hpez_tune_params* tp, void* h_out,
                                     uint64_t out_cap, uint64_t* h_out_size,
                                     void* stream);

HPEZ_API int hpez_tune(hpez_ctx* ctx, const float* d_in, int ndim,
                       const uint64_t* dims, int eb_mode, double eb,
                       const hpez_tune_params* tp, hpez_config* h_cfg,
                       uint8_t* h_blockmap, uint64_t blockmap_cap,
                       hpez_tune_report* h_report, void* stream);

/* ---- the quality-metric target and integer inputs ----
 * PSNR of y against x (Sec. 7.1.3): 20 log10(max x - min x) - 10 log10(MSE),
 * the squared errors summed exactly in the fixed-point unit `unit`:
 * q_i = rint((x_i - y_i) / unit) in double, sse = sum q_i^2 (64-bit
 * integer; its value does not depend on the order of the sum), MSE =
 * sse unit^2 / n; +inf when sse = 0.
 *   d_x, d_y  device, n floats each; h_psnr, h_sse host, optional
 * Errors: INVALID_ARG (n = 0, unit <= 0, |x_i - y_i| / unit > 2^16),
 * NONFINITE_INPUT (x not finite).  Synchronizes `stream`. */
HPEZ_API int hpez_psnr(hpez_ctx* ctx, const float* d_x, const float* d_y, uint64_t n,
                       double unit, double* h_psnr, uint64_t* h_sse, void* stream);

/* Eq. 1 (Sec. 3.1) with M = PSNR and target m0 = target_db: the largest
 * absolute bound the search finds whose auto-tuned round trip keeps
 * PSNR >= m0, and the stream compressed with it.  The search, in double:
 * from e_u = range sqrt(3) 10^(-m0/20) (uniform errors on [-e, e] give m0)
 * double or halve up to 6 times to bracket the target, then 8 geometric
 * bisection steps e = sqrt(lo hi) keeping PSNR(lo) >= m0; each probe is
 * hpez_compress_auto at the absolute bound e, hpez_decompress and
 * hpez_psnr in the unit (stored bound) / 2^16.  d_in finite, device.
 *   d_out, out_cap as hpez_compress; h_out_size, h_eb (the bound found) and
 *   h_psnr (its PSNR) on the host.  tp: tuning parameters (NULL: defaults).
 * Errors: as hpez_compress_auto, NONFINITE_INPUT.  Synchronizes. */
HPEZ_API int hpez_compress_psnr(hpez_ctx* ctx, const float* d_in, int ndim,
                                const uint64_t* dims, double target_db,
                                const hpez_tune_params* tp, void* d_out, uint64_t out_cap,
                                uint64_t* h_out_size, double* h_eb, double* h_psnr,
                                void* stream);

/* Integer inputs (the integer datasets of Sec. 7): int16, uint16 or int32
 * (|v| <= 2^24) fields are widened to binary32 on the device (exactly) and
 * compressed at the absolute float bound just below floor(e) + 1/2, e the
 * requested bound (REL: eb (max - min) of the integers); decompression
 * rounds to the nearest integer (ties to even) and clamps to the type's
 * range, so every value stays within floor(e) of its input (lossless when
 * e < 1).  The stream records the type in header byte 320 (0 = float32);
 * hpez_decompress of an integer stream returns the unrounded floats.
 *   d_in   device, N values of dtype; tune = 1: hpez_compress_auto with tp,
 *          else hpez_compress with cfg (NULL: default)
 * Errors: INVALID_ARG (an int32 beyond 2^24, a bound beyond 2^22, a
 * dtype that is not the stream's), and those of the calls it makes.
 * Uses a binary32 staging buffer of the context.  Synchronizes. */
#define HPEZ_DTYPE_F32 0
#define HPEZ_DTYPE_I16 1
#define HPEZ_DTYPE_U16 2
#define HPEZ_DTYPE_I32 3
HPEZ_API int hpez_compress_typed(hpez_ctx* ctx, const void* d_in, int dtype, int ndim,
                                 const uint64_t* dims, int eb_mode, double eb,
                                 const hpez_config* cfg, int tune,
                                 const hpez_tune_params* tp, void* d_out, uint64_t out_cap,
                                 uint64_t* h_out_size, void* stream);
HPEZ_API int hpez_decompress_typed(hpez_ctx* ctx, const void* d_in, uint64_t in_size,
                                   void* d_out, int dtype, uint64_t out_cap_elems,
                                   void* stream);

/* ---- the lossless stage after Huffman (Sec. 4, Step 5) ----
 * Read as run suppression of repeated 32-bit words of the stream body (the
 * bytes after the 512-byte header, zero-padded to whole words): per block of
 * 32 words a mask of the words that differ from the word before them (the
 * word before the first is 0), per group of 32 blocks a mask of the blocks
 * whose mask is not 0; only those masks and words are kept.  Output: the
 * header with flag bit 2 and the raw size at byte 328, four u64 counts
 * (words, kept words, kept block masks, 0), the group masks, the kept block
 * masks, the kept words.  When that would not be smaller, the stream is
 * copied unchanged.  hpez_decompress accepts either form (it undoes the
 * stage into a buffer of the context); hpez_decompress_noalloc refuses a
 * stream that went through it (HPEZ_ERR_UNSUPPORTED).
 *   d_in, d_out  device, 16-byte aligned, not overlapping; sizes in bytes
 * Errors: INVALID_ARG (an already encoded stream to encode, or a plain one
 * to decode), OUT_TOO_SMALL, CORRUPT_STREAM (counts or masks that do not
 * match the sizes).  Synchronize `stream`. */
HPEZ_API int hpez_lossless_encode(hpez_ctx* ctx, const void* d_in, uint64_t in_size,
                                  void* d_out, uint64_t out_cap, uint64_t* h_out_size,
                                  void* stream);
HPEZ_API int hpez_lossless_decode(hpez_ctx* ctx, const void* d_in, uint64_t in_size,
                                  void* d_out, uint64_t out_cap, uint64_t* h_out_size,
                                  void* stream);

/* Execution options of a context (the results never depend on them):
 *  HPEZ_OPT_FUSED_LEVELS  1 (default): a level of the 1D-style paradigm
 *                         runs as one tiled kernel; 0: one kernel per pass
 *  HPEZ_OPT_TILE_E0..2    tile extent of that slot of the level grid for
 *                         the fused kernel (0 = built-in heuristic)
 *  HPEZ_OPT_FUSED_SMEM    shared-memory cap in bytes for a fused tile
 *  HPEZ_OPT_LEVEL3D       1 (default): 3D levels in direction order 0,1,2
 *                         with one interpolator use the dedicated kernel
 *  HPEZ_OPT_STREAM_LEVELS 1 (default): the finest 3D level of the
 *                         multi-dimensional paradigm streams its planes
 *                         through shared memory in one launch (rows of a
 *                         multiple of 8 points); 0: two launches
 *  HPEZ_OPT_DROP_COPY     0 (default); n > 0: a test of the bounded device
 *                         waits -- the first CTA of the streamed level kernel
 *                         leaves out the copies of its n-th plane (of the
 *                         Lorenzo box-fed kernel: its first warp's n-th box),
 *                         its wait for them expires and the call returns
 *                         HPEZ_ERR_TIMEOUT (no copy stays in flight; the
 *                         context stays usable)
 *  HPEZ_OPT_WARP_LEVELS   1 (default): the finest 3D level of the
 *                         multi-dimensional paradigm runs one warp per strip
 *                         of rows and columns (rows of an even number of
 *                         points); 0: the streamed or two-launch kernels
 *  HPEZ_OPT_STREAM_CHUNKS 0 (default: as many chunks of planes as fill the
 *                         resident warps); n > 0: the finest-level kernels
 *                         cut dim 0 into n chunks, so a warp or CTA walks
 *                         more planes through its ring (what a large field
 *                         does)
 *  HPEZ_OPT_LORENZO_CTAS  0 (default: the resident CTAs); n > 0: at most n
 *                         persistent CTAs for the Lorenzo kernels, so each
 *                         streams more blocks back to back
 *  HPEZ_OPT_BATCH_CTAS    0 (default: the resident CTAs); n > 0: at most n
 *                         CTAs for each persistent level launch of the
 *                         batched and served forms, so each CTA walks more
 *                         tiles of the concatenated work list
 * Errors: INVALID_ARG for an unknown option or an out-of-range value. */
#define HPEZ_OPT_FUSED_LEVELS 1
#define HPEZ_OPT_TILE_E0 2
#define HPEZ_OPT_TILE_E1 3
#define HPEZ_OPT_TILE_E2 4
#define HPEZ_OPT_FUSED_SMEM 5
#define HPEZ_OPT_LEVEL3D 6
#define HPEZ_OPT_STREAM_LEVELS 7
#define HPEZ_OPT_DROP_COPY 8
#define HPEZ_OPT_STREAM_CHUNKS 9
#define HPEZ_OPT_LORENZO_CTAS 10
#define HPEZ_OPT_WARP_LEVELS 11
#define HPEZ_OPT_BATCH_CTAS 12
HPEZ_API int hpez_set_option(hpez_ctx* ctx, int option, int64_t value);

/* ---- measurement hooks (not part of the paper's method) ----
 * Phase timing: with profiling enabled, compress/decompress record a CUDA
 * event pair on the call's stream around each phase and accumulate the
 * elapsed times once the call has synchronized.  Phase ids: */
#define HPEZ_PH_RANGE 0     /* value range (relative bound) */
#define HPEZ_PH_ANCHORS 1   /* anchor gather */
#define HPEZ_PH_HIST 2      /* code histogram + outlier counts */
#define HPEZ_PH_CODEBOOK 3  /* canonical Huffman codebook */
#define HPEZ_PH_ENCODE 4    /* chunk lengths + offsets */
#define HPEZ_PH_PACK 5      /* bit packing */
#define HPEZ_PH_OUTLIERS 6  /* outlier gather */
#define HPEZ_PH_FINALIZE 7  /* header + static sections */
#define HPEZ_PH_DEC_PREP 8  /* chunk offsets + decode tables */
#define HPEZ_PH_DECODE 9    /* Huffman decode */
#define HPEZ_PH_SCATTER 10  /* outlier scatter */
#define HPEZ_PH_LEVEL 11    /* + (l-1): compress level l, l = 1..16 */
#define HPEZ_PH_DLEVEL 27   /* + (l-1): decompress level l */
#define HPEZ_PH_TUNE_STATS 43    /* tuner: Sec. 6.1 statistics */
#define HPEZ_PH_TUNE_LEVELS 44   /* tuner: Sec. 6.2 candidate tests */
#define HPEZ_PH_TUNE_EB 45       /* tuner: Sec. 6.4 (alpha, beta) tests */
#define HPEZ_PH_TUNE_LORENZO 46  /* tuner: Sec. 6.5 Lorenzo tests */
#define HPEZ_PH_TUNE_BLOCKS 47   /* tuner: Sec. 6.6 block-wise tests */
#define HPEZ_PROFILE_PHASES 48

/* Enable (1) or disable (0) phase timing; resets the accumulators and the
 * launch counter.  Errors: INVALID_ARG. */
HPEZ_API int hpez_profile_enable(hpez_ctx* ctx, int enable);
/* Accumulated milliseconds and number of timed occurrences of a phase. */
HPEZ_API int hpez_profile_get(hpez_ctx* ctx, int phase, double* total_ms,
                              uint64_t* count);
/* Static name of a phase id ("" if out of range). */
HPEZ_API const char* hpez_profile_phase_name(int phase);
/* Number of kernels this context launched since creation or the last
 * hpez_profile_enable call. */
HPEZ_API int hpez_launch_count(hpez_ctx* ctx, uint64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* HPEZ_H */
