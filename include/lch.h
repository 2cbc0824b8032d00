/*
 * lch.h - C ABI of the GB300 library for the transform in the Lin-Chung-Han
 * polynomial basis over GF(2^r) and the Reed-Solomon erasure code built on it
 * (S.-J. Lin, W.-H. Chung, Y. S. Han, "Novel Polynomial Basis and Its
 * Application to Reed-Solomon Erasure Codes").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Field.     `field` is LCH_GF8 (r = 8, reduction polynomial
 *            x^8+x^4+x^3+x^2+1) or LCH_GF16 (r = 16, x^16+x^12+x^3+x+1).
 *            The paper's basis v_0..v_{r-1} (Sec. II.A) is taken to be the
 *            polynomial basis v_j = x^j, so the point w_i is the field element
 *            whose bit pattern is i and w_a + w_b = w_{a xor b}.
 * Symbols.   A symbol is one shard: a row of `shard_bytes` bytes.  Each
 *            element offset inside the shards is an independent column that
 *            is transformed with the same factors.  GF(2^8) elements are
 *            bytes; GF(2^16) elements are little-endian uint16 (bit b is the
 *            coefficient of x^b).
 * Buffers.   Every data pointer is a DEVICE pointer to `rows x shard_bytes`
 *            bytes, row-major (row t starts at buf + t * shard_bytes), owned
 *            by the caller, 16-byte aligned.  `shard_bytes` must be a nonzero
 *            multiple of 16.
 * Streams.   `stream` is a cudaStream_t (NULL = the legacy default stream).
 *            Every call only enqueues work on it and returns; results are
 *            ready when the stream reaches that point.  The first call that
 *            uses a field on a context builds that field's tables and
 *            synchronises `stream` once.
 * Errors.    Arguments are checked on the host before anything is enqueued;
 *            a call that returns an error has modified no buffer.  Status 0 is
 *            success; see lch_strerror() and lch_last_error() for the rest.
 * Threads.   A context may be used from one host thread at a time.  Calls on
 *            one context that run concurrently on different streams race on
 *            the context's scratch memory; serialise them on one stream.
 */
#ifndef LCH_H
#define LCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LCH_API __attribute__((visibility("default")))
#else
#define LCH_API
#endif

/* Status codes. */
#define LCH_OK 0
#define LCH_EINVAL 1   /* an argument is out of range or misaligned */
#define LCH_ETOOMANY 2 /* rs_decode: more than n - k erasures */
#define LCH_ENOMEM 3   /* device or host allocation failed */
#define LCH_ECUDA 4    /* a CUDA runtime call failed (see lch_last_error) */
#define LCH_ETIMEDOUT 5 /* a batch task gave up waiting for its predecessors */

/* Fields. */
#define LCH_GF8 8
#define LCH_GF16 16

typedef struct lch_ctx lch_ctx;

/* Create a context bound to CUDA device `device`.  The context owns the
 * per-field tables (built lazily) and a scratch area that grows on demand.
 * On success *ctx receives the handle and LCH_OK is returned. */
LCH_API int lch_ctx_create(lch_ctx **ctx, int device);

/* Release a context and everything it owns.  Waits for the device first.
 * NULL is ignored. */
LCH_API void lch_ctx_destroy(lch_ctx *ctx);

/* Forward transform Psi_h^l (Sec. III, the set Psi(0,0,l) of Sec. III.C).
 * buf holds h rows: on entry row i is coefficient d_i of
 * [D_h](x) = sum_i d_i X_i(x) (Def. 1); on return row c is [D_h](w_c + w_l).
 * h: power of two, 1 <= h <= 2^r.  l: shift, 0 <= l < 2^r (any value; the
 * encoder uses multiples of h).  In place. */
LCH_API int lch_fft(lch_ctx *ctx, int field, uint32_t h, uint32_t l, void *buf, size_t shard_bytes,
                    void *stream);

/* Inverse transform (Psi_h^l)^{-1} (Sec. III.E): on entry row c holds the
 * value at w_c + w_l, on return row i holds d_i.  Same arguments as
 * lch_fft.  In place. */
LCH_API int lch_ifft(lch_ctx *ctx, int field, uint32_t h, uint32_t l, void *buf, size_t shard_bytes,
                     void *stream);

/* Formal derivative in the basis (Sec. IV, eqs. D'_h(x)-2 and XDhx3): on
 * entry buf holds the h coefficients of [D_h], on return the h coefficients
 * of [D_h]' (the last one is always zero).  h: power of two, 1 <= h <= 2^r.
 * In place; uses context scratch of h * shard_bytes bytes. */
LCH_API int lch_derivative(lch_ctx *ctx, int field, uint32_t h, void *buf, size_t shard_bytes,
                           void *stream);

/* lch_derivative without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * (a host application whose allocator owns the whole device heap, a plugin
 * that its host forbids to allocate, or a latency-critical loop that cannot
 * afford the implicit synchronisation of cudaMalloc/cudaFree).  It computes the
 * same result as lch_derivative but takes no context: its scratch (at most
 * 16 MiB, so h * shard_bytes <= 16777216 for h >= 2, else LCH_EINVAL; h = 1
 * only zeroes the row and has no size limit) and its B tables
 * are file-scope device arrays that every GPU loading the library keeps until
 * the process exits.  It runs on the current CUDA device.  The first call on a
 * device sets those arrays up and synchronises `stream` once; make that first
 * call before any stream capture.  All calls on a device share the scratch
 * (which keeps the last call's contents); calls that overlap on the GPU race.
 * Argument rules, layout and errors are otherwise those of lch_derivative. */
LCH_API int lch_derivative_noalloc(int field, uint32_t h, void *buf, size_t shard_bytes, void *stream);

/* Product of two polynomials in the basis (Sec. VI.A): with a and b holding
 * the h coefficients of [A_h] and [B_h] (h rows each), c (2h rows) receives
 * the 2h coefficients of [A_h](x) [B_h](x), computed as
 * (Psi_2h^0)^-1 [Psi_2h^0[A_2h] * Psi_2h^0[B_2h]] with A_2h, B_2h the inputs
 * padded with h zero rows.  h: power of two, 1 <= h <= 2^(r-1).  a, b and c
 * must not overlap.  Uses context scratch of 2 h shard_bytes bytes. */
LCH_API int lch_poly_mul(lch_ctx *ctx, int field, uint32_t h, const void *a, const void *b, void *c,
                         size_t shard_bytes, void *stream);

/* Systematic (n, k) Reed-Solomon encoding (Sec. V, Algorithm 1).
 * shards holds n rows; rows 0..k-1 are the message m_0..m_{k-1} and are only
 * read; rows k..n-1 are overwritten with F(w_k)..F(w_{n-1}), where F is the
 * polynomial of degree < k with F(w_i) = m_i (eq. F(i)=m_i).
 * n: power of two, 1 <= n <= 2^r.  1 <= k <= n.  When k is a power of two
 * Algorithm 1 runs as printed; otherwise the parity rows are recovered as
 * erasures of a codeword whose message rows are known (Algorithm 2 with
 * E = {k..n-1}), which yields the same unique F.  Uses context scratch of
 * up to 2 n shard_bytes bytes. */
LCH_API int rs_encode(lch_ctx *ctx, uint32_t n, uint32_t k, int field, void *shards, size_t shard_bytes,
                      void *stream);

/* Erasure decoding (Sec. V, Algorithm 2, with the Appendix locator).
 * shards holds the n rows of a received codeword.  erasure_mask is a HOST
 * array of n bytes; a nonzero byte marks that row as erased.  Surviving rows
 * are only read; each erased row j is overwritten with F(w_j).  With no
 * erasures the call returns LCH_OK and does nothing; with more than n - k it
 * returns LCH_ETOOMANY.  Rows that are not consistent with any codeword give
 * a deterministic but meaningless result (erasure-only code).  Same n, k
 * rules as rs_encode.  Uses context scratch of about 2 n shard_bytes bytes.
 * The mask is copied before the call returns. */
LCH_API int rs_decode(lch_ctx *ctx, uint32_t n, uint32_t k, int field, void *shards, size_t shard_bytes,
                      const uint8_t *erasure_mask, void *stream);

/* Erasure decoding from the received shards alone (Algorithm 2, as
 * rs_decode), without assembling the codeword: `received` (device) holds the
 * n - |E| surviving shards packed in increasing row order, and `recovered`
 * (device, |E| shard_bytes bytes) receives the erased shards packed in
 * increasing row order.  erasure_mask as in rs_decode; both pointers must be
 * 16-byte aligned.  With no erasures the call returns LCH_OK and touches
 * nothing; with more than n - k it returns LCH_ETOOMANY.  The received
 * shards are only read.  Uses context scratch of about 2 n shard_bytes
 * bytes. */
LCH_API int rs_decode_packed(lch_ctx *ctx, uint32_t n, uint32_t k, int field, const void *received,
                             void *recovered, size_t shard_bytes, const uint8_t *erasure_mask, void *stream);

/* ---- Batches: many independent codewords in one persistent launch -------
 * (Beyond the paper, which treats one codeword at a time: every stage of
 * Algorithms 1 and 2 is the same per codeword, so the stages of thousands of
 * codewords of different (n, k, field, shard size) are run as one queue of
 * tasks by a single persistent kernel.)
 *
 * A codeword: `shards` is a DEVICE pointer to n rows of shard_bytes (layout
 * and rules as for rs_encode/rs_decode, n <= 8192); `erasure_mask` is a HOST
 * array of n bytes (nonzero = erased) for decoding, ignored for encoding. */
typedef struct lch_codeword {
    uint32_t n;
    uint32_t k;
    int field;
    uint32_t reserved; /* must be 0 */
    size_t shard_bytes;
    void *shards;
    const uint8_t *erasure_mask;
} lch_codeword;

#define LCH_BATCH_ENCODE 0
#define LCH_BATCH_DECODE 1

typedef struct lch_batch lch_batch;

/* Plan a batch: validates every codeword (the first invalid one fails the
 * call with its index in lch_last_error), copies the erasure masks, builds the
 * task queue and allocates the batch's device memory (queue, counters and the
 * per-codeword scratch, about 2 n shard_bytes per decoded codeword and
 * k shard_bytes per encoded one).  The plan is tied to these buffers: running
 * it again recomputes the same codewords from the buffers' current contents.
 * Synchronises the device once.  Decoding a codeword without erasures is a
 * no-op; more than n - k erasures fail with LCH_ETOOMANY. */
LCH_API int lch_batch_create(lch_ctx *ctx, int op, const lch_codeword *cws, uint32_t count, lch_batch **out);

/* Device bytes (scratch, erasure bitmaps, task queue, counters) that
 * lch_batch_create_in needs for these codewords.  Host-only; validates like
 * lch_batch_create. */
LCH_API int lch_batch_bytes(lch_ctx *ctx, int op, const lch_codeword *cws, uint32_t count, size_t *bytes);

/* lch_batch_create without allocation: every device byte of the batch is
 * placed in the caller's block [mem, mem + bytes) (256-byte aligned, at least
 * lch_batch_bytes), and the plan is uploaded on `stream` without a device-wide
 * synchronisation, so a server can plan a new batch from a memory arena while
 * earlier batches still run.  The caller keeps the block, the shard buffers
 * and the batch alive until the batch's runs have completed on the device.
 * The first batch that uses a field or an n on the context still builds that
 * field's tables (allocating and synchronising once). */
LCH_API int lch_batch_create_in(lch_ctx *ctx, int op, const lch_codeword *cws, uint32_t count, void *mem,
                                size_t bytes, void *stream, lch_batch **out);

/* Enqueue one run of the batch on `stream`: a counter reset and one launch
 * of the persistent kernel.  Allocates nothing and does not synchronise, so
 * it can be recorded into a CUDA graph and replayed. */
LCH_API int lch_batch_run(lch_ctx *ctx, lch_batch *batch, void *stream);

/* Wait for the stream of the batch's last run and report whether that run
 * completed: LCH_OK, or LCH_ETIMEDOUT if a task gave up waiting for its
 * predecessors (the kernel then drains without finishing; the outputs are
 * undefined; the context and the batch stay usable). */
LCH_API int lch_batch_status(lch_ctx *ctx, lch_batch *batch);

/* How long one task of a batch run may wait for the tasks it depends on
 * before the run gives up (default 2 s; applies to runs enqueued later).
 * Every wait of the persistent kernel polls a completion counter and stops at
 * this limit, so a run never spins forever.  LCH_EINVAL for 0. */
LCH_API int lch_batch_set_wait_limit(lch_ctx *ctx, uint32_t wait_us);

/* Failure-path self-test (the paper has no counterpart): runs the batch
 * kernel on a one-task plan whose dependency is never met, so its wait must
 * give up after the context's wait limit.  Synchronises `stream`.  Returns
 * LCH_ETIMEDOUT when the wait gave up as designed (the expected result),
 * LCH_OK never, LCH_ENOMEM or LCH_ECUDA on other failures. */
LCH_API int lch_batch_selftest_stall(lch_ctx *ctx, void *stream);

/* Number of tasks in the plan (diagnostics). */
LCH_API uint32_t lch_batch_tasks(const lch_batch *batch);

LCH_API void lch_batch_destroy(lch_batch *batch);

/* ---- Row packing (the paper has no counterpart) ----------------------------
 * Utilities for callers that hold only some rows of a codeword, e.g. the
 * surviving shards before rs_decode or the recovered ones after it: they move
 * whole rows between a codeword buffer and a packed buffer of consecutive
 * rows.  idx is a DEVICE array of `count` uint32 row indices; src and dst are
 * device buffers of shard_bytes-byte rows (16-byte aligned, shard_bytes a
 * nonzero multiple of 16).  Indices are not checked against the buffers; they
 * must be in range, and for a scatter distinct.  Enqueued on `stream`; count 0
 * is a no-op.  No context needed.
 *   gather:  dst row i      = src row idx[i]
 *   scatter: dst row idx[i] = src row i */
LCH_API int lch_rows_gather(const void *src, void *dst, const uint32_t *idx, uint32_t count, size_t shard_bytes,
                            void *stream);
LCH_API int lch_rows_scatter(const void *src, void *dst, const uint32_t *idx, uint32_t count, size_t shard_bytes,
                             void *stream);

/* Static text for a status code. */
LCH_API const char *lch_strerror(int status);

/* Text of the last error raised on the calling host thread (never NULL). */
LCH_API const char *lch_last_error(void);

/* Number of kernels this context has launched so far (diagnostics). */
LCH_API uint64_t lch_launch_count(const lch_ctx *ctx);

/* Kernel kinds for the profiling counters. */
#define LCH_KIND_PASS 0     /* transform butterfly pass (Sec. III.C / III.E) */
#define LCH_KIND_DERIV 1    /* derivative neighbour sums (Sec. IV.B) */
#define LCH_KIND_ROWSCALE 2 /* per-row scaling: Phi, B, B^-1, final divide */
#define LCH_KIND_LOCATOR 3  /* FWHT locator (Appendix) */
#define LCH_KIND_COUNT 4

/* Diagnostics.  With profiling on, every kernel launch is bracketed by CUDA
 * events recorded on its own stream; lch_profile_read() returns, per kind,
 * the number of launches, their summed device time in milliseconds, the
 * algorithmic bytes they moved (each launch counts the rows it must read and
 * write once: 2 x rows x shard_bytes, plus rows x shard_bytes when it also
 * reads its output) and the algorithmic field multiplications they performed
 * (a transform pass over levels [L0, L0+q) of an h-point transform counts
 * (h/2) q per column, Sec. III.D; a row scaling counts one per element).
 * Enabling (or re-enabling) clears the counters.  Reading synchronises on the
 * recorded events. */
LCH_API int lch_profile_enable(lch_ctx *ctx, int on);
LCH_API int lch_profile_read(lch_ctx *ctx, int kind, uint64_t *launches, double *total_ms, uint64_t *bytes,
                             uint64_t *mults);

/* ---- Autotuning of the transform passes (the paper has no counterpart) ---
 * An h-point transform runs its lg h butterfly levels (Sec. III.C/E) in one
 * pass (lg h <= 8) or two: the low pass takes levels [0, split), the high pass
 * levels [split, lg h); each pass walks the shards in column tiles of
 * 2^lg_tile bytes.  The result never depends on the plan, only the speed.
 * A plan holds for one (field, h, shard_bytes) on the context that tuned or
 * received it and is used by lch_fft, lch_ifft, rs_encode, rs_decode,
 * lch_poly_mul and batches planned afterwards (lch_derivative keeps its own
 * passes). */
typedef struct lch_tuning {
    uint32_t split;        /* levels of the low pass; lg h when there is one pass */
    uint32_t lg_tile_low;  /* log2 column-tile bytes of the low pass, 4..12 */
    uint32_t lg_tile_high; /* ... of the high pass; 0 when there is one pass */
    float ms;              /* lch_autotune: device ms of one Psi plus one Psi^-1 */
} lch_tuning;

/* Time candidate plans for (field, h, shard_bytes) on `stream` and keep the
 * fastest on the context; *best receives it.  Candidates: the splits with
 * both passes <= 8 levels among {ceil(lg h/2), floor(lg h/2), lg h-8, 8}, and
 * for each pass the default tile width, one narrower and two wider ones that
 * fit in shared memory.  Each pass is timed with CUDA events, forward and inverse,
 * after one warm-up, on h * shard_bytes bytes of context scratch filled with a
 * fixed pattern (grown by cudaMalloc if needed; no caller data is touched).
 * Synchronises `stream`.  Errors: LCH_EINVAL (bad field, h not a power of two
 * in [2, 2^field], shard_bytes zero or not a multiple of 16, NULL pointer),
 * LCH_ENOMEM, LCH_ECUDA. */
LCH_API int lch_autotune(lch_ctx *ctx, int field, uint32_t h, size_t shard_bytes, void *stream, lch_tuning *best);

/* Install a plan for (field, h, shard_bytes), e.g. one read from a cache of
 * earlier lch_autotune results; plan NULL removes it (defaults again).  The
 * plan is checked (split, both passes <= 8 levels, widths in 4..12 and within
 * shared memory for these sizes); LCH_EINVAL if it is not valid, nothing
 * changed.  Not synchronised with work in flight: set plans before the calls
 * that should use them. */
LCH_API int lch_tune_set(lch_ctx *ctx, int field, uint32_t h, size_t shard_bytes, const lch_tuning *plan);

/* The plan installed on ctx for (field, h, shard_bytes) (ms is set to 0),
 * e.g. to give other contexts the same plans; LCH_EINVAL when there is none. */
LCH_API int lch_tune_get(lch_ctx *ctx, int field, uint32_t h, size_t shard_bytes, lch_tuning *plan);

/* Arithmetic of the GF(2^16) transform passes (the paper has no counterpart;
 * results are identical either way).  on == 0 (the default): every transform
 * uses the split-table passes and the plans above.  on != 0: when
 * shard_bytes is a multiple of 64, lch_fft, lch_ifft, lch_poly_mul and the
 * transforms inside rs_encode / rs_decode run as bit-sliced passes: each
 * 64-byte chunk of 32 elements is turned into 16 plane words, a product by a
 * butterfly factor becomes plane XORs selected by the factor's bits, and the
 * chunks are turned back when the transform's last pass stores them; the
 * tuned plans do not apply to those transforms.  On a GB300 the bit-sliced
 * passes are the slower of the two (about 1.3 against 1.9 T multiplies/s),
 * which is why they are not the default.  Codewords whose whole decode or
 * encode fits one tile (lg n <= 8, lg k <= 8), batches and GF(2^8) are not
 * affected.  Not synchronised with work in flight.  LCH_EINVAL for a NULL
 * ctx. */
LCH_API int lch_set_bitslice(lch_ctx *ctx, int on);

#ifdef __cplusplus
}
#endif

#endif /* LCH_H */
