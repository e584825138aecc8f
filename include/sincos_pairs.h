/*
 * sincos_pairs.h -- C ABI of the GB300 (sm_103a) sine-cosine pair library.
 *
 * The library computes single-precision sine-cosine pairs with the
 * branch-free method of M. H. Mendenhall, "A Fast, Vectorizable Algorithm
 * for Producing Single-Precision Sine-Cosine Pairs" (cs/0406049):
 *   - the angle is scaled by 1/(2 pi) and reduced onto [-1/2, 1/2] by
 *     rounding to nearest (ties to even) and subtracting (Sec. Methodology);
 *   - power series in the reduced value give the sine and cosine of the
 *     quarter angle (Sec. Methodology, the printed coefficient sets);
 *   - two double-angle steps of Eq. (1), s' = 2 s c and c' = c^2 - s^2,
 *     expand the pair to the full circle;
 *   - the amplitude drift is corrected by a factor computed from the
 *     half-angle pair (Sec. Methodology; Fig. 1).
 * Everything runs in hand-written CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   Memory     All array arguments are caller-owned.  Unless an entry point
 *              says otherwise they are device memory of the current CUDA
 *              device (cudaMalloc, or managed memory prefetched to that
 *              device: the bulk kernels move data with the copy engine of
 *              the SM, which is not used on pages that would first have to
 *              migrate).  Host arrays go to sincos_pairs_host.  No entry
 *              point allocates per call, except where stated (batched
 *              scratch, host-path streams).
 *   Layout     Structure of arrays: one contiguous array of angles in, one of
 *              sines and one of cosines out (the paper's `struct phase` holds
 *              the two vectors separately).  Element i of every array belongs
 *              to angle i.  Any 4-byte-aligned float pointer (2-byte for
 *              16-bit outputs) is accepted; the kernels peel to 16-byte
 *              alignment themselves.
 *   Streams    Every call is asynchronous and ordered on `stream` (NULL is the
 *              legacy default stream).  SINCOS_OK means "enqueued"; results
 *              are valid once the stream has reached that point.
 *   Errors     Invalid arguments are rejected on the host before anything is
 *              enqueued: SINCOS_EINVAL (null pointer with n > 0, a pointer
 *              not aligned to its element type, n < 0, bad enum),
 *              SINCOS_EOVERLAP (outputs overlap each other, or the
 *              input partially overlaps an output).  A failed CUDA call gives
 *              SINCOS_ECUDA and its text is kept for sincos_last_error().
 *              n == 0 (or count == 0) returns SINCOS_OK and enqueues nothing.
 *   Threads    Calls on different streams may run concurrently from any
 *              number of host threads.
 *   Device     All calls act on the calling thread's current CUDA device.
 */
#ifndef SINCOS_PAIRS_H
#define SINCOS_PAIRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared here so the header needs no CUDA headers. */
struct CUstream_st;
typedef struct CUstream_st *sincos_stream_t;

typedef enum {
    SINCOS_OK = 0,
    SINCOS_EINVAL = -1,       /* bad argument (null pointer, negative size, bad enum) */
    SINCOS_EOVERLAP = -2,     /* forbidden overlap between input and output arrays     */
    SINCOS_ECUDA = -3,        /* a CUDA runtime call failed; see sincos_last_error()  */
    SINCOS_EUNSUPPORTED = -4, /* the device is not an sm_103 GPU, or a size limit hit  */
    SINCOS_ECAPTURE = -5      /* the call would allocate or do first-use set-up while
                                 its stream is being captured                        */
} sincos_status;

/* Output element type.  BF16 and F16 results are the binary32 result rounded
 * to nearest, ties to even. */
typedef enum { SINCOS_F32 = 0, SINCOS_BF16 = 1, SINCOS_F16 = 2 } sincos_dtype;

/* Range reduction.
 * PLAIN        -- the paper's: x1 = fl(x * K), K = fl(1/(2*3.1415926536)),
 *                 q = x1 - rint(x1) (Sec. Methodology; Fig. 1).  The rounding
 *                 of x*K costs about 2 pi |x1| 2^-24 of angle for large |x|.
 * COMPENSATED  -- not in the paper: 1/(2 pi) split as Khi + Klo,
 *                 r = rint(fl(x*Khi)); q = fma(x, Khi, -r); q = fma(x, Klo, q);
 *                 q -= rint(q).  Within 7e-7 of FP64 for |x| <= 1e5. */
typedef enum { SINCOS_RED_PLAIN = 0, SINCOS_RED_COMPENSATED = 1 } sincos_reduction;

/* Series coefficients.
 * NORMALIZED -- the first method's least-squares sine/cosine series with the
 *               2 - s^2 - c^2 drift factor (Sec. Methodology, first method).
 * DAGGER     -- the second method's un-normalized series (fit to the angle)
 *               with the exact reciprocal 1/(s^2 + c^2) (Sec. Methodology,
 *               second method). */
typedef enum { SINCOS_COEF_NORMALIZED = 0, SINCOS_COEF_DAGGER = 1 } sincos_coef;

/* ------------------------------------------------------------------------ */
/* Forward                                                                   */
/* ------------------------------------------------------------------------ */

/* s[i], c[i] = sin(x[i]), cos(x[i]) for 0 <= i < n: binary32 in, binary32
 * out, plain reduction, normalized coefficients -- the method exactly as the
 * paper gives it (Sec. Methodology; Fig. 1).
 *   x  device, n floats, read only.  May be the same pointer as s or c (in
 *      place); any other overlap with s or c is SINCOS_EOVERLAP.
 *   s  device, n floats, written.  c  device, n floats, written.
 *      s and c must not overlap.
 * NaN or +-Inf angles give NaN; |fl(x*K)| >= 2^23 gives (0, 1). */
int sincos_pairs(const float *x, float *s, float *c, int64_t n, sincos_stream_t stream);

/* General forward: output dtype, reduction and coefficient set chosen by the
 * caller (Sec. Methodology; first and second methods).  s and c point to n
 * elements of `out_dtype` (4 or 2 bytes each).  In-place (x == s or x == c)
 * is allowed only for SINCOS_F32. */
int sincos_pairs_ex(const float *x, void *s, void *c, int64_t n, int out_dtype,
                    int reduction, int coef, sincos_stream_t stream);

/* exp(i x) = cos x + i sin x for 0 <= i < n as interleaved complex64:
 * z[2i] = c_i, z[2i+1] = s_i, the same pairs as sincos_pairs_ex with
 * SINCOS_F32 output (Sec. Methodology; the pair of the paper's struct
 * phase, written as one complex stream for FFT and phase-factor consumers).
 *   x  device, n floats, read only.
 *   z  device, 2n floats, written; must not overlap x.  Any 4-byte
 *      alignment works; the vector paths need z + 2h and x + h to share a
 *      16-byte grid for some small h (always true for complex64 storage and
 *      16-byte aligned x).
 * Uses the SINCOS_OP_EXPI launch plan (bulk or register path). */
int sincos_expi(const float *x, float *z, int64_t n, int reduction, int coef,
                sincos_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Fused consumer: Huygens-principle field sum                               */
/* ------------------------------------------------------------------------ */

/* The application the paper names (Sec. Conclusions: optical diffraction by
 * Huygens' principle), with every phase factor made by the method in
 * registers and never stored:
 *   u_i = sum_{j<n} a_j exp(i k r_ij) / r_ij,  r_ij = |p_i - q_j|,
 * in binary32 with this operation order per term:
 *   d = p_i - q_j;  r = sqrt(fma(dz, dz, fma(dy, dy, dx*dx)));  w = 1/r;
 *   (s, c) = the method's pair of k*r (normalized set, given reduction);
 *   u_re = fma(w, fma(ar_j, c, -(ai_j*s)), u_re);
 *   u_im = fma(w, fma(ar_j, s, ai_j*c), u_im);
 * and the terms of each point summed in source order j = 0, 1, ... from 0,
 * so the result is independent of the launch configuration.
 *   px, py, pz  device, m floats each: observation points.
 *   qx, qy, qz  device, n floats each: source points.
 *   ar, ai      device, n floats each: complex source amplitudes.
 *   k           wavenumber (2 pi / wavelength) in the coordinates' units.
 *   reduction   SINCOS_RED_COMPENSATED recommended: phases k*r are large.
 *   u           device, 2m floats, written as interleaved complex64; must not
 *               overlap any input.
 * A point that coincides with a source gives an infinite or NaN sum.
 * n == 0 writes zeros.  Plan: SINCOS_OP_HUYGENS (SINCOS_F32). */
int sincos_huygens(const float *px, const float *py, const float *pz, int64_t m,
                   const float *qx, const float *qy, const float *qz, const float *ar,
                   const float *ai, int64_t n, float k, int reduction, float *u,
                   sincos_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Backward                                                                  */
/* ------------------------------------------------------------------------ */

/* Gradient of L = sum(gs*sin(x) + gc*cos(x)) with respect to x, evaluated on
 * the forward's outputs: gx[i] = fma(gs[i], c[i], -(gc[i]*s[i])).  The method
 * has no seams inside (-pi, pi) (Sec. Methodology), so the analytic
 * derivative of the pair is the pair itself.
 *   gs, gc  device, n floats, read only; either may be NULL for an all-zero
 *           upstream gradient (gs == NULL: gx = -(gc*s); gc == NULL:
 *           gx = gs*c; both NULL: gx = +0).
 *   s, c    device, n floats: the forward's binary32 outputs, read only.
 *   gx      device, n floats, written; may be the same pointer as one of the
 *           inputs, no other overlap allowed. */
int sincos_backward(const float *gs, const float *gc, const float *s, const float *c,
                    float *gx, int64_t n, sincos_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batched: many arrays of uneven length in one persistent launch            */
/* ------------------------------------------------------------------------ */

/* One array of the batch: x has lens[i] floats; s and c have lens[i]
 * elements of the batch's output dtype.  All three are device pointers,
 * each aligned to its element type (4 bytes for x and binary32 outputs, 2
 * for 16-bit outputs).  The descriptors live on the device and are checked
 * there, by the kernels, before any array is touched: an array with
 * lens[i] > 0 and a null or misaligned x, s or c is skipped (its outputs are
 * not written) and counted, see sincos_device_bad_segments(); the same check
 * is available on the host as sincos_seg_check().  What no check can see is
 * whether a non-null, aligned pointer addresses lens[i] valid elements of
 * this device's memory; that remains the caller's responsibility. */
typedef struct {
    const float *x;
    void *s;
    void *c;
} sincos_seg;

/* The check the batched kernels apply to one descriptor, on the host: OK
 * when len <= 0, or when x, s and c are non-null, x is 4-byte aligned and s
 * and c are aligned to out_dtype's size; SINCOS_EINVAL otherwise (also for a
 * null seg or a bad dtype).  seg is a host pointer.  No paper counterpart. */
int sincos_seg_check(const sincos_seg *seg, int64_t len, int out_dtype);

/* The forward over `count` independent arrays: the method of Sec.
 * Methodology and Fig. 1 applied to each array (batching itself is not in
 * the paper).  Same per-element arithmetic as sincos_pairs_ex.  With the
 * default plan for binary32 outputs this is one persistent launch.  Each CTA
 * derives its own contiguous run of the concatenated element space from the
 * lengths (equal work per CTA to within one 8192-angle tile), then streams it
 * through a TMA-staged ring (4096-angle stages, two CTAs per SM, by default).
 * With a register plan (the default for 16-bit outputs) it is two launches: a
 * small schedule kernel over the lengths into the scratch below, then the
 * tile kernel.
 *   segs  device array of `count` descriptors, read by the kernels.
 *   lens  device array of `count` int64 lengths; a negative length counts
 *         as 0.  Both arrays are read when the kernels run, so they may be
 *         filled by earlier work on the same stream.
 * No output may overlap another segment's output or any segment's angles
 * (not checked: the descriptors live on the device).
 * Scratch (used by register plans): the library keeps one small device
 * buffer (count + 8195 int64) per (device, stream) pair, allocated with
 * cudaMalloc on the first call that needs a larger one.  A call that would
 * allocate while `stream` is being captured returns SINCOS_ECAPTURE; make one
 * uncaptured call first.
 * sincos_batched_release() frees all such buffers (call it only when no
 * batched work is in flight). */
int sincos_batched(const sincos_seg *segs, const int64_t *lens, int count,
                   sincos_stream_t stream);
int sincos_batched_ex(const sincos_seg *segs, const int64_t *lens, int count, int out_dtype,
                      int reduction, int coef, sincos_stream_t stream);
int sincos_batched_release(void);

/* The same batched forward for callers that cannot allocate device memory
 * (the paper has no counterpart; this is a deployment variant).  A plug-in
 * inside a host program that owns all device memory, a real-time thread that
 * must not risk the device-wide synchronization cudaMalloc/cudaFree can
 * trigger, or code under an allocation budget fixed at start-up cannot let
 * the library call cudaMalloc for scratch, as sincos_batched does on first
 * use.  This entry point allocates nothing: its schedule scratch (the
 * tile prefix of up to SINCOS_NOALLOC_MAX_SEGMENTS arrays and the start of
 * each CTA) is a fixed device array of SINCOS_NOALLOC_MAX_SEGMENTS + 8195
 * int64 (about 576 KiB) built into the library, present on every GPU that
 * loads it until the process exits.
 *   Arguments, layout, results and errors are those of sincos_batched_ex;
 *   count > SINCOS_NOALLOC_MAX_SEGMENTS returns SINCOS_EUNSUPPORTED before
 *   anything is enqueued.
 *   Only register plans (vec_bytes 16 or 32: the default for 16-bit outputs,
 *   or a plan set or tuned for binary32) use the array.  Bulk plans
 *   (vec_bytes 0, the binary32 default) run the ring kernel, which schedules
 *   itself and touches no scratch; sincos_batched_ex allocates nothing for
 *   them either.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current, which may load the
 *   library's device code onto the GPU; make that first call before
 *   capturing any stream into a graph.  A first call on a stream that is
 *   being captured returns SINCOS_ECAPTURE and enqueues nothing.
 *   All calls share the one array: calls under register plans whose work can
 *   overlap on the GPU (different streams without ordering between them)
 *   race and give wrong results.  Order them on one stream, or use
 *   sincos_batched instead.
 *   Each call rewrites every scratch entry it reads, so the contents left by
 *   an earlier call do not matter. */
#define SINCOS_NOALLOC_MAX_SEGMENTS 65536
int sincos_batched_noalloc(const sincos_seg *segs, const int64_t *lens, int count,
                           int out_dtype, int reduction, int coef, sincos_stream_t stream);

/* A batched launch captured once into a CUDA graph and replayed (launch
 * infrastructure around the batched form of Sec. Methodology / Fig. 1; no
 * paper counterpart).  The graph owns its scratch, if its plan needs one;
 * the segs/lens device arrays are read at every replay, so their contents
 * (not their addresses) may change between replays.  A replay launches the
 * kernels the graph holds (one for a ring plan, two for a register plan), and
 * sincos_launch_count() counts them at each replay, not at creation. */
typedef struct sincos_graph_s *sincos_graph;
int sincos_batched_graph_create(const sincos_seg *segs, const int64_t *lens, int count,
                                int out_dtype, int reduction, int coef, sincos_graph *out);
int sincos_batched_graph_launch(sincos_graph g, sincos_stream_t stream);
int sincos_batched_graph_destroy(sincos_graph g);

/* ------------------------------------------------------------------------ */
/* Host buffers: chunked, pipelined host -> device -> host                   */
/* ------------------------------------------------------------------------ */

/* The forward (Sec. Methodology, Fig. 1) on host arrays; the data movement
 * has no paper counterpart.  x_host holds n floats; s_host and c_host hold n
 * elements of out_dtype.
 *   If the device can reach all three buffers, one kernel reads x and writes
 *   s and c across the host link itself (zero-copy), and dev_ws is not used.
 *   It can reach page-locked buffers mapped into its address space
 *   (cudaHostAlloc, cudaMallocHost, cudaHostRegister with mapping), and, on a
 *   device that accesses pageable memory through the host's page tables
 *   (cudaDevAttrPageableMemoryAccess, as GB300 with Grace), ordinary pageable
 *   memory too.  Pageable pages that nothing has touched yet are populated
 *   by the system on the kernel's first access, which makes that first call
 *   slow (about 0.65 s for 2 GiB of fresh outputs on GB300; 12.4 ms per
 *   2^28-angle call afterwards, the same as page-locked buffers).  x may be
 *   s or c exactly (binary32 output); any other overlap returns
 *   SINCOS_EOVERLAP.
 *   Otherwise, or under SINCOS_HOST_ROUTE_PIPELINE, x is copied to the device
 *   in chunks, each chunk is computed, and s and c are copied back, with
 *   copies and kernels of different chunks overlapped on internal streams
 *   (pageable memory works, but the driver stages its copies).
 *   dev_ws   caller-owned device workspace of ws_bytes for the chunked path,
 *            used as three rotating chunk buffers; sincos_host_workspace_bytes()
 *            gives the size for a given chunk length.  Must be 256-byte
 *            aligned, and is required on both paths.
 * The call is ordered after earlier work on `stream`, and later work on
 * `stream` waits for all its reads and writes of the host buffers, which must
 * stay valid until then.  The library creates its internal streams and events
 * once per device, on first use of the chunked path. */
int sincos_pairs_host(const float *x_host, void *s_host, void *c_host, int64_t n,
                      int out_dtype, int reduction, int coef, void *dev_ws, size_t ws_bytes,
                      sincos_stream_t stream);
size_t sincos_host_workspace_bytes(int out_dtype, int64_t chunk_elems);

/* The route the calling thread's most recent sincos_pairs_host call took:
 * SINCOS_HOST_PATH_ZERO_COPY (one kernel on page-locked, mapped buffers),
 * SINCOS_HOST_PATH_ZERO_COPY_PAGEABLE (one kernel, at least one buffer
 * pageable memory reached through the host's page tables),
 * SINCOS_HOST_PATH_PIPELINE (chunked copies through dev_ws), or
 * SINCOS_HOST_PATH_NONE (no call yet on this thread, n == 0, or the call
 * returned an error).  Data movement only; the paper has no counterpart. */
typedef enum {
    SINCOS_HOST_PATH_NONE = 0,
    SINCOS_HOST_PATH_ZERO_COPY = 1,
    SINCOS_HOST_PATH_PIPELINE = 2,
    SINCOS_HOST_PATH_ZERO_COPY_PAGEABLE = 3
} sincos_host_path;
int sincos_host_last_path(void);

/* Which routes sincos_pairs_host may take, for the whole process:
 * SINCOS_HOST_ROUTE_AUTO (the default: zero-copy whenever the device can
 * reach all three buffers, else the copy pipeline) or
 * SINCOS_HOST_ROUTE_PIPELINE (always the copy pipeline through dev_ws, for
 * callers that want the host buffers touched only by copy engines).  Takes
 * effect for calls that start after it returns.  SINCOS_EINVAL for another
 * value. */
typedef enum { SINCOS_HOST_ROUTE_AUTO = 0, SINCOS_HOST_ROUTE_PIPELINE = 1 } sincos_host_route;
int sincos_host_route_set(int policy);

/* ------------------------------------------------------------------------ */
/* Launch plans and the autotuner                                            */
/* ------------------------------------------------------------------------ */

typedef enum {
    SINCOS_OP_PAIRS = 0,
    SINCOS_OP_BACKWARD = 1,
    SINCOS_OP_BATCHED = 2,
    SINCOS_OP_EXPI = 3,
    SINCOS_OP_HUYGENS = 4   /* plan: block = threads per CTA, unroll = points per thread
                               (1, 2 or 4), vec_bytes = 16 for one binary32 operation per
                               instruction, 32 for two sources per instruction on the
                               packed FP32 pipe (same results) */
} sincos_op;

/* A launch configuration.  The paper's only tuning knob is its 2-way
 * software interleave (Sec. Results); these plans are the GPU analogue and
 * have no other counterpart in it.
 * Register path (vec_bytes 16 or 32): threads per CTA, output vectors each
 * thread keeps in flight per iteration, resident CTAs per SM that the grid
 * is sized for, and the bytes of output one thread writes per vector and per
 * array (16: st.v4; 32: 256-bit st.v8).  A vector holds vec_bytes /
 * sizeof(out) pairs; a batched tile is block * unroll of them.
 * Bulk path (vec_bytes 0; forward, exp(ix) and batched): TMA bulk copies
 * stage 8192-angle chunks through a two-stage shared-memory ring and bulk
 * stores write the results (192 KB of shared memory for binary32 outputs,
 * one CTA per SM); block is 128, 256, 512 or 1024 and unroll is not used.
 * For the single-array forward and the batched ring kernel, ctas_per_sm >= 2
 * selects 4096-angle stages instead (96 KB for binary32 and 64 KB for 16-bit
 * outputs: two or three CTAs per SM as registers allow; block 128, 256 or
 * 512); for exp(ix) ctas_per_sm is not used.  The batched ring kernel runs
 * min(block, 512) consumer threads plus one producer warp.  Single arrays
 * shorter than one chunk, and the backward kernel, use the 16-byte register
 * path instead. */
typedef struct {
    int block;        /* 64 .. 1024, multiple of 32 */
    int unroll;       /* 1, 2, 4 or 8 */
    int ctas_per_sm;  /* 1 .. 32 */
    int vec_bytes;    /* 16 or 32 (register path) or 0 (bulk path) */
} sincos_plan;

/* The plan used for (op, out_dtype, n) on the current device: the tuned one
 * if the cache holds it for n's power-of-two bucket, else the default.  For
 * SINCOS_OP_BATCHED, n is the segment count.  The default for
 * SINCOS_OP_PAIRS depends on n: {256, 2, 2, 0} (4096-angle stages) below 2^24
 * angles, else {512, 2, 1, 0} for binary32 and {512, 2, 3, 0} for 16-bit
 * outputs; the other operations' defaults do not depend on n. */
int sincos_plan_get(int op, int out_dtype, int64_t n, sincos_plan *plan);
/* Store a plan for (op, out_dtype, n's bucket) on the current device. */
int sincos_plan_set(int op, int out_dtype, int64_t n, const sincos_plan *plan);

/* Time every candidate plan on the caller's own buffers (writes s and c; x
 * must not alias them), store the fastest for this (op, dtype, n bucket) and
 * return it in *best.  Timing: every candidate as the median of three bursts
 * of two launches, then the six fastest round-robin over nine passes of eight
 * back-to-back launches each; the lowest median wins.  Synchronizes
 * `stream`.  Must not be called while `stream` is captured. */
int sincos_autotune_pairs(const float *x, void *s, void *c, int64_t n, int out_dtype,
                          int reduction, int coef, sincos_stream_t stream, sincos_plan *best);
int sincos_autotune_backward(const float *gs, const float *gc, const float *s, const float *c,
                             float *gx, int64_t n, sincos_stream_t stream, sincos_plan *best);
/* Same for sincos_expi on the caller's x and z (plans filed under
 * SINCOS_OP_EXPI, dtype SINCOS_F32). */
int sincos_autotune_expi(const float *x, float *z, int64_t n, int reduction, int coef,
                         sincos_stream_t stream, sincos_plan *best);
/* Same for sincos_huygens on the caller's buffers (plans filed under
 * SINCOS_OP_HUYGENS, dtype SINCOS_F32, bucket of m). */
int sincos_autotune_huygens(const float *px, const float *py, const float *pz, int64_t m,
                            const float *qx, const float *qy, const float *qz, const float *ar,
                            const float *ai, int64_t n, float k, int reduction, float *u,
                            sincos_stream_t stream, sincos_plan *best);
/* Same for the batched launch, timed on the caller's batch (outputs are
 * written); the plan is stored under (SINCOS_OP_BATCHED, out_dtype, bucket
 * of `count`), which is also the key batched calls look up. */
int sincos_autotune_batched(const sincos_seg *segs, const int64_t *lens, int count,
                            int out_dtype, int reduction, int coef, sincos_stream_t stream,
                            sincos_plan *best);

/* Plan cache as a small JSON file, keyed by device name and SM count.
 * If the environment variable SINCOS_TUNE_CACHE names a file, it is loaded
 * on first use. */
int sincos_plan_cache_save(const char *path);
int sincos_plan_cache_load(const char *path);

/* ------------------------------------------------------------------------ */
/* Diagnostics (no paper counterpart: the paper's routine returns no status)  */
/* ------------------------------------------------------------------------ */

const char *sincos_strerror(int status);
/* Text of the last failed CUDA call on this host thread ("" if none). */
const char *sincos_last_error(void);
/* Bounded waits inside bulk-path kernels that gave up (an mbarrier that did
 * not complete within one second of wall-clock time) on the current device
 * since the previous call; the count is cleared by reading it.  Nonzero means
 * a launch stopped early and its outputs are incomplete (each thread that
 * gave up counts once).  Synchronizes the device. */
uint32_t sincos_device_wait_timeouts(void);
/* Batched arrays the kernels skipped because their descriptor failed the
 * check of sincos_seg_check (lens[i] > 0 with a null or misaligned pointer),
 * on the current device since the previous call; each skipped array of a
 * call counts once, and reading clears the count.  Synchronizes the
 * device. */
uint32_t sincos_device_bad_segments(void);
/* Self-test of the timeout path (the paper has no counterpart): one CTA waits
 * on a barrier nothing ever completes, giving up after limit_us microseconds
 * (1 .. 10^6) as the bulk kernels do after one second; the next
 * sincos_device_wait_timeouts() then reports one more timeout.  No fault, no
 * trap: the device stays usable. */
int sincos_selftest_wait_timeout(uint32_t limit_us, sincos_stream_t stream);
/* Kernel launches this library has enqueued since load (all threads); a
 * graph replay counts the kernels in the graph. */
uint64_t sincos_launch_count(void);
/* Library version, major * 10000 + minor * 100 + patch. */
int sincos_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SINCOS_PAIRS_H */
