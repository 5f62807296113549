/*
 * pbvd.h -- C ABI of the GB300 parallel block-based Viterbi decoder.
 *
 * The decoder implements the parallel block-based Viterbi decoding of
 * Peng, Liu, Hou, Zhao, "A Gb/s Parallel Block-based Viterbi Decoder for
 * Convolutional Codes on GPU" (arXiv 1608.00066):
 *   - the stream of n trellis stages is cut into blocks of D stages; block b
 *     decodes stages [bD, min((b+1)D, n)) (Sec. III-A, Fig. 1);
 *   - each block runs the forward add-compare-select recursion of Eq. (1)
 *     from L stages before its first stage ("truncation" stages, starting
 *     from all-zero metrics, or from the known encoder state S_0 when that
 *     range reaches stage 0) to L stages after its last stage;
 *   - it then traces back from state S_0 at its last forward stage, with no
 *     metric comparison (Sec. III-A, Algorithm 1), and emits its D bits.
 * Branch metrics are computed once per distinct codeword per stage and reused
 * by every butterfly of the same group (Sec. III-B, Eqs. (3)-(6)).
 *
 * Conventions
 *   state d = (D_{v-1} ... D_0)_2, v = K - 1; S_{2j}, S_{2j+1} move to S_j
 *   (input 0) and S_{j + 2^{v-1}} (input 1); decoded bit of a state = D_{v-1}.
 *   gens[r] holds generator r+1 as an integer whose bit K-1 is the tap on the
 *   input bit and bit 0 the tap on D_0 (octal 0171 = [1111001], Eq. (2)).
 *   Soft values are int8, positive favouring code bit 0; -128 is read as -127.
 *   Branch metric sum_r |lambda_r - mu(c_r)|, mu(0) = +127, mu(1) = -127.
 *   In Eq. (1) a tie keeps the predecessor S_{2j} (the upper branch).
 *   The known start gives S_0 metric 0 and every other state 8192.
 *   Streams and frames are zero-terminated: the last stage is traced back
 *   from S_0, which is exact when the encoder was flushed with v zero bits.
 *
 * Memory: every pointer named d_* is caller-owned device memory; every other
 * pointer is host memory.  The library never frees caller memory.  A context
 * owns its constant tables and a device workspace that grows on demand (it
 * holds the survivor bits of one launch); pbvd_destroy frees them.
 *
 * Errors: every call returns PBVD_OK (0) or a negative code; nothing aborts.
 * Calls are ordered on the CUDA stream passed in (NULL = legacy default
 * stream); device-side failures surface as PBVD_ECUDA on a later call.
 * A context is not thread-safe: do not use one context from two host
 * threads at once, nor in two streams whose work overlaps.
 */
#ifndef PBVD_H
#define PBVD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PBVD_API __attribute__((visibility("default")))
#else
#define PBVD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pbvd_ctx pbvd_ctx;

enum {
    PBVD_OK = 0,
    PBVD_EINVAL = -1,       /* bad argument */
    PBVD_ENOMEM = -2,       /* device or host allocation failed */
    PBVD_ECUDA = -3,        /* a CUDA call failed (see pbvd_last_cuda_error) */
    PBVD_EUNSUPPORTED = -4, /* valid, but no kernel is built for it */
    PBVD_ETIMEOUT = -5,     /* a bounded device wait ran out */
    PBVD_EBUSY = -6         /* resource in use (e.g. serving slots full) */
};

/* Creates a decoder context for an (R,1,K) convolutional code, optionally
 * punctured, decoded in blocks of D stages with L overlap stages per side.
 *   K          constraint length, 3 <= K <= 9 (N = 2^{K-1} states)
 *   R          number of generators (mother rate 1/R), 2 <= R <= 3
 *   gens       host array of R generator integers (see conventions); each
 *              must have its input tap (bit K-1) or its oldest tap (bit 0)
 *              set and no bit at or above K
 *   puncture   host array R x P, row-major, 0/1: code bit r of stage s is
 *              sent iff puncture[r*P + s % P]; NULL for no puncturing.
 *              Every column must send at least one bit.  1 <= P <= 32.
 *   D          decoded stages per block, a positive multiple of 8
 *   L          overlap (truncation and traceback) stages, 0 <= L <= 4096
 * Writes the new context to *out.  Returns PBVD_EINVAL for bad arguments,
 * PBVD_EUNSUPPORTED when no kernel is built for (K, gens), PBVD_ENOMEM. */
PBVD_API int pbvd_create(pbvd_ctx **out, int K, int R, const uint32_t *gens,
                const uint8_t *puncture, int P, int D, int L);

/* Decoding variants of a context (flags, 0 = the scheme of Sec. III-A):
 *   PBVD_MODE_ARGMIN      every block's traceback starts from the state with
 *                         the smallest path metric at its last forward stage
 *                         (the start state S_E of the classic VA, Sec. II;
 *                         the lowest state index on ties) instead of S_0;
 *                         suits streams that are not zero-terminated
 *   PBVD_MODE_TAILBITING  frames are tail-biting (not in the paper: the
 *                         encoder starts in the state its last K-1 message
 *                         bits leave it in; n stages, no tail): the frame is
 *                         read as a circle, block b's window is
 *                         [bD - L, min((b+1)D, n) + L - 1] with stage s taken
 *                         at s mod n, and every block starts from zero metrics
 *                         (no known start).  pbvd_decode then keeps a copy of
 *                         the frame with L wrapped stages on each side in a
 *                         buffer owned by the context (grown on first use of a
 *                         larger size).  Unpunctured codes only
 *                         (PBVD_EUNSUPPORTED otherwise).
 * The flags apply to pbvd_decode, pbvd_decode_packed and pbvd_autotune;
 * pbvd_decode_host and pbvd_decode_noalloc support PBVD_MODE_ARGMIN only;
 * batches and streams support neither (PBVD_EUNSUPPORTED).  PBVD_EINVAL for
 * unknown flags. */
#define PBVD_MODE_ARGMIN 1
#define PBVD_MODE_TAILBITING 2
PBVD_API int pbvd_set_mode(pbvd_ctx *ctx, int flags);

/* Reads the flags set by pbvd_set_mode. */
PBVD_API int pbvd_get_mode(const pbvd_ctx *ctx, int *flags);

/* Frees the context and its workspace.  Synchronises the device first if
 * work may still be in flight.  NULL is ignored. */
PBVD_API void pbvd_destroy(pbvd_ctx *ctx);

/* Decodes one terminated stream or frame of n_stages trellis stages.
 *   d_llr      device, int8 soft values as sent: n_stages * R values for an
 *              unpunctured code, otherwise the kept positions only, in stage
 *              order, code bits of a stage in ascending r
 *   n_stages   number of trellis stages, tail included (>= 1)
 *   d_out      device, ceil(n_stages / 8) bytes; bit s of the result is bit
 *              (s & 7) of byte (s >> 3), LSB first; the last v bits are the tail
 *   stream     a cudaStream_t (NULL = legacy default stream)
 * Asynchronous: returns after enqueueing.  Grows the context workspace on
 * first use of a larger n_stages (a device allocation that synchronises); call
 * once with the largest size before capturing a CUDA graph. */
PBVD_API int pbvd_decode(pbvd_ctx *ctx, const int8_t *d_llr, size_t n_stages,
                uint8_t *d_out, void *stream);

/* The paper's own two-kernel design (Sec. IV-A/IV-B, Algorithm 1, Table 1),
 * kept as an ablation of pbvd_decode: kernel K1 runs the forward procedure
 * with N_c threads per block of stages (one per group of butterflies sharing a
 * codeword alpha, Table 2), 32 blocks per thread block, path metrics in shared
 * memory laid out PM[N][32], and writes bit-packed survivor words to global
 * memory laid out SP[D+2L][N_c][N_t]; kernel K2 traces back with one thread
 * per block.  Same arguments, geometry and bits as pbvd_decode (32-bit path
 * metrics).  Built for the unpunctured K=7 (171,133) and K=9 (557,663,711)
 * codes and the plain mode (PBVD_EUNSUPPORTED otherwise).  The survivor
 * words live in the context workspace, (D+2L) N_c ceil(n_stages/D) words. */
PBVD_API int pbvd_decode_two_kernel(pbvd_ctx *ctx, const int8_t *d_llr, size_t n_stages, uint8_t *d_out,
                                    void *stream);

/* Decodes a stream held in HOST memory, in one of two ways.
 * Copy pipeline (segments >= 0), after the multi-stream scheme of Sec. IV-C
 * (Eq. (7)): the stream's blocks are cut into runs of whole pairs of blocks;
 * the soft values go host -> device in order on one copy stream, copy i
 * ending L stages into run i + 1 (the last stage that run i's blocks read),
 * each run is decoded on one of sixteen compute streams as soon as its copy
 * has arrived, and its packed bits go device -> host on the same compute
 * stream.  Runs decode concurrently, so the GPU fills up while later runs
 * are still being copied.
 * Direct access (segments = -1): both host buffers must be page-locked and
 * mapped into the device's address space (cudaHostAlloc / cudaMallocHost /
 * cudaHostRegister with unified addressing, as cudaPointerGetAttributes
 * reports); the decode kernel of pbvd_decode then reads the soft values
 * from host memory and writes the packed bits to host memory itself, over
 * the host-device link, with no staging copy and no device copy of the
 * stream (the halo stages of Sec. III-A cross the link twice).  Slower than
 * the copy pipeline on a GB300: the kernel's many small reads use the link
 * poorly.
 *   h_llr      host soft values, laid out as d_llr of pbvd_decode
 *   h_out      host, ceil(n_stages / 8) bytes, written as d_out of pbvd_decode
 *   segments   0 = copy pipeline with an automatic number of runs (up to 6
 *              runs of at least 1024 blocks); > 0 = copy pipeline with that
 *              many runs (at most 64); -1 = direct access (PBVD_EINVAL,
 *              nothing enqueued, when a buffer is not mapped page-locked
 *              memory).  Pageable memory works in the copy pipeline but is
 *              copied synchronously by the driver.
 *   stream     the caller's stream: the work starts after what is already
 *              queued on it, and work queued on it later waits for the whole
 *              decode, so h_out is complete once the stream reaches that point
 * The bits are exactly those of pbvd_decode with the same context.  The copy
 * pipeline uses the context's configuration with survivors in global
 * memory; the context owns the device copies of the stream, its copy and
 * compute streams and events, grown on first use of a larger size (device
 * allocations that synchronise).  Host buffers must stay valid until the
 * stream has passed the call; calls on one context must not overlap on the
 * GPU. */
PBVD_API int pbvd_decode_host(pbvd_ctx *ctx, const int8_t *h_llr, size_t n_stages,
                              uint8_t *h_out, int segments, void *stream);

/* Decodes soft values quantised to q bits and packed, as Sec. IV-C stores
 * them to shrink the input transfer (U_1 = 4R / floor(32/q) bytes per stage
 * instead of R): floor(32/q) values per 32-bit word, value i in word i / m
 * (m = floor(32/q)) at bits [q (i mod m), q (i mod m) + q) as a q-bit two's
 * complement number; q = 1 is hard decision (bit 1 = received code bit 1).
 *   d_words    device, ceil(count / m) words, count = pbvd_llr_count(n_stages)
 *              values in the order of pbvd_decode's d_llr (punctured codes:
 *              the sent values only)
 *   q          1..8
 * The branch metric is that of the paper with mu = +-Q, Q = 2^{q-1} - 1
 * (Q = 1 for q = 1: twice the Hamming distance); values below -Q read as -Q.
 * The values are unpacked on the device into a buffer owned by the context
 * (grown on first use of a larger size, a synchronising allocation), scaled
 * by floor(127 / Q) -- which changes every branch metric of a stage by the
 * same positive-affine map and therefore no decision -- and decoded as by
 * pbvd_decode.  d_out as for pbvd_decode. */
PBVD_API int pbvd_decode_packed(pbvd_ctx *ctx, const uint32_t *d_words, int q, size_t n_stages,
                                uint8_t *d_out, void *stream);

/* pbvd_decode_host with packed q-bit input (see pbvd_decode_packed): the
 * copy pipeline moves the packed words host -> device, unpacks each run's
 * values on the device as soon as its words have arrived, and decodes the
 * runs as pbvd_decode_host does.  segments >= 0 (direct access is not
 * offered for packed input); segments = 0 picks up to 2 runs for q <= 3 and
 * up to 4 for larger q. */
PBVD_API int pbvd_decode_host_packed(pbvd_ctx *ctx, const uint32_t *h_words, int q, size_t n_stages,
                                     uint8_t *h_out, int segments, void *stream);

/* pbvd_decode_packed with 8-bit path metrics (Sec. IV-C: with q-bit soft
 * values the branch metrics are at most BMmax = 2QR, Q = 2^{q-1} - 1, or 1
 * for q = 1, and the metrics of a block stay within (K - 1) BMmax of each
 * other, so they fit in bytes when K * BMmax < 127): four blocks per 32-bit
 * register, one or two threads per four blocks (two split the states of a
 * 64-state code between them; the context's pbvd_set_config threads_per_pair
 * picks 1 or 2, otherwise two while there are fewer than 64 four-block
 * groups per SM).  Same input format as
 * pbvd_decode_packed and the same decoded bits as that call, i.e. as the
 * block-based decoder on the q-bit branch metric.
 * Built for the K=7 (171,133) and (171,165,133) codes and the K=5 (23,35)
 * code, unpunctured, without pbvd_set_mode flags; q <= 3 for R = 2 at K = 7
 * and K = 5 and for R = 3 at K = 7.  PBVD_EUNSUPPORTED otherwise.  Grows two
 * context buffers on first use of a larger size (the values regrouped four
 * blocks to a word, 4 R min(D + 2L, n) bytes per four blocks, and the survivor
 * records, min(D + 2L, n) 2^{K-1} / 2 bytes per four blocks); asynchronous. */
PBVD_API int pbvd_decode_packed_pm8(pbvd_ctx *ctx, const uint32_t *d_words, int q, size_t n_stages,
                                    uint8_t *d_out, void *stream);

/* Number of soft values d_llr must hold for n_stages stages. */
PBVD_API int pbvd_llr_count(const pbvd_ctx *ctx, size_t n_stages, size_t *count);

/* One frame of a batched decode. */
typedef struct pbvd_batch_item {
    pbvd_ctx *ctx;        /* code and (D, L) of this frame */
    const int8_t *d_llr;  /* device soft values as for pbvd_decode */
    size_t n_stages;      /* stages of this frame, tail included */
    uint8_t *d_out;       /* device, ceil(n_stages / 8) bytes */
} pbvd_batch_item;

/* Decodes n_items independent frames of possibly different codes and lengths
 * in one persistent kernel launch (batching is not in the paper; every frame
 * is decoded exactly as pbvd_decode decodes it alone with its context).
 * One launch covers the K=7 (171,133) rate-1/2 code, the same code punctured
 * (any pattern) and the K=9 (557,663,711) rate-1/3 code; contexts of the same
 * code must agree on D, L and the puncture pattern (PBVD_EINVAL otherwise),
 * other codes give PBVD_EUNSUPPORTED.  items is a host array read during the
 * call.  The work list (blocks of all frames grouped by code, sorted by
 * length, paired and cut into tiles taken from a device queue) is built on the
 * host and uploaded into a workspace owned by the first item's context, which
 * must therefore not be used by another batch still in flight.  Output ranges
 * must not overlap.  Kernel shape: a batch of one code runs that code's own
 * kernel; a mixed batch runs the wide shape (four threads per pair of blocks
 * for K=7, sixteen for K=9), or the dense shape (two and eight) when the
 * configuration of an item's context (pbvd_set_config threads_per_pair)
 * names the dense shape's value for its code; the bits are the same. */
PBVD_API int pbvd_decode_batch(const pbvd_batch_item *items, size_t n_items, void *stream);

/* A prepared batch: the work list and workspace of pbvd_decode_batch, kept so
 * that the decode itself is one memset and one kernel launch (pbvd_batch_run),
 * which can be captured in a CUDA graph and replayed.  The item buffers must
 * stay valid and keep their addresses while the batch is in use. */
typedef struct pbvd_batch pbvd_batch;

/* Builds and uploads (on stream) the work list of items into a new batch. */
PBVD_API int pbvd_batch_prepare(pbvd_batch **out, const pbvd_batch_item *items, size_t n_items,
                                void *stream);

/* Replaces the items of a prepared batch, reusing its device buffers (they
 * grow, with a device synchronisation, only when the new work list is larger
 * than any before).  The upload is ordered on stream, so a previous run of
 * the batch must be on the same stream.  reserve_sms > 0 sizes the
 * persistent grid for that many SMs fewer (leaving room for other work, e.g.
 * stream pushes); 0 = fill the GPU.  For serving loops that decode a new set
 * of frames every iteration. */
PBVD_API int pbvd_batch_update(pbvd_batch *batch, const pbvd_batch_item *items, size_t n_items,
                               int reserve_sms, void *stream);

/* Decodes a prepared batch: resets the tile queue and launches the kernel. */
PBVD_API int pbvd_batch_run(pbvd_batch *batch, void *stream);

/* Frees a batch (synchronises the device first).  NULL is ignored. */
PBVD_API void pbvd_batch_destroy(pbvd_batch *batch);

/* Kernel configuration of a context (the tuning knobs).
 *   threads_per_pair  T: threads that share one pair of blocks (power of two,
 *                     N/T states per thread); 0 = automatic
 *   cta_threads       threads per CTA (multiple of 32, <= 256); 0 = automatic
 *   survivors_in_smem 1: survivor bits in shared memory, 0: in the device
 *                     workspace, -1 = automatic
 * Automatic: pbvd_decode (and the calls built on it) takes the fewest
 * threads per pair that give about 1.5 warps per SM scheduler, with at most
 * 64 states per thread (32 for codes of more than 64 states), in one-warp
 * CTAs when T <= 2 and 64-thread CTAs otherwise; pbvd_decode_host (its copy
 * pipeline and its direct access) aims at about 2 warps per scheduler in
 * CTAs of at least 64 threads, which shortens each run's dependency chain;
 * survivors go to shared memory when there are no more pairs than SMs. */
typedef struct pbvd_config {
    int threads_per_pair;
    int cta_threads;
    int survivors_in_smem;
} pbvd_config;

/* Sets the configuration used by later pbvd_decode calls on ctx.
 * PBVD_EUNSUPPORTED if the code has no kernel for that T. */
PBVD_API int pbvd_set_config(pbvd_ctx *ctx, const pbvd_config *cfg);

/* Reads back the configuration pbvd_decode would use for n_stages (with an
 * automatic configuration, pbvd_decode_host may use more threads per pair). */
PBVD_API int pbvd_get_config(const pbvd_ctx *ctx, size_t n_stages, pbvd_config *cfg);

/* Autotuner (not in the paper): decodes the caller's data with every built
 * threads-per-pair value, CTA size and survivor placement, timing each with
 * CUDA events on stream (reps timed runs after one warm-up; synchronises),
 * and keeps the fastest configuration in ctx (also written to best / best_ms
 * when non-NULL).  The decoded bits do not depend on the configuration.  D and
 * L, which do change the bits, are context parameters and are not tuned here. */
PBVD_API int pbvd_autotune(pbvd_ctx *ctx, const int8_t *d_llr, size_t n_stages, uint8_t *d_out,
                           void *stream, int reps, pbvd_config *best, float *best_ms);

/* Allocation-free variant of pbvd_decode (no counterpart in the paper).
 * For callers that must not allocate device memory while decoding: code
 * running under CUDA stream capture, real-time receive chains that reserve
 * all memory up front, hosts whose device memory belongs to their own pool.
 * pbvd_decode grows a context workspace with cudaMalloc; this call instead
 * keeps the survivor bits in one fixed array of
 * pbvd_noalloc_max_survivor_bytes() bytes (16 MiB) that every GPU loading the
 * library holds until exit, and calls no cudaMalloc, cudaFree or other
 * allocating routine.  Arguments and results are those of pbvd_decode; the
 * survivor bits live in shared memory when the context's configuration
 * places them there (as pbvd_decode would: few blocks, or survivors_in_smem
 * = 1), otherwise in that array.
 * With an automatic configuration it uses fewer threads per pair of blocks
 * (smaller survivor records) when that is what makes the bits fit.  Returns
 * PBVD_EINVAL when the launch would still need more survivor bytes than the
 * array holds (for the K=7 rate-1/2 code with D=512, L=42: about 1.9 million
 * stages) or when the current device is not the context's.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress), so
 * make it outside stream capture; the address is kept until the process
 * exits, so do not reset the device (cudaDeviceReset) while using the
 * library.  All calls share the array: calls whose work overlaps on the GPU
 * (other streams, other host threads) race on it.  Kernels the library
 * compiles at run time (codes without a built-in kernel, the decoding
 * variants of pbvd_set_mode) allocate device memory when they are first
 * loaded, so this call returns PBVD_EUNSUPPORTED until pbvd_decode has
 * launched the same kernel once (the same code, mode and configuration, and
 * a stream length for which the automatic configuration is the same). */
PBVD_API int pbvd_decode_noalloc(pbvd_ctx *ctx, const int8_t *d_llr, size_t n_stages,
                                 uint8_t *d_out, void *stream);

/* Size of the fixed survivor array of pbvd_decode_noalloc, in bytes. */
PBVD_API size_t pbvd_noalloc_max_survivor_bytes(void);

/* Continuous streams with device-resident path metrics (serving; the paper
 * decodes blocks only).  A stream of an unpunctured K=7 (171,133) or K=9
 * (557,663,711) code is decoded by Eq. (1) run once over all its stages with
 * the metrics carried in device memory between pushes; segment m of D stages
 * is released, once stage (m+1)D + L - 1 exists, by traceback from S_0 at that
 * stage; closing the stream (whose last v stages must be the zero tail)
 * releases the rest by traceback from S_0 at the last stage.  Bit s of the
 * stream goes to bit s & 7 of byte s >> 3 of d_out (device, caller-owned,
 * out_capacity stages).  Pushes are ordered on the CUDA stream given; a
 * stream object must not be pushed from two host threads at once. */
typedef struct pbvd_stream pbvd_stream;

/* Opens a stream on ctx accepting up to max_push stages per push; allocates
 * its device state (metrics, a survivor ring of max_push + D + L + 2P
 * records, a staging buffer). */
PBVD_API int pbvd_stream_open(pbvd_stream **out, pbvd_ctx *ctx, size_t max_push, uint8_t *d_out,
                              size_t out_capacity);

/* Appends n_stages stages (device soft values, R per stage) and decodes them. */
PBVD_API int pbvd_stream_push(pbvd_stream *s, const int8_t *d_llr, size_t n_stages, void *stream);

/* Pushes to count distinct streams of the same code, one kernel launch per
 * 128 streams; n_stages[i] may be 0, and d_llr and n_stages may both be NULL
 * when no stream receives stages.  With close != 0 every stream is closed
 * after its push.  A push decodes whole periods of P stages (P = 3 for K=7,
 * 4 for K=9 streams); the rest waits in the stream's carry buffer. */
PBVD_API int pbvd_stream_push_many(pbvd_stream *const *s, const int8_t *const *d_llr,
                                   const size_t *n_stages, size_t count, int close, void *stream);

/* Closes the stream: decodes what is left and releases every bit. */
PBVD_API int pbvd_stream_close(pbvd_stream *s, void *stream);

/* Number of leading stages whose bits are final in d_out once the pushes so
 * far have completed on their CUDA stream. */
PBVD_API int64_t pbvd_stream_released(const pbvd_stream *s);

/* Inspection of a stream's carried state (for tests and tools): copies the
 * N = 2^{K-1} path metrics the stream holds after its last decoded stage to
 * h_metrics (state order, host memory) and the number of stages decoded so
 * far (whole periods; a partial period waits in the carry buffer) to
 * *stages.  The metrics are renormalised 16-bit values: they equal Eq. (1)'s
 * exact metrics of those stages up to one common offset.  Waits for the work
 * queued on `stream` before the copy. */
PBVD_API int pbvd_stream_metrics(const pbvd_stream *s, int64_t *stages, int32_t *h_metrics, void *stream);

/* Frees the stream's device state (synchronises the device first). */
PBVD_API void pbvd_stream_destroy(pbvd_stream *s);

/* Measurement helper, not a decoding call: the integer issue rate of the
 * current device for one kind of instruction the decode kernels are built
 * from, in thread-level operations per clock per SM (a 16x2 operation counts
 * once).  op: 0 the 16x2 DPX add-min, 1 a three-input add, 2 a three-input
 * logic op, 3 a byte permute, 4 an integer multiply-add (FMA pipe), 5 logic
 * op and multiply-add interleaved, 6 16x2 add-min and multiply-add
 * interleaved.  Eight independent chains per thread, 2,048 threads per SM,
 * SM cycles from clock64; runs for a few milliseconds on the legacy default
 * stream and synchronises the device.  PBVD_EINVAL for another op,
 * PBVD_ENOMEM, PBVD_ECUDA. */
PBVD_API int pbvd_measure_int_rate(int op, double *ops_per_clk_per_sm);

/* Message for an error code (static string). */
PBVD_API const char *pbvd_strerror(int code);

/* Text of the last CUDA error seen by the library in this process. */
PBVD_API const char *pbvd_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PBVD_H */
