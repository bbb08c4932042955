/*
 * xorgens_gb300 -- C ABI of a GB300 (sm_103a) library of xorgens generators.
 *
 * The generator is the one of Nandapalan, Brent, Murray and Rendell,
 * "High-Performance Pseudo-Random Number Generation on Graphics Processing
 * Units" (arXiv:1108.0486):
 *   x_k = x_{k-r}(I + L^a)(I + R^b) xor x_{k-s}(I + L^c)(I + R^d)   (Sec. 2)
 *   w_k = w_{k-1} + omega mod 2^32                                   (Sec. 1.5)
 *   out_k = x_k + (w_k xor (w_k >> 16)) mod 2^32                     (Eq. 1)
 * with 32-bit words, r = 128 and one of two compile-time parameter sets:
 *   XG_PARAMS_DEFAULT  (r,s,a,b,c,d) = (128, 95, 17, 12, 13, 15)
 *   XG_PARAMS_PAPER    (r,s,a,b,c,d) = (128, 65, 15, 14, 12, 17)  (Sec. 2)
 * Each stream is one generator: r state words plus a Weyl word plus a
 * position (Sec. 2 counts the state the same way: the r words, the Weyl
 * word and the buffer index).  Many independent streams live in one context, resident in
 * device memory (Sec. 2, independent subsequences; Sec. 4, one seed per
 * block id).
 *
 * Conventions for every entry point:
 *   - Returns an xg_status; never throws or aborts.  On failure the
 *     thread-local message of xg_last_error() says why.
 *   - Device pointers are CUDA device memory of the current device (for
 *     example a torch tensor's data pointer); host pointers are ordinary
 *     (pageable or pinned) host memory.  The library never frees caller memory.
 *   - Work is enqueued on the context's CUDA stream and is asynchronous unless
 *     the entry point says otherwise.  Calls on one context must come from one
 *     host thread at a time, except the request server's calls (xg_submit,
 *     xg_submit_many, xg_poll, xg_wait, xg_release, xg_collect,
 *     xg_ticket_times, xg_server_stats_get), which several threads may make
 *     at once while the server runs; xg_server_start and xg_server_stop must
 *     not overlap any other call on the context.
 *   - Stream positions advance with every call, in call order.  Any split of
 *     a stream's output into consecutive calls concatenates to the same
 *     sequence as one call, for every output type and launch configuration.
 */
#ifndef XORGENS_GB300_H
#define XORGENS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xg_ctx xg_ctx; /* opaque, owned by the library */

typedef enum {
    XG_OK = 0,
    XG_EINVAL = 1,     /* bad argument: null pointer, range, alignment, size */
    XG_ENOMEM = 2,     /* device or host allocation failed */
    XG_EAGAIN = 3,     /* admission refused: the output memory cap is reached */
    XG_ETIMEDOUT = 4,  /* a bounded wait gave up */
    XG_ECUDA = 5,      /* a CUDA runtime call failed (message has the CUDA error) */
    XG_ENOTFOUND = 6,  /* unknown ticket */
    XG_EDEVICE = 7,    /* device-side state read back by the host is corrupt (xg_get_state),
                          a server request's batch failed to launch and never ran, or a
                          jump-ahead kernel on the tensor cores gave up one of its bounded
                          waits (xg_jump, xg_seed_substreams, a cut call: the streams being
                          advanced are not valid; reseed or restore them) */
    XG_ECANCELED = 8   /* the request was cancelled (xg_cancel) before it ran */
} xg_status;

typedef enum {
    XG_U32 = 0,         /* the output word itself, Eq. (1) */
    XG_UNIFORM_F32 = 1, /* (out >> 8) * 2^-24, exact, in [0, 1) */
    XG_NORMAL_F32 = 2   /* Box-Muller on consecutive word pairs (o1, o2):
                           u1 = ((o1 >> 8) + 1) 2^-24, u2 = (o2 >> 8) 2^-24,
                           z1 = sqrt(-2 ln u1) cos(2 pi u2),
                           z2 = sqrt(-2 ln u1) sin(2 pi u2).
                           n normals consume 2*ceil(n/2) words; pairs start at
                           the call's first word; when n is odd the last z2 is
                           dropped.  Within 4 ulp of the exact value. */
} xg_type;

enum { XG_PARAMS_DEFAULT = 0, XG_PARAMS_PAPER = 1 };

/* ---- contexts and state ------------------------------------------------- */

/* Create n_streams generators (all unseeded: call xg_seed before use).
 * param_set: XG_PARAMS_DEFAULT or XG_PARAMS_PAPER.  weyl_on: 1 for Eq. (1),
 * 0 to output the GF(2)-linear part x_k alone (for testing).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream) owned by the caller; it must
 * outlive the context.  Allocates the device state: 784 bytes per stream. */
xg_status xg_create_streams(xg_ctx** out, uint32_t n_streams, uint32_t param_set,
                            uint32_t weyl_on, void* cuda_stream);

/* Wait for the context's work, stop its server if running, free everything. */
xg_status xg_destroy(xg_ctx* ctx);

/* Change the CUDA stream later calls enqueue on (cudaStream_t). */
xg_status xg_set_stream(xg_ctx* ctx, void* cuda_stream);

/* Number of streams in the context. */
xg_status xg_num_streams(const xg_ctx* ctx, uint32_t* n_streams);

/* Seed streams [first, first+count) from host_seeds[0..count): expands each
 * 32-bit seed into r = 128 state words and a Weyl word with Marsaglia's
 * 64-bit xorshift (shift triple 13, 7, 17), then runs the generator for
 * 4r = 512 words and discards them (the paper defers seeding to the xorgens
 * package, Sec. 1.5 and Sec. 4; this is the library's own procedure).
 * Consecutive seeds (block ids, Sec. 4) give unrelated streams. */
xg_status xg_seed(xg_ctx* ctx, uint32_t first, uint32_t count, const uint32_t* host_seeds);

/* Checkpoint: the stream's r = 128 most recent state words, oldest first,
 * and its Weyl word, into host memory.  Synchronises the context's stream. */
xg_status xg_get_state(xg_ctx* ctx, uint32_t stream, uint32_t* host_ring128,
                       uint32_t* host_weyl);

/* Restore a state written by xg_get_state (or any nonzero state).  After it
 * the stream continues exactly as the checkpointed one did.  Synchronous. */
xg_status xg_set_state(xg_ctx* ctx, uint32_t stream, const uint32_t* host_ring128,
                       uint32_t weyl);

/* Bulk checkpoint of streams [first, first + count): host_rings receives
 * count x 128 words (stream after stream, each oldest first, as
 * xg_get_state), host_weyl count Weyl words, host_pos (may be NULL) count
 * positions (words consumed since seeding).  Synchronous; about 0.5 KiB per
 * stream through one kernel and three copies. */
xg_status xg_get_states(xg_ctx* ctx, uint32_t first, uint32_t count, uint32_t* host_rings,
                        uint32_t* host_weyl, uint64_t* host_pos);

/* Bulk restore of states written by xg_get_states (into this or another
 * context with the same parameter set): the streams continue exactly as the
 * checkpointed ones did.  Positions are restored when host_pos is not NULL,
 * else left as they are.  Synchronous. */
xg_status xg_set_states(xg_ctx* ctx, uint32_t first, uint32_t count, const uint32_t* host_rings,
                        const uint32_t* host_weyl, const uint64_t* host_pos);

/* ---- plain generation (one kernel launch per call) --------------------- */

/* Write n_per_stream outputs of each stream in [first, first+nstreams) to
 * out + (i - first) * ld (elements), stream-major.  ld >= n_per_stream.
 * out may be device memory (asynchronous on the context's stream) or host
 * memory (the library generates into its own device buffer in chunks and
 * copies them to the host, overlapping both; returns when the data is there).
 * The fast path needs out and ld*4 bytes 16-byte aligned; other alignments
 * are accepted and use scalar stores.  Calls on at most 64 streams with at
 * least 2^18 outputs each go through the batch path, which cuts them into
 * pieces generated at once (see xg_set_batch_split; 1 turns this off); the
 * outputs are the same. */
xg_status xg_generate_u32(xg_ctx* ctx, uint32_t first, uint32_t nstreams,
                          uint64_t n_per_stream, uint32_t* out, uint64_t ld);
xg_status xg_generate_uniform(xg_ctx* ctx, uint32_t first, uint32_t nstreams,
                              uint64_t n_per_stream, float* out, uint64_t ld);
xg_status xg_generate_normal(xg_ctx* ctx, uint32_t first, uint32_t nstreams,
                             uint64_t n_per_stream, float* out, uint64_t ld);

/* Fused mode: generate n_per_stream normals per stream exactly as
 * xg_generate_normal would (the streams advance the same way) but write only
 * their FP32 sum per stream to d_sums[i - first] (device memory).  The sum
 * order is fixed by the launch configuration (xg_get_launch): each lane adds
 * its own values in sequence order, then the lanes of a stream are combined
 * by a butterfly over lane offsets TPG/2, ..., 1. */
xg_status xg_generate_normal_sum(xg_ctx* ctx, uint32_t first, uint32_t nstreams,
                                 uint64_t n_per_stream, float* d_sums);

/* Conversions alone: apply the XG_UNIFORM_F32 / XG_NORMAL_F32 transform to
 * n words already in device memory (d_words), writing n floats to d_out.
 * For the normal transform, n must be even (pairs (d_words[2i],
 * d_words[2i+1])). */
xg_status xg_transform_uniform(xg_ctx* ctx, const uint32_t* d_words, uint64_t n, float* d_out);
xg_status xg_transform_normal(xg_ctx* ctx, const uint32_t* d_words, uint64_t n, float* d_out);

/* ---- batched generation ------------------------------------------------ */

typedef struct {
    uint32_t stream; /* stream index in the context */
    uint32_t type;   /* xg_type */
    uint64_t count;  /* outputs */
    void* out;       /* device memory for count 4-byte outputs (16-byte
                        alignment takes the vector-store path) */
} xg_item;

/* Run n_items generation calls with ONE launch of the persistent batch
 * kernel, replayed from a CUDA graph (a copy of the batch description into
 * device scratch, then the kernel); when long calls are cut into pieces (see
 * xg_set_batch_split), a jump-ahead prologue of a few small launches comes
 * first.  Items may have different types and very
 * different lengths.  Items of the same stream run in array order, exactly as
 * consecutive xg_generate_* calls would; different streams run concurrently,
 * one warp per stream, the longest stream first.  Asynchronous on the
 * context's stream; the items array may be reused when the call returns.
 * This is the independent-subsequence scheme of Sec. 2: each stream is one
 * generator with its own state. */
xg_status xg_generate_batch(xg_ctx* ctx, const xg_item* items, uint32_t n_items);

/* The same batched generation for callers that must not allocate memory
 * while they run -- for example an application whose device memory is owned
 * by another allocator, or a latency-critical loop that cannot take
 * cudaMalloc's implicit device synchronisation.  (The paper has no
 * counterpart: this is a property of the library, not of the method.)
 * Calls no cudaMalloc, cudaFree or other allocating routine: the batch
 * description is assembled in a fixed host buffer inside the library (about
 * 86 KiB; calls from several threads take turns on it, and nothing large
 * goes on the caller's stack) and goes with one cudaMemcpyAsync to a fixed
 * device array inside the library (about 48 KiB, held by every GPU that
 * loads the library until the process exits); the persistent batch kernel
 * of xg_generate_batch runs on it.  Results are identical to
 * xg_generate_batch's.
 *   - At most 1024 items per call; more is XG_EINVAL.
 *   - The context's device must be current.  The array's device address is
 *     looked up, and the module holding it loaded, by xg_create_streams
 *     (once per device), so no call of this function loads code or memory.
 *   - The array is shared by every call and keeps the last call's batch; each
 *     call rewrites its header, including the work counter that starts at
 *     zero.  Calls whose kernels overlap on the GPU (different CUDA streams,
 *     other contexts on the same device, other threads) race on the array:
 *     order them on one stream or synchronise between them. */
xg_status xg_generate_batch_noalloc(xg_ctx* ctx, const xg_item* items, uint32_t n_items);

/* Launch shape of the persistent batch kernel for calls of one output type
 * (the threads-per-generator choice of Sec. 2's parallel scheme).  Calls of
 * that type that are alone on their stream in a batch (and pieces of cut
 * calls) with a 16-byte aligned output run
 *   (tpg, wpl) = (32, 2): one stream per warp, 2 words per lane per round,
 *                         64-bit stores;
 *                (16, 4): two streams per warp side by side, 4 words per lane,
 *                         128-bit stores;
 *                (8, 4):  four streams per warp, 128-bit stores.
 * The batch groups calls of similar length, and only calls of at most 1/8
 * of a resident warp's share of the batch's words (a group runs each of its
 * calls at 1/2 or 1/4 of a warp's rate, so a group of long calls would
 * become the batch's tail).  Other calls (longer ones, several calls on one
 * stream in a batch, unaligned outputs) run (32, 2), and so do normals
 * (their transform needs the registers a wider group would take).  Applies
 * to xg_generate_batch, the request server and cut calls.  The results do
 * not depend on the shape.  Default: (32, 2) for every type.  The
 * environment variable XG_BATCH_GROUP_MAX_WORDS=<n> replaces the 1/8 rule
 * by a fixed limit of n words.  XG_EINVAL for another pair, or for normals
 * other than (32, 2). */
xg_status xg_set_batch_shape(xg_ctx* ctx, xg_type type, uint32_t tpg, uint32_t wpl);
xg_status xg_get_batch_shape(xg_ctx* ctx, xg_type type, uint32_t* tpg, uint32_t* wpl);

/* Autotune the batch kernel's shape per output type on the caller's own
 * batch: for each type present in items, the calls of that type are run as
 * one batch with every shape (one warm-up and three timed launches, the
 * median kept), and the fastest shape is kept for the context.  The stream
 * states are restored afterwards, so the streams do not advance; the items'
 * output buffers are written.  Synchronous; allocates a copy of the stream
 * state.  tpg, wpl, ms: arrays of 3 (indexed by xg_type) or null; a type
 * absent from the batch keeps its shape and reports ms = 0. */
xg_status xg_autotune_batch(xg_ctx* ctx, const xg_item* items, uint32_t n_items, uint32_t* tpg, uint32_t* wpl,
                            float* ms);

/* Cutting long calls in batches: a call that is alone on its stream in a
 * batch (xg_generate_batch and the request server) and has at least twice
 * piece_words words is cut into pieces of piece_words words that different
 * warps generate at once; each piece starts from the stream's state jumped
 * ahead by its offset (see xg_jump), so the output is exactly that of the
 * uncut call.  piece_words: 0 = automatic (about the batch's words per
 * resident warp, between 2^15 and 2^22), 1 = never cut, else a power of two
 * >= 64. */
xg_status xg_set_batch_split(xg_ctx* ctx, uint64_t piece_words);

/* Jump-ahead: advance streams [first, first+nstreams) by `words` positions
 * without generating them, exactly as if that many words had been drawn
 * (the recurrence of Sec. 2 is linear over GF(2) on the 4096-bit ring, so
 * the jump is a product of precomputed powers M^(2^k) of its transition
 * matrix, one per set bit of `words`; the Weyl word advances by
 * words * omega).  The first use of each power builds it on the GPU (2 MiB
 * each, kept until exit).  Synchronous.  Useful for provably disjoint
 * substreams: stream i jumped by i * 2^64 would never overlap, here by any
 * 64-bit distance. */
xg_status xg_jump(xg_ctx* ctx, uint32_t first, uint32_t nstreams, uint64_t words);

/* Seed streams [first, first+count) as consecutive, disjoint blocks of ONE
 * sequence: stream first + i starts at position i * 2^log2_spacing of the
 * sequence that xg_seed gives for `seed` (its ring, Weyl word and position
 * are those of that sequence there), so no two of them draw a common word
 * until one has drawn 2^log2_spacing words -- the independent subsequences
 * of Sec. 2 taken from one period instead of from different seeds.  Built
 * with log2(count) doubling steps of the jump-ahead matrices (one matrix
 * application per stream).  Requires (count - 1) * 2^log2_spacing < 2^64,
 * else XG_EINVAL; also XG_EINVAL for a stream range out of bounds or a
 * running server.  Synchronous. */
xg_status xg_seed_substreams(xg_ctx* ctx, uint32_t first, uint32_t count, uint32_t seed, uint32_t log2_spacing);

/* ---- serving: continuous batching of requests --------------------------- */

typedef struct {
    uint64_t mem_cap_bytes; /* cap on outstanding output bytes (pool buffers and
                               caller buffers alike); 0 = 16 GiB.  The pool is
                               one device allocation of this size. */
    uint32_t max_batch;     /* requests per batch launch; 0 = 1024 */
    uint32_t lanes;         /* batches in flight at once, each on its own CUDA
                               stream; 0 = 48, at most 64 */
} xg_server_config;

typedef struct {
    uint32_t stream; /* stream index in the context */
    uint32_t type;   /* xg_type */
    uint64_t count;  /* outputs (> 0) */
    void* d_out;     /* device memory for count outputs, or NULL: the library
                        carves a buffer from its pool, valid until xg_release */
} xg_request;

typedef struct {
    uint64_t submitted, completed, refused, queued, in_flight, batches, items_launched;
    uint64_t outstanding_bytes;
    uint64_t now_ns; /* the server clock (steady, ns) that xg_ticket_times uses */
    uint64_t host_launch_ns; /* host time the server thread spent launching batches */
} xg_server_stats;

/* Start the request server on a context.  From then on the context's streams
 * belong to the server: plain generate, seed and set_state calls return
 * XG_EINVAL until xg_server_stop.  A host thread admits requests, keeps a
 * FIFO per stream (a stream has at most one request on the GPU, so its
 * requests run in submission order and read consecutive words), and whenever
 * one of the lanes is free launches the oldest ready requests as one batch
 * (one replay of the persistent batch kernel's graph).  Batches on different
 * lanes run concurrently, so requests that arrive while others are on the
 * GPU start as soon as a lane and memory free up; while the GPU already has
 * about 1.5 ms of work in flight, new requests wait and gather into larger
 * batches, and long requests are cut into fewer, longer pieces (jump-ahead
 * work only pays while the GPU would otherwise idle).  Each result is identical
 * to the same request run alone.  Start-up allocates the pool, each lane's
 * buffers and the jump-ahead powers (about 70 MiB) so that serving itself
 * does not allocate.  A request whose batch fails to launch is
 * reported as XG_EDEVICE by xg_poll / xg_wait and leaves its stream where it
 * was; the server keeps serving.  (For testing that path without a GPU
 * fault, the environment variable XG_INJECT_LAUNCH_FAILURES=N, read at
 * start, makes the first N batch launches fail on the host.)  Tracing:
 * XG_SERVER_TRACE=<path>, read at start, records every batch (lane, items,
 * units, words, host launch time, GPU time between events around the launch)
 * and the scheduler loop's time split, written as CSV by xg_server_stop. */
xg_status xg_server_start(xg_ctx* ctx, const xg_server_config* cfg);

/* Stop the server thread after the batches in flight finish; frees the pool
 * (pool results become invalid). */
xg_status xg_server_stop(xg_ctx* ctx);

/* Non-blocking.  Ticket numbers are nonzero and grow in submission order
 * (not consecutively).  XG_EAGAIN when admitting the request would put the
 * outstanding output bytes above the cap (retry later, after xg_release);
 * XG_EINVAL for a request larger than the cap itself, which could never be
 * admitted. */
xg_status xg_submit(xg_ctx* ctx, const xg_request* req, uint64_t* ticket);

/* Non-blocking bulk submission: admits reqs[0 .. n) in order, as n calls of
 * xg_submit would, taking the server's lock once.  tickets[i] receives the
 * ticket of each admitted request and *n_accepted how many were admitted.
 * XG_OK when all were; XG_EAGAIN when the cap (or the pool) refused request
 * *n_accepted, the ones before it staying admitted (resubmit the rest later);
 * XG_EINVAL, with nothing admitted, when any request is invalid. */
xg_status xg_submit_many(xg_ctx* ctx, const xg_request* reqs, uint32_t n, uint64_t* tickets,
                         uint32_t* n_accepted);

/* Non-blocking.  *done = 1 once the request's outputs are in device memory
 * and visible to later work on any stream; *d_result is then its output
 * pointer.  XG_EDEVICE if the request's batch failed to run. */
xg_status xg_poll(xg_ctx* ctx, uint64_t ticket, int* done, void** d_result);

/* Poll until done or timeout_ms elapses (XG_ETIMEDOUT). */
xg_status xg_wait(xg_ctx* ctx, uint64_t ticket, uint32_t timeout_ms, void** d_result);

/* Forget a finished (or cancelled) ticket and return its bytes (and pool
 * buffer) to the cap. */
xg_status xg_release(xg_ctx* ctx, uint64_t ticket);

/* Cancel a request that has not been launched yet: it will never run, its
 * stream does not advance for it (the stream's later requests read the words
 * it would have read), and xg_poll / xg_wait report XG_ECANCELED for it from
 * now on (xg_collect too, once the scheduler has dropped it); release it as
 * any other ticket.  XG_EINVAL if the request is already on the GPU or
 * finished (it then completes normally), XG_ENOTFOUND for an unknown ticket. */
xg_status xg_cancel(xg_ctx* ctx, uint64_t ticket);

/* Server clock timestamps of a ticket: submission, batch launch, completion
 * as seen by the host (0 while pending). */
xg_status xg_ticket_times(xg_ctx* ctx, uint64_t ticket, uint64_t* t_submit_ns,
                          uint64_t* t_launch_ns, uint64_t* t_done_ns);

xg_status xg_server_stats_get(xg_ctx* ctx, xg_server_stats* out);

typedef struct {
    uint64_t ticket;
    uint64_t t_submit_ns, t_launch_ns, t_done_ns; /* server clock */
    int32_t status;                               /* XG_OK, XG_EDEVICE if its batch failed,
                                                     XG_ECANCELED if it was cancelled */
    uint32_t pad;
    void* d_result;                               /* output pointer (NULL once released) */
} xg_completion;

/* Drain finished requests in bulk: up to max of them, oldest completion
 * first, into out[0 .. *n_out).  With release != 0 each is also released as
 * by xg_release (a pool buffer is then gone: use it only for requests whose
 * output went to caller memory, or whose data is no longer needed).  Each
 * finished ticket is reported once; tickets released by their owner before
 * they are collected are skipped. */
xg_status xg_collect(xg_ctx* ctx, xg_completion* out, uint32_t max, uint32_t* n_out, int release);

/* ---- launch configuration --------------------------------------------- */

/* Threads per generator (tpg) and words per thread per round (wpl) used for
 * an output type; tpg*wpl is the round width (32 or 64 words, never more than
 * s, so that every word of a round depends only on earlier rounds, Sec. 2).
 * Supported pairs: (4,8) (8,4) (16,2) (16,4) (32,2).  0,0 = autotune. */
xg_status xg_set_launch(xg_ctx* ctx, xg_type type, uint32_t tpg, uint32_t wpl);
xg_status xg_get_launch(const xg_ctx* ctx, xg_type type, uint32_t* tpg, uint32_t* wpl);

/* Autotuner: time every supported (tpg, wpl) with 32, 64, 128 and 256
 * threads per block on a slice of the workload (nstreams streams -- 0 = all
 * -- by up to n_per_stream outputs, at most 2^28 outputs in all; the median
 * of five launches each), keep the fastest for later calls of this type and
 * return it (outputs may be NULL; best_ms is that median).
 * The streams do not advance: their state is saved and restored around the
 * timing runs.  Synchronous; allocates a temporary buffer for the slice. */
xg_status xg_autotune(xg_ctx* ctx, xg_type type, uint32_t nstreams, uint64_t n_per_stream,
                      uint32_t* tpg, uint32_t* wpl, uint32_t* block, float* best_ms);

/* ---- errors ------------------------------------------------------------- */

/* Thread-local description of the last failure on this thread ("" if none). */
const char* xg_last_error(void);

/* Library version string. */
const char* xg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* XORGENS_GB300_H */
