/*
 * xorgens_gb300, 64-bit words -- C ABI of the w = 64 member of the xorgens
 * family with FP64 uniforms (arXiv:1108.0486, Sec. 1.5: periods 2^n - 1 for
 * n = r w a power of two up to 4096; the Weyl generator and Eq. (1) are
 * stated for a general word length w).
 *
 *   x_k = x_{k-r}(I + L^a)(I + R^b) xor x_{k-s}(I + L^c)(I + R^d)   (Sec. 2)
 *   w_k = w_{k-1} + omega mod 2^64, omega = 0x9E3779B97F4A7C15      (Sec. 1.5)
 *   out_k = x_k + (w_k xor (w_k >> 32)) mod 2^64                    (Eq. 1)
 *
 * (r,s,a,b,c,d) = (64, 55, 42, 27, 25, 22): r w = 4096 state bits as in the
 * 32-bit sets.  The paper gives no 64-bit set; this one comes from this
 * library's own search and its characteristic polynomial is primitive
 * (period 2^4096 - 1 of the linear part; with the Weyl word, 2^64 times more).
 *
 * Seeding: v = seed * 2^32 + (~seed mod 2^32); 64 outputs of Marsaglia's
 * xorshift64 (13, 7, 17) are discarded, the next 64 fill the ring (oldest
 * first), the next one is the Weyl word; an all-zero ring gets x = 1 in its
 * oldest word; then 4r = 256 words are generated and discarded.
 *
 * FP64 uniform: (out >> 11) * 2^-53, exact, in [0, 1).
 *
 * Conventions are those of xorgens_gb300.h (status codes, xg_last_error(),
 * device or host outputs, asynchronous on the context's CUDA stream, calls on
 * one context from one host thread at a time, and any split of a stream's
 * outputs into consecutive calls concatenating to one call's output).
 * Contexts of this header are distinct from xg_ctx: batching and the request
 * server are for the 32-bit generators only; jump-ahead (xg_w64_jump) exists
 * for both.
 */
#ifndef XORGENS_W64_H
#define XORGENS_W64_H

#include <stddef.h>
#include <stdint.h>

#include "xorgens_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xg_w64_ctx xg_w64_ctx; /* opaque, owned by the library */

typedef enum {
    XG_W64_U64 = 0,         /* the output word itself, Eq. (1) */
    XG_W64_UNIFORM_F64 = 1  /* (out >> 11) * 2^-53 */
} xg_w64_type;

/* The parameter set (r, s, a, b, c, d) and omega compiled into the kernels. */
xg_status xg_w64_params(uint32_t* host_rsabcd6, uint64_t* omega);

/* Create n_streams 64-bit generators on the current device, state resident
 * in device memory (96 words + Weyl word + position per stream, 788 bytes),
 * all zero until seeded.  weyl_on: 1 for Eq. (1), 0 for the bare recurrence.
 * cuda_stream: the CUDA stream for all work (NULL: legacy default stream). */
xg_status xg_w64_create(xg_w64_ctx** out, uint32_t n_streams, uint32_t weyl_on, void* cuda_stream);
xg_status xg_w64_destroy(xg_w64_ctx* ctx);
xg_status xg_w64_set_stream(xg_w64_ctx* ctx, void* cuda_stream);

/* Seed streams [first, first + count) with host_seeds[0 .. count) (see the
 * seeding above); positions restart at 0.  Asynchronous. */
xg_status xg_w64_seed(xg_w64_ctx* ctx, uint32_t first, uint32_t count, const uint32_t* host_seeds);

/* Copy one stream's state to the host: host_ring64 receives the 64 ring
 * words oldest first (the next word computed is from these), *weyl the Weyl
 * word of the last consumed output.  Synchronises the context's stream. */
xg_status xg_w64_get_state(xg_w64_ctx* ctx, uint32_t stream, uint64_t* host_ring64, uint64_t* weyl);
/* Restore a state of xg_w64_get_state (or any state with a nonzero ring).
 * Synchronises the context's stream. */
xg_status xg_w64_set_state(xg_w64_ctx* ctx, uint32_t stream, const uint64_t* host_ring64, uint64_t weyl);

/* n_per_stream outputs from each of streams [first, first + nstreams), row t
 * (stream first + t) at out + t * ld (elements of 8 bytes; ld >= n_per_stream
 * when nstreams > 1).  out: device memory (8-byte aligned; rows 16-byte
 * aligned for the vector store path) or host memory (staged through device
 * buffers; returns when the data is on the host).  Streams advance by
 * n_per_stream. */
xg_status xg_w64_generate_u64(xg_w64_ctx* ctx, uint32_t first, uint32_t nstreams, uint64_t n_per_stream,
                              uint64_t* out, uint64_t ld);
xg_status xg_w64_generate_uniform_f64(xg_w64_ctx* ctx, uint32_t first, uint32_t nstreams,
                                      uint64_t n_per_stream, double* out, uint64_t ld);

/* The FP64 uniform conversion alone: d_out[i] = (d_words[i] >> 11) * 2^-53
 * for n given 64-bit words (device memory, 8-byte aligned; may not overlap).
 * Asynchronous. */
xg_status xg_w64_transform_uniform_f64(xg_w64_ctx* ctx, const uint64_t* d_words, uint64_t n, double* d_out);

/* Launch shape per output type: tpg lanes per stream x wpl words per lane,
 * tpg * wpl = 32: (4,8) (8,4) (16,2) (32,1); (0,0) restores the automatic
 * choice.  block 0 = the configuration's default threads per block. */
xg_status xg_w64_set_launch(xg_w64_ctx* ctx, xg_w64_type type, uint32_t tpg, uint32_t wpl, uint32_t block);
/* Time every launch shape and block size on nstreams x n_per_stream (a
 * bounded slice of it) and keep the fastest for this type.  Stream states are
 * saved and restored.  Synchronous.  Outputs may be NULL. */
xg_status xg_w64_autotune(xg_w64_ctx* ctx, xg_w64_type type, uint32_t nstreams, uint64_t n_per_stream,
                          uint32_t* tpg, uint32_t* wpl, uint32_t* block, float* best_ms);

/* Long calls on few streams (at most 16 streams, at least 2^18 words each,
 * device output) are cut into pieces that run on many warps at once, each
 * starting from the stream's state jumped ahead by its offset (xg_w64_jump's
 * matrices); the output and the stream's final state are exactly those of
 * the uncut call.  piece_words: 0 = automatic (about four pieces per SM
 * sub-partition in all, at least 2^16 words), 1 = never cut, else a power of
 * two >= 64.  XG_EINVAL for other values. */
xg_status xg_w64_set_split(xg_w64_ctx* ctx, uint64_t piece_words);

/* Jump-ahead: advance streams [first, first+nstreams) by `words` positions
 * without generating them, exactly as if that many words had been drawn.
 * The recurrence is linear over GF(2) on the 4096-bit ring (Sec. 2), so the
 * jump is a product of powers M^(2^k) of its transition matrix, one per set
 * bit of `words`; the Weyl word advances by words * omega mod 2^64 (Sec. 1.5).
 * The first use of each power builds it on the GPU (2 MiB each, kept until
 * the process exits).  Synchronous.  Errors: XG_EINVAL for a null context or
 * a stream range out of bounds, XG_ENOMEM / XG_ECUDA from the device. */
xg_status xg_w64_jump(xg_w64_ctx* ctx, uint32_t first, uint32_t nstreams, uint64_t words);

/* Seed streams [first, first+count) as consecutive, disjoint blocks of one
 * sequence: stream first + i starts at position i * 2^log2_spacing of the
 * sequence that xg_w64_seed gives for `seed` (as xg_seed_substreams does for
 * the 32-bit generators).  Requires (count - 1) * 2^log2_spacing < 2^64, else
 * XG_EINVAL; also XG_EINVAL for a stream range out of bounds.  Synchronous. */
xg_status xg_w64_seed_substreams(xg_w64_ctx* ctx, uint32_t first, uint32_t count, uint32_t seed,
                                 uint32_t log2_spacing);

#ifdef __cplusplus
}
#endif

#endif /* XORGENS_W64_H */
