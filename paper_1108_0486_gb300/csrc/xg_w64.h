// Internal interface of the 64-bit-word generator (w = 64) between the host
// runtime (xg_runtime64.cpp) and its kernels (xg_w64.cu).  Plain C++.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace xg64 {

// (r, s, a, b, c, d): r = 64 words of 64 bits, so n = r w = 4096 as for the
// 32-bit sets.  The paper gives no 64-bit set; this one was found by a search
// over s odd in [41, 55] and shifts in [16, 48] and has a primitive
// characteristic polynomial of degree 4096 (period 2^4096 - 1 of the linear
// part, Sec. 1.5).
constexpr int kR = 64, kS = 55, kA = 42, kB = 27, kC = 25, kD = 22;
// Weyl increment: the odd integer nearest 2^63 (sqrt 5 - 1) (Sec. 1.5).
constexpr uint64_t kOmega = 0x9E3779B97F4A7C15ull;
// Output shift gamma = w / 2 (Eq. 1).
constexpr int kGamma = 32;

// Rounds are 32 words (a round reads words at least s >= 32 back), so the
// per-stream window holds the 64-word ring and up to 31 pending words:
// ring = window[kRingBase - pend, kRingBase - pend + 64).
constexpr int kRW = 32;
constexpr int kWin = kR + kRW;
constexpr int kRingBase = kRW;

struct State {
    uint64_t* win;   // [n][kWin]
    uint64_t* weyl;  // [n] Weyl word at the consumed position
    uint32_t* pend;  // [n] words computed beyond the consumed position (< 32)
    uint64_t* pos;   // [n] words consumed since seeding
};

enum OutKind { kU64 = 0, kUniformF64 = 1 };

struct GenArgs {
    State st;
    uint32_t first;
    uint32_t nstreams;
    uint64_t n;       // outputs per stream
    void* out;        // stream-major, 8-byte elements
    uint64_t ld;      // elements between consecutive streams' outputs
    uint64_t omega;   // kOmega, or 0 with the Weyl generator off
};

// Launch configurations: lanes per stream x words per lane = 32.
struct LaunchCfg {
    int tpg, wpl, block;
};
constexpr int kNumCfgs = 4;
extern const LaunchCfg kCfgs[kNumCfgs];  // (4,8) (8,4) (16,2) (32,1)
int cfg_index(int tpg, int wpl);

cudaError_t launch_seed(const State& st, const uint32_t* d_seeds, uint32_t first, uint32_t count,
                        cudaStream_t s);
cudaError_t launch_gen(int cfg, int kind, bool vec, int block, const GenArgs& a, cudaStream_t s);
cudaError_t launch_transform_uniform(const uint64_t* in, uint64_t n, uint64_t* out, int sms, cudaStream_t s);

// Jump-ahead.  The 64-word ring is a 4096-bit state like the 32-bit sets'
// 128-word ring (bit j = bit j mod 64 of word j / 64, the same bits as
// 32-bit word j / 32 on a little-endian device), so the GF(2) matrix powers
// and their application are shared with the 32-bit generators.
// Columns of the one-step matrix: column j (64 words) = one step from e_j.
cudaError_t launch_step_columns(uint64_t* cols, cudaStream_t s);
// rings[k] = ring of stream first + k (64 words, oldest first).
cudaError_t launch_gather_rings(const State& st, uint32_t first, uint32_t n, uint64_t* rings, cudaStream_t s);
// Stream first + k takes rings[k] as its ring (pend = 0), its Weyl word
// advanced by jump * omega and its position by jump.
cudaError_t launch_scatter_rings(const State& st, uint32_t first, uint32_t n, const uint64_t* rings, uint64_t jump,
                                 uint64_t omega, cudaStream_t s);
// Substreams: stream first + m takes rings[m] (pend = 0), the Weyl word
// *w0 advanced by m 2^q omega, and position m 2^q.
cudaError_t launch_substream_scatter(const State& st, uint32_t first, uint32_t n, const uint64_t* rings,
                                     const uint64_t* w0, int q, uint64_t omega, cudaStream_t s);

// Cut calls: a long call on stream first + i is generated as K pieces of L
// words, piece m by stream i K + m of a scratch state `pieces` whose ring is
// rings[i K + m] (the real ring advanced m L words) and whose Weyl word is
// the real one advanced by m L omega.
cudaError_t launch_init_pieces(const State& real, uint32_t first, uint32_t nstreams, uint32_t K, uint64_t L,
                               const uint64_t* rings, const State& pieces, uint64_t omega, cudaStream_t s);
// After the pieces ran: stream first + i takes the state of its last piece
// (window, Weyl word, pending words) and its position advances by n.
cudaError_t launch_adopt_last_piece(const State& real, uint32_t first, uint32_t nstreams, uint32_t K,
                                    const State& pieces, uint64_t n, cudaStream_t s);

}  // namespace xg64
