// Internal interface between the host runtime and the kernel translation
// units.  Plain C++ (no device code), included by both sides.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace xg {

// Per-stream window of recent words kept in device memory.  The ring that
// the next call starts from is window[kRingBase - pend, kRingBase - pend + 128),
// where pend (< 64, less than one round) counts words already computed past the
// stream's consumed position; they are recomputed, identically, by the next
// call, so every call starts its rounds at its own first word.
constexpr int kWin = 192;
constexpr int kRingBase = 64;

// Device-resident state of a context (structure of arrays).
struct State {
    uint32_t* win;   // [n][kWin]
    uint32_t* weyl;  // [n]  Weyl word at the consumed position
    uint32_t* pend;  // [n]  words computed beyond the consumed position
    uint64_t* pos;   // [n]  words consumed since seeding
};

enum OutKind { kU32 = 0, kUniform = 1, kNormal = 2, kNormalSum = 3 };

struct GenArgs {
    State st;
    uint32_t first;     // first stream
    uint32_t nstreams;  // streams in the call
    uint64_t n;         // outputs per stream
    void* out;          // stream-major outputs (4-byte elements)
    uint64_t ld;        // elements between consecutive streams' outputs
    float* sums;        // fused normal sum: one per stream
    uint32_t omega;     // Weyl increment, 0 when the Weyl generator is off
};

// Launch configurations: lanes per generator (tpg) x words per lane (wpl).
struct LaunchCfg {
    int tpg;
    int wpl;
    int block;  // threads per block
};
constexpr int kNumCfgs = 5;
extern const LaunchCfg kCfgs[kNumCfgs];  // (4,8) (8,4) (16,2) (16,4) (32,2)
int cfg_index(int tpg, int wpl);          // -1 if unsupported

// Launchers (return the launch error, if any).
cudaError_t launch_seed(int param_set, const State& st, const uint32_t* d_seeds,
                        uint32_t first, uint32_t count, cudaStream_t s);
cudaError_t launch_gen(int param_set, int cfg, int out_kind, bool vec, int block,
                       const GenArgs& a, cudaStream_t s);
cudaError_t launch_transform(int out_kind, const uint32_t* in, uint64_t n, float* out,
                             cudaStream_t s);

// Per parameter set (defined in xg_inst_default.cu / xg_inst_paper.cu).
cudaError_t launch_seed_default(const State&, const uint32_t*, uint32_t, uint32_t, cudaStream_t);
cudaError_t launch_seed_paper(const State&, const uint32_t*, uint32_t, uint32_t, cudaStream_t);
cudaError_t launch_gen_default(int cfg, int out_kind, bool vec, int block, const GenArgs&, cudaStream_t);
cudaError_t launch_gen_paper(int cfg, int out_kind, bool vec, int block, const GenArgs&, cudaStream_t);

}  // namespace xg
