// Internal interface between the host runtime and the kernel translation
// units.  Plain C++ (no device code), included by both sides.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#if defined(__CUDACC__)
#define XG_HD __host__ __device__
#else
#define XG_HD
#endif

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

// ---- batches: work items of the persistent batch kernel -----------------
constexpr uint32_t kNoItem = 0xFFFFFFFFu;

struct BatchItem {
    uint32_t stream;   // stream index in the context
    uint32_t kind;     // kU32, kUniform or kNormal
    uint64_t count;    // outputs
    void* out;         // device output (count 4-byte elements)
    uint32_t* flag;    // device-visible completion counter (+1 per finished unit), or null
    uint32_t next;     // next item of the same stream (kNoItem: none)
    uint32_t piece;    // 0: a whole call; k+1: piece k of a split call (BatchPiece k)
};

// A piece of a long call cut at multiples of a power-of-two length: its start
// ring and Weyl word come from the jump-ahead prologue, not from the stream.
struct BatchPiece {
    const uint32_t* ring;   // 128-word start ring, oldest first
    const uint32_t* weyl0;  // Weyl word just before the piece's first word
    uint64_t item_words;    // words of the whole call (the last piece adds them to pos)
    uint32_t last;          // 1: the call's last piece, which writes the stream state back
    uint32_t pad;
};

// Scratch layout of one batch: header, chain heads (u32, longest chain
// first), then the items at batch_items_offset(capacity).
struct BatchHeader {
    uint32_t counter;   // next head to take (reset to 0 by every launch)
    uint32_t n_heads;
    uint32_t n_items;
    uint32_t capacity;  // items the scratch can hold
};

XG_HD inline size_t batch_items_offset(uint32_t capacity)
{
    return (sizeof(BatchHeader) + (size_t)capacity * 4 + 15) / 16 * 16;
}
XG_HD inline size_t batch_pieces_offset(uint32_t capacity)
{
    return batch_items_offset(capacity) + (size_t)capacity * sizeof(BatchItem);
}
XG_HD inline size_t batch_scratch_bytes(uint32_t capacity)
{
    return batch_pieces_offset(capacity) + (size_t)capacity * sizeof(BatchPiece);
}

struct BatchArgs {
    State st;
    BatchHeader* hdr;   // device scratch
    uint32_t omega;
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

// Bulk checkpoint and restore of streams [first, first + n) (128-word rings).
cudaError_t launch_export_states(const State& st, uint32_t first, uint32_t n, uint32_t* rings, uint32_t* weyl,
                                 uint64_t* pos, cudaStream_t s);
cudaError_t launch_import_states(const State& st, uint32_t first, uint32_t n, const uint32_t* rings,
                                 const uint32_t* weyl, const uint64_t* pos, uint32_t weyl_on, cudaStream_t s);
const void* batch_kernel_ptr(int param_set);

// Per parameter set (defined in xg_inst_default.cu / xg_inst_paper.cu).
cudaError_t launch_seed_default(const State&, const uint32_t*, uint32_t, uint32_t, cudaStream_t);
cudaError_t launch_seed_paper(const State&, const uint32_t*, uint32_t, uint32_t, cudaStream_t);
cudaError_t launch_gen_default(int cfg, int out_kind, bool vec, int block, const GenArgs&, cudaStream_t);
cudaError_t launch_gen_paper(int cfg, int out_kind, bool vec, int block, const GenArgs&, cudaStream_t);
const void* batch_kernel_ptr_default();
const void* batch_kernel_ptr_paper();

}  // namespace xg
