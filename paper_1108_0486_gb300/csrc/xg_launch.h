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

// Tasks of the persistent batch kernel.  A warp takes one task at a time.
// A task word is (shape << 28) | first, `first` indexing the member list:
//   kShapeChain: members[first] heads one chain (the calls on one stream, in
//                order, possibly of different types), 32 lanes per stream,
//                two words per lane per round (64-bit stores);
//   kShape16x4:  members[first .. first+2) are single-call chains of one
//                type, 16 lanes each, four words per lane (128-bit stores);
//   kShape8x4:   members[first .. first+4), 8 lanes each, four words per lane.
// A group's unused member slots hold kNoItem.  Every grouped unit's output
// is 16-byte aligned.
constexpr uint32_t kShapeChain = 0;
constexpr uint32_t kShape16x4 = 1;
constexpr uint32_t kShape8x4 = 2;
constexpr int kNumShapes = 3;
XG_HD inline uint32_t shape_tpg(uint32_t shape) { return shape == kShape16x4 ? 16u : shape == kShape8x4 ? 8u : 32u; }
XG_HD inline uint32_t shape_wpl(uint32_t shape) { return shape == kShapeChain ? 2u : 4u; }
XG_HD inline uint32_t shape_group(uint32_t shape) { return 32u / shape_tpg(shape); }
XG_HD inline uint32_t task_word(uint32_t shape, uint32_t first) { return (shape << 28) | first; }
constexpr uint32_t kTaskFirstMask = 0x0FFFFFFFu;
// Member slots beyond the unit capacity: the partly filled last group of
// each type adds at most 3 empty slots.
constexpr uint32_t kMemberSlack = 16;

// Scratch layout of one batch: header, task words (costliest first), member
// list, then the units at batch_items_offset(capacity) and the pieces.
struct BatchHeader {
    uint32_t counter;   // next task to take (reset to 0 by every launch)
    uint32_t n_tasks;
    uint32_t n_items;
    uint32_t capacity;  // units the scratch can hold
};

XG_HD constexpr size_t batch_members_offset(uint32_t capacity)
{
    return sizeof(BatchHeader) + (size_t)capacity * 4;
}
XG_HD constexpr size_t batch_items_offset(uint32_t capacity)
{
    return (batch_members_offset(capacity) + ((size_t)capacity + kMemberSlack) * 4 + 15) / 16 * 16;
}
XG_HD constexpr size_t batch_pieces_offset(uint32_t capacity)
{
    return batch_items_offset(capacity) + (size_t)capacity * sizeof(BatchItem);
}
XG_HD constexpr size_t batch_scratch_bytes(uint32_t capacity)
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
// The persistent batch kernel of a parameter set; groups: the variant with
// the group-task paths.
const void* batch_kernel_ptr(int param_set, bool groups);

// Per parameter set (defined in xg_inst_default.cu / xg_inst_paper.cu).
cudaError_t launch_seed_default(const State&, const uint32_t*, uint32_t, uint32_t, cudaStream_t);
cudaError_t launch_seed_paper(const State&, const uint32_t*, uint32_t, uint32_t, cudaStream_t);
cudaError_t launch_gen_default(int cfg, int out_kind, bool vec, int block, const GenArgs&, cudaStream_t);
cudaError_t launch_gen_paper(int cfg, int out_kind, bool vec, int block, const GenArgs&, cudaStream_t);
const void* batch_kernel_ptr_default(bool groups);
const void* batch_kernel_ptr_paper(bool groups);

}  // namespace xg
