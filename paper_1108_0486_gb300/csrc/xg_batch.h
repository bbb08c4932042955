// Batch launcher: a CUDA graph of two nodes -- copy the batch description
// from pinned host staging into device scratch, then the persistent batch
// kernel -- instantiated once per launcher and updated (copy size, grid) per
// launch.  Long calls alone on their stream are cut into pieces whose start
// states come from a jump-ahead prologue launched just before the graph.
#pragma once

#include <cstdint>
#include <vector>

#include "xg_launch.h"
#include "xorgens_gb300.h"

struct xg_ctx;

namespace xg {

struct HostItem {
    uint32_t stream;
    uint32_t kind;
    uint64_t count;
    void* out;
    uint32_t* flag;  // device pointer of a completion counter, or null
};

struct BatchPlan {
    std::vector<BatchItem> units;        // device items (whole calls and pieces)
    std::vector<uint32_t> heads;         // chain heads, costliest chain first
    std::vector<uint32_t> tasks;         // task words (shape << 28 | first member), costliest first
    std::vector<uint32_t> members;       // chain heads by task; kNoItem fills a group's unused slots
    std::vector<uint64_t> chain_words;   // estimated cost per chain, same order
    std::vector<BatchPiece> pieces;      // ring/weyl pointers filled at launch
    std::vector<uint32_t> piece_stream;  // stream of each piece
    std::vector<uint64_t> piece_skip;    // words of its call before each piece
    std::vector<uint32_t> piece_index;   // m: the piece starts m * 2^split_log2 words in
    std::vector<uint32_t> units_per_item;
    int split_log2 = 0;                  // piece length 2^split_log2 (when pieces exist)
    // dense per-stream scratch, all zero between calls
    std::vector<uint32_t> items_of_stream, last_unit, chain_of;
    // the head ordering's buffers, reused between calls
    std::vector<uint32_t> sort_start, sort_key, sort_heads;
    std::vector<uint64_t> sort_cost;
};

// Plan a batch.  piece_len: 0 = cut nothing, else a power of two; calls alone
// on their stream with at least 2 * piece_len words are cut into pieces of
// piece_len words (the last one shorter).  shapes (per output type, null =
// kShapeChain for all): the task shape for single-call chains of that type
// whose output is 16-byte aligned; every other chain is a chain task.
void plan_batch(const HostItem* items, uint32_t n, uint64_t piece_len, uint32_t n_streams, BatchPlan& plan,
                const uint8_t* shapes = nullptr, uint64_t group_max_words = ~uint64_t(0));
// Tasks from the ordered heads: consecutive single-call chains of one type
// (hence of similar cost) with at most group_max_words words fill groups of
// that type's shape; longer units stay chains, so that a group (which runs
// each of its units at 1/G of a warp's rate) never becomes the batch's tail.
void plan_tasks(BatchPlan& plan, const uint8_t* shapes, uint64_t group_max_words);

class BatchLauncher {
public:
    ~BatchLauncher();
    // Grow to hold `capacity` units (re-creates the graph when it grows).
    xg_status reserve(xg_ctx* c, uint32_t capacity);
    // Plan, stage, run the jump prologue if needed, and replay the graph on
    // stream s.  Waits first for this launcher's previous replay to finish
    // reading its staging buffers.  units_per_item (optional, n entries)
    // receives how many completion increments each item will produce.
    // min_piece: the shortest piece the automatic choice may cut (a caller
    // that knows the GPU is already busy raises it: cutting buys latency at
    // the price of jump-ahead work, about 2.2e4 words' worth per piece).
    xg_status launch(xg_ctx* c, const HostItem* items, uint32_t n, cudaStream_t s,
                     uint32_t* units_per_item = nullptr, uint64_t min_piece = kMinPiece);
    // 2^15: on an idle GPU the serving p99 is lowest there (2^14 and 2^13 add
    // more jump-ahead than they save; 2^16 leaves longer chains)
    static constexpr uint64_t kMinPiece = uint64_t(1) << 15;
    // Preallocate the jump prologue's buffers for up to `pieces` pieces (so
    // that a later launch does not allocate).
    xg_status reserve_jump(uint32_t pieces, uint32_t pairs);
    size_t scratch_bytes() const { return bytes_; }
    cudaEvent_t done_event() const { return done_; }
    bool busy() const;

private:
    xg_status build_graph(xg_ctx* c);
    xg_status prologue(xg_ctx* c, cudaStream_t s);
    xg_status grow_jump(size_t want);
    uint64_t choose_piece_len(const xg_ctx* c, const HostItem* items, uint32_t n, uint64_t min_piece) const;
    uint32_t capacity_ = 0;
    size_t bytes_ = 0;
    void* h_staging_ = nullptr;   // pinned
    void* d_scratch_ = nullptr;
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    cudaGraphNode_t copy_node_ = nullptr;
    cudaGraphNode_t kernel_node_ = nullptr;
    cudaEvent_t done_ = nullptr;
    bool launched_ = false;
    BatchArgs args_{};
    int max_grid_ = 0;          // resident blocks of the variant without group paths
    int max_grid_g_[2] = {0, 0};  // per variant (without, with group paths)
    BatchPlan plan_;
    // jump-ahead prologue buffers
    void* h_jstage_ = nullptr;
    void* d_jbuf_ = nullptr;
    size_t jbytes_ = 0;
};

}  // namespace xg
