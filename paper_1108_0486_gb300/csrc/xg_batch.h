// Batch launcher: a CUDA graph of two nodes -- copy the batch description
// from pinned host staging into device scratch, then the persistent batch
// kernel -- instantiated once per launcher and updated (copy size, grid) per
// launch.
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
    uint32_t* flag;  // device pointer of a completion flag, or null
};

class BatchLauncher {
public:
    ~BatchLauncher();
    // Grow to hold `capacity` items (re-creates the graph when it grows).
    xg_status reserve(xg_ctx* c, uint32_t capacity);
    // Build chains (items of one stream, in order), sort chain heads longest
    // first, stage, and replay the graph on stream s.  Waits first for this
    // launcher's previous replay to finish reading its staging buffer.
    xg_status launch(xg_ctx* c, const HostItem* items, uint32_t n, cudaStream_t s);
    // Scratch the kernel uses (device), for callers that want its size.
    size_t scratch_bytes() const { return bytes_; }
    cudaEvent_t done_event() const { return done_; }
    bool busy() const;

private:
    xg_status build_graph(xg_ctx* c);
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
    int max_grid_ = 0;
    std::vector<uint32_t> heads_;
    std::vector<uint64_t> chain_words_;
};

// Plan a batch on the host: items -> device items with chain links, and the
// chain heads sorted by total words (longest first).  Exposed for tests.
void plan_batch(const HostItem* items, uint32_t n, std::vector<BatchItem>& out_items,
                std::vector<uint32_t>& heads, std::vector<uint64_t>& chain_words);

}  // namespace xg
