// The library's context object (the C ABI's opaque xg_ctx).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "xg_launch.h"
#include "xorgens_gb300.h"

namespace xg {
class Server;
class BatchLauncher;
// Set the calling thread's xg_last_error() message and return st.
xg_status fail(xg_status st, const char* fmt, ...);
xg_status cuda_fail(cudaError_t e, const char* what);
// Device set-up of xg_generate_batch_noalloc (its scratch array's address and
// the batch kernel's grid), done once per device by xg_create_streams.
xg_status noalloc_setup(int dev, int sm_count);
}

struct xg_ctx {
    int device = 0;
    int sm_count = 148;
    uint32_t n = 0;            // streams
    uint32_t param_set = 0;    // 0: (128,95,17,12,13,15), 1: (128,65,15,14,12,17)
    uint32_t weyl_on = 1;
    cudaStream_t stream = nullptr;  // caller-owned
    void* state_mem = nullptr;
    xg::State st{};
    int cfg[3] = {-1, -1, -1};      // per output type; -1 = automatic
    int blk[3] = {0, 0, 0};         // tuned threads per block per output type; 0 = the cfg's default
    int block[xg::kNumCfgs] = {};   // threads per block per configuration
    // host-output staging: kStage device buffers, each with its own copy stream
    static constexpr int kStage = 4;
    void* staging[kStage] = {};
    size_t staging_bytes = 0;
    cudaStream_t copy_stream[kStage] = {};
    cudaEvent_t ev_gen[kStage] = {};
    cudaEvent_t ev_copy[kStage] = {};
    std::mutex mu;
    xg::Server* server = nullptr;
    xg::BatchLauncher* batch[2] = {nullptr, nullptr};
    int batch_next = 0;
    uint64_t split_words = 0;  // batch piece length: 0 automatic, 1 never, else forced
    // batch kernel task shape per output type (xg::kShape*): single-call
    // chains of that type are grouped; set by xg_set_batch_shape or
    // xg_autotune_batch
    uint8_t batch_shape[3] = {xg::kShapeChain, xg::kShapeChain, xg::kShapeChain};

    // xg_jump's workspace (grow-only, freed by xg_destroy)
    void* jump_ws = nullptr;
    size_t jump_ws_bytes = 0;

    int pick_cfg(int kind, uint32_t nstreams) const;
    int pick_block(int kind, int cfg) const;
    xg_status ensure_staging(size_t bytes);
    xg_status ensure_jump_ws(size_t bytes);
    void shutdown_server();
};

namespace xg {
using Ctx = xg_ctx;
}
