// Batched generation that allocates nothing.
//
// xg_generate_batch keeps its batch description in device scratch that it
// allocates (cudaMalloc, pinned staging) the first time it needs it or when a
// batch outgrows it.  Some callers cannot allow that once they are running:
// an application whose memory is entirely managed by another allocator (a
// framework's caching allocator that owns the device budget), or a
// latency-critical loop where cudaMalloc's implicit device synchronisation is
// not acceptable.  For them, xg_generate_batch_noalloc runs the same
// persistent batch kernel with its scratch in the file-scope device array
// below instead.  Every GPU that loads this library holds that array (about
// 48 KiB) until the process exits.
//
// The batch description is assembled in a file-scope host buffer (about
// 86 KiB with the planner's tables), not on the caller's stack, so threads
// with small stacks can call this; calls from different threads take turns
// on that buffer.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "xg_kernels.cuh"
#include "xg_runtime.h"

namespace {

// At most this many items per call.
constexpr uint32_t kNoallocMaxItems = 1024;
constexpr size_t kNoallocItemsOffset = xg::batch_items_offset(kNoallocMaxItems);
constexpr size_t kNoallocScratchBytes = kNoallocItemsOffset + (size_t)kNoallocMaxItems * sizeof(xg::BatchItem);

// The scratch: header (with the work counter), task words, chain heads,
// items.  Shared by every call on a device and left holding the last call's
// batch.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device
int g_max_grid[kMaxDevices][2] = {};     // persistent grid per device and parameter set

// Host-side planning buffers, one set for the process (guarded by g_stage_mu).
constexpr uint32_t kSlots = 2 * kNoallocMaxItems;  // stream -> chain, open addressing
struct Stage {
    alignas(16) unsigned char desc[kNoallocScratchBytes];  // image of the device scratch
    uint64_t chain_words[kNoallocMaxItems];
    uint32_t head_pos[kNoallocMaxItems];
    uint32_t sorted[kNoallocMaxItems];
    uint32_t slot_stream[kSlots], slot_last[kSlots], slot_head[kSlots];
    bool slot_used[kSlots];
};
std::mutex g_stage_mu;
Stage g_stage;

uint64_t item_words(uint32_t type, uint64_t count)
{
    return type == XG_NORMAL_F32 ? count + (count & 1u) : count;
}

}  // namespace

namespace xg {

// Once per device, with that device current: the device address of the
// array (the host-side symbol is only a stand-in) and the kernel's grid.
// Called by xg_create_streams, so that the module holding the array and the
// kernel is loaded there and not by the first xg_generate_batch_noalloc.
xg_status noalloc_setup(int dev, int sm_count)
{
    if (dev < 0 || dev >= kMaxDevices) return XG_OK;  // such a device is refused at call time
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (g_scratch_addr[dev]) return XG_OK;
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return xg::cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    for (int ps = 0; ps < 2; ++ps) {
        int blocks = 0;
        const void* fn = ps == 1 ? reinterpret_cast<const void*>(&xg::batch_kernel<xg::ParamsPaper, false>)
                                 : reinterpret_cast<const void*>(&xg::batch_kernel<xg::ParamsDefault, false>);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, 128, 0);
        if (e != cudaSuccess) return xg::cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        g_max_grid[dev][ps] = std::max(1, blocks) * sm_count;
    }
    g_scratch_addr[dev] = ptr;
    return XG_OK;
}

}  // namespace xg

extern "C" xg_status xg_generate_batch_noalloc(xg_ctx* ctx, const xg_item* items, uint32_t n_items)
{
    using xg::fail;
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (n_items == 0) return XG_OK;
    if (!items) return fail(XG_EINVAL, "null items");
    if (n_items > kNoallocMaxItems)
        return fail(XG_EINVAL, "xg_generate_batch_noalloc takes at most %u items per call (got %u)",
                    kNoallocMaxItems, n_items);
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return fail(XG_EINVAL, "device %d unsupported", ctx->device);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != ctx->device)
        return fail(XG_EINVAL, "the context's device (%d) must be current (it is %d)", ctx->device, cur);

    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->server) return fail(XG_EINVAL, "the request server owns this context; use xg_submit");
    if (xg_status st = xg::noalloc_setup(ctx->device, ctx->sm_count)) return st;  // no-op after create

    std::lock_guard<std::mutex> lk_stage(g_stage_mu);
    Stage& S = g_stage;
    auto* hdr = reinterpret_cast<xg::BatchHeader*>(S.desc);
    auto* tasks = reinterpret_cast<uint32_t*>(S.desc + sizeof(xg::BatchHeader));
    auto* heads = reinterpret_cast<uint32_t*>(S.desc + xg::batch_members_offset(kNoallocMaxItems));
    auto* dev_items = reinterpret_cast<xg::BatchItem*>(S.desc + kNoallocItemsOffset);
    std::memset(S.slot_used, 0, sizeof S.slot_used);
    uint32_t n_heads = 0;
    for (uint32_t i = 0; i < n_items; ++i) {
        const xg_item& it = items[i];
        if (it.stream >= ctx->n) return fail(XG_EINVAL, "item %u: stream %u out of range", i, it.stream);
        if (it.type > XG_NORMAL_F32) return fail(XG_EINVAL, "item %u: unknown type %u", i, it.type);
        if (it.count > 0 && !it.out) return fail(XG_EINVAL, "item %u: null output", i);
        if (reinterpret_cast<uintptr_t>(it.out) & 3u) return fail(XG_EINVAL, "item %u: output not 4-byte aligned", i);
        dev_items[i] = xg::BatchItem{it.stream, it.type, it.count, it.out, nullptr, xg::kNoItem, 0u};
        uint32_t h = (it.stream * 2654435761u) & (kSlots - 1);
        while (S.slot_used[h] && S.slot_stream[h] != it.stream) h = (h + 1) & (kSlots - 1);
        if (!S.slot_used[h]) {
            S.slot_used[h] = true;
            S.slot_stream[h] = it.stream;
            S.slot_last[h] = i;
            S.slot_head[h] = n_heads;
            heads[n_heads] = i;
            S.chain_words[n_heads] = item_words(it.type, it.count);
            ++n_heads;
        } else {
            dev_items[S.slot_last[h]].next = i;
            S.slot_last[h] = i;
            S.chain_words[S.slot_head[h]] += item_words(it.type, it.count);
        }
    }
    // longest chain first (ties in submission order)
    for (uint32_t k = 0; k < n_heads; ++k) S.head_pos[k] = k;
    std::sort(S.head_pos, S.head_pos + n_heads, [&](uint32_t a, uint32_t b) {
        return S.chain_words[a] != S.chain_words[b] ? S.chain_words[a] > S.chain_words[b] : a < b;
    });
    for (uint32_t k = 0; k < n_heads; ++k) S.sorted[k] = heads[S.head_pos[k]];
    std::memcpy(heads, S.sorted, (size_t)n_heads * 4);
    // one chain task per head (one stream per warp)
    for (uint32_t k = 0; k < n_heads; ++k) tasks[k] = xg::task_word(xg::kShapeChain, k);
    // the work counter starts at zero on every call
    *hdr = xg::BatchHeader{0u, n_heads, n_items, kNoallocMaxItems};

    void* scratch = g_scratch_addr[ctx->device];
    const size_t used = kNoallocItemsOffset + (size_t)n_items * sizeof(xg::BatchItem);
    // from pageable host memory: returns once the source has been read, so
    // the buffer may be reused as soon as this call returns
    cudaError_t e = cudaMemcpyAsync(scratch, S.desc, used, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return xg::cuda_fail(e, "cudaMemcpyAsync(noalloc batch)");
    xg::BatchArgs a{};
    a.st = ctx->st;
    a.hdr = static_cast<xg::BatchHeader*>(scratch);
    a.omega = ctx->weyl_on ? 0x9E3779B9u : 0u;
    const int ps = ctx->param_set == 1 ? 1 : 0;
    const unsigned grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((uint64_t)g_max_grid[ctx->device][ps], (n_heads + 3) / 4));
    if (ps == 1) xg::batch_kernel<xg::ParamsPaper, false><<<grid, 128, 0, ctx->stream>>>(a);
    else xg::batch_kernel<xg::ParamsDefault, false><<<grid, 128, 0, ctx->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return xg::cuda_fail(e, "noalloc batch kernel launch");
    return XG_OK;
}
