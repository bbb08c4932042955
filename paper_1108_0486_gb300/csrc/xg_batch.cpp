// Batched generation: host planning, the graph launcher, xg_generate_batch.
#include "xg_batch.h"

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <unordered_map>

#include "xg_runtime.h"

namespace xg {

static uint64_t words_of(uint32_t kind, uint64_t count)
{
    return kind == kNormal ? count + (count & 1u) : count;
}

void plan_batch(const HostItem* items, uint32_t n, std::vector<BatchItem>& out,
                std::vector<uint32_t>& heads, std::vector<uint64_t>& chain_words)
{
    out.resize(n);
    heads.clear();
    std::unordered_map<uint32_t, uint32_t> last;   // stream -> last item index
    std::unordered_map<uint32_t, uint32_t> head_of;  // stream -> position in heads
    last.reserve(n * 2);
    head_of.reserve(n * 2);
    std::vector<uint64_t> words;
    for (uint32_t i = 0; i < n; ++i) {
        const HostItem& h = items[i];
        out[i] = BatchItem{h.stream, h.kind, h.count, h.out, h.flag, kNoItem, 0u};
        auto it = last.find(h.stream);
        if (it == last.end()) {
            head_of[h.stream] = (uint32_t)heads.size();
            heads.push_back(i);
            words.push_back(words_of(h.kind, h.count));
            last[h.stream] = i;
        } else {
            out[it->second].next = i;
            it->second = i;
            words[head_of[h.stream]] += words_of(h.kind, h.count);
        }
    }
    std::vector<uint32_t> order(heads.size());
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return words[a] > words[b]; });
    std::vector<uint32_t> sorted(heads.size());
    chain_words.resize(heads.size());
    for (size_t k = 0; k < order.size(); ++k) {
        sorted[k] = heads[order[k]];
        chain_words[k] = words[order[k]];
    }
    heads.swap(sorted);
}

BatchLauncher::~BatchLauncher()
{
    if (done_) cudaEventSynchronize(done_);
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    if (done_) cudaEventDestroy(done_);
    if (h_staging_) cudaFreeHost(h_staging_);
    if (d_scratch_) cudaFree(d_scratch_);
}

bool BatchLauncher::busy() const
{
    if (!launched_) return false;
    return cudaEventQuery(done_) == cudaErrorNotReady;
}

xg_status BatchLauncher::build_graph(xg_ctx* c)
{
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    exec_ = nullptr;
    graph_ = nullptr;
    if (cudaGraphCreate(&graph_, 0) != cudaSuccess) return XG_ECUDA;
    if (cudaGraphAddMemcpyNode1D(&copy_node_, graph_, nullptr, 0, d_scratch_, h_staging_, bytes_,
                                 cudaMemcpyHostToDevice) != cudaSuccess)
        return XG_ECUDA;
    args_.st = c->st;
    args_.hdr = static_cast<BatchHeader*>(d_scratch_);
    args_.omega = c->weyl_on ? 0x9E3779B9u : 0u;
    void* params[] = {&args_};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(batch_kernel_ptr((int)c->param_set));
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(128);
    kp.sharedMemBytes = 0;
    kp.kernelParams = params;
    if (cudaGraphAddKernelNode(&kernel_node_, graph_, &copy_node_, 1, &kp) != cudaSuccess) return XG_ECUDA;
    if (cudaGraphInstantiate(&exec_, graph_, 0) != cudaSuccess) return XG_ECUDA;
    return XG_OK;
}

xg_status BatchLauncher::reserve(xg_ctx* c, uint32_t capacity)
{
    if (capacity <= capacity_ && exec_) return XG_OK;
    if (done_ && launched_) cudaEventSynchronize(done_);
    uint32_t cap = std::max<uint32_t>(64, capacity_);
    while (cap < capacity) cap *= 2;
    if (h_staging_) cudaFreeHost(h_staging_);
    if (d_scratch_) cudaFree(d_scratch_);
    h_staging_ = nullptr;
    d_scratch_ = nullptr;
    capacity_ = 0;
    bytes_ = batch_scratch_bytes(cap);
    if (cudaHostAlloc(&h_staging_, bytes_, cudaHostAllocDefault) != cudaSuccess) return XG_ENOMEM;
    if (cudaMalloc(&d_scratch_, bytes_) != cudaSuccess) return XG_ENOMEM;
    if (!done_ && cudaEventCreateWithFlags(&done_, cudaEventDisableTiming) != cudaSuccess) return XG_ECUDA;
    capacity_ = cap;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_kernel_ptr((int)c->param_set), 128, 0) !=
        cudaSuccess)
        return XG_ECUDA;
    max_grid_ = std::max(1, blocks) * c->sm_count;
    return build_graph(c);
}

xg_status BatchLauncher::launch(xg_ctx* c, const HostItem* items, uint32_t n, cudaStream_t s)
{
    if (xg_status st = reserve(c, n)) return st;
    if (launched_ && cudaEventSynchronize(done_) != cudaSuccess) return XG_ECUDA;
    std::vector<BatchItem> dev_items;
    plan_batch(items, n, dev_items, heads_, chain_words_);
    char* base = static_cast<char*>(h_staging_);
    BatchHeader hdr{0u, (uint32_t)heads_.size(), n, capacity_};
    std::memcpy(base, &hdr, sizeof hdr);
    std::memcpy(base + sizeof hdr, heads_.data(), heads_.size() * 4);
    std::memcpy(base + batch_items_offset(capacity_), dev_items.data(), (size_t)n * sizeof(BatchItem));
    const size_t used = batch_items_offset(capacity_) + (size_t)n * sizeof(BatchItem);
    if (cudaGraphExecMemcpyNodeSetParams1D(exec_, copy_node_, d_scratch_, h_staging_, used,
                                           cudaMemcpyHostToDevice) != cudaSuccess)
        return XG_ECUDA;
    const unsigned grid = (unsigned)std::min<uint64_t>(max_grid_, (heads_.size() + 3) / 4);
    args_.st = c->st;
    void* params[] = {&args_};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(batch_kernel_ptr((int)c->param_set));
    kp.gridDim = dim3(std::max(1u, grid));
    kp.blockDim = dim3(128);
    kp.sharedMemBytes = 0;
    kp.kernelParams = params;
    if (cudaGraphExecKernelNodeSetParams(exec_, kernel_node_, &kp) != cudaSuccess) return XG_ECUDA;
    if (cudaGraphLaunch(exec_, s) != cudaSuccess) return XG_ECUDA;
    if (cudaEventRecord(done_, s) != cudaSuccess) return XG_ECUDA;
    launched_ = true;
    return XG_OK;
}

}  // namespace xg

extern "C" xg_status xg_generate_batch(xg_ctx* ctx, const xg_item* items, uint32_t n_items)
{
    using namespace xg;
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (n_items == 0) return XG_OK;
    if (!items) return fail(XG_EINVAL, "null items");
    if (ctx->server) return fail(XG_EINVAL, "the request server owns this context; use xg_submit");
    std::vector<HostItem> h(n_items);
    for (uint32_t i = 0; i < n_items; ++i) {
        const xg_item& it = items[i];
        if (it.stream >= ctx->n) return fail(XG_EINVAL, "item %u: stream %u out of range", i, it.stream);
        if (it.type > XG_NORMAL_F32) return fail(XG_EINVAL, "item %u: unknown type %u", i, it.type);
        if (it.count > 0 && !it.out) return fail(XG_EINVAL, "item %u: null output", i);
        if (reinterpret_cast<uintptr_t>(it.out) & 3u) return fail(XG_EINVAL, "item %u: output not 4-byte aligned", i);
        h[i] = HostItem{it.stream, it.type, it.count, it.out, nullptr};
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    BatchLauncher*& L = ctx->batch[ctx->batch_next];
    ctx->batch_next ^= 1;
    if (!L) L = new (std::nothrow) BatchLauncher();
    if (!L) return fail(XG_ENOMEM, "host allocation failed");
    xg_status st = L->launch(ctx, h.data(), n_items, ctx->stream);
    if (st != XG_OK) {
        cudaError_t e = cudaGetLastError();
        return fail(st, "batch launch failed (%s)", cudaGetErrorString(e));
    }
    return XG_OK;
}
