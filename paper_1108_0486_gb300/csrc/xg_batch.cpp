// Batched generation: host planning, the graph launcher, xg_generate_batch.
#include "xg_batch.h"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>

#include "xg_gf2_tc.h"
#include "xg_jump.h"
#include "xg_runtime.h"

namespace xg {

// Threads per block of the persistent batch kernel: one warp, so that a
// block retires as soon as its warp finds no more work.  With several batch
// kernels in flight (the server's lanes) a block of four warps would hold
// the registers of all four until its slowest warp ended.
constexpr int kBatchBlock = 32;
constexpr int kWarpsPerBlock = kBatchBlock / 32;

static uint64_t words_of(uint32_t kind, uint64_t count)
{
    return kind == kNormal ? count + (count & 1u) : count;
}

// Relative GPU cost of a word by output kind (GB300 batch kernel: u32 5.3 ms,
// uniforms 6.2 ms, normals 11.6 ms for the same 7.3e9-word batch), used to
// order units longest-running first.
static uint64_t cost_of(uint32_t kind, uint64_t words)
{
    return words * (kind == kNormal ? 18u : kind == kUniform ? 9u : 8u);
}

// Units and pieces of a batch, chains linked, one cost per chain head; the
// heads are not yet ordered (plan_order does that).
static void plan_units(const HostItem* items, uint32_t n, uint64_t piece_len, uint32_t n_streams, BatchPlan& plan)
{
    plan.units.clear();
    plan.heads.clear();
    plan.chain_words.clear();
    plan.pieces.clear();
    plan.piece_stream.clear();
    plan.piece_skip.clear();
    plan.piece_index.clear();
    plan.units_per_item.assign(n, 1u);
    plan.split_log2 = 0;
    if (piece_len) {
        while ((uint64_t(1) << plan.split_log2) < piece_len) ++plan.split_log2;
        piece_len = uint64_t(1) << plan.split_log2;
    }
    if (plan.items_of_stream.size() < n_streams) {
        plan.items_of_stream.assign(n_streams, 0u);
        plan.last_unit.assign(n_streams, 0u);
        plan.chain_of.assign(n_streams, 0u);
    }
    // stream -> items in this batch; last unit of its chain + 1; its chain + 1
    auto& count = plan.items_of_stream;
    auto& last = plan.last_unit;
    auto& chain = plan.chain_of;
    for (uint32_t i = 0; i < n; ++i) ++count[items[i].stream];
    size_t npieces_all = 0;
    if (piece_len) {
        for (uint32_t i = 0; i < n; ++i) {
            const uint64_t w = words_of(items[i].kind, items[i].count);
            if (count[items[i].stream] == 1 && w >= 2 * piece_len) npieces_all += (w + piece_len - 1) / piece_len;
        }
    }
    plan.units.reserve(n + npieces_all);
    plan.heads.reserve(n + npieces_all);
    plan.chain_words.reserve(n + npieces_all);
    plan.pieces.reserve(npieces_all);
    plan.piece_stream.reserve(npieces_all);
    plan.piece_skip.reserve(npieces_all);
    plan.piece_index.reserve(npieces_all);
    auto& words = plan.chain_words;  // cost per head, in head order until plan_order
    for (uint32_t i = 0; i < n; ++i) {
        const HostItem& h = items[i];
        const uint64_t w = words_of(h.kind, h.count);
        if (piece_len && count[h.stream] == 1 && w >= 2 * piece_len) {
            // cut into pieces; each piece is a one-unit chain of its own
            const uint64_t npieces = (w + piece_len - 1) / piece_len;
            plan.units_per_item[i] = (uint32_t)npieces;
            for (uint64_t m = 0; m < npieces; ++m) {
                const uint64_t skip = m * piece_len;
                const uint64_t cnt = std::min<uint64_t>(piece_len, h.count - skip);
                const uint32_t k = (uint32_t)plan.pieces.size();
                BatchPiece pc{};
                pc.item_words = w;
                pc.last = (m + 1 == npieces) ? 1u : 0u;
                plan.pieces.push_back(pc);
                plan.piece_stream.push_back(h.stream);
                plan.piece_skip.push_back(skip);
                plan.piece_index.push_back((uint32_t)m);
                char* out = static_cast<char*>(h.out) + skip * 4;
                plan.heads.push_back((uint32_t)plan.units.size());
                words.push_back(cost_of(h.kind, words_of(h.kind, cnt)));
                plan.units.push_back(BatchItem{h.stream, h.kind, cnt, out, h.flag, kNoItem, k + 1});
            }
            continue;
        }
        const uint32_t u = (uint32_t)plan.units.size();
        plan.units.push_back(BatchItem{h.stream, h.kind, h.count, h.out, h.flag, kNoItem, 0u});
        if (last[h.stream] == 0) {
            chain[h.stream] = (uint32_t)plan.heads.size() + 1;
            plan.heads.push_back(u);
            words.push_back(cost_of(h.kind, w));
        } else {
            plan.units[last[h.stream] - 1].next = u;
            words[chain[h.stream] - 1] += cost_of(h.kind, w);
        }
        last[h.stream] = u + 1;
    }
    for (uint32_t i = 0; i < n; ++i) {
        count[items[i].stream] = 0;
        last[items[i].stream] = 0;
        chain[items[i].stream] = 0;
    }
}

// Order the chain heads costliest first by a counting sort on the cost
// rounded down to 7 significant bits (exponent and 6 bits below the leading
// one: within 1.6% of the exact order); equal keys keep submission order.
// Linear in the number of heads, which runs to tens of thousands when long
// calls are cut.
static uint32_t cost_key(uint64_t c)
{
    if (c < 64) return (uint32_t)c;
    const int e = 63 - __builtin_clzll(c);               // 6 .. 63
    return (uint32_t)((e - 5) << 6) | (uint32_t)((c >> (e - 6)) & 63u);
}

static void plan_order(BatchPlan& plan)
{
    constexpr uint32_t kKeys = 59u << 6;   // cost_key < 58 * 64 + 64
    const size_t nh = plan.heads.size();
    // buffers kept in the plan between calls (no allocation once grown)
    std::vector<uint32_t>& start = plan.sort_start;
    std::vector<uint32_t>& key = plan.sort_key;
    std::vector<uint32_t>& sorted = plan.sort_heads;
    std::vector<uint64_t>& cost = plan.sort_cost;
    start.assign(kKeys + 1, 0u);
    key.resize(nh);
    for (size_t k = 0; k < nh; ++k) {
        key[k] = cost_key(plan.chain_words[k]);
        ++start[kKeys - 1 - key[k]];   // descending
    }
    uint32_t acc = 0;
    for (uint32_t b = 0; b <= kKeys; ++b) {
        const uint32_t v = start[b];
        start[b] = acc;
        acc += v;
    }
    sorted.resize(nh);
    cost.resize(nh);
    for (size_t k = 0; k < nh; ++k) {
        const uint32_t pos = start[kKeys - 1 - key[k]]++;
        sorted[pos] = plan.heads[k];
        cost[pos] = plan.chain_words[k];
    }
    plan.heads.swap(sorted);
    plan.chain_words.swap(cost);
}

void plan_tasks(BatchPlan& plan, const uint8_t* shapes, uint64_t group_max_words)
{
    plan.tasks.clear();
    plan.members.clear();
    plan.tasks.reserve(plan.heads.size());
    plan.members.reserve(plan.heads.size() + kMemberSlack);
    uint32_t pending[3][4];
    uint32_t npend[3] = {0, 0, 0};
    auto emit_group = [&](uint32_t kind) {
        const uint32_t sh = shapes[kind];
        plan.tasks.push_back(task_word(sh, (uint32_t)plan.members.size()));
        for (uint32_t g = 0; g < shape_group(sh); ++g) plan.members.push_back(g < npend[kind] ? pending[kind][g] : kNoItem);
        npend[kind] = 0;
    };
    for (const uint32_t u : plan.heads) {
        const BatchItem& it = plan.units[u];
        // normals always run as chains (see batch_kernel)
        const uint32_t sh = shapes && it.kind < kNormal ? shapes[it.kind] : kShapeChain;
        const bool aligned = (reinterpret_cast<uintptr_t>(it.out) & 15u) == 0;
        if (sh == kShape16x4 || sh == kShape8x4) {
            if (it.next == kNoItem && aligned && words_of(it.kind, it.count) <= group_max_words) {
                pending[it.kind][npend[it.kind]++] = u;
                if (npend[it.kind] == shape_group(sh)) emit_group(it.kind);
                continue;
            }
        }
        plan.tasks.push_back(task_word(kShapeChain, (uint32_t)plan.members.size()));
        plan.members.push_back(u);
    }
    for (uint32_t k = 0; k < 3; ++k)
        if (npend[k]) emit_group(k);
}

void plan_batch(const HostItem* items, uint32_t n, uint64_t piece_len, uint32_t n_streams, BatchPlan& plan,
                const uint8_t* shapes, uint64_t group_max_words)
{
    plan_units(items, n, piece_len, n_streams, plan);
    plan_order(plan);
    plan_tasks(plan, shapes, group_max_words);
}

BatchLauncher::~BatchLauncher()
{
    if (done_) cudaEventSynchronize(done_);
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    if (done_) cudaEventDestroy(done_);
    if (h_staging_) cudaFreeHost(h_staging_);
    if (d_scratch_) cudaFree(d_scratch_);
    if (h_jstage_) cudaFreeHost(h_jstage_);
    if (d_jbuf_) cudaFree(d_jbuf_);
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
    kp.func = const_cast<void*>(batch_kernel_ptr((int)c->param_set, false));
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(kBatchBlock);
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
    for (int g = 0; g < 2; ++g) {
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_kernel_ptr((int)c->param_set, g == 1),
                                                          kBatchBlock, 0) != cudaSuccess)
            return XG_ECUDA;
        max_grid_g_[g] = std::max(1, blocks) * c->sm_count;
    }
    max_grid_ = max_grid_g_[0];
    return build_graph(c);
}

uint64_t BatchLauncher::choose_piece_len(const xg_ctx* c, const HostItem* items, uint32_t n,
                                         uint64_t min_piece) const
{
    if (c->split_words == 1) return 0;  // never cut
    if (c->split_words > 1) return c->split_words;
    // automatic: aim at units no longer than the batch's words per resident
    // warp, so that a long call stops being the last warp still running
    uint64_t total = 0, longest = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t w = words_of(items[i].kind, items[i].count);
        total += w;
        longest = std::max(longest, w);
    }
    const uint64_t warps = (uint64_t)std::max(1, max_grid_) * kWarpsPerBlock;
    uint64_t per_warp = std::max<uint64_t>(1, total / warps);
    uint64_t len = kMinPiece;
    while (len < min_piece) len *= 2;
    // about two units per resident warp
    while (len * 4 <= per_warp && len < (uint64_t(1) << 22)) len *= 2;
    return longest >= 2 * len ? len : 0;
}

xg_status BatchLauncher::grow_jump(size_t want)
{
    if (want <= jbytes_) return XG_OK;
    if (launched_ && cudaEventSynchronize(done_) != cudaSuccess) return XG_ECUDA;
    if (h_jstage_) cudaFreeHost(h_jstage_);
    if (d_jbuf_) cudaFree(d_jbuf_);
    h_jstage_ = nullptr;
    d_jbuf_ = nullptr;
    jbytes_ = 0;
    if (cudaHostAlloc(&h_jstage_, want, cudaHostAllocDefault) != cudaSuccess) return XG_ENOMEM;
    if (cudaMalloc(&d_jbuf_, want) != cudaSuccess) return XG_ENOMEM;
    jbytes_ = want;
    return XG_OK;
}

xg_status BatchLauncher::reserve_jump(uint32_t pieces, uint32_t pairs)
{
    // the layout of prologue(): rings, weyls, streams, skips, pair lists,
    // then the tensor-core operand of one doubling step (at most all pieces)
    return grow_jump((size_t)pieces * (512 + 4 + 4 + 8 + 64) + (size_t)pairs * 8 + 4096 + gf2_tc_scratch_bytes(pieces));
}

// Start rings of the pieces.  Piece 0 of a call gets the stream's ring
// (gather).  Then, doubling: step b gives every piece m in [2^b, 2^(b+1)) the
// ring of piece m - 2^b advanced by 2^b pieces, i.e. C_{q+b} applied to it
// (q = log2 of the piece length).  Each piece costs one application and a
// call cut into K pieces needs ceil(log2 K) steps.
xg_status BatchLauncher::prologue(xg_ctx* c, cudaStream_t s)
{
    const uint32_t P = (uint32_t)plan_.pieces.size();
    if (P == 0) return XG_OK;
    // per step b: (src, dst) piece pairs; pieces of one call are consecutive.
    // Count them per step first, then write the lists straight into staging.
    uint32_t per_step[32] = {0};
    int nsteps = 0;
    for (uint32_t k = 0; k < P; ++k) {
        const uint32_t m = plan_.piece_index[k];
        if (m == 0) continue;
        const int b = 31 - __builtin_clz(m);
        ++per_step[b];
        nsteps = std::max(nsteps, b + 1);
    }
    size_t npairs = 0;
    for (int b = 0; b < nsteps; ++b) npairs += per_step[b];
    // device buffer: rings | weyls | gather streams | gather skips | pair lists
    const size_t off_rings = 0;
    const size_t off_weyl = off_rings + (size_t)P * 512;
    const size_t off_streams = (off_weyl + (size_t)P * 4 + 15) / 16 * 16;
    const size_t off_skip = (off_streams + (size_t)P * 4 + 15) / 16 * 16;
    const size_t off_lists = off_skip + (size_t)P * 8;
    uint32_t most = 0;
    for (int b = 0; b < nsteps; ++b) most = std::max(most, per_step[b]);
    const size_t tc_bytes = gf2_apply_scratch(c->device, most);  // tensor-core operand, when used
    const size_t off_tc = (off_lists + 2 * npairs * 4 + 16 + 255) / 256 * 256;
    const size_t total = off_tc + tc_bytes;
    if (total > jbytes_) {
        if (xg_status st = grow_jump(total + total / 2)) return st;
    }
    char* hb = static_cast<char*>(h_jstage_);
    char* db = static_cast<char*>(d_jbuf_);
    // every piece's Weyl word comes from the gather (its own skip); its ring
    // from the gather (m = 0) or a doubling step
    std::memcpy(hb + off_streams, plan_.piece_stream.data(), (size_t)P * 4);
    std::memcpy(hb + off_skip, plan_.piece_skip.data(), (size_t)P * 8);
    size_t src_off[32], dst_off[32];
    uint32_t* src_w[32];
    uint32_t* dst_w[32];
    size_t o = off_lists;
    for (int b = 0; b < nsteps; ++b) {
        src_off[b] = o;
        src_w[b] = reinterpret_cast<uint32_t*>(hb + o);
        o += (size_t)per_step[b] * 4;
        dst_off[b] = o;
        dst_w[b] = reinterpret_cast<uint32_t*>(hb + o);
        o += (size_t)per_step[b] * 4;
    }
    for (uint32_t k = 0; k < P; ++k) {
        const uint32_t m = plan_.piece_index[k];
        if (m == 0) continue;
        const int b = 31 - __builtin_clz(m);
        *src_w[b]++ = k - (1u << b);
        *dst_w[b]++ = k;
    }
    for (uint32_t k = 0; k < P; ++k) {
        plan_.pieces[k].ring = reinterpret_cast<const uint32_t*>(db + off_rings + (size_t)k * 512);
        plan_.pieces[k].weyl0 = reinterpret_cast<const uint32_t*>(db + off_weyl + (size_t)k * 4);
    }
    // matrices first (the first use builds them and synchronises)
    const uint64_t* mats[32] = {nullptr};
    for (int b = 0; b < nsteps; ++b) {
        if (per_step[b] == 0) continue;
        xg_status st = XG_OK;
        mats[b] = jump_matrix(c->device, (int)c->param_set, plan_.split_log2 + (int)b, s, &st);
        if (!mats[b]) return st;
    }
    if (cudaMemcpyAsync(db + off_streams, hb + off_streams, o - off_streams, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return XG_ECUDA;
    // piece 0 of each call gets its stream's ring, the others (nonzero skip)
    // a zero ring, into which their doubling step XORs
    if (launch_gather_rings(c->st, reinterpret_cast<const uint32_t*>(db + off_streams), P,
                            reinterpret_cast<uint32_t*>(db + off_rings),
                            reinterpret_cast<const uint64_t*>(db + off_skip),
                            reinterpret_cast<uint32_t*>(db + off_weyl), 1u, c->weyl_on ? 0x9E3779B9u : 0u,
                            s) != cudaSuccess)
        return XG_ECUDA;
    uint8_t* tc_scratch = tc_bytes ? reinterpret_cast<uint8_t*>(db + off_tc) : nullptr;
    for (int b = 0; b < nsteps; ++b) {
        if (per_step[b] == 0) continue;
        xg_status st = XG_OK;
        if (gf2_apply(c->device, (int)c->param_set, plan_.split_log2 + b, reinterpret_cast<uint32_t*>(db + off_rings),
                      per_step[b], reinterpret_cast<const uint32_t*>(db + src_off[b]),
                      reinterpret_cast<const uint32_t*>(db + dst_off[b]), tc_scratch, c->sm_count, s,
                      &st, true) != cudaSuccess)
            return st != XG_OK ? st : XG_ECUDA;
    }
    return XG_OK;
}

xg_status BatchLauncher::launch(xg_ctx* c, const HostItem* items, uint32_t n, cudaStream_t s,
                                uint32_t* units_per_item, uint64_t min_piece)
{
    if (!exec_) {
        if (xg_status st = reserve(c, std::max<uint32_t>(n, 64))) return st;
    }
    if (launched_ && cudaEventSynchronize(done_) != cudaSuccess) return XG_ECUDA;
    // a tensor-core jump-ahead that gave up waiting (in any earlier prologue)
    // made its pieces' outputs invalid: report it here, the first point at
    // which the host has synchronised with it
    if (launched_ && gf2_tc_take_failure()) return XG_EDEVICE;
    // the jump prologue needs only the pieces: enqueue it before ordering the
    // heads, so that the GPU starts while the host finishes the plan
    plan_units(items, n, choose_piece_len(c, items, n, min_piece), c->n, plan_);
    const uint32_t nu = (uint32_t)plan_.units.size();
    if (xg_status st = reserve(c, nu)) return st;
    if (xg_status st = prologue(c, s)) return st;
    plan_order(plan_);
    // group only units of at most 1/8 of a resident warp's share of the
    // batch (XG_BATCH_GROUP_MAX_WORDS=<n> sets the limit instead)
    uint64_t group_max = 0;
    if (const char* env = std::getenv("XG_BATCH_GROUP_MAX_WORDS")) group_max = std::strtoull(env, nullptr, 10);
    if (group_max == 0) {
        uint64_t total = 0;
        for (const BatchItem& u : plan_.units) total += words_of(u.kind, u.count);
        const uint64_t warps = (uint64_t)std::max(1, max_grid_g_[1]) * kWarpsPerBlock;
        group_max = std::max<uint64_t>(64, total / warps / 8);
    }
    plan_tasks(plan_, c->batch_shape, group_max);
    if (units_per_item) std::memcpy(units_per_item, plan_.units_per_item.data(), (size_t)n * 4);
    char* base = static_cast<char*>(h_staging_);
    BatchHeader hdr{0u, (uint32_t)plan_.tasks.size(), nu, capacity_};
    std::memcpy(base, &hdr, sizeof hdr);
    std::memcpy(base + sizeof hdr, plan_.tasks.data(), plan_.tasks.size() * 4);
    std::memcpy(base + batch_members_offset(capacity_), plan_.members.data(), plan_.members.size() * 4);
    std::memcpy(base + batch_items_offset(capacity_), plan_.units.data(), (size_t)nu * sizeof(BatchItem));
    size_t used = batch_items_offset(capacity_) + (size_t)nu * sizeof(BatchItem);
    if (!plan_.pieces.empty()) {
        std::memcpy(base + batch_pieces_offset(capacity_), plan_.pieces.data(),
                    plan_.pieces.size() * sizeof(BatchPiece));
        used = batch_pieces_offset(capacity_) + plan_.pieces.size() * sizeof(BatchPiece);
    }
    if (cudaGraphExecMemcpyNodeSetParams1D(exec_, copy_node_, d_scratch_, h_staging_, used,
                                           cudaMemcpyHostToDevice) != cudaSuccess)
        return XG_ECUDA;
    // the variant with the group paths only when the plan has group tasks
    bool groups = false;
    for (const uint32_t t : plan_.tasks) groups = groups || (t >> 28) != kShapeChain;
    const unsigned grid = (unsigned)std::min<uint64_t>(
        max_grid_g_[groups ? 1 : 0], (plan_.tasks.size() + kWarpsPerBlock - 1) / kWarpsPerBlock);
    args_.st = c->st;
    void* params[] = {&args_};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(batch_kernel_ptr((int)c->param_set, groups));
    kp.gridDim = dim3(std::max(1u, grid));
    kp.blockDim = dim3(kBatchBlock);
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

namespace {

int shape_of(uint32_t tpg, uint32_t wpl)
{
    for (uint32_t sh = 0; sh < (uint32_t)xg::kNumShapes; ++sh)
        if (xg::shape_tpg(sh) == tpg && xg::shape_wpl(sh) == wpl) return (int)sh;
    return -1;
}

}  // namespace

extern "C" xg_status xg_set_batch_shape(xg_ctx* ctx, xg_type type, uint32_t tpg, uint32_t wpl)
{
    using namespace xg;
    if (!ctx) return fail(XG_EINVAL, "null context");
    if ((unsigned)type > XG_NORMAL_F32) return fail(XG_EINVAL, "unknown output type");
    const int sh = shape_of(tpg, wpl);
    if (sh < 0) return fail(XG_EINVAL, "batch shape (%u, %u) unsupported: (32,2), (16,4) or (8,4)", tpg, wpl);
    if (type == XG_NORMAL_F32 && sh != (int)kShapeChain)
        return fail(XG_EINVAL, "normals run (32,2) in batches");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->batch_shape[type] = (uint8_t)sh;
    return XG_OK;
}

extern "C" xg_status xg_get_batch_shape(xg_ctx* ctx, xg_type type, uint32_t* tpg, uint32_t* wpl)
{
    using namespace xg;
    if (!ctx || !tpg || !wpl) return fail(XG_EINVAL, "null argument");
    if ((unsigned)type > XG_NORMAL_F32) return fail(XG_EINVAL, "unknown output type");
    std::lock_guard<std::mutex> lk(ctx->mu);
    *tpg = shape_tpg(ctx->batch_shape[type]);
    *wpl = shape_wpl(ctx->batch_shape[type]);
    return XG_OK;
}

extern "C" xg_status xg_autotune_batch(xg_ctx* ctx, const xg_item* items, uint32_t n_items, uint32_t* tpg,
                                       uint32_t* wpl, float* ms)
{
    using namespace xg;
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (n_items > 0 && !items) return fail(XG_EINVAL, "null items");
    if (ctx->server) return fail(XG_EINVAL, "the request server owns this context; stop it first");
    std::vector<HostItem> by_kind[3];
    for (uint32_t i = 0; i < n_items; ++i) {
        const xg_item& it = items[i];
        if (it.stream >= ctx->n) return fail(XG_EINVAL, "item %u: stream %u out of range", i, it.stream);
        if (it.type > XG_NORMAL_F32) return fail(XG_EINVAL, "item %u: unknown type %u", i, it.type);
        if (it.count > 0 && !it.out) return fail(XG_EINVAL, "item %u: null output", i);
        if (reinterpret_cast<uintptr_t>(it.out) & 3u) return fail(XG_EINVAL, "item %u: output not 4-byte aligned", i);
        by_kind[it.type].push_back(HostItem{it.stream, it.type, it.count, it.out, nullptr});
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    BatchLauncher*& L = ctx->batch[0];
    if (!L) L = new (std::nothrow) BatchLauncher();
    if (!L) return fail(XG_ENOMEM, "host allocation failed");
    const size_t state_bytes = (size_t)((char*)(ctx->st.pos + ctx->n) - (char*)ctx->state_mem);
    void* saved = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&saved, state_bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(saved, ctx->state_mem, state_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    xg_status st = e == cudaSuccess ? XG_OK : cuda_fail(e, "batch autotune set-up");
    float best_ms[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < 3 && st == XG_OK; ++k) {
        if (by_kind[k].empty()) continue;
        const std::vector<HostItem>& h = by_kind[k];
        int best = ctx->batch_shape[k];
        float best_t = 1e30f;
        const int n_shapes = k == XG_NORMAL_F32 ? 1 : kNumShapes;   // normals: (32,2) only
        for (int sh = 0; sh < n_shapes && st == XG_OK; ++sh) {
            ctx->batch_shape[k] = (uint8_t)sh;
            float t[3] = {0.f, 0.f, 0.f};
            for (int r = -1; r < 3 && st == XG_OK; ++r) {
                if (r >= 0) cudaEventRecord(e0, ctx->stream);
                st = L->launch(ctx, h.data(), (uint32_t)h.size(), ctx->stream);
                if (st != XG_OK) {
                    st = fail(st, "batch autotune launch failed (%s)", cudaGetErrorString(cudaGetLastError()));
                    break;
                }
                if (r >= 0) {
                    cudaEventRecord(e1, ctx->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        st = cuda_fail(cudaGetLastError(), "batch autotune timing");
                        break;
                    }
                    cudaEventElapsedTime(&t[r], e0, e1);
                }
            }
            if (st != XG_OK) break;
            std::sort(t, t + 3);
            if (t[1] < best_t) {
                best_t = t[1];
                best = sh;
            }
        }
        ctx->batch_shape[k] = (uint8_t)best;
        best_ms[k] = best_t;
    }
    if (saved) {
        cudaStreamSynchronize(ctx->stream);
        cudaMemcpyAsync(ctx->state_mem, saved, state_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        cudaFree(saved);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != XG_OK) return st;
    for (int k = 0; k < 3; ++k) {
        if (tpg) tpg[k] = shape_tpg(ctx->batch_shape[k]);
        if (wpl) wpl[k] = shape_wpl(ctx->batch_shape[k]);
        if (ms) ms[k] = best_ms[k];
    }
    return XG_OK;
}

extern "C" xg_status xg_set_batch_split(xg_ctx* ctx, uint64_t piece_words)
{
    using namespace xg;
    if (!ctx) return fail(XG_EINVAL, "null context");
    if (piece_words > 1 && (piece_words < 64 || (piece_words & (piece_words - 1))))
        return fail(XG_EINVAL, "piece length must be 0, 1 or a power of two >= 64");
    ctx->split_words = piece_words;
    return XG_OK;
}
