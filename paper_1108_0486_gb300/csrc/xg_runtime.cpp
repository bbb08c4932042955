// Host runtime of the xorgens library: contexts with device-resident stream
// state, argument checking, launch selection, host-buffer staging, and the
// extern "C" entry points declared in include/xorgens_gb300.h.
#include "xorgens_gb300.h"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "xg_batch.h"
#include "xg_launch.h"
#include "xg_runtime.h"

namespace {
thread_local std::string g_err;
}  // namespace

namespace xg {

xg_status fail(xg_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

xg_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(XG_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

}  // namespace xg

using xg::fail;
using xg::cuda_fail;

namespace {

#define XG_CUDA(call, what)                        \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr uint32_t kOmegaHost = 0x9E3779B9u;  // odd integer nearest 2^31 (sqrt 5 - 1), Sec. 1.5

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

int xg_ctx::pick_cfg(int kind, uint32_t nstreams) const
{
    const int fixed = cfg[kind == xg::kNormalSum ? xg::kNormal : kind];
    if (fixed >= 0) return fixed;
    // Without a tuned choice: many streams -> few lanes per stream (fewer
    // shuffles and 128-bit stores); few streams -> more lanes per stream.
    const uint64_t lanes_wanted = (uint64_t)sm_count * 32 * 24;  // ~24 resident warps per SM
    if ((uint64_t)nstreams * 8 >= lanes_wanted / 2) return xg::cfg_index(8, 4);
    if ((uint64_t)nstreams * 16 >= lanes_wanted / 2) return xg::cfg_index(16, 2);
    return xg::cfg_index(32, 2);
}

int xg_ctx::pick_block(int kind, int c) const
{
    const int t = kind == xg::kNormalSum ? xg::kNormal : kind;
    return (cfg[t] == c && blk[t] > 0) ? blk[t] : block[c];
}

xg_status xg_ctx::ensure_jump_ws(size_t bytes)
{
    if (jump_ws_bytes >= bytes) return XG_OK;
    if (jump_ws) {
        cudaStreamSynchronize(stream);
        cudaFree(jump_ws);
    }
    jump_ws = nullptr;
    jump_ws_bytes = 0;
    if (cudaMalloc(&jump_ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return xg::fail(XG_ENOMEM, "cudaMalloc(jump workspace, %zu bytes) failed", bytes);
    }
    jump_ws_bytes = bytes;
    return XG_OK;
}

xg_status xg_ctx::ensure_staging(size_t bytes)
{
    if (staging_bytes >= bytes) return XG_OK;
    for (int b = 0; b < kStage; ++b) {
        if (staging[b]) cudaFree(staging[b]);
        staging[b] = nullptr;
    }
    staging_bytes = 0;
    for (int b = 0; b < kStage; ++b) XG_CUDA(cudaMalloc(&staging[b], bytes), "cudaMalloc(staging)");
    staging_bytes = bytes;
    return XG_OK;
}

using xg::Ctx;

static xg_status check_ctx(const xg_ctx* c)
{
    if (!c) return fail(XG_EINVAL, "null context");
    return XG_OK;
}

static xg_status enqueue_gen(Ctx* c, int kind, uint32_t first, uint32_t nstreams, uint64_t n,
                             void* d_out, uint64_t ld, float* d_sums, cudaStream_t s,
                             int force_cfg = -1, int force_block = 0)
{
    xg::GenArgs a{};
    a.st = c->st;
    a.first = first;
    a.nstreams = nstreams;
    a.n = n;
    a.out = d_out;
    a.ld = ld;
    a.sums = d_sums;
    a.omega = c->weyl_on ? kOmegaHost : 0u;
    const int cfg = force_cfg >= 0 ? force_cfg : c->pick_cfg(kind, nstreams);
    const bool vec = kind == xg::kNormalSum ||
                     (((reinterpret_cast<uintptr_t>(d_out) & 15u) == 0) && (ld % 4 == 0));
    const int block = force_block > 0 ? force_block : c->pick_block(kind, cfg);
    cudaError_t e = xg::launch_gen(c->param_set, cfg, kind, vec, block, a, s);
    if (e != cudaSuccess) return cuda_fail(e, "generate kernel launch");
    return XG_OK;
}

constexpr uint32_t kCutMaxStreams = 64;
constexpr uint64_t kCutMinWords = uint64_t(1) << 18;

static xg_status generate_cut(Ctx* c, int kind, uint32_t first, uint32_t nstreams, uint64_t n, void* out,
                              uint64_t ld)
{
    std::vector<xg::HostItem> items(nstreams);
    for (uint32_t i = 0; i < nstreams; ++i)
        items[i] = xg::HostItem{first + i, (uint32_t)kind, n, static_cast<char*>(out) + (uint64_t)i * ld * 4,
                                nullptr};
    xg::BatchLauncher*& L = c->batch[c->batch_next];
    c->batch_next ^= 1;
    if (!L) L = new (std::nothrow) xg::BatchLauncher();
    if (!L) return fail(XG_ENOMEM, "host allocation failed");
    xg_status st = L->launch(c, items.data(), nstreams, c->stream);
    if (st != XG_OK) {
        cudaError_t e = cudaGetLastError();
        return fail(st, "cut generation failed (%s)", cudaGetErrorString(e));
    }
    return XG_OK;
}

static bool is_device_pointer(const void* p)
{
    cudaPointerAttributes attr{};
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Host output: generate piece by piece into kStage device buffers and copy
// each piece out on that buffer's own CUDA stream while the next pieces are
// generated (several copies in flight keep the host link busy).  Pieces split
// the stream range and, for long requests, each stream's length; the stream
// positions make consecutive pieces of one stream continue each other.
static xg_status generate_to_host(Ctx* c, int kind, uint32_t first, uint32_t nstreams, uint64_t n,
                                  void* h_out, uint64_t ld)
{
    const size_t kPieceBytes = size_t(128) << 20;
    xg_status st = c->ensure_staging(kPieceBytes);
    if (st != XG_OK) return st;
    const uint64_t words_per_piece = kPieceBytes / 4;
    // normals: keep pieces even so that pairs never straddle pieces
    uint64_t ncols = std::min<uint64_t>(n, words_per_piece);
    if (kind == xg::kNormal && ncols < n && (ncols & 1)) ncols -= 1;
    ncols = std::max<uint64_t>(ncols, 1);
    const uint64_t ld_stage = align_up(ncols, 4);
    const uint32_t rows_per_piece = (uint32_t)std::max<uint64_t>(1, words_per_piece / ld_stage);
    int b = 0;
    for (uint32_t r0 = 0; r0 < nstreams; r0 += rows_per_piece) {
        const uint32_t rows = std::min<uint32_t>(rows_per_piece, nstreams - r0);
        for (uint64_t c0 = 0; c0 < n; c0 += ncols) {
            const uint64_t cols = std::min<uint64_t>(ncols, n - c0);
            XG_CUDA(cudaStreamWaitEvent(c->stream, c->ev_copy[b], 0), "cudaStreamWaitEvent");
            st = enqueue_gen(c, kind, first + r0, rows, cols, c->staging[b], ld_stage, nullptr, c->stream);
            if (st != XG_OK) return st;
            XG_CUDA(cudaEventRecord(c->ev_gen[b], c->stream), "cudaEventRecord");
            XG_CUDA(cudaStreamWaitEvent(c->copy_stream[b], c->ev_gen[b], 0), "cudaStreamWaitEvent");
            char* dst = static_cast<char*>(h_out) + ((uint64_t)r0 * ld + c0) * 4;
            if (ld == ld_stage && cols == ld) {
                XG_CUDA(cudaMemcpyAsync(dst, c->staging[b], (size_t)rows * cols * 4, cudaMemcpyDeviceToHost,
                                        c->copy_stream[b]),
                        "cudaMemcpyAsync(device to host)");
            } else {
                XG_CUDA(cudaMemcpy2DAsync(dst, ld * 4, c->staging[b], ld_stage * 4, cols * 4, rows,
                                          cudaMemcpyDeviceToHost, c->copy_stream[b]),
                        "cudaMemcpy2DAsync(device to host)");
            }
            XG_CUDA(cudaEventRecord(c->ev_copy[b], c->copy_stream[b]), "cudaEventRecord");
            b = (b + 1) % xg_ctx::kStage;
        }
    }
    for (int k = 0; k < xg_ctx::kStage; ++k)
        XG_CUDA(cudaStreamSynchronize(c->copy_stream[k]), "cudaStreamSynchronize(copy)");
    return XG_OK;
}

static xg_status generate_common(xg_ctx* ctx, int kind, uint32_t first, uint32_t nstreams,
                                 uint64_t n, void* out, uint64_t ld)
{
    if (xg_status s = check_ctx(ctx)) return s;
    Ctx* c = ctx;
    if ((uint64_t)first + nstreams > c->n)
        return fail(XG_EINVAL, "streams [%u, %u) out of range (context has %u)", first,
                    first + nstreams, c->n);
    if (nstreams == 0 || n == 0) return XG_OK;
    if (!out) return fail(XG_EINVAL, "null output pointer");
    if (nstreams > 1 && ld < n) return fail(XG_EINVAL, "ld (%llu) < n_per_stream (%llu)",
                                            (unsigned long long)ld, (unsigned long long)n);
    if (nstreams == 1 && ld < n) ld = n;
    if (ld > (UINT64_MAX / 8) / nstreams) return fail(XG_EINVAL, "output extent overflows");
    if (reinterpret_cast<uintptr_t>(out) & 3u) return fail(XG_EINVAL, "output must be 4-byte aligned");
    if (c->server) return fail(XG_EINVAL, "the request server owns this context; use xg_submit");
    std::lock_guard<std::mutex> lk(c->mu);
    if (is_device_pointer(out)) {
        // few streams, long calls: a single stream is one serial chain (one
        // warp, ~1.5e9 words/s), so cut each call into pieces that run on
        // many warps at once (jump-ahead; the output is the same)
        if (nstreams <= kCutMaxStreams && n >= kCutMinWords && c->split_words != 1)
            return generate_cut(c, kind, first, nstreams, n, out, ld);
        return enqueue_gen(c, kind, first, nstreams, n, out, ld, nullptr, c->stream);
    }
    return generate_to_host(c, kind, first, nstreams, n, out, ld);
}

extern "C" {

const char* xg_last_error(void) { return g_err.c_str(); }

const char* xg_version(void) { return "xorgens_gb300 0.1 (sm_103a)"; }

xg_status xg_create_streams(xg_ctx** out, uint32_t n_streams, uint32_t param_set, uint32_t weyl_on,
                            void* cuda_stream)
{
    if (!out) return fail(XG_EINVAL, "null output handle");
    *out = nullptr;
    if (n_streams == 0) return fail(XG_EINVAL, "n_streams must be positive");
    if (param_set > 1) return fail(XG_EINVAL, "unknown parameter set %u", param_set);
    Ctx* c = new (std::nothrow) Ctx();
    if (!c) return fail(XG_ENOMEM, "host allocation failed");
    c->n = n_streams;
    c->param_set = param_set;
    c->weyl_on = weyl_on ? 1u : 0u;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    for (int i = 0; i < xg::kNumCfgs; ++i) c->block[i] = xg::kCfgs[i].block;
    const size_t nw = (size_t)n_streams * xg::kWin * 4;
    const size_t off_weyl = align_up(nw, 256);
    const size_t off_pend = align_up(off_weyl + (size_t)n_streams * 4, 256);
    const size_t off_pos = align_up(off_pend + (size_t)n_streams * 4, 256);
    const size_t total = off_pos + (size_t)n_streams * 8;
    if (e == cudaSuccess) e = cudaMalloc(&c->state_mem, total);
    if (e != cudaSuccess) {
        xg_status st = e == cudaErrorMemoryAllocation ? fail(XG_ENOMEM, "cudaMalloc(state, %zu bytes) failed", total)
                                                      : cuda_fail(e, "create");
        cudaGetLastError();
        delete c;
        return st;
    }
    char* base = static_cast<char*>(c->state_mem);
    c->st.win = reinterpret_cast<uint32_t*>(base);
    c->st.weyl = reinterpret_cast<uint32_t*>(base + off_weyl);
    c->st.pend = reinterpret_cast<uint32_t*>(base + off_pend);
    c->st.pos = reinterpret_cast<uint64_t*>(base + off_pos);
    e = cudaMemsetAsync(c->state_mem, 0, total, c->stream);
    for (int b = 0; b < xg_ctx::kStage && e == cudaSuccess; ++b)
        e = cudaStreamCreateWithFlags(&c->copy_stream[b], cudaStreamNonBlocking);
    for (int b = 0; b < xg_ctx::kStage && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&c->ev_gen[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_copy[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        xg_status st = cuda_fail(e, "create");
        xg_destroy(c);
        return st;
    }
    if (xg_status st = xg::noalloc_setup(c->device, c->sm_count)) {
        xg_destroy(c);
        return st;
    }
    *out = c;
    return XG_OK;
}

xg_status xg_destroy(xg_ctx* ctx)
{
    if (!ctx) return XG_OK;
    Ctx* c = ctx;
    c->shutdown_server();
    for (int b = 0; b < 2; ++b) {
        delete c->batch[b];
        c->batch[b] = nullptr;
    }
    if (c->stream || c->state_mem) cudaStreamSynchronize(c->stream);
    for (int b = 0; b < xg_ctx::kStage; ++b) {
        if (c->copy_stream[b]) {
            cudaStreamSynchronize(c->copy_stream[b]);
            cudaStreamDestroy(c->copy_stream[b]);
        }
    }
    for (int b = 0; b < xg_ctx::kStage; ++b) {
        if (c->ev_gen[b]) cudaEventDestroy(c->ev_gen[b]);
        if (c->ev_copy[b]) cudaEventDestroy(c->ev_copy[b]);
        if (c->staging[b]) cudaFree(c->staging[b]);
    }
    if (c->jump_ws) cudaFree(c->jump_ws);
    if (c->state_mem) cudaFree(c->state_mem);
    delete c;
    return XG_OK;
}

xg_status xg_set_stream(xg_ctx* ctx, void* cuda_stream)
{
    if (xg_status s = check_ctx(ctx)) return s;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return XG_OK;
}

xg_status xg_num_streams(const xg_ctx* ctx, uint32_t* n)
{
    if (xg_status s = check_ctx(ctx)) return s;
    if (!n) return fail(XG_EINVAL, "null output");
    *n = ctx->n;
    return XG_OK;
}

xg_status xg_seed(xg_ctx* ctx, uint32_t first, uint32_t count, const uint32_t* host_seeds)
{
    if (xg_status s = check_ctx(ctx)) return s;
    Ctx* c = ctx;
    if ((uint64_t)first + count > c->n) return fail(XG_EINVAL, "seed range out of bounds");
    if (count == 0) return XG_OK;
    if (!host_seeds) return fail(XG_EINVAL, "null seeds");
    if (c->server) return fail(XG_EINVAL, "the request server owns this context; stop it first");
    std::lock_guard<std::mutex> lk(c->mu);
    uint32_t* d = nullptr;
    XG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), (size_t)count * 4, c->stream), "cudaMallocAsync(seeds)");
    cudaError_t e = cudaMemcpyAsync(d, host_seeds, (size_t)count * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = xg::launch_seed(c->param_set, c->st, d, first, count, c->stream);
    cudaError_t e2 = cudaFreeAsync(d, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "seed");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync(seeds)");
    if (!c->weyl_on) {
        // the Weyl word is unused; keep it zero so that its combination is the identity
        XG_CUDA(cudaMemsetAsync(c->st.weyl + first, 0, (size_t)count * 4, c->stream), "cudaMemsetAsync");
    }
    return XG_OK;
}

xg_status xg_get_state(xg_ctx* ctx, uint32_t stream, uint32_t* ring, uint32_t* weyl)
{
    if (xg_status s = check_ctx(ctx)) return s;
    Ctx* c = ctx;
    if (stream >= c->n) return fail(XG_EINVAL, "stream %u out of range", stream);
    if (!ring || !weyl) return fail(XG_EINVAL, "null output");
    std::lock_guard<std::mutex> lk(c->mu);
    uint32_t win[xg::kWin], pend = 0, w = 0;
    XG_CUDA(cudaMemcpyAsync(win, c->st.win + (size_t)stream * xg::kWin, sizeof win, cudaMemcpyDeviceToHost, c->stream), "get_state");
    XG_CUDA(cudaMemcpyAsync(&pend, c->st.pend + stream, 4, cudaMemcpyDeviceToHost, c->stream), "get_state");
    XG_CUDA(cudaMemcpyAsync(&w, c->st.weyl + stream, 4, cudaMemcpyDeviceToHost, c->stream), "get_state");
    XG_CUDA(cudaStreamSynchronize(c->stream), "get_state");
    if (pend >= (uint32_t)xg::kRingBase) return fail(XG_EDEVICE, "corrupt stream state (pend %u)", pend);
    std::memcpy(ring, win + xg::kRingBase - pend, 128 * 4);
    *weyl = w;
    return XG_OK;
}

xg_status xg_set_state(xg_ctx* ctx, uint32_t stream, const uint32_t* ring, uint32_t weyl)
{
    if (xg_status s = check_ctx(ctx)) return s;
    Ctx* c = ctx;
    if (stream >= c->n) return fail(XG_EINVAL, "stream %u out of range", stream);
    if (!ring) return fail(XG_EINVAL, "null ring");
    if (c->server) return fail(XG_EINVAL, "the request server owns this context; stop it first");
    std::lock_guard<std::mutex> lk(c->mu);
    uint32_t win[xg::kWin] = {0};
    std::memcpy(win + xg::kRingBase, ring, 128 * 4);
    const uint32_t pend = 0, w = c->weyl_on ? weyl : 0u;
    XG_CUDA(cudaMemcpyAsync(c->st.win + (size_t)stream * xg::kWin, win, sizeof win, cudaMemcpyHostToDevice, c->stream), "set_state");
    XG_CUDA(cudaMemcpyAsync(c->st.pend + stream, &pend, 4, cudaMemcpyHostToDevice, c->stream), "set_state");
    XG_CUDA(cudaMemcpyAsync(c->st.weyl + stream, &w, 4, cudaMemcpyHostToDevice, c->stream), "set_state");
    XG_CUDA(cudaStreamSynchronize(c->stream), "set_state");
    return XG_OK;
}

xg_status xg_get_states(xg_ctx* ctx, uint32_t first, uint32_t count, uint32_t* rings, uint32_t* weyl,
                        uint64_t* pos)
{
    if (xg_status s = check_ctx(ctx)) return s;
    Ctx* c = ctx;
    if ((uint64_t)first + count > c->n) return fail(XG_EINVAL, "streams [%u, %u) out of range", first, first + count);
    if (count == 0) return XG_OK;
    if (!rings || !weyl) return fail(XG_EINVAL, "null output");
    std::lock_guard<std::mutex> lk(c->mu);
    const size_t rb = (size_t)count * 128 * 4, wb = (size_t)count * 4, pb = (size_t)count * 8;
    char* d = nullptr;
    XG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), rb + wb + pb + 16, c->stream), "cudaMallocAsync(states)");
    uint32_t* d_rings = reinterpret_cast<uint32_t*>(d);
    uint32_t* d_weyl = reinterpret_cast<uint32_t*>(d + rb);
    uint64_t* d_pos = reinterpret_cast<uint64_t*>(d + (rb + wb + 7) / 8 * 8);
    cudaError_t e = xg::launch_export_states(c->st, first, count, d_rings, d_weyl, d_pos, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rings, d_rings, rb, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(weyl, d_weyl, wb, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && pos) e = cudaMemcpyAsync(pos, d_pos, pb, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? XG_OK : cuda_fail(e, "xg_get_states");
}

xg_status xg_set_states(xg_ctx* ctx, uint32_t first, uint32_t count, const uint32_t* rings, const uint32_t* weyl,
                        const uint64_t* pos)
{
    if (xg_status s = check_ctx(ctx)) return s;
    Ctx* c = ctx;
    if ((uint64_t)first + count > c->n) return fail(XG_EINVAL, "streams [%u, %u) out of range", first, first + count);
    if (count == 0) return XG_OK;
    if (!rings || !weyl) return fail(XG_EINVAL, "null input");
    if (c->server) return fail(XG_EINVAL, "the request server owns this context; stop it first");
    std::lock_guard<std::mutex> lk(c->mu);
    const size_t rb = (size_t)count * 128 * 4, wb = (size_t)count * 4, pb = (size_t)count * 8;
    char* d = nullptr;
    XG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), rb + wb + pb + 16, c->stream), "cudaMallocAsync(states)");
    uint32_t* d_rings = reinterpret_cast<uint32_t*>(d);
    uint32_t* d_weyl = reinterpret_cast<uint32_t*>(d + rb);
    uint64_t* d_pos = reinterpret_cast<uint64_t*>(d + (rb + wb + 7) / 8 * 8);
    cudaError_t e = cudaMemcpyAsync(d_rings, rings, rb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_weyl, weyl, wb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && pos) e = cudaMemcpyAsync(d_pos, pos, pb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = xg::launch_import_states(c->st, first, count, d_rings, d_weyl, pos ? d_pos : nullptr, c->weyl_on,
                                     c->stream);
    cudaFreeAsync(d, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host arrays are caller-owned
    return e == cudaSuccess ? XG_OK : cuda_fail(e, "xg_set_states");
}

xg_status xg_generate_u32(xg_ctx* ctx, uint32_t first, uint32_t nstreams, uint64_t n, uint32_t* out, uint64_t ld)
{
    return generate_common(ctx, xg::kU32, first, nstreams, n, out, ld);
}

xg_status xg_generate_uniform(xg_ctx* ctx, uint32_t first, uint32_t nstreams, uint64_t n, float* out, uint64_t ld)
{
    return generate_common(ctx, xg::kUniform, first, nstreams, n, out, ld);
}

xg_status xg_generate_normal(xg_ctx* ctx, uint32_t first, uint32_t nstreams, uint64_t n, float* out, uint64_t ld)
{
    return generate_common(ctx, xg::kNormal, first, nstreams, n, out, ld);
}

xg_status xg_generate_normal_sum(xg_ctx* ctx, uint32_t first, uint32_t nstreams, uint64_t n, float* d_sums)
{
    if (xg_status s = check_ctx(ctx)) return s;
    Ctx* c = ctx;
    if ((uint64_t)first + nstreams > c->n) return fail(XG_EINVAL, "streams out of range");
    if (nstreams == 0) return XG_OK;
    if (!d_sums) return fail(XG_EINVAL, "null sums");
    if (!is_device_pointer(d_sums)) return fail(XG_EINVAL, "sums must be device memory");
    if (c->server) return fail(XG_EINVAL, "the request server owns this context; use xg_submit");
    std::lock_guard<std::mutex> lk(c->mu);
    return enqueue_gen(c, xg::kNormalSum, first, nstreams, n, nullptr, 0, d_sums, c->stream);
}

xg_status xg_transform_uniform(xg_ctx* ctx, const uint32_t* d_words, uint64_t n, float* d_out)
{
    if (xg_status s = check_ctx(ctx)) return s;
    if (n == 0) return XG_OK;
    if (!d_words || !d_out) return fail(XG_EINVAL, "null pointer");
    if ((reinterpret_cast<uintptr_t>(d_words) | reinterpret_cast<uintptr_t>(d_out)) & 3u)
        return fail(XG_EINVAL, "buffers must be 4-byte aligned");
    cudaError_t e = xg::launch_transform(xg::kUniform, d_words, n, d_out, ctx->stream);
    return e == cudaSuccess ? XG_OK : cuda_fail(e, "transform_uniform");
}

xg_status xg_transform_normal(xg_ctx* ctx, const uint32_t* d_words, uint64_t n, float* d_out)
{
    if (xg_status s = check_ctx(ctx)) return s;
    if (n == 0) return XG_OK;
    if (!d_words || !d_out) return fail(XG_EINVAL, "null pointer");
    if (n & 1) return fail(XG_EINVAL, "normal transform needs an even word count");
    if ((reinterpret_cast<uintptr_t>(d_words) | reinterpret_cast<uintptr_t>(d_out)) & 7u)
        return fail(XG_EINVAL, "buffers must be 8-byte aligned");
    cudaError_t e = xg::launch_transform(xg::kNormal, d_words, n, d_out, ctx->stream);
    return e == cudaSuccess ? XG_OK : cuda_fail(e, "transform_normal");
}

xg_status xg_set_launch(xg_ctx* ctx, xg_type type, uint32_t tpg, uint32_t wpl)
{
    if (xg_status s = check_ctx(ctx)) return s;
    if ((unsigned)type > XG_NORMAL_F32) return fail(XG_EINVAL, "unknown output type");
    ctx->blk[type] = 0;
    if (tpg == 0 && wpl == 0) {
        ctx->cfg[type] = -1;
        return XG_OK;
    }
    const int ci = xg::cfg_index((int)tpg, (int)wpl);
    if (ci < 0) return fail(XG_EINVAL, "unsupported launch (tpg %u, wpl %u)", tpg, wpl);
    ctx->cfg[type] = ci;
    return XG_OK;
}

xg_status xg_get_launch(const xg_ctx* ctx, xg_type type, uint32_t* tpg, uint32_t* wpl)
{
    if (xg_status s = check_ctx(ctx)) return s;
    if ((unsigned)type > XG_NORMAL_F32 || !tpg || !wpl) return fail(XG_EINVAL, "bad argument");
    const int ci = ctx->cfg[type];
    if (ci < 0) {
        *tpg = 0;
        *wpl = 0;
    } else {
        *tpg = (uint32_t)xg::kCfgs[ci].tpg;
        *wpl = (uint32_t)xg::kCfgs[ci].wpl;
    }
    return XG_OK;
}

xg_status xg_autotune(xg_ctx* ctx, xg_type type, uint32_t nstreams, uint64_t n_per_stream,
                      uint32_t* tpg, uint32_t* wpl, uint32_t* block, float* best_ms)
{
    if (xg_status s = check_ctx(ctx)) return s;
    Ctx* c = ctx;
    if ((unsigned)type > XG_NORMAL_F32) return fail(XG_EINVAL, "unknown output type");
    if (c->server) return fail(XG_EINVAL, "the request server owns this context; stop it first");
    if (nstreams == 0 || nstreams > c->n) nstreams = c->n;
    if (n_per_stream == 0) return fail(XG_EINVAL, "n_per_stream must be positive");
    // a slice of the workload: every stream, at most 2^28 outputs in all (a
    // smaller slice ranked block sizes differently from the full size)
    uint64_t nt = std::min<uint64_t>(n_per_stream, std::max<uint64_t>(256, (uint64_t(1) << 28) / nstreams));
    nt = align_up(nt, 64);
    std::lock_guard<std::mutex> lk(c->mu);
    const size_t state_bytes = (size_t)((char*)(c->st.pos + c->n) - (char*)c->state_mem);
    void* saved = nullptr;
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    xg_status st = XG_OK;
    int best_cfg = -1, best_block = 0;
    float best = 1e30f;
    auto cleanup = [&]() {
        if (saved) {
            cudaMemcpyAsync(c->state_mem, saved, state_bytes, cudaMemcpyDeviceToDevice, c->stream);
            cudaStreamSynchronize(c->stream);
            cudaFree(saved);
        }
        if (out) cudaFree(out);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&saved, state_bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(saved, c->state_mem, state_bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)nstreams * nt * 4);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return cuda_fail(e, "autotune set-up");
    }
    static const int kBlocks[] = {32, 64, 128, 256};
    for (int ci = 0; ci < xg::kNumCfgs && st == XG_OK; ++ci) {
        for (int b : kBlocks) {
            st = enqueue_gen(c, type, 0, nstreams, nt, out, nt, nullptr, c->stream, ci, b);
            if (st != XG_OK) break;
            // the median of five timed launches
            float t[5];
            for (int r = 0; r < 5 && st == XG_OK; ++r) {
                cudaEventRecord(e0, c->stream);
                st = enqueue_gen(c, type, 0, nstreams, nt, out, nt, nullptr, c->stream, ci, b);
                cudaEventRecord(e1, c->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    st = cuda_fail(cudaGetLastError(), "autotune timing");
                    break;
                }
                t[r] = 0.f;
                cudaEventElapsedTime(&t[r], e0, e1);
            }
            if (st != XG_OK) break;
            std::sort(t, t + 5);
            const float ms = t[2];
            if (ms < best) {
                best = ms;
                best_cfg = ci;
                best_block = b;
            }
        }
    }
    cleanup();
    if (st != XG_OK) return st;
    c->cfg[type] = best_cfg;
    c->blk[type] = best_block;
    if (tpg) *tpg = (uint32_t)xg::kCfgs[best_cfg].tpg;
    if (wpl) *wpl = (uint32_t)xg::kCfgs[best_cfg].wpl;
    if (block) *block = (uint32_t)best_block;
    if (best_ms) *best_ms = best;
    return XG_OK;
}

}  // extern "C"
