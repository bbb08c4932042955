// Host runtime of the 64-bit-word generators: contexts with device-resident
// state, argument checking, launch choice, host-output staging, autotuning,
// and the extern "C" entry points of include/xorgens_w64.h.
#include "xorgens_w64.h"

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "xg_gf2_tc.h"
#include "xg_jump.h"
#include "xg_runtime.h"
#include "xg_w64.h"

using xg::cuda_fail;
using xg::fail;

struct xg_w64_ctx {
    int device = 0;
    int sm_count = 148;
    uint32_t n = 0;
    uint32_t weyl_on = 1;
    cudaStream_t stream = nullptr;
    void* state_mem = nullptr;
    size_t state_bytes = 0;
    xg64::State st{};
    int cfg[2] = {-1, -1};
    int blk[2] = {0, 0};
    void* staging = nullptr;
    size_t staging_bytes = 0;
    uint64_t split_words = 0;   // cut calls: 0 automatic, 1 never, else the piece length
    std::mutex mu;
};

namespace {

#define XG_CUDA(call, what)                                \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool is_device_pointer(const void* p)
{
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

int pick_cfg(const xg_w64_ctx* c, int kind, uint32_t nstreams)
{
    if (c->cfg[kind] >= 0) return c->cfg[kind];
    // many streams: few lanes per stream (fewer shuffles, 16-byte stores)
    const uint64_t lanes_wanted = (uint64_t)c->sm_count * 32 * 24;
    if ((uint64_t)nstreams * 8 >= lanes_wanted / 2) return xg64::cfg_index(8, 4);
    if ((uint64_t)nstreams * 16 >= lanes_wanted / 2) return xg64::cfg_index(16, 2);
    return xg64::cfg_index(32, 1);
}

xg_status enqueue(xg_w64_ctx* c, int kind, uint32_t first, uint32_t nstreams, uint64_t n, void* d_out,
                  uint64_t ld, int force_cfg = -1, int force_block = 0)
{
    xg64::GenArgs a{};
    a.st = c->st;
    a.first = first;
    a.nstreams = nstreams;
    a.n = n;
    a.out = d_out;
    a.ld = ld;
    a.omega = c->weyl_on ? xg64::kOmega : 0;
    const int cfg = force_cfg >= 0 ? force_cfg : pick_cfg(c, kind, nstreams);
    int block = force_block;
    if (block <= 0) block = (c->cfg[kind] == cfg && c->blk[kind] > 0) ? c->blk[kind] : xg64::kCfgs[cfg].block;
    const bool vec = ((reinterpret_cast<uintptr_t>(d_out) & 15u) == 0) && (nstreams == 1 || ld % 2 == 0);
    cudaError_t e = xg64::launch_gen(cfg, kind, vec, block, a, c->stream);
    return e == cudaSuccess ? XG_OK : cuda_fail(e, "64-bit generate kernel launch");
}

// Few streams, long calls: one stream is one serial chain (one warp), so the
// call is cut into K pieces of L = 2^q words per stream whose start states
// come from the jump-ahead matrices (piece m = the stream advanced m L
// words), generated as K streams of a scratch state, and the stream then
// takes the state of its last piece.  The output is exactly the uncut call's.
constexpr uint32_t kCutMaxStreams = 16;
constexpr uint64_t kCutMinWords = uint64_t(1) << 18;

xg_status generate_cut(xg_w64_ctx* c, int kind, uint32_t first, uint32_t nstreams, uint64_t n, void* d_out,
                       uint64_t ld)
{
    // piece length: about four pieces per SM sub-partition in all, at least 2^16
    int q = 16;
    if (c->split_words > 1) {
        while ((uint64_t(1) << q) < c->split_words) ++q;
    } else {
        const uint64_t target = std::max<uint64_t>(1, (uint64_t)c->sm_count * 4 / nstreams);
        while (q < 40 && (uint64_t(1) << q) * target < n) ++q;
    }
    const uint64_t L = uint64_t(1) << q;
    const uint64_t K64 = (n + L - 1) / L;
    if (K64 < 2 || K64 * nstreams > (uint64_t(1) << 20)) return enqueue(c, kind, first, nstreams, n, d_out, ld);
    const uint32_t K = (uint32_t)K64;
    const uint32_t P = nstreams * K;
    cudaStream_t s = c->stream;
    int steps = 0;   // doubling steps: bits of K - 1
    while (((uint64_t)(K - 1) >> steps)) ++steps;
    xg_status st = XG_OK;
    for (int b = 0; b < steps; ++b)
        if (!xg::jump_matrix(c->device, xg::kJumpSetW64, q + b, s, &st)) return st;
    // pair lists per step b: sources i K + m - 2^b, destinations i K + m
    std::vector<uint32_t> h;
    std::vector<size_t> src_off(steps), dst_off(steps);
    std::vector<uint32_t> cnt(steps);
    for (int b = 0; b < steps; ++b) {
        const uint32_t lo = 1u << b, hi = (uint32_t)std::min<uint64_t>((uint64_t)lo << 1, K);
        cnt[b] = (hi - lo) * nstreams;
        src_off[b] = h.size();
        for (uint32_t i = 0; i < nstreams; ++i)
            for (uint32_t m = lo; m < hi; ++m) h.push_back(i * K + m - lo);
        dst_off[b] = h.size();
        for (uint32_t i = 0; i < nstreams; ++i)
            for (uint32_t m = lo; m < hi; ++m) h.push_back(i * K + m);
    }
    // scratch: rings[P][64] | piece state (window, Weyl, pend, pos) | lists
    const size_t off_win = (size_t)P * xg64::kR * 8;
    const size_t off_weyl = off_win + (size_t)P * xg64::kWin * 8;
    const size_t off_pos = off_weyl + (size_t)P * 8;
    const size_t off_pend = off_pos + (size_t)P * 8;
    const size_t off_lists = align_up(off_pend + (size_t)P * 4, 16);
    const uint32_t most = steps ? *std::max_element(cnt.begin(), cnt.end()) : 0u;
    const size_t tc_bytes = xg::gf2_apply_scratch(c->device, most);  // tensor-core operand, when used
    const size_t off_tc = align_up(off_lists + h.size() * 4 + 4, 256);
    const size_t total = off_tc + tc_bytes;
    char* scratch = nullptr;
    XG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&scratch), total, s), "cut scratch");
    uint64_t* rings = reinterpret_cast<uint64_t*>(scratch);
    uint32_t* rings32 = reinterpret_cast<uint32_t*>(scratch);
    uint32_t* lists = reinterpret_cast<uint32_t*>(scratch + off_lists);
    xg64::State pieces{reinterpret_cast<uint64_t*>(scratch + off_win), reinterpret_cast<uint64_t*>(scratch + off_weyl),
                       reinterpret_cast<uint32_t*>(scratch + off_pend), reinterpret_cast<uint64_t*>(scratch + off_pos)};
    cudaError_t e = cudaSuccess;
    if (!h.empty()) e = cudaMemcpyAsync(lists, h.data(), h.size() * 4, cudaMemcpyHostToDevice, s);
    // every ring zeroed once (the doubling steps XOR into the pieces m > 0),
    // then piece 0 of each stream: the stream's own ring (one stream at a time)
    if (e == cudaSuccess) e = cudaMemsetAsync(rings, 0, off_win, s);
    for (uint32_t i = 0; i < nstreams && e == cudaSuccess; ++i)
        e = xg64::launch_gather_rings(c->st, first + i, 1, rings + (size_t)i * K * xg64::kR, s);
    uint8_t* tc_scratch = tc_bytes ? reinterpret_cast<uint8_t*>(scratch + off_tc) : nullptr;
    for (int b = 0; b < steps && e == cudaSuccess; ++b)
        e = xg::gf2_apply(c->device, xg::kJumpSetW64, q + b, rings32, cnt[b], lists + src_off[b], lists + dst_off[b],
                          tc_scratch, c->sm_count, s, &st, true);
    const uint64_t omega = c->weyl_on ? xg64::kOmega : 0;
    if (e == cudaSuccess) e = xg64::launch_init_pieces(c->st, first, nstreams, K, L, rings, pieces, omega, s);
    xg_status gst = XG_OK;
    if (e == cudaSuccess) {
        // the full pieces of each stream as K - 1 streams with ld = L, then its last piece
        xg_w64_ctx view = {};
        view.sm_count = c->sm_count;
        view.stream = s;
        view.st = pieces;
        view.weyl_on = c->weyl_on;
        view.cfg[0] = c->cfg[0];
        view.cfg[1] = c->cfg[1];
        view.blk[0] = c->blk[0];
        view.blk[1] = c->blk[1];
        const uint64_t last = n - (uint64_t)(K - 1) * L;
        for (uint32_t i = 0; i < nstreams && gst == XG_OK; ++i) {
            char* row = static_cast<char*>(d_out) + (uint64_t)i * ld * 8;
            gst = enqueue(&view, kind, i * K, K - 1, L, row, L);
            if (gst == XG_OK) gst = enqueue(&view, kind, i * K + K - 1, 1, last, row + (uint64_t)(K - 1) * L * 8, last);
        }
        if (gst == XG_OK) e = xg64::launch_adopt_last_piece(c->st, first, nstreams, K, pieces, n, s);
    }
    cudaFreeAsync(scratch, s);
    if (gst != XG_OK) return gst;
    if (e != cudaSuccess) return cuda_fail(e, "64-bit cut generation");
    return XG_OK;
}

// Host output: generate into one device buffer piece by piece and copy each
// piece out (synchronously); pieces split the stream range and, for long
// requests, each stream's length.
xg_status to_host(xg_w64_ctx* c, int kind, uint32_t first, uint32_t nstreams, uint64_t n, void* h_out,
                  uint64_t ld)
{
    const size_t kPieceBytes = size_t(128) << 20;
    if (c->staging_bytes < kPieceBytes) {
        if (c->staging) cudaFree(c->staging);
        c->staging = nullptr;
        c->staging_bytes = 0;
        XG_CUDA(cudaMalloc(&c->staging, kPieceBytes), "cudaMalloc(staging)");
        c->staging_bytes = kPieceBytes;
    }
    const uint64_t words = kPieceBytes / 8;
    const uint64_t ncols = std::max<uint64_t>(1, std::min<uint64_t>(n, words));
    const uint64_t ld_stage = align_up(ncols, 2);
    const uint32_t rows_per = (uint32_t)std::max<uint64_t>(1, words / ld_stage);
    for (uint32_t r0 = 0; r0 < nstreams; r0 += rows_per) {
        const uint32_t rows = std::min<uint32_t>(rows_per, nstreams - r0);
        for (uint64_t c0 = 0; c0 < n; c0 += ncols) {
            const uint64_t cols = std::min<uint64_t>(ncols, n - c0);
            xg_status st = enqueue(c, kind, first + r0, rows, cols, c->staging, ld_stage);
            if (st != XG_OK) return st;
            char* dst = static_cast<char*>(h_out) + ((uint64_t)r0 * ld + c0) * 8;
            XG_CUDA(cudaMemcpy2DAsync(dst, ld * 8, c->staging, ld_stage * 8, cols * 8, rows,
                                      cudaMemcpyDeviceToHost, c->stream),
                    "cudaMemcpy2DAsync(device to host)");
        }
    }
    XG_CUDA(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return XG_OK;
}

xg_status generate(xg_w64_ctx* c, int kind, uint32_t first, uint32_t nstreams, uint64_t n, void* out,
                   uint64_t ld)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if ((uint64_t)first + nstreams > c->n)
        return fail(XG_EINVAL, "streams [%u, %u) out of range (context has %u)", first, first + nstreams, c->n);
    if (nstreams == 0 || n == 0) return XG_OK;
    if (!out) return fail(XG_EINVAL, "null output pointer");
    if (nstreams > 1 && ld < n)
        return fail(XG_EINVAL, "ld (%llu) < n_per_stream (%llu)", (unsigned long long)ld, (unsigned long long)n);
    if (nstreams == 1 && ld < n) ld = n;
    if (ld > (UINT64_MAX / 16) / nstreams) return fail(XG_EINVAL, "output extent overflows");
    if (reinterpret_cast<uintptr_t>(out) & 7u) return fail(XG_EINVAL, "output must be 8-byte aligned");
    std::lock_guard<std::mutex> lk(c->mu);
    if (is_device_pointer(out)) {
        if (nstreams <= kCutMaxStreams && n >= kCutMinWords && c->split_words != 1)
            return generate_cut(c, kind, first, nstreams, n, out, ld);
        return enqueue(c, kind, first, nstreams, n, out, ld);
    }
    return to_host(c, kind, first, nstreams, n, out, ld);
}

}  // namespace

extern "C" {

xg_status xg_w64_params(uint32_t* rsabcd, uint64_t* omega)
{
    if (!rsabcd || !omega) return fail(XG_EINVAL, "null output");
    const uint32_t v[6] = {xg64::kR, xg64::kS, xg64::kA, xg64::kB, xg64::kC, xg64::kD};
    std::memcpy(rsabcd, v, sizeof v);
    *omega = xg64::kOmega;
    return XG_OK;
}

xg_status xg_w64_create(xg_w64_ctx** out, uint32_t n_streams, uint32_t weyl_on, void* cuda_stream)
{
    if (!out) return fail(XG_EINVAL, "null output handle");
    *out = nullptr;
    if (n_streams == 0) return fail(XG_EINVAL, "n_streams must be positive");
    xg_w64_ctx* c = new (std::nothrow) xg_w64_ctx();
    if (!c) return fail(XG_ENOMEM, "host allocation failed");
    c->n = n_streams;
    c->weyl_on = weyl_on ? 1u : 0u;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    const size_t off_weyl = align_up((size_t)n_streams * xg64::kWin * 8, 256);
    const size_t off_pend = align_up(off_weyl + (size_t)n_streams * 8, 256);
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
    c->state_bytes = total;
    char* base = static_cast<char*>(c->state_mem);
    c->st.win = reinterpret_cast<uint64_t*>(base);
    c->st.weyl = reinterpret_cast<uint64_t*>(base + off_weyl);
    c->st.pend = reinterpret_cast<uint32_t*>(base + off_pend);
    c->st.pos = reinterpret_cast<uint64_t*>(base + off_pos);
    e = cudaMemsetAsync(c->state_mem, 0, total, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        xg_status st = cuda_fail(e, "create");
        xg_w64_destroy(c);
        return st;
    }
    *out = c;
    return XG_OK;
}

xg_status xg_w64_destroy(xg_w64_ctx* c)
{
    if (!c) return XG_OK;
    if (c->state_mem) cudaStreamSynchronize(c->stream);
    if (c->staging) cudaFree(c->staging);
    if (c->state_mem) cudaFree(c->state_mem);
    delete c;
    return XG_OK;
}

xg_status xg_w64_set_stream(xg_w64_ctx* c, void* cuda_stream)
{
    if (!c) return fail(XG_EINVAL, "null context");
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    return XG_OK;
}

xg_status xg_w64_seed(xg_w64_ctx* c, uint32_t first, uint32_t count, const uint32_t* host_seeds)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if ((uint64_t)first + count > c->n) return fail(XG_EINVAL, "seed range out of bounds");
    if (count == 0) return XG_OK;
    if (!host_seeds) return fail(XG_EINVAL, "null seeds");
    std::lock_guard<std::mutex> lk(c->mu);
    uint32_t* d = nullptr;
    XG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), (size_t)count * 4, c->stream), "cudaMallocAsync(seeds)");
    cudaError_t e = cudaMemcpyAsync(d, host_seeds, (size_t)count * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = xg64::launch_seed(c->st, d, first, count, c->stream);
    cudaError_t e2 = cudaFreeAsync(d, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "seed");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync(seeds)");
    if (!c->weyl_on)
        XG_CUDA(cudaMemsetAsync(c->st.weyl + first, 0, (size_t)count * 8, c->stream), "cudaMemsetAsync");
    return XG_OK;
}

xg_status xg_w64_get_state(xg_w64_ctx* c, uint32_t stream, uint64_t* ring, uint64_t* weyl)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if (stream >= c->n) return fail(XG_EINVAL, "stream %u out of range", stream);
    if (!ring || !weyl) return fail(XG_EINVAL, "null output");
    std::lock_guard<std::mutex> lk(c->mu);
    uint64_t win[xg64::kWin], w = 0;
    uint32_t pend = 0;
    XG_CUDA(cudaMemcpyAsync(win, c->st.win + (size_t)stream * xg64::kWin, sizeof win, cudaMemcpyDeviceToHost,
                            c->stream), "get_state");
    XG_CUDA(cudaMemcpyAsync(&pend, c->st.pend + stream, 4, cudaMemcpyDeviceToHost, c->stream), "get_state");
    XG_CUDA(cudaMemcpyAsync(&w, c->st.weyl + stream, 8, cudaMemcpyDeviceToHost, c->stream), "get_state");
    XG_CUDA(cudaStreamSynchronize(c->stream), "get_state");
    if (pend >= (uint32_t)xg64::kRingBase) return fail(XG_EDEVICE, "corrupt stream state (pend %u)", pend);
    std::memcpy(ring, win + xg64::kRingBase - pend, xg64::kR * 8);
    *weyl = w;
    return XG_OK;
}

xg_status xg_w64_set_state(xg_w64_ctx* c, uint32_t stream, const uint64_t* ring, uint64_t weyl)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if (stream >= c->n) return fail(XG_EINVAL, "stream %u out of range", stream);
    if (!ring) return fail(XG_EINVAL, "null ring");
    std::lock_guard<std::mutex> lk(c->mu);
    uint64_t win[xg64::kWin] = {0};
    std::memcpy(win + xg64::kRingBase, ring, xg64::kR * 8);
    const uint32_t pend = 0;
    const uint64_t w = c->weyl_on ? weyl : 0;
    XG_CUDA(cudaMemcpyAsync(c->st.win + (size_t)stream * xg64::kWin, win, sizeof win, cudaMemcpyHostToDevice,
                            c->stream), "set_state");
    XG_CUDA(cudaMemcpyAsync(c->st.pend + stream, &pend, 4, cudaMemcpyHostToDevice, c->stream), "set_state");
    XG_CUDA(cudaMemcpyAsync(c->st.weyl + stream, &w, 8, cudaMemcpyHostToDevice, c->stream), "set_state");
    XG_CUDA(cudaStreamSynchronize(c->stream), "set_state");
    return XG_OK;
}

xg_status xg_w64_generate_u64(xg_w64_ctx* c, uint32_t first, uint32_t nstreams, uint64_t n, uint64_t* out,
                              uint64_t ld)
{
    return generate(c, xg64::kU64, first, nstreams, n, out, ld);
}

xg_status xg_w64_generate_uniform_f64(xg_w64_ctx* c, uint32_t first, uint32_t nstreams, uint64_t n, double* out,
                                      uint64_t ld)
{
    return generate(c, xg64::kUniformF64, first, nstreams, n, out, ld);
}

xg_status xg_w64_set_split(xg_w64_ctx* c, uint64_t piece_words)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if (piece_words > 1 && (piece_words < 64 || (piece_words & (piece_words - 1))))
        return fail(XG_EINVAL, "piece length must be 0, 1 or a power of two >= 64");
    c->split_words = piece_words;
    return XG_OK;
}

xg_status xg_w64_jump(xg_w64_ctx* c, uint32_t first, uint32_t nstreams, uint64_t words)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if ((uint64_t)first + nstreams > c->n) return fail(XG_EINVAL, "streams out of range");
    if (nstreams == 0 || words == 0) return XG_OK;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t s = c->stream;
    int top = 63;
    while (!((words >> top) & 1)) --top;
    xg_status st = XG_OK;
    for (int k = 0; k <= top; ++k)
        if (((words >> k) & 1) && !xg::jump_matrix(c->device, xg::kJumpSetW64, k, s, &st)) return st;
    // one allocation: rings[0, n) hold the states, rings[n, 2n) the second
    // buffer (the shared GF(2) kernels work on 4096-bit states as 128 32-bit
    // words); index lists (0 .. n-1, then 0 .. 2n-1, built on the device);
    // the jump's work area
    const size_t rings_bytes = (size_t)2 * nstreams * xg64::kR * 8;
    const size_t work_off = (rings_bytes + (size_t)3 * nstreams * 4 + 255) / 256 * 256;
    const size_t wbytes = xg::gf2_jump_work_bytes(c->device, nstreams, words);
    const size_t tc_bytes = xg::gf2_apply_scratch(c->device, nstreams);
    char* ws = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), work_off + wbytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "xg_w64_jump scratch");
    uint64_t* rings = reinterpret_cast<uint64_t*>(ws);
    uint32_t* rings32 = reinterpret_cast<uint32_t*>(ws);
    uint32_t* ids = reinterpret_cast<uint32_t*>(ws + rings_bytes);
    const uint32_t* lo_idx = ids + nstreams;  // 0 .. 2n-1
    e = xg::launch_jump_index(ids, nstreams, 0u, s);
    if (e == cudaSuccess) e = xg64::launch_gather_rings(c->st, first, nstreams, rings, s);
    bool hi = false;
    if (e == cudaSuccess)
        e = xg::gf2_jump_states(c->device, xg::kJumpSetW64, words, rings32, nstreams, lo_idx,
                                reinterpret_cast<uint8_t*>(ws + work_off), c->sm_count, s, &st, &hi);
    const bool in_lo = !hi;
    if (e == cudaSuccess) {
        const uint64_t* res = in_lo ? rings : rings + (size_t)nstreams * xg64::kR;
        e = xg64::launch_scatter_rings(c->st, first, nstreams, res, words, c->weyl_on ? xg64::kOmega : 0, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(ws, s);
    if (st != XG_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "xg_w64_jump");
    if (tc_bytes && xg::gf2_tc_take_failure())
        return fail(XG_EDEVICE, "xg_w64_jump: a tensor-core kernel gave up waiting; the streams are not valid");
    return XG_OK;
}

xg_status xg_w64_seed_substreams(xg_w64_ctx* c, uint32_t first, uint32_t count, uint32_t seed,
                                 uint32_t log2_spacing)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if ((uint64_t)first + count > c->n) return fail(XG_EINVAL, "streams out of range");
    if (count == 0) return XG_OK;
    int steps = 0;   // doubling steps: bits of count - 1
    while (steps < 32 && ((uint64_t)(count - 1) >> steps)) ++steps;
    if (log2_spacing > 63 || (count > 1 && (int)log2_spacing + steps > 64))
        return fail(XG_EINVAL, "(count - 1) * 2^%u does not fit in 64 bits", log2_spacing);
    if (xg_status s = xg_w64_seed(c, first, 1, &seed)) return s;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t s = c->stream;
    const int q = (int)log2_spacing;
    xg_status st = XG_OK;
    for (int b = 0; b < steps; ++b)
        if (!xg::jump_matrix(c->device, xg::kJumpSetW64, q + b, s, &st)) return st;
    // step b takes the states m - 2^b to the states m, m in [2^b, min(2^(b+1), count)):
    // its sources are the identity list from 0 and its destinations the same
    // list from 2^b, so one device-built list 0 .. 2 count - 1 serves every step
    uint32_t most = 0;
    for (int b = 0; b < steps; ++b) {
        const uint32_t lo = 1u << b, hi = (uint32_t)std::min<uint64_t>((uint64_t)lo << 1, count);
        most = std::max(most, hi - lo);
    }
    // one workspace: rings of all count states; the index lists (0 .. count - 1,
    // then 0 .. 2 count - 1); the base Weyl word (8-byte aligned); the
    // tensor-core operand (256-byte aligned, when used)
    const size_t rings_bytes = (size_t)count * xg64::kR * 8;
    const size_t ids_off = rings_bytes;
    const size_t w0_off = (ids_off + (size_t)3 * count * 4 + 7) / 8 * 8;
    const size_t tc_off = (w0_off + 8 + 255) / 256 * 256;
    const size_t tc_bytes = xg::gf2_apply_scratch(c->device, most);
    char* ws = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), tc_off + tc_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "xg_w64_seed_substreams scratch");
    uint64_t* rings = reinterpret_cast<uint64_t*>(ws);
    uint32_t* ids = reinterpret_cast<uint32_t*>(ws + ids_off);
    const uint32_t* iota = ids + count;
    uint64_t* d_w0 = reinterpret_cast<uint64_t*>(ws + w0_off);
    uint8_t* tc_scratch = tc_bytes ? reinterpret_cast<uint8_t*>(ws + tc_off) : nullptr;
    uint32_t* rings32 = reinterpret_cast<uint32_t*>(rings);
    e = xg::launch_jump_index(ids, count, 0u, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_w0, c->st.weyl + first, 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = xg64::launch_gather_rings(c->st, first, 1, rings, s);
    // the destinations 1 .. count - 1, zeroed once for all the steps
    if (e == cudaSuccess && count > 1)
        e = cudaMemsetAsync(rings + xg64::kR, 0, (size_t)(count - 1) * xg64::kR * 8, s);
    for (int b = 0; b < steps && e == cudaSuccess; ++b) {
        const uint32_t lo = 1u << b, hi = (uint32_t)std::min<uint64_t>((uint64_t)lo << 1, count);
        e = xg::gf2_apply(c->device, xg::kJumpSetW64, q + b, rings32, hi - lo, iota, iota + lo, tc_scratch,
                          c->sm_count, s, &st, true);
    }
    if (e == cudaSuccess)
        e = xg64::launch_substream_scatter(c->st, first, count, rings, d_w0, q, c->weyl_on ? xg64::kOmega : 0, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(ws, s);
    if (st != XG_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "xg_w64_seed_substreams");
    if (tc_bytes && xg::gf2_tc_take_failure())
        return fail(XG_EDEVICE, "xg_w64_seed_substreams: a tensor-core kernel gave up waiting; the streams are not valid");
    return XG_OK;
}

xg_status xg_w64_transform_uniform_f64(xg_w64_ctx* c, const uint64_t* d_words, uint64_t n, double* d_out)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if (n == 0) return XG_OK;
    if (!d_words || !d_out) return fail(XG_EINVAL, "null pointer");
    if ((reinterpret_cast<uintptr_t>(d_words) | reinterpret_cast<uintptr_t>(d_out)) & 7u)
        return fail(XG_EINVAL, "buffers must be 8-byte aligned");
    cudaError_t e = xg64::launch_transform_uniform(d_words, n, reinterpret_cast<uint64_t*>(d_out), c->sm_count,
                                                   c->stream);
    return e == cudaSuccess ? XG_OK : cuda_fail(e, "64-bit transform_uniform");
}

xg_status xg_w64_set_launch(xg_w64_ctx* c, xg_w64_type type, uint32_t tpg, uint32_t wpl, uint32_t block)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if ((unsigned)type > XG_W64_UNIFORM_F64) return fail(XG_EINVAL, "unknown output type");
    if (block > 1024 || (block & 31u)) return fail(XG_EINVAL, "block must be a multiple of 32, at most 1024");
    if (tpg == 0 && wpl == 0) {
        c->cfg[type] = -1;
        c->blk[type] = 0;
        return XG_OK;
    }
    const int ci = xg64::cfg_index((int)tpg, (int)wpl);
    if (ci < 0) return fail(XG_EINVAL, "unsupported launch (tpg %u, wpl %u)", tpg, wpl);
    c->cfg[type] = ci;
    c->blk[type] = (int)block;
    return XG_OK;
}

xg_status xg_w64_autotune(xg_w64_ctx* c, xg_w64_type type, uint32_t nstreams, uint64_t n_per_stream,
                          uint32_t* tpg, uint32_t* wpl, uint32_t* block, float* best_ms)
{
    if (!c) return fail(XG_EINVAL, "null context");
    if ((unsigned)type > XG_W64_UNIFORM_F64) return fail(XG_EINVAL, "unknown output type");
    if (nstreams == 0 || nstreams > c->n) nstreams = c->n;
    if (n_per_stream == 0) return fail(XG_EINVAL, "n_per_stream must be positive");
    uint64_t nt = std::min<uint64_t>(n_per_stream, std::max<uint64_t>(128, (uint64_t(1) << 26) / nstreams));
    nt = align_up(nt, 32);
    std::lock_guard<std::mutex> lk(c->mu);
    void* saved = nullptr;
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (saved) {
            cudaMemcpyAsync(c->state_mem, saved, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
            cudaStreamSynchronize(c->stream);
            cudaFree(saved);
        }
        if (out) cudaFree(out);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&saved, c->state_bytes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(saved, c->state_mem, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)nstreams * nt * 8);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return cuda_fail(e, "autotune set-up");
    }
    static const int kBlocks[] = {32, 64, 128, 256};
    int best_cfg = -1, best_block = 0;
    float best = 1e30f;
    xg_status st = XG_OK;
    for (int ci = 0; ci < xg64::kNumCfgs && st == XG_OK; ++ci) {
        for (int b : kBlocks) {
            st = enqueue(c, type, 0, nstreams, nt, out, nt, ci, b);
            if (st != XG_OK) break;
            cudaEventRecord(e0, c->stream);
            for (int r = 0; r < 3 && st == XG_OK; ++r) st = enqueue(c, type, 0, nstreams, nt, out, nt, ci, b);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = cuda_fail(cudaGetLastError(), "autotune timing");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
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
    if (tpg) *tpg = (uint32_t)xg64::kCfgs[best_cfg].tpg;
    if (wpl) *wpl = (uint32_t)xg64::kCfgs[best_cfg].wpl;
    if (block) *block = (uint32_t)best_block;
    if (best_ms) *best_ms = best;
    return XG_OK;
}

}  // extern "C"
