// Jump-ahead for xorgens streams.
//
// The recurrence of Sec. 2 is linear over GF(2) on the 4096-bit state (the
// 128-word ring): one step maps a state v to M v.  A stream advanced by J
// words is M^J v, and with the powers C_k = M^(2^k) at hand, M^J v is the
// product of the C_k for the set bits of J.  This lets one long stream be cut
// into pieces that run on different warps (Sec. 2's independent subsequences,
// here exact consecutive pieces of one sequence) and lets xg_jump skip ahead
// without generating.  The Weyl word needs no matrix: w + J omega.
//
// Matrices are kept in column form: column j of C is the state reached from
// the unit state e_j (bit j of ring word j/32).  Applying C to v is the XOR of
// the columns selected by v's bits; squaring is applying C to its own columns.
// The columns of M itself are one step of the recurrence applied to e_j.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "xg_gf2_tc.h"
#include "xg_jump.h"
#include "xg_kernels.cuh"
#include "xg_runtime.h"
#include "xg_w64.h"

namespace xg {

constexpr int kBits = 4096;      // state bits
constexpr int kWords64 = 64;     // uint64 words per state
constexpr int kApplyVecs = 16;   // states per block in gf2_apply_kernel

// Columns of M for parameter set P: column j = one step from e_j.
template <class P>
__global__ void __launch_bounds__(128) step_columns_kernel(uint32_t* __restrict__ cols)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kBits) return;
    const int wj = j >> 5, bj = j & 31;
    uint32_t* out = cols + (size_t)j * kR;
    // the ring shifts by one word: word w of the result is word w+1 of e_j
    for (int w = 0; w < kR - 1; ++w) out[w] = (w + 1 == wj) ? (1u << bj) : 0u;
    // the new word: x_{k-r} is ring word 0, x_{k-s} is ring word r - s
    uint32_t t = (wj == 0) ? (1u << bj) : 0u;
    uint32_t u = (wj == kR - P::S) ? (1u << bj) : 0u;
    t ^= t << P::A;
    t ^= t >> P::B;
    u ^= u << P::C;
    u ^= u >> P::D;
    out[kR - 1] = t ^ u;
}

// out[i] = C in[i] for the n states listed in idx (or 0..n-1 when idx is
// null).  64 threads per block, thread t owns uint64 word t of the results;
// each column of C is loaded once per block and shared by its 16 states.
// in and out may be the same array: a block reads its states before writing.
__global__ void __launch_bounds__(64) gf2_apply_kernel(const uint64_t* __restrict__ C, const uint64_t* in,
                                                       uint64_t* out, uint32_t n, const uint32_t* __restrict__ idx)
{
    __shared__ uint64_t vin[kApplyVecs][kWords64];
    const int t = threadIdx.x;
    const uint32_t base = blockIdx.x * kApplyVecs;
    const int nv = (int)umin((uint32_t)kApplyVecs, n - base);
    for (int v = 0; v < nv; ++v) {
        const uint32_t i = idx ? idx[base + v] : base + v;
        vin[v][t] = in[(size_t)i * kWords64 + t];
    }
    __syncthreads();
    uint64_t acc[kApplyVecs];
#pragma unroll
    for (int v = 0; v < kApplyVecs; ++v) acc[v] = 0;
    for (int w = 0; w < kWords64; ++w) {
        uint64_t bits[kApplyVecs];
        uint64_t any = 0;
#pragma unroll
        for (int v = 0; v < kApplyVecs; ++v) {
            bits[v] = v < nv ? vin[v][w] : 0ull;
            any |= bits[v];
        }
        while (any) {
            const int b = __ffsll((long long)any) - 1;
            any &= any - 1;
            const uint64_t col = C[(size_t)(w * 64 + b) * kWords64 + t];
#pragma unroll
            for (int v = 0; v < kApplyVecs; ++v) acc[v] ^= col & (0ull - ((bits[v] >> b) & 1ull));
        }
    }
#pragma unroll
    for (int v = 0; v < kApplyVecs; ++v) {
        if (v < nv) {
            const uint32_t i = idx ? idx[base + v] : base + v;
            out[(size_t)i * kWords64 + t] = acc[v];
        }
    }
}

// dst[i] ^= C src[i] for n (src, dst) pairs, dst zeroed beforehand.  Block
// (x, y): pairs [48x, 48x+48), columns [y*cols, (y+1)*cols); 128 threads,
// thread t owns 32-bit word t of every result.  Columns go four at a time:
// each thread tabulates the 16 XOR combinations of its word of the four
// columns (in shared memory, its own column of the table, so no barrier is
// needed), and a state then costs one lookup and one XOR per four columns.
// Partial results are folded into dst with one atomic XOR per pair.  The
// shared-memory traffic of the lookups and of building the tables bounds the
// kernel, so many states per block (NV = 48) spread each table over more
// lookups: on GB300, 16384 states x 8 applications take 3.3 ms against
// 5.1 ms with 16 (64 gains no more and needs 168 registers a thread).  Few
// states take NV = 16, which pads less.
template <int kPairVecs>
// rings and out are the same array (sources are read, distinct destinations
// are written), so neither is declared __restrict__.
__global__ void __launch_bounds__(128) gf2_apply_pairs_kernel(const uint32_t* __restrict__ C,
                                                              const uint32_t* rings,
                                                              const uint32_t* __restrict__ src,
                                                              const uint32_t* __restrict__ dst, uint32_t n,
                                                              uint32_t* out, int cols)
{
    __shared__ uint32_t vbits[kPairVecs][kR];
    __shared__ uint32_t tbl[16][kR];
    const int t = threadIdx.x;
    const uint32_t base = blockIdx.x * kPairVecs;
    const int nv = (int)umin((uint32_t)kPairVecs, n - base);
    for (int v = 0; v < kPairVecs; ++v)
        vbits[v][t] = v < nv ? rings[(size_t)src[base + v] * kR + t] : 0u;
    __syncthreads();
    uint32_t acc[kPairVecs];
#pragma unroll
    for (int v = 0; v < kPairVecs; ++v) acc[v] = 0;
    const int w0 = blockIdx.y * (cols / 32), w1 = w0 + cols / 32;
    for (int w = w0; w < w1; ++w) {  // 32 columns per input word
        const uint32_t* colw = C + (size_t)w * 32 * kR + t;
        uint32_t col[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) col[b] = __ldg(colw + (size_t)b * kR);
        uint32_t bw[kPairVecs];
#pragma unroll
        for (int v = 0; v < kPairVecs; ++v) bw[v] = vbits[v][w];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const uint32_t c0 = col[4 * g], c1 = col[4 * g + 1], c2 = col[4 * g + 2], c3 = col[4 * g + 3];
            const uint32_t c01 = c0 ^ c1, c23 = c2 ^ c3;
            tbl[0][t] = 0u;        tbl[1][t] = c0;         tbl[2][t] = c1;         tbl[3][t] = c01;
            tbl[4][t] = c2;        tbl[5][t] = c2 ^ c0;    tbl[6][t] = c2 ^ c1;    tbl[7][t] = c2 ^ c01;
            tbl[8][t] = c3;        tbl[9][t] = c3 ^ c0;    tbl[10][t] = c3 ^ c1;   tbl[11][t] = c3 ^ c01;
            tbl[12][t] = c23;      tbl[13][t] = c23 ^ c0;  tbl[14][t] = c23 ^ c1;  tbl[15][t] = c23 ^ c01;
#pragma unroll
            for (int v = 0; v < kPairVecs; ++v) acc[v] ^= tbl[(bw[v] >> (4 * g)) & 15u][t];
        }
    }
#pragma unroll
    for (int v = 0; v < kPairVecs; ++v)
        if (v < nv && acc[v]) atomicXor(&out[(size_t)dst[base + v] * kR + t], acc[v]);
}

__global__ void zero_listed_kernel(uint32_t* __restrict__ rings, const uint32_t* __restrict__ idx, uint32_t n)
{
    const uint32_t j = blockIdx.x;
    if (j < n) rings[(size_t)idx[j] * kR + threadIdx.x] = 0u;
}

// Copy each listed stream's current ring (window at its pend offset) into
// rings[k]; also rings' Weyl words advanced by skip[k] words.  With skips,
// an entry with a nonzero skip gets a zero ring instead: its ring is the
// result of a later jump-ahead step, which XORs into it.
__global__ void gather_rings_kernel(State st, const uint32_t* __restrict__ streams, uint32_t n,
                                    uint32_t* __restrict__ rings, const uint64_t* __restrict__ skip,
                                    uint32_t* __restrict__ weyl0, uint32_t weyl0_stride, uint32_t omega)
{
    const uint32_t k = blockIdx.x;
    if (k >= n) return;
    const uint32_t s = streams[k];
    const uint32_t pend = st.pend[s];
    const uint32_t* src = st.win + (size_t)s * kWin + (kRingBase - pend);
    const bool zero = skip && skip[k] != 0;
    for (int w = threadIdx.x; w < kR; w += blockDim.x) rings[(size_t)k * kR + w] = zero ? 0u : src[w];
    if (threadIdx.x == 0 && weyl0)
        weyl0[(size_t)k * weyl0_stride] = st.weyl[s] + (uint32_t)(skip ? skip[k] : 0) * omega;
}

// Write jumped rings back as the streams' state (pend = 0; the ring sits at
// window[kRingBase, kWin)).
__global__ void scatter_rings_kernel(State st, uint32_t first, uint32_t n, const uint32_t* __restrict__ rings,
                                     uint64_t jump, uint32_t omega)
{
    const uint32_t k = blockIdx.x;
    if (k >= n) return;
    const uint32_t s = first + k;
    uint32_t* dst = st.win + (size_t)s * kWin + kRingBase;
    for (int w = threadIdx.x; w < kR; w += blockDim.x) dst[w] = rings[(size_t)k * kR + w];
    if (threadIdx.x == 0) {
        st.weyl[s] += (uint32_t)jump * omega;
        st.pend[s] = 0;
        st.pos[s] += jump;
    }
}

// Substreams: stream first + m takes rings[m] (its ring after m * 2^q words
// of the seeded sequence), the Weyl word w0 + m 2^q omega and position m 2^q.
__global__ void substream_scatter_kernel(State st, uint32_t first, uint32_t n, const uint32_t* __restrict__ rings,
                                         const uint32_t* __restrict__ w0, int q, uint32_t omega)
{
    const uint32_t m = blockIdx.x;
    if (m >= n) return;
    const uint32_t s = first + m;
    uint32_t* dst = st.win + (size_t)s * kWin + kRingBase;
    for (int w = threadIdx.x; w < kR; w += blockDim.x) dst[w] = rings[(size_t)m * kR + w];
    if (threadIdx.x == 0) {
        const uint64_t off = (uint64_t)m << q;
        st.weyl[s] = *w0 + (uint32_t)off * omega;
        st.pend[s] = 0;
        st.pos[s] = off;
    }
}

// ---------------------------------------------------------------------------

namespace {
struct Tables {
    uint64_t* mat[kMaxPow] = {};  // C_k: 4096 columns x 64 uint64 (2 MiB), allocated when built
    int built = 0;                // C_0 .. C_{built-1} are valid
};
std::mutex g_tab_mu;
Tables g_tabs[64][3];  // per device, per matrix family
}  // namespace

const uint64_t* jump_matrix(int device, int param_set, int k, cudaStream_t s, xg_status* st)
{
    *st = XG_OK;
    if (device < 0 || device >= 64 || k < 0 || k >= kMaxPow || param_set < 0 || param_set > kJumpSetW64) {
        *st = fail(XG_EINVAL, "jump power %d out of range", k);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_tab_mu);
    Tables& T = g_tabs[device][param_set];
    const size_t mat_bytes = (size_t)kBits * kWords64 * 8;
    bool built_now = false;
    while (T.built <= k) {
        const int b = T.built;
        cudaError_t e = cudaMalloc(&T.mat[b], mat_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            T.mat[b] = nullptr;
            *st = fail(XG_ENOMEM, "jump tables: cudaMalloc(2 MiB) failed for power %d", b);
            return nullptr;
        }
        if (b == 0) {
            if (param_set == kJumpSetW64)
                e = xg64::launch_step_columns(T.mat[0], s);
            else if (param_set == 1)
                step_columns_kernel<ParamsPaper><<<kBits / 128, 128, 0, s>>>(reinterpret_cast<uint32_t*>(T.mat[0]));
            else
                step_columns_kernel<ParamsDefault><<<kBits / 128, 128, 0, s>>>(reinterpret_cast<uint32_t*>(T.mat[0]));
        } else {
            gf2_apply_kernel<<<kBits / kApplyVecs, 64, 0, s>>>(T.mat[b - 1], T.mat[b - 1], T.mat[b], kBits, nullptr);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "jump table build");
            return nullptr;
        }
        T.built = b + 1;
        built_now = true;
    }
    // other CUDA streams may use the tables next: make the build complete
    if (built_now && cudaStreamSynchronize(s) != cudaSuccess) {
        *st = cuda_fail(cudaGetLastError(), "jump table build");
        return nullptr;
    }
    return T.mat[k];
}

namespace {
// FP8 copies of the powers for the tensor-core path: 16 MiB each, built on
// first use and kept until exit.
std::mutex g_tc_mu;
uint8_t* g_tc_mats[64][3][kMaxPow] = {};

const uint8_t* jump_matrix_tc(int device, int family, int k, cudaStream_t s, xg_status* st)
{
    const uint64_t* C = jump_matrix(device, family, k, s, st);
    if (!C) return nullptr;
    std::lock_guard<std::mutex> lk(g_tc_mu);
    uint8_t*& A = g_tc_mats[device][family][k];
    if (A) return A;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, (size_t)kGf2Bits * kGf2Bits);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *st = fail(XG_ENOMEM, "jump tables: cudaMalloc(16 MiB) failed for the FP8 power %d", k);
        return nullptr;
    }
    e = gf2_tc_expand_matrix(C, static_cast<uint8_t*>(p), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // other CUDA streams may use it next
    if (e != cudaSuccess) {
        cudaFree(p);
        *st = cuda_fail(e, "jump tables: FP8 expansion");
        return nullptr;
    }
    A = static_cast<uint8_t*>(p);
    return A;
}
}  // namespace

bool gf2_use_tc(int device, uint32_t n)
{
    // read on every call (a few hundred nanoseconds against a matrix application)
    const char* off = std::getenv("XG_JUMP_TENSOR_CORES");
    if (off && std::strcmp(off, "0") == 0) return false;
    const char* v = std::getenv("XG_GF2_TC_MIN_STATES");
    const uint32_t min_states = v ? (uint32_t)std::strtoul(v, nullptr, 10) : 1024u;
    return n >= std::max(1u, min_states) && gf2_tc_available(device);
}

size_t gf2_apply_scratch(int device, uint32_t n)
{
    return gf2_use_tc(device, n) ? gf2_tc_scratch_bytes(n) : 0;
}

cudaError_t gf2_apply(int device, int family, int k, uint32_t* rings, uint32_t n, const uint32_t* d_src,
                      const uint32_t* d_dst, uint8_t* scratch, int sm_count, cudaStream_t s, xg_status* st,
                      bool dst_zeroed)
{
    *st = XG_OK;
    if (n == 0) return cudaSuccess;
    if (scratch && gf2_use_tc(device, n)) {
        const uint8_t* A = jump_matrix_tc(device, family, k, s, st);
        if (!A) return cudaErrorMemoryAllocation;
        return gf2_tc_apply(device, A, rings, d_src, n, rings, d_dst, scratch, s);
    }
    const uint64_t* C = jump_matrix(device, family, k, s, st);
    if (!C) return cudaErrorMemoryAllocation;
    cudaError_t e = dst_zeroed ? cudaSuccess : zero_rings(rings, d_dst, n, s);
    if (e == cudaSuccess) e = launch_gf2_apply_pairs(C, rings, n, d_src, d_dst, sm_count, s);
    return e;
}

// rings[dst[i]] = P rings[src[i]] for a matrix P in column form that is not
// one of the cached powers; A_buf (16 MiB) receives its FP8 copy when the
// tensor cores are used.
static cudaError_t gf2_apply_explicit(int device, const uint64_t* P, uint8_t* A_buf, uint32_t* rings, uint32_t n,
                                      const uint32_t* d_src, const uint32_t* d_dst, uint8_t* scratch, int sm_count,
                                      cudaStream_t s)
{
    if (scratch && A_buf && gf2_use_tc(device, n)) {
        cudaError_t e = gf2_tc_expand_matrix(P, A_buf, s);
        if (e == cudaSuccess) e = gf2_tc_apply(device, A_buf, rings, d_src, n, rings, d_dst, scratch, s);
        return e;
    }
    cudaError_t e = zero_rings(rings, d_dst, n, s);
    if (e == cudaSuccess) e = launch_gf2_apply_pairs(P, rings, n, d_src, d_dst, sm_count, s);
    return e;
}

static bool jump_combines(uint64_t words, uint32_t n)
{
    return __builtin_popcountll(words) >= 2 && n > (uint32_t)kGf2Bits;
}

size_t gf2_jump_work_bytes(int device, uint32_t n, uint64_t words)
{
    // the tensor-core operand (the product of powers, n > 4096, applies to
    // 4096 columns, fewer than n), then the product matrix pair and its FP8
    // copy when the powers are multiplied first
    size_t b = (gf2_apply_scratch(device, n) + 255) / 256 * 256;
    if (jump_combines(words, n)) {
        b += (size_t)2 * kBits * kR * 4;
        if (gf2_use_tc(device, n)) b += (size_t)kGf2Bits * kGf2Bits;
    }
    return b;
}

cudaError_t gf2_jump_states(int device, int family, uint64_t words, uint32_t* rings, uint32_t n,
                            const uint32_t* d_idx, uint8_t* work, int sm_count, cudaStream_t s, xg_status* st,
                            bool* result_hi)
{
    *st = XG_OK;
    *result_hi = false;
    const uint32_t* lo = d_idx;       // 0 .. n-1
    const uint32_t* hi = d_idx + n;   // n .. 2n-1
    const size_t sbytes = gf2_apply_scratch(device, n);
    uint8_t* scratch = sbytes ? work : nullptr;
    if (!jump_combines(words, n)) {
        bool in_lo = true;
        for (int k = 0; k < 64; ++k) {
            if (!((words >> k) & 1)) continue;
            cudaError_t e = gf2_apply(device, family, k, rings, n, in_lo ? lo : hi, in_lo ? hi : lo, scratch, sm_count, s, st);
            if (e != cudaSuccess) return e;
            in_lo = !in_lo;
        }
        *result_hi = !in_lo;
        return cudaSuccess;
    }
    // multiply the powers first (they commute: all are powers of one
    // matrix): b - 1 applications to the 4096 columns of a matrix in column
    // form, then one to the states -- (b - 1) 4096 + n state applications
    // instead of b n.  The identity list runs to 2n - 1 > 8191.
    uint8_t* w = work + (sbytes + 255) / 256 * 256;
    uint32_t* prod = reinterpret_cast<uint32_t*>(w);   // two 4096-column matrices (ping-pong)
    uint8_t* abuf = scratch ? w + (size_t)2 * kBits * kR * 4 : nullptr;  // FP8 copy of the product
    cudaError_t e = cudaSuccess;
    bool p_lo = true, first_bit = true;
    for (int k = 0; k < 64 && e == cudaSuccess; ++k) {
        if (!((words >> k) & 1)) continue;
        if (first_bit) {
            const uint64_t* C = jump_matrix(device, family, k, s, st);
            e = C ? cudaMemcpyAsync(prod, C, (size_t)kBits * kR * 4, cudaMemcpyDeviceToDevice, s)
                  : cudaErrorMemoryAllocation;
            first_bit = false;
            continue;
        }
        e = gf2_apply(device, family, k, prod, kBits, p_lo ? lo : lo + kBits, p_lo ? lo + kBits : lo, scratch,
                      sm_count, s, st);
        p_lo = !p_lo;
    }
    if (e == cudaSuccess) {
        const uint64_t* P = reinterpret_cast<const uint64_t*>(p_lo ? prod : prod + (size_t)kBits * kR);
        e = gf2_apply_explicit(device, P, abuf, rings, n, lo, hi, scratch, sm_count, s);
        *result_hi = true;
    }
    return e;
}

// ids[i] = first + i for i < n, then ids[n + j] = j for j < 2n.
__global__ void jump_index_kernel(uint32_t* __restrict__ ids, uint32_t n, uint32_t first)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ids[i] = first + (uint32_t)i;
    else if (i < (uint64_t)3 * n) ids[i] = (uint32_t)(i - n);
}

cudaError_t launch_jump_index(uint32_t* ids, uint32_t n, uint32_t first, cudaStream_t s)
{
    const uint64_t total = (uint64_t)3 * n;
    jump_index_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ids, n, first);
    return cudaGetLastError();
}

template <int NV>
static cudaError_t launch_pairs(const uint64_t* C, uint32_t* rings, uint32_t n, const uint32_t* d_src,
                                const uint32_t* d_dst, int sm_count, cudaStream_t s)
{
    const uint32_t groups = (n + NV - 1) / NV;
    // enough blocks for about 8 per SM, splitting the 4096 columns if needed
    // (down to one 32-column input word per block: with few states the
    // matrix read is the cost, spread over up to 128 blocks)
    int chunks = 1;
    while (chunks < kBits / 32 && (uint64_t)groups * chunks < (uint64_t)8 * sm_count) chunks *= 2;
    gf2_apply_pairs_kernel<NV><<<dim3(groups, chunks), 128, 0, s>>>(reinterpret_cast<const uint32_t*>(C), rings,
                                                                   d_src, d_dst, n, rings, kBits / chunks);
    return cudaGetLastError();
}

cudaError_t launch_gf2_apply_pairs(const uint64_t* C, uint32_t* rings, uint32_t n, const uint32_t* d_src,
                                   const uint32_t* d_dst, int sm_count, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    return n >= 4 * 48 ? launch_pairs<48>(C, rings, n, d_src, d_dst, sm_count, s)
                       : launch_pairs<16>(C, rings, n, d_src, d_dst, sm_count, s);
}

cudaError_t zero_rings(uint32_t* rings, const uint32_t* d_idx, uint32_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    zero_listed_kernel<<<n, kR, 0, s>>>(rings, d_idx, n);
    return cudaGetLastError();
}

cudaError_t launch_gather_rings(const State& st, const uint32_t* d_streams, uint32_t n, uint32_t* d_rings,
                                const uint64_t* d_skip, uint32_t* d_weyl0, uint32_t weyl0_stride, uint32_t omega,
                                cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    gather_rings_kernel<<<n, 128, 0, s>>>(st, d_streams, n, d_rings, d_skip, d_weyl0, weyl0_stride, omega);
    return cudaGetLastError();
}

}  // namespace xg

extern "C" xg_status xg_jump(xg_ctx* ctx, uint32_t first, uint32_t nstreams, uint64_t words)
{
    using namespace xg;
    if (!ctx) return fail(XG_EINVAL, "null context");
    if ((uint64_t)first + nstreams > ctx->n) return fail(XG_EINVAL, "streams out of range");
    if (ctx->server) return fail(XG_EINVAL, "the request server owns this context; stop it first");
    if (nstreams == 0 || words == 0) return XG_OK;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t s = ctx->stream;
    int top = 63;
    while (!((words >> top) & 1)) --top;
    xg_status st = XG_OK;
    for (int k = 0; k <= top; ++k)
        if (((words >> k) & 1) && !jump_matrix(ctx->device, (int)ctx->param_set, k, s, &st)) return st;
    // workspace kept in the context (grow-only): rings[0, n) hold the
    // states, rings[n, 2n) receive the results; index lists (stream ids for
    // the gather, then 0 .. 2n-1); the jump's own work area
    const size_t rings_bytes = (size_t)2 * nstreams * kR * 4;
    const size_t ids_off = rings_bytes;
    const size_t work_off = (ids_off + (size_t)3 * nstreams * 4 + 255) / 256 * 256;
    const size_t wbytes = gf2_jump_work_bytes(ctx->device, nstreams, words);
    if (xg_status g = ctx->ensure_jump_ws(work_off + wbytes)) return g;
    char* ws = static_cast<char*>(ctx->jump_ws);
    uint32_t* rings = reinterpret_cast<uint32_t*>(ws);
    uint32_t* ids = reinterpret_cast<uint32_t*>(ws + ids_off);
    const uint32_t* lo_idx = ids + nstreams;  // 0 .. 2n-1
    cudaError_t e = launch_jump_index(ids, nstreams, first, s);
    if (e == cudaSuccess) e = launch_gather_rings(ctx->st, ids, nstreams, rings, nullptr, nullptr, 0, 0, s);
    bool hi = false;
    if (e == cudaSuccess)
        e = gf2_jump_states(ctx->device, (int)ctx->param_set, words, rings, nstreams, lo_idx,
                            reinterpret_cast<uint8_t*>(ws + work_off), ctx->sm_count, s, &st, &hi);
    const bool in_lo = !hi;
    if (e == cudaSuccess) {
        const uint32_t* res = in_lo ? rings : rings + (size_t)nstreams * kR;
        scatter_rings_kernel<<<nstreams, 128, 0, s>>>(ctx->st, first, nstreams, res, words,
                                                      ctx->weyl_on ? 0x9E3779B9u : 0u);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const size_t sbytes = gf2_apply_scratch(ctx->device, nstreams);
    if (st != XG_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "xg_jump");
    if (sbytes && gf2_tc_take_failure())
        return fail(XG_EDEVICE, "xg_jump: a tensor-core kernel gave up waiting; the streams are not valid");
    return XG_OK;
}

extern "C" xg_status xg_seed_substreams(xg_ctx* ctx, uint32_t first, uint32_t count, uint32_t seed,
                                        uint32_t log2_spacing)
{
    using namespace xg;
    if (!ctx) return fail(XG_EINVAL, "null context");
    if ((uint64_t)first + count > ctx->n) return fail(XG_EINVAL, "streams out of range");
    if (count == 0) return XG_OK;
    if (ctx->server) return fail(XG_EINVAL, "the request server owns this context; stop it first");
    // the last stream starts at (count - 1) * 2^q, which must fit in 64 bits
    int steps = 0;   // doubling steps: bits of count - 1
    while (steps < 32 && ((uint64_t)(count - 1) >> steps)) ++steps;
    if (log2_spacing > 63 || (count > 1 && (int)log2_spacing + steps > 64))
        return fail(XG_EINVAL, "(count - 1) * 2^%u does not fit in 64 bits", log2_spacing);
    if (xg_status s = xg_seed(ctx, first, 1, &seed)) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t s = ctx->stream;
    const int q = (int)log2_spacing;
    xg_status st = XG_OK;
    for (int b = 0; b < steps; ++b)
        if (!jump_matrix(ctx->device, (int)ctx->param_set, q + b, s, &st)) return st;
    // step b takes the states m - 2^b to the states m, m in [2^b, min(2^(b+1), count)):
    // its sources are the identity list from 0 and its destinations the same
    // list from 2^b, so one device-built list 0 .. 2 count - 1 serves every step
    uint32_t most = 0;
    for (int b = 0; b < steps; ++b) {
        const uint32_t lo = 1u << b, hi = (uint32_t)std::min<uint64_t>((uint64_t)lo << 1, count);
        most = std::max(most, hi - lo);
    }
    // workspace kept in the context (grow-only): rings of all count states;
    // the index lists (first + i, then 0 .. 2 count - 1); the gathered Weyl
    // word; the tensor-core operand (when used)
    const size_t rings_bytes = (size_t)count * kR * 4;
    const size_t ids_off = rings_bytes;
    const size_t w0_off = ids_off + (size_t)3 * count * 4;
    const size_t scratch_off = (w0_off + 4 + 255) / 256 * 256;
    const size_t sbytes = gf2_apply_scratch(ctx->device, most);
    if (xg_status g = ctx->ensure_jump_ws(scratch_off + sbytes)) return g;
    char* ws = static_cast<char*>(ctx->jump_ws);
    uint32_t* rings = reinterpret_cast<uint32_t*>(ws);
    uint32_t* ids = reinterpret_cast<uint32_t*>(ws + ids_off);
    const uint32_t* iota = ids + count;
    uint32_t* d_w0 = reinterpret_cast<uint32_t*>(ws + w0_off);
    uint8_t* scratch = sbytes ? reinterpret_cast<uint8_t*>(ws + scratch_off) : nullptr;
    cudaError_t e = launch_jump_index(ids, count, first, s);
    if (e == cudaSuccess) e = launch_gather_rings(ctx->st, ids, 1, rings, nullptr, d_w0, 1, 0u, s);
    // the destinations 1 .. count - 1, zeroed once for all the steps
    if (e == cudaSuccess && count > 1) e = cudaMemsetAsync(rings + kR, 0, (size_t)(count - 1) * kR * 4, s);
    for (int b = 0; b < steps && e == cudaSuccess; ++b) {
        const uint32_t lo = 1u << b, hi = (uint32_t)std::min<uint64_t>((uint64_t)lo << 1, count);
        e = gf2_apply(ctx->device, (int)ctx->param_set, q + b, rings, hi - lo, iota, iota + lo, scratch,
                      ctx->sm_count, s, &st, true);
    }
    if (e == cudaSuccess) {
        substream_scatter_kernel<<<count, 128, 0, s>>>(ctx->st, first, count, rings, d_w0, q,
                                                       ctx->weyl_on ? 0x9E3779B9u : 0u);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st != XG_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "xg_seed_substreams");
    if (sbytes && gf2_tc_take_failure())
        return fail(XG_EDEVICE, "xg_seed_substreams: a tensor-core kernel gave up waiting; the streams are not valid");
    return XG_OK;
}
