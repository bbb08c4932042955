// GF(2) matrix applications on the tensor cores (tcgen05, sm_103a).
//
// The recurrence of Sec. 2 is linear over GF(2) on the 4096-bit state, so a
// jump-ahead applies a 4096 x 4096 bit matrix C to many states: y = C x.
// Over the integers, with 0/1 entries, (C x)_i counts the set bits of row i
// of C that meet set bits of x; the GF(2) result is that count's parity.  The
// counts are at most 4096, which an FP32 accumulator holds exactly, and 0/1
// are exact in FP8 E4M3, so the product of the matrix and a batch of states
// is a plain FP8 GEMM with an FP32 accumulator:
//   D[i][s] = sum_k A[i][k] B[s][k],  A[i][k] = C[i][k],  B[s][k] = bit k of x_s
// (M = 4096 output bits, N = states, K = 4096 input bits, both operands
// K-major), followed by a parity epilogue that packs bits back into 32-bit
// ring words.
//
// Kernel: persistent, one CTA per SM, 128 x 256 output tiles.  Warp 0 (one
// lane) streams 128-byte-wide K blocks of A and B into a 4-stage
// shared-memory ring with TMA (128B swizzle, mbarrier transaction counts);
// warp 1 (one lane) issues tcgen05.mma (kind::f8f6f4, E4M3 x E4M3 -> F32,
// 128 x 256 x 32 each) into one of two TMEM accumulators and frees each
// stage with tcgen05.commit; four epilogue warps read the other accumulator
// with tcgen05.ld (32 TMEM lanes = 32 output bits each), take each count's
// parity and pack the 32 lanes' bits with a warp ballot: one ballot is one
// ring word of one state.
//
// Every wait is bounded (2 s of %globaltimer); a wait that gives up records
// a failure in a host-visible status word, the CTA waits (bounded) for its
// own TMA copies still in flight, frees its TMEM and returns.  To test that
// path, XG_TC_TEST_STALL=1 in the environment makes CTA 0 arm its first
// stage's barrier without starting the stage's copies: the waits on that
// stage run out (no fault, no unbounded wait) and the call reports it.
#include <cuda.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "xg_gf2_tc.h"
#include "xg_runtime.h"

namespace xg {
namespace {

constexpr int kBM = 128;                  // output bits per tile (TMEM lanes)
constexpr int kBN = 256;                  // states per tile (TMEM columns)
constexpr int kBK = 128;                  // K per stage: one 128-byte swizzle row
constexpr int kKBlocks = kGf2Bits / kBK;  // 32
constexpr int kStages = 4;
constexpr int kABytes = kBM * kBK;        // 16 KiB
constexpr int kBBytes = kBN * kBK;        // 32 KiB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /* barriers */ + 1024 /* alignment */;
constexpr int kEpilogueWarps = 4;
constexpr int kThreads = 32 * (2 + kEpilogueWarps);
constexpr uint8_t kOneE4M3 = 0x38;        // 1.0 in FP8 E4M3
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Wait for the phase with the given parity to complete; false if it has not
// after the deadline.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t deadline)
{
    const uint32_t a = smem_addr(bar);
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 255u && global_ns() > deadline) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major, 128B swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart, version 1.
__device__ __forceinline__ uint64_t smem_desc(const void* p)
{
    const uint64_t addr = smem_addr(p);
    return ((addr & 0x3FFFFull) >> 4)        // start address, bits 0-13
           | (1ull << 16)                    // leading byte offset (unused for swizzled K-major)
           | ((1024ull >> 4) << 32)          // stride byte offset: 8 rows x 128 B
           | (1ull << 46)                    // descriptor version
           | (2ull << 61);                   // layout: 128-byte swizzle
}

// Instruction descriptor, kind::f8f6f4: D F32, A and B E4M3, both K-major,
// N = kBN, M = kBM.
constexpr uint32_t kInstrDesc = (1u << 4)                    // D format F32
                                | (0u << 7) | (0u << 10)     // A, B: E4M3
                                | ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kInstrDesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive columns of this warp's 32 TMEM lanes: v[j] = column col + j.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool failed(const volatile int* flag) { return *flag != 0; }

// out[dst[s]] = C x_s for the n states of the B operand (rows >= n of B are
// zero padding).  Persistent: CTA b takes tiles b, b + gridDim.x, ... of the
// (4096 / kBM) x (n_pad / kBN) tiles, M fastest (consecutive tiles share a B
// tile in L2).  192 threads: warp 0 = TMA producer, warp 1 = TMEM owner and
// MMA issuer, warps 2-5 = epilogue (warp w reads TMEM lanes 32 (w mod 4) ..).
// Two accumulators of kBN columns alternate, so that the epilogue of one
// tile overlaps the MMAs of the next.
__global__ void __launch_bounds__(kThreads, 1) gf2_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB, uint32_t n,
                                                              uint32_t n_tiles, const uint32_t* __restrict__ dst,
                                                              uint32_t* rings, uint32_t* status, uint32_t stall)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sa = smem;
    uint8_t* sb = smem + kStages * kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sb + kStages * kBBytes);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;   // [2] accumulator ready (MMA commit)
    uint64_t* tempty = tfull + 2;        // [2] accumulator drained (4 epilogue warps)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
    __shared__ volatile int s_failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t kMTiles = kGf2Bits / kBM;
    const uint32_t total = kMTiles * n_tiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], kEpilogueWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_failed = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"((uint32_t)(2 * kBN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    uint32_t issued = 0;  // producer: K blocks whose copies were started
    if (warp == 0) {
        if (lane == 0) {
            for (uint32_t t = blockIdx.x; t < total && !failed(&s_failed); t += gridDim.x) {
                const int mt = (int)(t % kMTiles), nt = (int)(t / kMTiles);
                for (int kb = 0; kb < kKBlocks; ++kb, ++issued) {
                    const uint32_t s = issued % kStages, u = issued / kStages;
                    if (issued >= (uint32_t)kStages && !mbar_wait(&empty[s], (u & 1) ^ 1, global_ns() + kWaitLimitNs)) {
                        s_failed = 1;
                        break;
                    }
                    mbar_expect_tx(&full[s], kStageBytes);
                    if (stall && blockIdx.x == 0 && issued == 0) continue;   // the failure-path test
                    tma_load_2d(sa + s * kABytes, &tmA, &full[s], kb * kBK, mt * kBM);
                    tma_load_2d(sb + s * kBBytes, &tmB, &full[s], kb * kBK, nt * kBN);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, lt = 0;
            for (uint32_t t = blockIdx.x; t < total && !failed(&s_failed); t += gridDim.x, ++lt) {
                const uint32_t acc = lt & 1, v = lt >> 1;
                if (lt >= 2 && !mbar_wait(&tempty[acc], (v & 1) ^ 1, global_ns() + kWaitLimitNs)) {
                    s_failed = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + acc * kBN;
                for (int kb = 0; kb < kKBlocks; ++kb, ++it) {
                    const uint32_t s = it % kStages, u = it / kStages;
                    if (!mbar_wait(&full[s], u & 1, global_ns() + kWaitLimitNs)) {
                        s_failed = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = smem_desc(sa + s * kABytes);
                    const uint64_t bd = smem_desc(sb + s * kBBytes);
#pragma unroll
                    for (int kk = 0; kk < kBK / 32; ++kk)  // K = 32 bytes per instruction: +2 in 16-byte units
                        mma_f8(d, ad + 2 * kk, bd + 2 * kk, (kb | kk) != 0);
                    mma_commit(&empty[s]);
                }
                mma_commit(&tfull[acc]);  // arrives once this tile's MMAs have completed
            }
        }
        __syncwarp();
    } else {
        // epilogue: this warp's 32 TMEM lanes = output bits 32 q .. 32 q + 31 of a tile
        const uint32_t q = (uint32_t)(warp & 3);
        uint32_t lt = 0;
        for (uint32_t t = blockIdx.x; t < total; t += gridDim.x, ++lt) {
            const uint32_t acc = lt & 1, v = lt >> 1;
            if (!mbar_wait(&tfull[acc], v & 1, global_ns() + kWaitLimitNs)) {
                s_failed = 1;
                break;
            }
            tc_fence_after();
            if (failed(&s_failed)) break;
            const uint32_t mt = t % kMTiles, nt = t / kMTiles;
            const uint32_t word = mt * (kBM / 32) + q;  // ring word of these 32 bits
            for (int c = 0; c < kBN; c += 32) {
                uint32_t vals[32];
                tmem_ld32(tmem + ((q * 32) << 16) + acc * kBN + (uint32_t)c, vals);
                uint32_t mine = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    // the count is an integer <= 4096: adding 2^23 puts its parity in the last bit
                    const uint32_t bit = __float_as_uint(__uint_as_float(vals[j]) + 8388608.0f) & 1u;
                    const uint32_t b = __ballot_sync(0xFFFFFFFFu, bit);
                    if (lane == j) mine = b;
                }
                const uint32_t st = nt * kBN + (uint32_t)c + (uint32_t)lane;
                if (st < n) rings[(size_t)dst[st] * kGf2Words + word] = mine;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (failed(&s_failed)) {
        if (warp == 0 && lane == 0) {
            // the copies of the last (at most kStages) started K blocks may still be in flight
            for (uint32_t kb = issued > (uint32_t)kStages ? issued - kStages : 0u; kb < issued; ++kb)
                (void)mbar_wait(&full[kb % kStages], (kb / kStages) & 1, global_ns() + kWaitLimitNs);
        }
        if (threadIdx.x == 0) {
            *reinterpret_cast<volatile uint32_t*>(status) = 1u;
            __threadfence_system();
        }
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * kBN))
                     : "memory");
    }
}

// A[i][k] = bit i of column k of C (column form: column k = 128 ring words).
// Thread (k, w): one word of one column, 32 rows of A.
__global__ void expand_matrix_kernel(const uint32_t* __restrict__ cols, uint8_t* __restrict__ A)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t w = blockIdx.y;
    if (k >= (uint32_t)kGf2Bits) return;
    const uint32_t word = cols[(size_t)k * kGf2Words + w];
#pragma unroll 8
    for (int b = 0; b < 32; ++b) A[(size_t)(32 * w + b) * kGf2Bits + k] = ((word >> b) & 1u) ? kOneE4M3 : 0;
}

// Four bits to four E4M3 bytes (byte b = 1.0 when bit b is set).
__device__ __forceinline__ uint32_t spread4(uint32_t x)
{
    return ((x & 1u) | ((x & 2u) << 7) | ((x & 4u) << 14) | ((x & 8u) << 21)) * (uint32_t)kOneE4M3;
}

// B[s][k] = bit k of state src[s] (s < n), 0 for n <= s < n_pad.  Thread =
// one ring word = 32 bytes of B.
__global__ void expand_states_kernel(const uint32_t* __restrict__ rings, const uint32_t* __restrict__ src,
                                     uint32_t n, uint32_t n_pad, uint8_t* __restrict__ B)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n_pad * kGf2Words) return;
    const uint32_t s = (uint32_t)(t / kGf2Words), w = (uint32_t)(t % kGf2Words);
    uint32_t x = 0;
    if (s < n) x = rings[(size_t)(src ? src[s] : s) * kGf2Words + w];
    uint4 lo, hi;
    lo.x = spread4(x);
    lo.y = spread4(x >> 4);
    lo.z = spread4(x >> 8);
    lo.w = spread4(x >> 12);
    hi.x = spread4(x >> 16);
    hi.y = spread4(x >> 20);
    hi.z = spread4(x >> 24);
    hi.w = spread4(x >> 28);
    uint4* out = reinterpret_cast<uint4*>(B + (size_t)s * kGf2Bits + 32 * w);
    out[0] = lo;
    out[1] = hi;
}

// ---- host side -------------------------------------------------------------

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_mu;
EncodeTiled g_encode = nullptr;
bool g_probed = false;
uint32_t* g_status_host = nullptr;  // mapped pinned word shared by every launch
uint32_t* g_status_dev = nullptr;
bool g_attr_set[64] = {};

bool init_locked()
{
    if (g_probed) return g_encode != nullptr && g_status_dev != nullptr;
    g_probed = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    g_encode = reinterpret_cast<EncodeTiled>(fn);
    void* h = nullptr;
    if (cudaHostAlloc(&h, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        g_encode = nullptr;
        return false;
    }
    g_status_host = static_cast<uint32_t*>(h);
    *g_status_host = 0;
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
        cudaGetLastError();
        g_encode = nullptr;
        return false;
    }
    g_status_dev = static_cast<uint32_t*>(d);
    return true;
}

bool make_map(CUtensorMap* m, const uint8_t* base, uint64_t rows, uint32_t box_rows)
{
    const cuuint64_t dims[2] = {(cuuint64_t)kGf2Bits, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kGf2Bits};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gf2_tc_available(int device)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!init_locked()) return false;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return major == 10 && minor == 3;
}

uint32_t gf2_tc_padded(uint32_t n) { return (n + kBN - 1) / kBN * kBN; }

size_t gf2_tc_scratch_bytes(uint32_t n) { return (size_t)gf2_tc_padded(n) * kGf2Bits; }

cudaError_t gf2_tc_expand_matrix(const uint64_t* C, uint8_t* A, cudaStream_t s)
{
    expand_matrix_kernel<<<dim3(kGf2Bits / 128, kGf2Words), 128, 0, s>>>(reinterpret_cast<const uint32_t*>(C), A);
    return cudaGetLastError();
}

cudaError_t gf2_tc_apply(int device, const uint8_t* A, const uint32_t* rings_in, const uint32_t* src, uint32_t n,
                         uint32_t* rings_out, const uint32_t* dst, uint8_t* scratch, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint32_t n_pad = gf2_tc_padded(n);
    CUtensorMap ma, mb;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!init_locked()) return cudaErrorNotSupported;
        if (!make_map(&ma, A, kGf2Bits, kBM) || !make_map(&mb, scratch, n_pad, kBN)) return cudaErrorInvalidValue;
        if (device >= 0 && device < 64 && !g_attr_set[device]) {
            cudaError_t e = cudaFuncSetAttribute(gf2_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
            if (e != cudaSuccess) return e;
            g_attr_set[device] = true;
        }
    }
    const uint64_t words = (uint64_t)n_pad * kGf2Words;
    expand_states_kernel<<<(unsigned)((words + 255) / 256), 256, 0, s>>>(rings_in, src, n, n_pad, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint32_t n_tiles = n_pad / kBN;
    const uint32_t tiles = (kGf2Bits / kBM) * n_tiles;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) sms = 1;
    const unsigned grid = (unsigned)std::min<uint32_t>(tiles, (uint32_t)sms);
    const char* stall = std::getenv("XG_TC_TEST_STALL");
    gf2_tc_kernel<<<grid, kThreads, kSmemBytes, s>>>(ma, mb, n, n_tiles, dst, rings_out, g_status_dev,
                                                     (stall && stall[0] == '1') ? 1u : 0u);
    return cudaGetLastError();
}

bool gf2_tc_take_failure()
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_host) return false;
    const uint32_t v = *reinterpret_cast<volatile uint32_t*>(g_status_host);
    if (v) *reinterpret_cast<volatile uint32_t*>(g_status_host) = 0;
    return v != 0;
}

}  // namespace xg
