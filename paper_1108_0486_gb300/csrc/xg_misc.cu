// Stand-alone conversion kernels and the parameter-set dispatch.
#include "xg_device.cuh"
#include "xg_launch.h"

namespace xg {

const LaunchCfg kCfgs[kNumCfgs] = {{4, 8, 64}, {8, 4, 64}, {16, 2, 64}, {16, 4, 64}, {32, 2, 64}};

int cfg_index(int tpg, int wpl)
{
    for (int i = 0; i < kNumCfgs; ++i)
        if (kCfgs[i].tpg == tpg && kCfgs[i].wpl == wpl) return i;
    return -1;
}

// Uniform conversion of n words, 4 per thread when both buffers are 16-byte
// aligned (vec), one per thread otherwise.
__global__ void __launch_bounds__(256) transform_uniform_kernel(const uint32_t* __restrict__ in,
                                                                 uint64_t n, float* __restrict__ out,
                                                                 bool vec)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n4 = vec ? n / 4 : 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const uint4 w = reinterpret_cast<const uint4*>(in)[i];
        reinterpret_cast<float4*>(out)[i] =
            make_float4(to_uniform(w.x), to_uniform(w.y), to_uniform(w.z), to_uniform(w.w));
    }
    for (uint64_t i = 4 * n4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = to_uniform(in[i]);
}

// Box-Muller on pairs (in[2i], in[2i+1]) -> (out[2i], out[2i+1]): two pairs
// per thread through the packed transform the generation kernels use (the
// same bits as normal_pair), the odd last pair alone.
__global__ void __launch_bounds__(256) transform_normal_kernel(const uint32_t* __restrict__ in,
                                                                uint64_t npairs, float* __restrict__ out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t nquads = npairs / 2;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nquads; i += stride) {
        const uint2 a = reinterpret_cast<const uint2*>(in)[2 * i];
        const uint2 b = reinterpret_cast<const uint2*>(in)[2 * i + 1];
        float z1a, z2a, z1b, z2b;
        normal_pair2(a.x, a.y, b.x, b.y, z1a, z2a, z1b, z2b);
        reinterpret_cast<float2*>(out)[2 * i] = make_float2(z1a, z2a);
        reinterpret_cast<float2*>(out)[2 * i + 1] = make_float2(z1b, z2b);
    }
    if ((npairs & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const uint2 w = reinterpret_cast<const uint2*>(in)[npairs - 1];
        float z1, z2;
        normal_pair(w.x, w.y, z1, z2);
        reinterpret_cast<float2*>(out)[npairs - 1] = make_float2(z1, z2);
    }
}

cudaError_t launch_transform(int out_kind, const uint32_t* in, uint64_t n, float* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int block = 256;
    if (out_kind == kUniform) {
        const bool aligned = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
        uint64_t work = aligned ? (n + 3) / 4 : n;
        uint64_t grid = (work + block - 1) / block;
        if (grid > (uint64_t)sms * 16) grid = (uint64_t)sms * 16;
        transform_uniform_kernel<<<(unsigned)grid, block, 0, s>>>(in, n, out, aligned);
    } else if (out_kind == kNormal) {
        const uint64_t npairs = n / 2;
        uint64_t grid = (npairs + block - 1) / block;
        if (grid > (uint64_t)sms * 16) grid = (uint64_t)sms * 16;
        transform_normal_kernel<<<(unsigned)grid, block, 0, s>>>(in, npairs, out);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Bulk checkpoint: stream first + k's ring (oldest first), Weyl word and
// position into rings[k], weyl[k], pos[k].
__global__ void __launch_bounds__(128) export_states_kernel(State st, uint32_t first, uint32_t n,
                                                            uint32_t* __restrict__ rings,
                                                            uint32_t* __restrict__ weyl,
                                                            uint64_t* __restrict__ pos)
{
    const uint32_t k = blockIdx.x;
    if (k >= n) return;
    const uint32_t s = first + k;
    const uint32_t* src = st.win + (size_t)s * kWin + (kRingBase - st.pend[s]);
    for (int w = threadIdx.x; w < 128; w += blockDim.x) rings[(size_t)k * 128 + w] = src[w];
    if (threadIdx.x == 0) {
        weyl[k] = st.weyl[s];
        pos[k] = st.pos[s];
    }
}

// Bulk restore: the ring at window[kRingBase, kWin), pend = 0, the Weyl word
// (0 with the Weyl generator off), and the position when pos is given.
__global__ void __launch_bounds__(128) import_states_kernel(State st, uint32_t first, uint32_t n,
                                                            const uint32_t* __restrict__ rings,
                                                            const uint32_t* __restrict__ weyl,
                                                            const uint64_t* __restrict__ pos, uint32_t weyl_on)
{
    const uint32_t k = blockIdx.x;
    if (k >= n) return;
    const uint32_t s = first + k;
    uint32_t* dst = st.win + (size_t)s * kWin + kRingBase;
    for (int w = threadIdx.x; w < 128; w += blockDim.x) dst[w] = rings[(size_t)k * 128 + w];
    if (threadIdx.x == 0) {
        st.weyl[s] = weyl_on ? weyl[k] : 0u;
        st.pend[s] = 0;
        if (pos) st.pos[s] = pos[k];
    }
}

cudaError_t launch_export_states(const State& st, uint32_t first, uint32_t n, uint32_t* rings, uint32_t* weyl,
                                 uint64_t* pos, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    export_states_kernel<<<n, 128, 0, s>>>(st, first, n, rings, weyl, pos);
    return cudaGetLastError();
}

cudaError_t launch_import_states(const State& st, uint32_t first, uint32_t n, const uint32_t* rings,
                                 const uint32_t* weyl, const uint64_t* pos, uint32_t weyl_on, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    import_states_kernel<<<n, 128, 0, s>>>(st, first, n, rings, weyl, pos, weyl_on);
    return cudaGetLastError();
}

cudaError_t launch_seed(int param_set, const State& st, const uint32_t* d_seeds, uint32_t first,
                        uint32_t count, cudaStream_t s)
{
    return param_set == 1 ? launch_seed_paper(st, d_seeds, first, count, s)
                          : launch_seed_default(st, d_seeds, first, count, s);
}

cudaError_t launch_gen(int param_set, int cfg, int out_kind, bool vec, int block, const GenArgs& a,
                       cudaStream_t s)
{
    return param_set == 1 ? launch_gen_paper(cfg, out_kind, vec, block, a, s)
                          : launch_gen_default(cfg, out_kind, vec, block, a, s);
}

const void* batch_kernel_ptr(int param_set, bool groups)
{
    return param_set == 1 ? batch_kernel_ptr_paper(groups) : batch_kernel_ptr_default(groups);
}

}  // namespace xg
