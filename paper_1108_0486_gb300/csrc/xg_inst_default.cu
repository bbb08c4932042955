// Kernels of the default parameter set (r,s,a,b,c,d) = (128,95,17,12,13,15).
#include "xg_kernels.cuh"

namespace xg {

cudaError_t launch_seed_default(const State& st, const uint32_t* d_seeds, uint32_t first,
                                uint32_t count, cudaStream_t s)
{
    return launch_seed_impl<ParamsDefault, 32, 2>(st, d_seeds, first, count, s);
}

cudaError_t launch_gen_default(int cfg, int out_kind, bool vec, int block, const GenArgs& a,
                               cudaStream_t s)
{
    return launch_gen_impl<ParamsDefault>(cfg, out_kind, vec, block, a, s);
}

const void* batch_kernel_ptr_default(bool groups) { return batch_kernel_ptr<ParamsDefault>(groups); }

}  // namespace xg
