// Kernels of the parameter set of the paper, (r,s,a,b,c,d) = (128,65,15,14,12,17) (Sec. 2).
#include "xg_kernels.cuh"

namespace xg {

cudaError_t launch_seed_paper(const State& st, const uint32_t* d_seeds, uint32_t first,
                                uint32_t count, cudaStream_t s)
{
    return launch_seed_impl<ParamsPaper, 32, 2>(st, d_seeds, first, count, s);
}

cudaError_t launch_gen_paper(int cfg, int out_kind, bool vec, int block, const GenArgs& a,
                               cudaStream_t s)
{
    return launch_gen_impl<ParamsPaper>(cfg, out_kind, vec, block, a, s);
}

const void* batch_kernel_ptr_paper(bool groups) { return batch_kernel_ptr<ParamsPaper>(groups); }

}  // namespace xg
