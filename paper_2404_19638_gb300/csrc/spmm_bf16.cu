// SpMM instantiations whose gathered operand B is BF16.
#include "spmm_impl.cuh"

namespace spk {

cudaError_t launch_spmm_bf16(const Launch& L, const SpmmArgs& a, cudaStream_t s)
{
    return launch_spmm_t<DT_BF16>(L, a, s);
}

}  // namespace spk
