// SpMM instantiations whose gathered operand B is F16.
#include "spmm_impl.cuh"

namespace spk {

cudaError_t launch_spmm_f16(const Launch& L, const SpmmArgs& a, cudaStream_t s)
{
    return launch_spmm_t<DT_F16>(L, a, s);
}

}  // namespace spk
