// SpMM instantiations whose gathered operand B is F32.
#include "spmm_impl.cuh"

namespace spk {

cudaError_t launch_spmm_f32(const Launch& L, const SpmmArgs& a, cudaStream_t s)
{
    return launch_spmm_t<DT_F32>(L, a, s);
}

}  // namespace spk
