// SpMM instantiations whose gathered operand B is E4M3.
#include "spmm_impl.cuh"

namespace spk {

cudaError_t launch_spmm_e4m3(const Launch& L, const SpmmArgs& a, cudaStream_t s)
{
    return launch_spmm_t<DT_E4M3>(L, a, s);
}

}  // namespace spk
