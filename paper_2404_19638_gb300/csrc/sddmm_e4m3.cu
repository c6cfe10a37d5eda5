// SDDMM instantiations whose gathered operand B is E4M3.
#include "sddmm_impl.cuh"

namespace spk {

cudaError_t launch_sddmm_e4m3(int dta, const Launch& L, const SddmmArgs& a, cudaStream_t s)
{
    if (dta == DT_E4M3) return launch_sddmm_t<DT_E4M3, DT_E4M3>(L, a, s);
    return cudaErrorInvalidValue;
}

}  // namespace spk
