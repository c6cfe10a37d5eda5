// SDDMM instantiations whose gathered operand B is F32.
#include "sddmm_impl.cuh"

namespace spk {

cudaError_t launch_sddmm_f32(int dta, const Launch& L, const SddmmArgs& a, cudaStream_t s)
{
    if (dta == DT_F32) return launch_sddmm_t<DT_F32, DT_F32>(L, a, s);
    return cudaErrorInvalidValue;
}

}  // namespace spk
