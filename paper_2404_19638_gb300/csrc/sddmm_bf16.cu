// SDDMM instantiations whose gathered operand B is BF16.
#include "sddmm_impl.cuh"

namespace spk {

cudaError_t launch_sddmm_bf16(int dta, const Launch& L, const SddmmArgs& a, cudaStream_t s)
{
    if (dta == DT_BF16) return launch_sddmm_t<DT_BF16, DT_BF16>(L, a, s);
    if (dta == DT_F32) return launch_sddmm_t<DT_F32, DT_BF16>(L, a, s);
    return cudaErrorInvalidValue;
}

}  // namespace spk
