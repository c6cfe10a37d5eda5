// Multi-head SDDMM launch (sddmm_mh.cu).
#pragma once
#include "common.cuh"

namespace spk {

// Heads of NH 16-byte vectors each, on the SDDMM ring shape (G, NV, U) whose
// lane blocks cover the whole row (K = G * NV vectors).
bool sddmm_mh_supported(int dt, int G, int NV, int U, int NH);
cudaError_t launch_sddmm_mh(int dt, int G, int NV, int U, int NH, const SddmmArgs& a, cudaStream_t s);

}  // namespace spk
