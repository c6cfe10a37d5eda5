// FusedMM launches beyond the ones common.cuh declares (fused.cu).
#pragma once
#include "common.cuh"

namespace spk {

// All heads in one lane group of G lanes, NV (1 or 2) adjacent 16-byte
// vectors a lane: G * NV vectors cover a row of K, heads are blocks of
// G / heads lanes.
cudaError_t launch_fused_mh_nv(int dt, int G, int NV, const FusedArgs& a, cudaStream_t s);

}  // namespace spk
