// Host interface of the TMA-fed FMG interpolation with the first refinement
// residual (resid_tma.cu).
#pragma once

#include <cuda_runtime.h>

#include "fmg_device.cuh"

namespace mlqmc_resid {

// Level sides the TMA form handles (64 x 32 fine tiles, every box within the
// level's extent).
bool supported(int n);

// Raise the dynamic shared-memory limit; once per process.
bool prepare();

// Mixed forms, the refinement step that opens level t (n cells per side) for
// samples 0..B-1 of A: u64 = P u_(t-1) (the FP32 copy of the coarse solution
// interpolated in FP32, widened) and bc = 1 - A u64 rounded to FP32 from FP32
// error-free pairs; inactive samples skipped. The same arithmetic, operand
// for operand, as the grid-stride form in mlqmc_cuda.cu. interp32: the
// interpolant is stored as FP32 in the level's field array k (whose field is
// no longer read once the faces are formed) instead of widened into u64.
// Returns false when a tensor map cannot be encoded or the launch fails.
bool launch(const mlqmc_dev::FmgArgs& A, int t, int n, int B, bool interp32, int sm_count, cudaStream_t st);

}  // namespace mlqmc_resid
