// Host interface of the whole-sample red-black smoother (rbgs_whole.cu).
#pragma once

#include <cuda_runtime.h>

#include "fmg_device.cuh"

namespace mlqmc_whole {

// Level sides whose whole grid one team stages in shared memory (n <= 64).
bool supported(int n, bool fp64);

// Raise the dynamic shared-memory limit of every instance; once per process.
bool prepare();

// ns red-black sweeps of level t (n cells per side) for samples 0..B-1 of A,
// u updated in place; fp64: the FP64 form's arrays (the stored 1/D is used). first: colour of the first half sweep (0 red:
// (i1 + i2) even). ones: right-hand side 1, else bc of level t. post: add
// the coarse-grid correction P u_{t-1} to u before the sweeps. pre:
// afterwards write bc of level t-1 = mean over the 4 children of b - A u.
// zin: u is zero on entry (pre-smoothing of a correction; not with post): it is
// cleared in shared memory instead of read.
bool launch(const mlqmc_dev::FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool pre, bool post,
            bool zin, bool fp64, cudaStream_t st);

}  // namespace mlqmc_whole
