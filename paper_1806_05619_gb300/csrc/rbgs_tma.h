// Host interface of the TMA-fed tiled red-black smoother (rbgs_tma.cu).
#pragma once

#include <cuda_runtime.h>

#include "fmg_device.cuh"

namespace mlqmc_tma {

// Level sides the tiled smoother handles (FP32 arrays, 32 x 32 tiles, n >= 64).
bool supported(int n);

// Raise the dynamic shared-memory limit of every instance; once per process.
bool prepare();

// ns (1 or 2) red-black sweeps of level t (n cells per side) for samples
// 0..B-1 of A, read from u and written to u2 (the caller swaps the two).
// first: colour of the first half sweep (0 red: (i1 + i2) even). ones:
// right-hand side 1, else bc of level t. post: add the coarse-grid correction
// P u_{t-1} to the staged u before the sweeps. Returns false when a tensor
// map cannot be encoded or the launch fails.
// zin: u is zero on entry (pre-smoothing of a correction; not with post): its
// tiles are cleared in shared memory instead of copied.
// rr (not with post): also write the restricted residual of the swept u,
// bc of level t-1 = mean over each coarse cell's 4 children of b - A u.
bool launch(const mlqmc_dev::FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool post, bool zin,
            bool rr, int sm_count, cudaStream_t st);

}  // namespace mlqmc_tma
