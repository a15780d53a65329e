// Internal declarations shared by the library's host and CUDA translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mlqmc.h"

#define MLQMC_MAX_LEVELS 12
#define MLQMC_MAX_MODES 4096

// ---- host precompute (mlqmc_host.cpp) -----------------------------------
namespace mlqmc {

// Closed-form 1D KL eigenpairs of exp(-|x-x'|/corr_len) on [0,1] (eq. inteq).
struct Eig1D {
    std::vector<double> omega, theta, norm;  // root, eigenvalue, squared norm of the unnormalised psi
};
Eig1D kl_eigen_1d(double corr_len, int K);

// Top-s separable 2D modes: theta_ab = sigma^2 theta_a theta_b, ordered by
// theta (rounded to 40 mantissa bits) descending, then a, then b.
struct Modes {
    std::vector<int> a, b;
    std::vector<double> theta;
    int K1 = 0;  // 1 + max(a, b)
};
Modes select_modes(double corr_len, double sigma, int s);

// psi_k at the cell centres of an n-cell axis, k-major: out[k*n + i].
void psi_table(const Eig1D& e, double corr_len, int K1, int n, std::vector<double>& out);

// Algorithm 1 driver (host control around mlqmc_sample_levels).
mlqmc_status run_estimate(mlqmc_ctx* c, double eps, const mlqmc_run_opts* o, mlqmc_result* out);

}  // namespace mlqmc

// ---- device-side sample descriptor ---------------------------------------
struct SampleDesc {
    int64_t n;      // lattice / MC index
    int32_t r;      // shift
    int32_t level;  // finest FMG level of this sample
    int32_t canon;  // position in work order (output index)
    int32_t pad;
};

// Per-level offsets inside one workspace slot (bytes from the slot base).
struct LevelOffsets {
    int n;
    size_t u, bc, kx, ky, idiag, k, G;  // working precision arrays
    size_t u64, kx64, ky64;             // FP64 arrays of the mixed forms
};

struct SlotLayout {
    int n_levels = 0;
    LevelOffsets lv[MLQMC_MAX_LEVELS];
    size_t bytes = 0;
};

struct mlqmc_ctx {
    mlqmc_problem p{};
    int device = 0;
    int sm_count = 0;
    std::vector<uint32_t> z;
    mlqmc::Modes modes;
    mlqmc::Eig1D eig;
    int Ka = 0;  // 1 + max a over the kept modes

    // device tables
    double* d_psi = nullptr;  // per level: K1 x n_t doubles
    float* d_psi32 = nullptr;
    size_t psi_off[MLQMC_MAX_LEVELS] = {};
    int* d_grp_start = nullptr;  // Ka+1: modes grouped by a
    int* d_grp_b = nullptr;
    int* d_grp_m = nullptr;
    double* d_grp_sqrt = nullptr;
    uint32_t* d_z = nullptr;

    // per-call buffers
    int64_t max_samples = 0;
    SampleDesc* d_samples = nullptr;  // queue order (largest level first)
    int2* d_canon = nullptr;          // (level, r) in work order
    double* d_Y = nullptr;            // max_samples x s normals
    double* d_dF = nullptr;           // max_samples x n_levels
    SampleDesc* h_samples = nullptr;  // pinned staging
    int2* h_canon = nullptr;
    cudaEvent_t staged = nullptr;     // recorded after the last copy out of the staging buffers

    // FMG workspace: `slots` slots of `layout.bytes`
    unsigned char* d_work = nullptr;
    int slots = 0;
    int fmg_threads = 256;
    size_t fmg_smem = 0;
    SlotLayout layout;

    // optional per-kernel event timing
    bool profiling = false;
    struct Mark {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;       // recorded, not yet read
    std::vector<cudaEvent_t> pool; // free events
    double prof_ms[3] = {0, 0, 0};
    int64_t prof_n[3] = {0, 0, 0};

    int* d_status = nullptr;  // deferred device status bits
    int* d_queue = nullptr;   // work-queue counter
    int64_t launches = 0;
};
