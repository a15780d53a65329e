// Internal declarations shared by the library's host and CUDA translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mlqmc.h"
#include "kl_tcgen05.h"

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
mlqmc_status run_estimate_mlmc(mlqmc_ctx* c, double eps, const mlqmc_run_opts* o, mlqmc_result* out);

// A round's reuse sums (n doubles, device -> host) and the deferred device
// status in one synchronisation of `st`; the status word is cleared on `st`
// after it is read. Returns what mlqmc_get_device_status would.
mlqmc_status fetch_round(mlqmc_ctx* c, const double* d_sums, double* h_sums, size_t n, cudaStream_t st);

}  // namespace mlqmc

// ---- device-side sample descriptor ---------------------------------------
struct SampleDesc {
    int64_t n;      // lattice / MC index
    int64_t gidx;   // position in work order across the whole call (output index)
    int32_t r;      // shift
    int32_t level;  // finest FMG level of this sample
    int32_t canon;  // position inside its chunk (index of its normals)
    int32_t pad;
};

// Kinds of kernels for the optional per-kind event timing.
enum ProfKind {
    kProfPoints = 0,   // normals
    kProfSmall = 1,    // per-sample level-0 factor and exact solve
    kProfSynth = 2,    // batched KL field, faces, inverse diagonal
    kProfSmooth = 3,   // batched red-black sweeps
    kProfTransfer = 4, // batched residual/restriction, prolongation, FP64 refinement updates
    kProfSmallV = 5,   // coarse solves of the V-cycles (one thread per sample)
    kProfReduce = 6,   // QoI, norms, reuse sums, outputs
    kProfKlTc = 7,     // KL contraction on the tensor cores
    kProfKinds = 8
};

// Below this many samples in a call a level follows its small-batch schedule.
constexpr int kSmallBatch = 256;

// Profile buckets per grid level; the last holds launches of no single level
// (normals, reuse sums, outputs).
constexpr int kProfLevels = MLQMC_MAX_LEVELS + 1;
constexpr int kProfNoLevel = MLQMC_MAX_LEVELS;
static_assert(kProfLevels == MLQMC_PROFILE_LEVELS, "profile level buckets of the C ABI");

struct ProfCell {
    double ms = 0.0, bytes = 0.0, f64 = 0.0, f32 = 0.0, ftc = 0.0;
    int64_t n = 0;
};

// Pool of per-sample arrays of one level: array a of sample i lives at
// mem + off[a] + i * stride[a].
enum PoolArr { kU = 0, kBc, kKx, kKy, kIdiag, kK, kG, kU64, kU2, kPoolArrs };

struct LevelPool {
    unsigned char* mem = nullptr;
    int64_t cap = 0;
    size_t off[kPoolArrs] = {};
    size_t stride[kPoolArrs] = {};
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
    uint64_t* d_shift = nullptr;  // lattice shifts [(level * R + r) * s + j] (null: Philox per point)
    int* d_ma = nullptr;               // modes in order: first index a
    int* d_mb = nullptr;               // second index b
    double* d_sqrt_theta = nullptr;    // sqrt(theta_m)
    // Matern covariance: every level's modes at its cell centres, FP64,
    // cell-major (n_t^2 x s), level t at d_psi_dense + dense_off[t]
    float* d_c32 = nullptr;  // mixed forms: FP32 KL coefficients of the chunk's samples (max_samples x s)
    bool c32_ready = false;  // d_c32 holds the current chunk's coefficients (set inside run_chunk)
    bool matern = false;
    uint64_t psi_hash = 0;  // Matern: hash of the caller's nodal eigenfunctions
    double* d_psi_dense = nullptr;
    size_t dense_off[MLQMC_MAX_LEVELS] = {};

    // tensor-core KL (mixed forms): Psi per level (rows padded to 128-cell tiles), C per chunk
    bool kl_tc = false;
    void* d_psi_tc[MLQMC_MAX_LEVELS] = {};  // Psi operand per level (FP32 or split BF16 rows)
    void* d_C = nullptr;   // C operand of the contraction (FP32 or split BF16 rows)
    mlqmc_kl::Variant kl_variant = mlqmc_kl::Variant::TF32;
    mlqmc_kl::TensorMaps kl_maps[MLQMC_MAX_LEVELS];

    // per-chunk buffers (max_samples entries)
    int64_t max_samples = 0;
    SampleDesc* d_samples = nullptr;  // rank order (finest level descending)
    double* d_Y = nullptr;            // normals, s per sample
    double* d_F = nullptr;            // F_t per sample, n_levels each
    double* d_chol = nullptr;         // banded level-0 factor per sample (interleaved by sample)
    float* d_chol32 = nullptr;        // its FP32 copy (mixed forms)
    double* d_norms = nullptr;
    double* d_part = nullptr;  // partial residual sums of the converged forms (samples x chunks), grown on demand
    int64_t part_cap = 0;
    double* d_qpart = nullptr;  // QoI partial sums of the large levels (samples x chunks), grown on demand
    int64_t qpart_cap = 0;
    // multi-index runs (mlqmc_sample_mixed): per-sample QoI in work order and
    // a throw-away sums buffer for the inner mlqmc_sample_levels call, the
    // work-item table on the device; grown on demand
    double* d_mix_F = nullptr;
    double* d_mix_S = nullptr;
    int64_t mix_cap = 0;
    void* d_mix_W = nullptr;
    int mix_wcap = 0;
    int* d_active = nullptr;
    int* d_count = nullptr;
    SampleDesc* h_samples = nullptr;  // pinned staging
    int* h_count = nullptr;           // pinned
    int* h_status = nullptr;          // pinned: the status word read with a round's sums
    cudaEvent_t staged = nullptr;     // recorded after the last copy out of the staging buffer
    // level 0 (its field, faces and banded factorisation) runs on a second
    // stream beside the other levels' fields: fork and join by events; with
    // every field from the tensor cores the factorisation waits for ev_fields
    // (the other levels' contractions issued) and runs beside their faces
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fields = nullptr;
    size_t chol_stride = 0;

    // level pools, grown on demand; chunks are cut to fit pool_budget bytes
    LevelPool pools[MLQMC_MAX_LEVELS];
    size_t pool_budget = 0;

    // optional per-kernel event timing
    bool profiling = false;
    struct Mark {
        int kind, level, nk;  // kernel kind, grid level (kProfNoLevel: none), kernels inside the bracket
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;        // recorded, not yet read
    std::vector<cudaEvent_t> pool;  // free events
    // per kernel kind and grid level: device time and launches of the read
    // brackets, and the algorithmic work of the launches since mlqmc_profile(1)
    // (bytes each launch must move with every array it touches once; FP64 /
    // FP32 / tensor-core FLOPs)
    ProfCell prof[kProfKinds][kProfLevels];
    int prof_level = kProfNoLevel;  // level that the next brackets belong to

    // smoother of each level's V-cycle sweeps (MLQMC_SMOOTHER_*), picked by
    // the autotuner at creation (mixed forms) or fixed by mlqmc_set_smoother;
    // tune_ms: the tuner's time per candidate (ms, 0 when not timed)
    int smoother[MLQMC_MAX_LEVELS] = {};
    double tune_ms[MLQMC_MAX_LEVELS][5] = {};
    // batch-size schedule of the autotuner: a level with fewer than
    // kSmallBatch samples in a call uses smoother_small (tuned on 64 samples)
    // instead of smoother (tuned on 1024); the tensor-core KL takes kl_nt[t][0]
    // or kl_nt[t][1] samples per tile (128 or 256), tuned on 64 and 256
    // samples (tune_kl_ms[t][class][0: 128, 1: 256])
    int smoother_small[MLQMC_MAX_LEVELS] = {};
    double tune_small_ms[MLQMC_MAX_LEVELS][5] = {};
    int kl_nt[MLQMC_MAX_LEVELS][2] = {};
    double tune_kl_ms[MLQMC_MAX_LEVELS][2][2] = {};

    // Replay of repeated identical calls of the fixed-cycle forms as one CUDA
    // graph: the second call with the same ranked samples, outputs and pools
    // is captured (on a stream of the library's own, since the caller's may
    // be the legacy stream), later ones replay it.
    struct GraphCache {
        bool enabled = true;
        cudaStream_t stream = nullptr;
        cudaEvent_t in = nullptr, out = nullptr;  // caller stream -> graph stream -> caller stream
        SampleDesc* h_samples = nullptr;          // pinned descriptors the graph's upload reads
        std::vector<SampleDesc> key;              // ranked samples of the pending / captured call
        double* sums = nullptr;
        double* F = nullptr;
        uint64_t epoch = 0;
        bool profiled = false;
        int seen = 0;  // 1: key seen once, 2: captured
        cudaGraphExec_t exec = nullptr;
        std::vector<Mark> marks;  // events recorded inside the graph (profiling)
        ProfCell work[kProfKinds][kProfLevels];  // algorithmic work of one replay
        int64_t launches = 0;
        int64_t replays = 0;
        bool capturing = false;  // event brackets become graph event-record nodes
        // Round graphs: a call that is not a repeat (an adaptive round of
        // Algorithm 1) is captured as one graph, the converged forms'
        // refinement loops as conditional WHILE nodes driven by the device,
        // and launched once; an instantiated graph of the same launch shape
        // is updated in place (cudaGraphExecUpdate) instead of rebuilt.
        int rounds = 2;               // 0 off, 1 on, 2 on in the converged forms only (the default)
        bool round_capture = false;   // capturing a round: loops run on the device
        bool in_body = false;         // capturing a conditional body (no memset nodes)
        cudaStream_t body = nullptr;  // captures the loop bodies
        struct RoundExec {
            std::vector<int32_t> key;
            cudaGraphExec_t exec;
        };
        std::vector<RoundExec> round_execs;
        int64_t round_launches = 0, round_updates = 0, round_instantiations = 0;
    } graph;
    uint64_t pool_epoch = 0;  // bumped whenever a pool or device buffer is reallocated

    int* d_status = nullptr;  // deferred device status bits
    int host_status = 0;      // deferred status found on the host (converged-form loops)
    int last_iters[MLQMC_MAX_LEVELS] = {};  // extra cycles / refinement steps per level, last converged-form call
    int* d_queue = nullptr;   // work-queue counter
    // device-side refinement loops (round graphs): per level the current
    // iteration [t] and the largest iteration reached since the last
    // mlqmc_last_iterations [MLQMC_MAX_LEVELS + t]
    int* d_iters = nullptr;
    int64_t launches = 0;
};
