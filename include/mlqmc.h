/*
 * mlqmc.h -- C ABI of the GB300 (sm_103a) library for the multigrid multilevel
 * (quasi-)Monte Carlo method with sample recycling of Robbe, Nuyens and
 * Vandewalle (arXiv 1806.05619).
 *
 * Per sample the library draws y (a randomly shifted rank-1 lattice point
 * mapped to standard normals, Sec. 3.2, or Monte Carlo normals), synthesises
 * the lognormal Karhunen-Loeve field a = exp(z_s) on every grid level
 * (eq. truncatedKL, Sec. 5), solves -div(a grad u) = 1 on (0,1)^2 with zero
 * Dirichlet data by Full Multigrid (Sec. 4, Fig. FMG), and recycles the
 * solution of every level of that FMG into the level differences of the
 * MG-MLQMC estimator (eqs. Upsilon-reuse, MGMLQMC, var_of_mgmlqmc).
 *
 * Conventions for every entry point:
 *  - Plain C types only. "Device" pointers are CUDA global-memory addresses
 *    on the current device; "host" pointers are ordinary CPU memory.
 *  - The caller owns every pointer it passes; the library never frees them and
 *    keeps no reference after the call returns (genvec is copied).
 *  - A context owns all library scratch in device memory (tables, workspace).
 *  - Streams are passed as void* holding a cudaStream_t (NULL = legacy stream).
 *  - Every call returns an mlqmc_status; nothing throws across the ABI and
 *    nothing traps on the device. Errors raised inside kernels are recorded in
 *    a per-context device status word read by mlqmc_get_device_status.
 *  - One context must not be used from two host threads at once.
 */
#ifndef MLQMC_H
#define MLQMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MLQMC_OK = 0,
    MLQMC_ERR_INVALID_ARG = 1,      /* a size, index or option is out of range */
    MLQMC_ERR_CUDA = 2,             /* a CUDA runtime call failed */
    MLQMC_ERR_OOM = 3,              /* device or host allocation failed */
    MLQMC_ERR_POINTS_EXHAUSTED = 4, /* lattice index n >= 2^log2_nmax requested */
    MLQMC_ERR_NOT_CONVERGED = 5,    /* a level missed refine_rtol within refine_max_iter */
    MLQMC_ERR_TIMEOUT = 6,          /* a bounded device wait gave up */
    MLQMC_ERR_DEVICE_STATUS = 7,    /* a kernel reported an internal check failure */
    MLQMC_ERR_UNSUPPORTED = 8,      /* option combination not built */
    MLQMC_ERR_SCRATCH_LIMIT = 9     /* larger than mlqmc_fmg_fields_noalloc's static scratch */
} mlqmc_status;

typedef enum {
    MLQMC_FP64 = 0,         /* every step in FP64 */
    MLQMC_MIXED_TF32 = 1,   /* KL contraction in TF32 (FP32 accumulate), FP32 V-cycles,
                               FP64 outer residual/correction */
    MLQMC_MIXED_BF16X3 = 2  /* as MIXED_TF32 with a three-term split-bf16 contraction */
} mlqmc_precision;

typedef enum { MLQMC_QOI_CENTER = 0, MLQMC_QOI_MEAN = 1 } mlqmc_qoi;

/* Smoother of a level's red-black sweeps (all compute the same sweeps). */
typedef enum {
    MLQMC_SMOOTHER_GS = 0,     /* one launch per colour (FP64 form) */
    MLQMC_SMOOTHER_TILE = 1,   /* shared-memory tiles staged by plain loads (FP32: two sweeps per launch, FP64: one) */
    MLQMC_SMOOTHER_STREAM = 2, /* row wavefront with bulk-copy rings, residual/correction fused (n <= 256) */
    MLQMC_SMOOTHER_TMA = 3,    /* 32 x 32 tiles staged by TMA tensor copies, double-buffered (n >= 64) */
    MLQMC_SMOOTHER_WHOLE = 4   /* the whole grid of a sample in shared memory, residual/correction fused (n <= 64) */
} mlqmc_smoother;
typedef enum { MLQMC_SAMPLER_MC = 0, MLQMC_SAMPLER_LATTICE = 1 } mlqmc_sampler;
typedef enum {
    MLQMC_COV_SEPARABLE_EXP = 0, /* sigma^2 exp(-|x1-x1'|/l - |x2-x2'|/l), closed-form eigenpairs */
    MLQMC_COV_MATERN = 1         /* Matern (eq. matern) with Nystrom eigenpairs (Sec. 5) */
} mlqmc_covariance;

/*
 * Problem statement (Sec. 1 eq. PDE; Sec. 6 set-up restated on a cell-centred
 * finite-volume grid).
 *  n_levels      L+1 grid levels; level t has (coarse_cells * 2^t)^2 cells.
 *  coarse_cells  cells per side on level 0 (even, >= 2).
 *  n_modes       s, KL terms kept (eq. truncatedKL), 1..4096.
 *  sigma, corr_len  separable exponential covariance
 *                sigma^2 exp(-|x1-x1'|/corr_len - |x2-x2'|/corr_len).
 *  qoi           MLQMC_QOI_CENTER: mean of the four cells around (1/2,1/2)
 *                (the point value of Sec. 6 on a cell-centred grid);
 *                MLQMC_QOI_MEAN: mean of u over the domain.
 *  mu0, nu1, nu2 FMG cycles per level and pre/post red-black Gauss-Seidel sweeps
 *                (Sec. 4: mu0, mu1, mu2).
 *  precision     mlqmc_precision.
 *  refine_rtol   0: FMG with exactly mu0 V-cycles per level (fixed work).
 *                >0: after the mu0 cycles each level is iterated until
 *                ||b - A u||_2 / ||b||_2 <= refine_rtol (FP64 residual; in the
 *                mixed forms each correction is an FP32 V-cycle solve).
 *  refine_max_iter cap on extra cycles / refinement steps per level.
 *  sampler       mlqmc_sampler.
 *  seed          Philox key: random shifts (lattice) or the normals (MC).
 *  n_shifts      R independent shifts (or MC replicates), 1..4096.
 *  genvec        host array of n_modes odd generating-vector entries (lattice
 *                only; copied at create time); see mlqmc_cbc_genvec.
 *  log2_nmax     lattice sequence length 2^log2_nmax (0..32).
 *  reuse         1: MG-ML(Q)MC, every FMG level feeds its difference (eq.
 *                MGMLMC); 0: plain ML(Q)MC, only the finest difference counts.
 *  covariance    mlqmc_covariance (0 when the fields below are left zero).
 *  MLQMC_COV_MATERN (eq. matern, variance sigma^2, correlation length
 *  corr_len, smoothness matern_nu in {0.5, 1, 1.5, 2, 2.5}; half-integer nu in
 *  closed form, nu = 1, 2 through K_nu by the trapezoidal rule on its integral
 *  representation, tabulated with cubic Hermite interpolation): the KL modes are the Nystrom eigenpairs (eqs. discrinteq,
 *  matrixequation) on the cell centres of an nystrom_m x nystrom_m grid with
 *  midpoint weights 1/nystrom_m^2 (2..128), as mlqmc_nystrom_modes returns
 *  them: nystrom_theta (n_modes eigenvalues, positive) and nystrom_psi
 *  (nystrom_m^2 x n_modes, node-major, the eigenfunctions at the nodes,
 *  normalised to sum_q w_q psi_j(x_q)^2 = 1), host arrays copied at create
 *  time. Every level's cell-centre values come from the Nystrom
 *  interpolation formula (Sec. 5), evaluated once at create time in FP64.
 */
typedef struct {
    int32_t n_levels;
    int32_t coarse_cells;
    int32_t n_modes;
    int32_t pad0;
    double sigma;
    double corr_len;
    int32_t qoi;
    int32_t mu0, nu1, nu2;
    int32_t precision;
    int32_t pad1;
    double refine_rtol;
    int32_t refine_max_iter;
    int32_t sampler;
    uint64_t seed;
    int32_t n_shifts;
    int32_t pad2;
    const uint32_t* genvec;
    int32_t log2_nmax;
    int32_t reuse;
    int32_t covariance;
    int32_t nystrom_m;
    double matern_nu;
    const double* nystrom_theta;
    const double* nystrom_psi;
} mlqmc_problem;

/*
 * One block of samples (Algorithm 1, SampleAndSolve): samples whose FMG ends
 * at `level`, lattice (or MC) indices n_begin..n_end-1, shifts r_begin..r_end-1.
 * Samples are ordered item by item, then by r, then by n.
 */
typedef struct {
    int32_t level;
    int32_t pad;
    int64_t n_begin, n_end;
    int32_t r_begin, r_end;
} mlqmc_work;

typedef struct mlqmc_ctx mlqmc_ctx;

/* Adaptive run options (Algorithm 1). */
typedef struct {
    int32_t max_rounds;   /* cap on SampleAndSolve calls (0 -> 1000) */
    int32_t cost_model;   /* 0: C_l = sum_{t<=l} n_t^2 (deterministic); 1: measured GPU time */
    int32_t batched;      /* 0: one level per round (exact Algorithm 1);
                             1: every level with V_l/C_l >= max/2 doubles in one launch */
    int32_t pad;
} mlqmc_run_opts;

typedef struct {
    double Q;             /* eq. MGMLQMC */
    double varQ;          /* eq. var_of_mgmlqmc */
    double bias;          /* eq. bias, |Ybar_L| / (2^alpha + 1) */
    double alpha;         /* least-squares rate of |Ybar_l|, l = 1..L */
    int32_t L;            /* finest level used */
    int32_t rounds;       /* SampleAndSolve calls */
    int32_t run_status;   /* 0 done; 7 stopped at the finest available level; 8 round cap */
    int32_t alpha_clamped;
    double wall_seconds;  /* host wall time of the whole run */
    double gpu_seconds;   /* device time of all sample launches (CUDA events) */
    int64_t N[32];        /* samples whose FMG ended at each level */
    double Ybar[32];      /* eq. Upsilon-reuse-bar */
    double Vell[32];      /* eq. sample_variances */
    double C[32];         /* cost per sample used by the level choice */
} mlqmc_result;

/*
 * Create a context: validates the problem, builds the KL eigenpairs in closed
 * form (eq. inteq for the exponential kernel), the mode table, the per-level
 * 1D eigenfunction tables, and allocates device workspace for
 * max_samples_per_call samples per mlqmc_sample_levels call (0 -> 65536).
 * The current CUDA device at this call is the context's device.
 * Errors: INVALID_ARG (bad sizes, even genvec entry, NULL out), OOM, CUDA.
 */
mlqmc_status mlqmc_create(const mlqmc_problem* p, int64_t max_samples_per_call, mlqmc_ctx** out);

/*
 * Nystrom eigenpairs of the Matern covariance (Sec. 5, eqs. discrinteq and
 * matrixequation): nodes x_q at the cell centres of an m x m grid on the unit
 * square (q = k2*m + k1), weights w_q = 1/m^2, B = sqrt(W) Sigma sqrt(W) with
 * Sigma_kq = C(x_k, x_q) (eq. matern, variance sigma^2), all eigenpairs of B
 * by the dense symmetric eigensolver of cuSOLVER in FP64 on the current
 * device, the s largest returned in descending order:
 *  theta_out  host, s eigenvalues;
 *  psi_out    host, m*m x s (node-major): psi_j(x_q) = v_qj / sqrt(w_q), so
 *             that sum_q w_q psi_j(x_q) psi_i(x_q) = delta_ij.
 * Within an eigenvalue of multiplicity > 1 the basis is the solver's; an
 * eigenvector's sign is the solver's. nu in {0.5, 1, 1.5, 2, 2.5}; 2 <= m <= 128;
 * 1 <= s <= m*m. Blocking. Errors: INVALID_ARG, OOM, CUDA (solver failure).
 */
mlqmc_status mlqmc_nystrom_modes(double nu, double corr_len, double sigma, int32_t m, int32_t s,
                                 double* theta_out, double* psi_out);

/* Release everything the context owns. NULL is a no-op. */
void mlqmc_destroy(mlqmc_ctx* c);

/*
 * Run SampleAndSolve (Algorithm 1) for a list of sample blocks on `stream`
 * and ACCUMULATE the level-difference sums (eq. Upsilon-reuse numerators):
 *   d_sums[(t*R + r)*2 + 0] += sum of dF_t,  [.. + 1] += sum of dF_t^2
 * over the samples of shift r whose FMG level k >= t (reuse) or k == t (no
 * reuse), dF_t = F_t - F_{t-1}, F_{-1} = 0.
 *  d_sums  device, n_levels * R * 2 doubles, caller-owned, not cleared.
 *  d_F     device or NULL: per sample (in work order) n_levels doubles,
 *          F_0..F_level then zeros.
 * Asynchronous: returns after enqueueing. Host-side validation errors
 * (INVALID_ARG, POINTS_EXHAUSTED, more samples than max_samples_per_call)
 * are returned at once; device-side failures (NOT_CONVERGED) are recorded
 * for mlqmc_get_device_status. Sums are deterministic for a given input.
 */
mlqmc_status mlqmc_sample_levels(mlqmc_ctx* c, const mlqmc_work* work, int32_t n_work,
                                 double* d_sums, double* d_F, void* stream);

/*
 * Algorithm 1 (MG-MLQMC(eps)): adaptive levels and sample doubling until the
 * variance estimate is <= eps^2/2 and the bias estimate is <= eps/sqrt(2).
 * Blocking; the result is in host memory. Uses its own stream. After each
 * round the reuse sums and the context's deferred device status come back in
 * one synchronisation (the status word is then cleared, as by
 * mlqmc_get_device_status); a device error ends the run with its status.
 */
mlqmc_status mlqmc_estimate(mlqmc_ctx* c, double eps, const mlqmc_run_opts* opts, mlqmc_result* out);

/*
 * Plain MLMC, the baseline of the paper's comparison (Sec. 2; Tab. speedup,
 * S1 and S2): independent Monte Carlo samples per level, no recycling, one
 * replicate (shift index 0 only), the mean-square error split into variance
 * and squared bias, each at most eps^2/2 (eq. MSE). Levels are added one at
 * a time from L = 0; a new level first takes 32 samples; after each round
 * the sample counts are raised to eq. nopt,
 *   N_l = ceil(2/eps^2 sqrt(V_l/C_l) sum_{t<=L} sqrt(V_t C_t)),
 * with V_l the sample variance of F_l - F_{l-1} (ddof 1) and C_l as in
 * mlqmc_estimate (opts->cost_model), all levels short of their count sampled
 * in one mlqmc_sample_levels call; when no level is short, the bias test of
 * mlqmc_estimate (least-squares alpha over levels 1..L, |Ybar_L|/(2^alpha+1))
 * decides between stopping and adding a level (L >= 2 first).
 * The context must use the Monte Carlo sampler and no recycling
 * (MLQMC_ERR_INVALID_ARG otherwise); opts->batched is ignored.
 * Result: Q = sum of the level means, varQ = sum V_l/N_l (eq. vardecomp),
 * N[l] samples of level l, Ybar[l] their mean difference, Vell[l] = V_l,
 * C[l]; rounds = mlqmc_sample_levels calls; run_status 7 when the finest
 * level is reached with the bias test failing, 8 at max_rounds.
 * Blocking; uses its own stream.
 */
mlqmc_status mlqmc_estimate_mlmc(mlqmc_ctx* c, double eps, const mlqmc_run_opts* opts, mlqmc_result* out);

/*
 * Multi-index variant: the second refinement direction is the number of
 * V-cycles of the FMG solve (the outlook of Sec. 7, multi-index Monte Carlo
 * with levels x V-cycles). Index (t, m): grid level t and the cycle count of
 * a context c_m. For one sample y the mixed difference is
 *   D_{t,m}(y) = [F_t^{hi}(y) - F_{t-1}^{hi}(y)] - [F_t^{lo}(y) - F_{t-1}^{lo}(y)]
 * with F^{hi}, F^{lo} the QoI of the FMG solves of that y by c_hi and c_lo
 * (F_{-1} = 0); with c_lo = NULL (m = 0) the second bracket is zero and D is
 * the level difference of mlqmc_sample_levels. An FMG that ends at level k
 * yields D_{t,m} for every t <= k, and these are recycled exactly as in eq.
 * Upsilon-reuse.
 *
 * Runs mlqmc_sample_levels for `work` on c_hi and on c_lo (the same y: both
 * contexts draw the same points and shifts), then on `stream`
 *   d_sums[(t*R + r)*2 + 0] += sum of D_{t,m},  [.. + 1] += sum of D_{t,m}^2
 * over the samples of shift r whose FMG level k >= t (reuse) or k == t.
 *  d_sums  device, n_levels * R * 2 doubles, caller-owned, not cleared.
 *  d_D     device or NULL: per sample in work order n_levels doubles,
 *          D_{0..level,m} then zeros.
 * c_lo, when given, must equal c_hi in every problem field, the generating
 * vector and the modes, except mu0, which must be smaller (else INVALID_ARG).
 * Work is validated as in mlqmc_sample_levels. Scratch for the per-sample
 * QoI of both contexts (n_levels doubles per sample each) is grown on demand
 * inside the contexts. Asynchronous like mlqmc_sample_levels; deterministic.
 * Errors: INVALID_ARG, POINTS_EXHAUSTED, OOM, CUDA.
 */
mlqmc_status mlqmc_sample_mixed(mlqmc_ctx* c_hi, mlqmc_ctx* c_lo, const mlqmc_work* work, int32_t n_work,
                                double* d_sums, double* d_D, void* stream);

#define MLQMC_MIMC_MAX_M 8
/* Result of mlqmc_estimate_mimc; index (t, m) is stored at [m*32 + t]. */
typedef struct {
    double Q;             /* sum over {0..L} x {0..K-1} of the recycled mean mixed differences */
    double varQ;          /* variance of Q from the R shift replicates of the whole estimator */
    double bias;          /* eq. bias on the level direction: |Ybar_L| / (2^alpha + 1), Ybar_l = sum_m Ybar_{l,m} */
    double alpha;         /* least-squares rate of |Ybar_l|, l = 1..L */
    double bias_cycles;   /* indicator of the cycle direction: sum_t |Ybar_{t,K-1}| (not tested) */
    int32_t L;            /* finest level used */
    int32_t K;            /* number of cycle counts (contexts) */
    int32_t rounds;       /* rounds of sample doubling */
    int32_t run_status;   /* 0 done; 7 finest available level reached with the bias test failing; 8 round cap */
    int32_t alpha_clamped;
    int32_t pad;
    double wall_seconds;  /* host wall time of the whole run */
    double gpu_seconds;   /* device time of all sample launches (CUDA events) */
    int64_t N[MLQMC_MIMC_MAX_M * 32];   /* samples whose FMG ended at level t, direction m */
    double Ybar[MLQMC_MIMC_MAX_M * 32]; /* recycled mean of D_{t,m} over shifts (eq. Upsilon-reuse-bar) */
    double Vell[MLQMC_MIMC_MAX_M * 32]; /* its variance from the replicates (eq. sample_variances) */
    double C[MLQMC_MIMC_MAX_M * 32];    /* cost per sample used by the index choice */
} mlqmc_mimc_result;

/*
 * Multi-index MLQMC, levels x cycle counts: ctx[0..K-1] are compatible
 * contexts (as for mlqmc_sample_mixed) with strictly increasing mu0; direction
 * m uses ctx[m] and ctx[m-1]. Algorithm 1 with the level direction adaptive
 * and the cycle direction complete: levels are added one at a time from
 * L = 0; for the index set {0..L} x {0..K-1}, each round doubles N_{t,m}
 * (0 -> 1 point x R shifts) of the index with the largest V_{t,m} / C_{t,m}
 * (unsampled first, ties -> smallest m, then smallest t; opts->batched: every
 * index with at least half the largest ratio) until varQ <= eps^2/2; then,
 * for L >= 2, the bias test of mlqmc_estimate on Ybar_l = sum_m Ybar_{l,m}
 * (the level differences of the largest cycle count, by telescoping in m)
 * decides between stopping and adding a level. Cost: opts->cost_model 0
 * gives C_{t,m} = (sum_{t'<=t} n_t'^2) (mu0_m + mu0_{m-1}) (mu0_{-1} = 0), 1
 * the measured GPU time per sample. K in 1..MLQMC_MIMC_MAX_M; with K = 1 this
 * is mlqmc_estimate. opts->max_rounds caps the rounds (0 -> 1000).
 * Blocking; uses its own stream. Errors: INVALID_ARG, OOM, CUDA, and the
 * device status of the contexts.
 */
mlqmc_status mlqmc_estimate_mimc(mlqmc_ctx* const* ctx, int32_t K, double eps, const mlqmc_run_opts* opts,
                                 mlqmc_mimc_result* out);

/*
 * The estimator from reuse sums (host only, no context or device needed): for
 * levels t = 0..L and shifts r < R, sums[(t*R + r)*2 + 0] = sum of dF_t over
 * the samples that enter level t's difference ([.. + 1] the sum of squares,
 * not used here), N[t] = samples whose FMG ended at level t. Writes Q (eq.
 * MGMLQMC), varQ (eq. var_of_mgmlqmc) and, when non-NULL, Ybar[t] (eq.
 * Upsilon-reuse-bar) and Vell[t] (eq. sample_variances), L+1 entries each.
 * With reuse = 0 the difference of level t averages over N[t] samples (plain
 * ML(Q)MC), else over N[t] + ... + N[L] (eq. Upsilon-reuse). This is how
 * sums all-reduced over ranks that ran disjoint shift ranges become one
 * estimate. Errors: INVALID_ARG (L outside 0..31, R < 1, negative N, NULL).
 */
mlqmc_status mlqmc_estimator_from_sums(int32_t L, int32_t R, int32_t reuse, const int64_t* N, const double* sums,
                                       double* Q, double* varQ, double* Ybar, double* Vell);

/* Synchronise `stream`, return and clear the deferred device status. */
mlqmc_status mlqmc_get_device_status(mlqmc_ctx* c, void* stream);

/* Static text for a status code. */
const char* mlqmc_status_string(mlqmc_status s);

/*
 * Generating vector by component-by-component construction (Sec. 3.2 cites
 * Nuyens-Cools): N = 2^m points, product weights gamma (host, s entries),
 * criterion e^2 = -1 + N^-1 sum_k prod_j (1 + gamma_j B2({k z_j/N})),
 * B2(x) = x^2 - x + 1/6; z_1 = 1; candidates odd z <= N/2, ties -> smallest.
 * Host only, multi-threaded. z_out: s entries; e2_out (may be NULL): the
 * criterion after each component. Errors: INVALID_ARG (s < 1, m < 1, m > 24).
 */
mlqmc_status mlqmc_cbc_genvec(int32_t s, int32_t m, const double* gamma, uint32_t* z_out,
                              double* e2_out);

/* ---- Introspection of intermediate steps (parity tests and tools) ------- */

/* The context's modes (eq. truncatedKL ordering): host arrays of n_modes. */
mlqmc_status mlqmc_modes(const mlqmc_ctx* c, int32_t* a, int32_t* b, double* theta);

/*
 * Lattice bits (Sec. 3.2): d_bits[i*s + j] = ((bitrev32(n_i) z_j mod 2^32) << 32)
 * + S_{level,r,j} mod 2^64 for n_i = n_begin + i, i < count (device uint64).
 * MC sampler: the 64 Philox bits of coordinate j instead.
 */
mlqmc_status mlqmc_point_bits(mlqmc_ctx* c, int32_t level, int32_t r, int64_t n_begin,
                              int32_t count, uint64_t* d_bits, void* stream);

/* Normals y = Phi^{-1}(u) for the same samples: d_y[i*s + j], device doubles;
 * u = ((bits >> 11) + 1/2) 2^-53. FP64 form: Phi^{-1} in FP64. Mixed forms
 * (whose normals only enter FP32 and tensor-core arithmetic): Phi^{-1} in
 * FP32 of u (u < 1/2) or of 1 - u (negated), so both tails keep float
 * resolution; these are the normals the mixed forms' samples use. */
mlqmc_status mlqmc_normals(mlqmc_ctx* c, int32_t level, int32_t r, int64_t n_begin,
                           int32_t count, double* d_y, void* stream);

/*
 * Field on grid level t for `count` normal vectors d_y[i*s + j] (device):
 * d_k[i*n_t^2 + i2*n_t + i1] = exp(z_s) at cell centres, FP64 output, computed
 * in the context's precision (FP64 form: FP64 synthesis; mixed forms: the
 * tensor-core contraction, rounded to FP32, widened). MLQMC_ERR_INVALID_ARG
 * when count exceeds max_samples or count x n_t (n_t + 1) reaches 2^31.
 */
mlqmc_status mlqmc_fields(mlqmc_ctx* c, int32_t t, const double* d_y, int32_t count, double* d_k,
                          void* stream);

/*
 * One sample (level, r, n): the solutions of all its FMG levels, concatenated
 * level 0..level, FP64, device (sum_t n_t^2 doubles), and F_0..F_level into
 * d_F (device, level+1 doubles).
 */
mlqmc_status mlqmc_sample_solution(mlqmc_ctx* c, int32_t level, int32_t r, int64_t n, double* d_u,
                                   double* d_F, void* stream);

/*
 * Allocation-free FMG solve from caller-supplied coefficient fields. The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- plug-ins whose host application owns all device memory
 * and hands them only their inputs and outputs, and real-time loops that must
 * not wait on the allocator or risk an allocation failing mid-run. It needs
 * no context (mlqmc_create allocates) and allocates nothing: its scratch is one static
 * device array of MLQMC_NOALLOC_SLOTS slots of MLQMC_NOALLOC_SLOT_BYTES
 * (16 x 1.25 MiB = 20 MiB) that every GPU loading this library holds until
 * the process exits.
 *
 * It runs the same FMG as mlqmc_sample_levels (FP64 form, fixed mu0
 * V(nu1,nu2)-cycles per level, exact level-0 solve) for `count` samples:
 *  d_k  device, per sample the FP64 coefficient k = exp(z) of levels 0..L
 *       concatenated, level t being (coarse_cells*2^t)^2 values row-major
 *       [i2*n + i1]; samples follow each other.
 *  d_F  device, count x n_levels FP64 outputs F_0..F_L (qoi as in mlqmc_qoi).
 * Limits: coarse_cells even in 2..16, finest level at most
 * MLQMC_NOALLOC_MAX_CELLS = 128 cells per side, n_levels <= 7; larger
 * problems return MLQMC_ERR_SCRATCH_LIMIT without launching anything.
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. Every call shares the one array: calls whose
 * kernels overlap on the GPU (other streams, other host threads) race and
 * corrupt each other; order them on one stream. Nothing in the array needs
 * to start at zero -- each solve writes every value it reads.
 */
#define MLQMC_NOALLOC_SLOTS 16
#define MLQMC_NOALLOC_SLOT_BYTES (1280 * 1024)
#define MLQMC_NOALLOC_MAX_CELLS 128
mlqmc_status mlqmc_fmg_fields_noalloc(int32_t coarse_cells, int32_t n_levels, int32_t qoi, int32_t mu0,
                                      int32_t nu1, int32_t nu2, int32_t count, const double* d_k, double* d_F,
                                      void* stream);

/*
 * Converged form: for each level (host array of n_levels), the largest
 * number of cycles (FP64 form) or refinement steps (mixed forms) beyond the
 * first mu0 that any sample of the calls since the previous query needed on
 * the batched path. Reading clears the counters.
 */
mlqmc_status mlqmc_last_iterations(mlqmc_ctx* c, int32_t* out);

/*
 * Test of the device-side timeout path (no counterpart in the paper): launches
 * one kernel that waits, with the bounded mbarrier wait the TMA-fed kernels
 * use, on a barrier that nothing arrives on, and gives up after limit_ns
 * nanoseconds (0..1e8); the give-up records MLQMC_ERR_TIMEOUT in the context's
 * device status (read by mlqmc_get_device_status). The kernel issues no copy
 * and holds no tensor memory, so nothing is in flight when it gives up.
 * Asynchronous on `stream`. Errors: INVALID_ARG, CUDA.
 */
mlqmc_status mlqmc_test_wait_timeout(mlqmc_ctx* c, int64_t limit_ns, void* stream);

/* Kernel launches issued by this context since creation (all entry points). */
int64_t mlqmc_launch_count(const mlqmc_ctx* c);

/*
 * Smoother per level of the V-cycles. mlqmc_create picks
 * one per level: where more than one smoother can run a level, an autotuner
 * times one V-cycle visit of that level (pre-smoothing with the restricted
 * residual, correction and post-smoothing) of each on 1024 samples of
 * scratch data and keeps the fastest (mixed forms; the choice changes results
 * by FP32 rounding only).
 * mlqmc_smoother_info: kind (host, n_levels int32, MLQMC_SMOOTHER_*; level 0
 * has no sweeps and reports 0) and tuned_ms (host, n_levels x 5 doubles,
 * [level][kind] milliseconds of the tuning visit, 0 where not timed); either
 * may be NULL. The FP64 form takes a fixed rule, so that every context gives
 * the same bits: MLQMC_SMOOTHER_WHOLE for n <= 64, MLQMC_SMOOTHER_GS above
 * (both multiply by the stored FP64 1/D and agree to rounding).
 * MLQMC_SMOOTHER_TILE also runs the FP64 form (one sweep per launch on
 * 32 x 32 tiles, sides 8, 16 or a multiple of 32; kb_gs's operations in
 * kb_gs's order) but is slower there, FP64 issue being the limit on GB300;
 * the wavefront and TMA smoothers are FP32 only.
 * mlqmc_set_smoother: force `kind` on `level` (1 <= level < n_levels) for
 * later calls; MLQMC_ERR_INVALID_ARG if that smoother cannot run the level
 * in the context's form (GS in a mixed form, an FP32-only smoother in the
 * FP64 form, or a side it does not handle).
 */
mlqmc_status mlqmc_smoother_info(const mlqmc_ctx* c, int32_t* kind, double* tuned_ms);
mlqmc_status mlqmc_set_smoother(mlqmc_ctx* c, int32_t level, int32_t kind);

/*
 * Batch-size schedule of the autotuner (mixed forms). The sample count of a
 * level varies from call to call (Algorithm 1's rounds start at one point
 * per shift and double), and the best kernel shape changes with it. A call
 * with fewer than 256 samples on a level uses that level's small-batch
 * choices, tuned on 64 samples; larger calls use the choices of
 * mlqmc_smoother_info (tuned on 1024). For the tensor-core KL contraction the
 * autotuner also times tiles of 128 and of 256 samples per CTA on up to
 * 262,144 of the level's cells, for 64 and for 256 samples, and keeps the
 * faster width per class. mlqmc_set_smoother forces a smoother for every
 * batch size. Outputs (host, any may be NULL): smoother_small (n_levels
 * int32, MLQMC_SMOOTHER_*; 0 for level 0); tuned_small_ms (n_levels x 5, as
 * tuned_ms); kl_nt (n_levels x 2: [level][small, large] samples per tile; 0
 * where the level has no tensor-core contraction); tuned_kl_ms (n_levels x 2
 * x 2: [level][class][128, 256] milliseconds).
 */
mlqmc_status mlqmc_schedule_info(const mlqmc_ctx* c, int32_t* smoother_small, double* tuned_small_ms, int32_t* kl_nt,
                                 double* tuned_kl_ms);

/*
 * Graph replay (on by default). In the fixed-cycle forms (refine_rtol = 0) a
 * call of mlqmc_sample_levels that fits one chunk and repeats the previous
 * call exactly (same ranked samples, same d_sums and d_F, no pool
 * reallocated or smoother changed since) is captured as one CUDA graph:
 * the upload of the sample descriptors and every launch of the call. Later
 * identical calls replay that graph on a stream of the library's own,
 * ordered after the caller's earlier work on `stream` and before its later
 * work by events. Results equal those of the launch-by-launch path (same
 * kernels, same order). With profiling on, the graph records its brackets
 * and each replay adds them to the totals (the call then waits for the
 * replay). mlqmc_set_graphs(c, 0) drops the graph and turns replay off;
 * mlqmc_graph_replays counts replays since creation.
 */
mlqmc_status mlqmc_set_graphs(mlqmc_ctx* c, int32_t enable);
int64_t mlqmc_graph_replays(const mlqmc_ctx* c);

/*
 * Round graphs (with graph replay on). A call of mlqmc_sample_levels that is
 * not a repeat -- one adaptive round of Algorithm 1 (Sec. 3.3), whose sample
 * counts differ from the previous round's -- runs as one graph launch when
 * round graphs apply to it (mlqmc_set_round_graphs), it fits one chunk and
 * profiling is off: the descriptors are uploaded by one
 * copy, then the call's kernels are captured into a graph, an instantiated
 * graph of the same launch shape (the levels that run, their smoothers, the
 * outputs asked for) is updated in place (cudaGraphExecUpdate) or a new one
 * instantiated, and the graph is launched once. In the converged forms
 * (refine_rtol > 0) each level's refinement loop becomes a conditional WHILE
 * node: its body (the masked mu0 V-cycles, u64 += e, the residual norms and
 * the loop decision) repeats on the device with no host round trip, taking
 * the same decisions as the host loop (stop when no sample is above the
 * tolerance; NOT_CONVERGED after refine_max_iter passes). Results equal those
 * of the launch-by-launch path (same kernels, same order).
 * mlqmc_graph_stats: out (host, 4 int64): repeat-graph replays, round-graph
 * launches, in-place updates, instantiations since creation.
 */
mlqmc_status mlqmc_graph_stats(const mlqmc_ctx* c, int64_t* out);

/*
 * Which calls run as round graphs: mode 0 none, 1 every call that is not a
 * repeat, 2 (the default) such calls of the converged forms (refine_rtol > 0),
 * where the refinement loops then run on the device without a host round
 * trip per pass. A one-off call of a fixed-cycle form has no such loop: there
 * the capture and update of its graph (host work while the GPU waits) cost
 * more than launching its kernels one by one. Errors: INVALID_ARG.
 */
mlqmc_status mlqmc_set_round_graphs(mlqmc_ctx* c, int32_t mode);

/*
 * Per-kernel device timing of mlqmc_sample_levels (off by default). With
 * enable = 1 every later launch is bracketed by CUDA events recorded on the
 * launch stream; enable = 0 stops recording. Either call clears the totals.
 */
mlqmc_status mlqmc_profile(mlqmc_ctx* c, int32_t enable);

/*
 * Totals since the last mlqmc_profile call, per kernel kind (8 entries):
 * 0 normals, 1 level-0 banded factor and exact solve (per sample), 2 KL field
 * and faces, 3 red-black sweeps, 4 residual/restriction, prolongation and
 * FP64 refinement updates, 5 coarse solves of the V-cycles, 6 QoI, norms,
 * reuse sums and outputs, 7 KL contraction on the tensor cores.
 * out_ms: device milliseconds (host, 8 doubles); out_n: launches (host, 8
 * int64). Waits for the recorded events.
 */
mlqmc_status mlqmc_profile_read(mlqmc_ctx* c, double* out_ms, int64_t* out_n);

/*
 * Algorithmic work of the launches recorded since the last mlqmc_profile
 * call, per kernel kind (same 8 kinds; host arrays of 8 doubles each):
 * out_bytes: bytes the launches must move when every array a launch touches
 * is read or written exactly once (halo re-reads, cache misses and
 * redundant tile work not counted); out_f64 / out_f32: FP64 and FP32 FLOPs of
 * the method's arithmetic (stencil updates 10 per cell, residual 10-12,
 * restriction 1, prolongation 8, harmonic faces 3 per face, banded Cholesky
 * N0 n0^2 per sample; exp and divisions counted as one); out_ftc: FLOPs of
 * the KL contraction on the tensor cores (2 M s B per level). These are the
 * numerators of the roofline fractions. Recorded only while profiling is on.
 */
mlqmc_status mlqmc_profile_work(mlqmc_ctx* c, double* out_bytes, double* out_f64, double* out_f32, double* out_ftc);

/*
 * The totals of mlqmc_profile_read and mlqmc_profile_work split by grid
 * level, so that one kernel on one grid size can be put against its
 * roofline: every output is a host array of 8 x MLQMC_PROFILE_LEVELS entries,
 * entry [kind * MLQMC_PROFILE_LEVELS + t] for level t (0..MLQMC_PROFILE_LEVELS-2);
 * the last column holds the launches that belong to no single level (normals,
 * reuse sums, per-sample outputs). out_ms: device milliseconds; out_n:
 * launches; out_bytes, out_f64, out_f32, out_ftc: algorithmic work as in
 * mlqmc_profile_work. Any output may be NULL. Waits for the recorded events.
 */
#define MLQMC_PROFILE_LEVELS 13
mlqmc_status mlqmc_profile_read_levels(mlqmc_ctx* c, double* out_ms, int64_t* out_n, double* out_bytes,
                                       double* out_f64, double* out_f32, double* out_ftc);

#ifdef __cplusplus
}
#endif

#endif /* MLQMC_H */
