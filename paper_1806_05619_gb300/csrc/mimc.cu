// Multi-index variant of MG-MLQMC: grid level x number of V-cycles (the
// outlook of Sec. 7: multi-index Monte Carlo whose second direction is the
// cycle count of the multigrid solver).
//
// Index (t, m): grid level t, cycle count mu_m (the mu0 of context m). One
// sample y at FMG level k gives, from the FMG solves of y by the contexts of
// direction m and m-1, the mixed differences
//   D_{t,m}(y) = [F_t^m(y) - F_{t-1}^m(y)] - [F_t^{m-1}(y) - F_{t-1}^{m-1}(y)]
// for every t <= k (F_{-1} = 0, F^{-1} = 0), recycled over t as in eq.
// Upsilon-reuse. Summed over the full index set they telescope to F_L of the
// largest cycle count, so the estimator keeps the MG-MLQMC mean of that
// count while spending fewer samples on the expensive cycle counts.
//
// The FMG solves are mlqmc_sample_levels calls on the two contexts (per-sample
// QoI into context scratch); the mixed differences and their sums are formed
// by the kernels below, in a fixed order.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "mlqmc_internal.h"

namespace {

// One work item on the device: samples off .. off + count*(r_end-r_begin)-1 in
// work order (item by item, then r, then n).
struct MixItem {
    int32_t level, r_begin, r_end, pad;
    int64_t count, off;
};

// Sum over the block in a fixed order (warp tree, then warps in order).
__device__ __forceinline__ double mix_block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
        red[32] = s;
    }
    __syncthreads();
    const double s = red[32];
    __syncthreads();
    return s;
}

__device__ __forceinline__ double mixed_diff(const double* __restrict__ Fh, const double* __restrict__ Fl,
                                             size_t q, int n_levels, int t)
{
    const double* fh = Fh + q * n_levels;
    double v = fh[t] - (t > 0 ? fh[t - 1] : 0.0);
    if (Fl) {
        const double* fl = Fl + q * n_levels;
        v -= fl[t] - (t > 0 ? fl[t - 1] : 0.0);
    }
    return v;
}

// Sums of D_{t,m} and D_{t,m}^2 per (level t, shift r): one block each.
// blockDim.x is a multiple of 32 and at most 1024.
__global__ void k_mixed_sums(const MixItem* __restrict__ items, int n_items, const double* __restrict__ Fh,
                             const double* __restrict__ Fl, int n_levels, int R, int reuse, double* __restrict__ sums)
{
    __shared__ double red[33];
    const int t = blockIdx.x / R;
    const int r = blockIdx.x - t * R;
    double a = 0.0, a2 = 0.0;
    for (int i = 0; i < n_items; ++i) {
        const MixItem w = items[i];
        // uniform over the block: depends on i, t, r only
        if (!(reuse ? w.level >= t : w.level == t) || r < w.r_begin || r >= w.r_end) continue;
        const int64_t base = w.off + static_cast<int64_t>(r - w.r_begin) * w.count;
        for (int64_t j = threadIdx.x; j < w.count; j += blockDim.x) {
            const double v = mixed_diff(Fh, Fl, static_cast<size_t>(base + j), n_levels, t);
            a += v;
            a2 += v * v;
        }
    }
    a = mix_block_sum(a, red);
    a2 = mix_block_sum(a2, red);
    if (threadIdx.x == 0) {
        sums[(static_cast<size_t>(t) * R + r) * 2 + 0] += a;
        sums[(static_cast<size_t>(t) * R + r) * 2 + 1] += a2;
    }
}

// Per-sample D_{0..level,m} (zeros above) in work order.
__global__ void k_mixed_out(const MixItem* __restrict__ items, int n_items, const double* __restrict__ Fh,
                            const double* __restrict__ Fl, int n_levels, int64_t total, double* __restrict__ D)
{
    const int64_t n = total * n_levels;
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < n;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t q = idx / n_levels;
        const int t = static_cast<int>(idx - q * n_levels);
        int level = -1;
        for (int i = 0; i < n_items; ++i) {
            const MixItem w = items[i];
            const int64_t size = w.count * (w.r_end - w.r_begin);
            if (q >= w.off && q < w.off + size) {
                level = w.level;
                break;
            }
        }
        D[idx] = t <= level ? mixed_diff(Fh, Fl, static_cast<size_t>(q), n_levels, t) : 0.0;
    }
}

bool compatible(const mlqmc_ctx* hi, const mlqmc_ctx* lo)
{
    const mlqmc_problem& p = hi->p;
    const mlqmc_problem& q = lo->p;
    return hi != lo && hi->device == lo->device && q.mu0 < p.mu0 && p.n_levels == q.n_levels &&
           p.coarse_cells == q.coarse_cells && p.n_modes == q.n_modes && p.sigma == q.sigma &&
           p.corr_len == q.corr_len && p.qoi == q.qoi && p.nu1 == q.nu1 && p.nu2 == q.nu2 &&
           p.precision == q.precision && p.refine_rtol == q.refine_rtol && p.refine_max_iter == q.refine_max_iter &&
           p.sampler == q.sampler && p.seed == q.seed && p.n_shifts == q.n_shifts && p.log2_nmax == q.log2_nmax &&
           p.reuse == q.reuse && p.covariance == q.covariance && p.nystrom_m == q.nystrom_m &&
           p.matern_nu == q.matern_nu && hi->z == lo->z && hi->modes.theta == lo->modes.theta &&
           hi->modes.a == lo->modes.a && hi->modes.b == lo->modes.b && hi->matern == lo->matern &&
           hi->psi_hash == lo->psi_hash;
}

// Per-sample QoI scratch (n_levels doubles per sample) and the throw-away sums.
mlqmc_status ensure_mix(mlqmc_ctx* c, int64_t total)
{
    const size_t nl = static_cast<size_t>(c->p.n_levels);
    if (!c->d_mix_S &&
        cudaMalloc(&c->d_mix_S, nl * static_cast<size_t>(c->p.n_shifts) * 2 * sizeof(double)) != cudaSuccess)
        return MLQMC_ERR_OOM;
    if (total > c->mix_cap) {
        const int64_t cap = std::max(total, 2 * c->mix_cap);
        cudaFree(c->d_mix_F);
        c->d_mix_F = nullptr;
        c->mix_cap = 0;
        if (cudaMalloc(&c->d_mix_F, static_cast<size_t>(cap) * nl * sizeof(double)) != cudaSuccess)
            return MLQMC_ERR_OOM;
        c->mix_cap = cap;
    }
    return MLQMC_OK;
}

}  // namespace

extern "C" mlqmc_status mlqmc_sample_mixed(mlqmc_ctx* hi, mlqmc_ctx* lo, const mlqmc_work* work, int32_t n_work,
                                           double* d_sums, double* d_D, void* stream)
{
    if (!hi || n_work < 0 || (n_work > 0 && !work) || !d_sums) return MLQMC_ERR_INVALID_ARG;
    if (lo && !compatible(hi, lo)) return MLQMC_ERR_INVALID_ARG;
    const mlqmc_problem& p = hi->p;
    std::vector<MixItem> items(static_cast<size_t>(n_work));
    int64_t total = 0;
    for (int i = 0; i < n_work; ++i) {
        const mlqmc_work& w = work[i];
        if (w.level < 0 || w.level >= p.n_levels || w.n_begin < 0 || w.n_end < w.n_begin || w.r_begin < 0 ||
            w.r_end < w.r_begin || w.r_end > p.n_shifts)
            return MLQMC_ERR_INVALID_ARG;
        items[i].level = w.level;
        items[i].r_begin = w.r_begin;
        items[i].r_end = w.r_end;
        items[i].pad = 0;
        items[i].count = w.n_end - w.n_begin;
        items[i].off = total;
        total += items[i].count * (w.r_end - w.r_begin);
    }
    if (total == 0) return MLQMC_OK;
    mlqmc_status s = ensure_mix(hi, total);
    if (s == MLQMC_OK && lo) s = ensure_mix(lo, total);
    if (s != MLQMC_OK) return s;
    if (n_work > hi->mix_wcap) {
        cudaFree(hi->d_mix_W);
        hi->d_mix_W = nullptr;
        hi->mix_wcap = 0;
        if (cudaMalloc(&hi->d_mix_W, sizeof(MixItem) * static_cast<size_t>(n_work)) != cudaSuccess)
            return MLQMC_ERR_OOM;
        hi->mix_wcap = n_work;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t sums_bytes = static_cast<size_t>(p.n_levels) * p.n_shifts * 2 * sizeof(double);
    // pageable source: the call returns once the items are staged, so the
    // vector may go out of scope afterwards
    if (cudaMemcpyAsync(hi->d_mix_W, items.data(), sizeof(MixItem) * items.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(hi->d_mix_S, 0, sums_bytes, st) != cudaSuccess ||
        (lo && cudaMemsetAsync(lo->d_mix_S, 0, sums_bytes, st) != cudaSuccess))
        return MLQMC_ERR_CUDA;
    s = mlqmc_sample_levels(hi, work, n_work, hi->d_mix_S, hi->d_mix_F, stream);
    if (s != MLQMC_OK) return s;
    if (lo) {
        s = mlqmc_sample_levels(lo, work, n_work, lo->d_mix_S, lo->d_mix_F, stream);
        if (s != MLQMC_OK) return s;
    }
    const MixItem* d_items = static_cast<const MixItem*>(hi->d_mix_W);
    const double* Fl = lo ? lo->d_mix_F : nullptr;
    k_mixed_sums<<<p.n_levels * p.n_shifts, 256, 0, st>>>(d_items, n_work, hi->d_mix_F, Fl, p.n_levels, p.n_shifts,
                                                          p.reuse, d_sums);
    if (d_D) {
        const int64_t n = total * p.n_levels;
        const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 8 * std::max(hi->sm_count, 1)));
        k_mixed_out<<<grid, 256, 0, st>>>(d_items, n_work, hi->d_mix_F, Fl, p.n_levels, total, d_D);
    }
    return cudaGetLastError() == cudaSuccess ? MLQMC_OK : MLQMC_ERR_CUDA;
}

// ---- multi-index driver ---------------------------------------------------

namespace {

struct MixEst {
    double Q = 0.0, varQ = std::numeric_limits<double>::infinity();
    std::vector<double> Ybar, V;  // [m * 32 + t]
};

// eqs. Upsilon-reuse, Upsilon-reuse-bar and sample_variances per index; the
// variance of Q from the shift replicates of the whole estimator (eq.
// var_of_mgmlqmc), which covers the correlation between indices that share
// points.
MixEst mix_finalize(int L, int K, int R, bool reuse, const std::vector<int64_t>& N,
                    const std::vector<std::vector<double>>& sums)
{
    MixEst e;
    e.Ybar.assign(static_cast<size_t>(MLQMC_MIMC_MAX_M) * 32, 0.0);
    e.V.assign(static_cast<size_t>(MLQMC_MIMC_MAX_M) * 32, 0.0);
    std::vector<double> Qr(R, 0.0), U(R);
    for (int m = 0; m < K; ++m)
        for (int t = 0; t <= L; ++t) {
            int64_t cnt = 0;
            if (reuse) {
                for (int i = t; i <= L; ++i) cnt += N[m * 32 + i];
            } else {
                cnt = N[m * 32 + t];
            }
            double mean = 0.0;
            for (int r = 0; r < R; ++r) {
                U[r] = cnt > 0 ? sums[m][(static_cast<size_t>(t) * R + r) * 2] / static_cast<double>(cnt) : 0.0;
                Qr[r] += U[r];
                mean += U[r];
            }
            mean /= R;
            double v = 0.0;
            for (int r = 0; r < R; ++r) v += (U[r] - mean) * (U[r] - mean);
            e.Ybar[m * 32 + t] = mean;
            e.V[m * 32 + t] = R > 1 ? v / (static_cast<double>(R) * (R - 1)) : std::numeric_limits<double>::infinity();
        }
    double qm = 0.0;
    for (int r = 0; r < R; ++r) qm += Qr[r];
    qm /= R;
    double v = 0.0;
    for (int r = 0; r < R; ++r) v += (Qr[r] - qm) * (Qr[r] - qm);
    e.Q = qm;
    e.varQ = R > 1 ? v / (static_cast<double>(R) * (R - 1)) : std::numeric_limits<double>::infinity();
    return e;
}

}  // namespace

extern "C" mlqmc_status mlqmc_estimate_mimc(mlqmc_ctx* const* ctx, int32_t K, double eps, const mlqmc_run_opts* o,
                                            mlqmc_mimc_result* out)
{
    if (!ctx || !out || K < 1 || K > MLQMC_MIMC_MAX_M || !(eps > 0.0)) return MLQMC_ERR_INVALID_ARG;
    for (int m = 0; m < K; ++m)
        if (!ctx[m]) return MLQMC_ERR_INVALID_ARG;
    for (int m = 1; m < K; ++m)
        if (!compatible(ctx[m], ctx[m - 1])) return MLQMC_ERR_INVALID_ARG;
    mlqmc_run_opts opts{};
    if (o) opts = *o;
    if (opts.max_rounds <= 0) opts.max_rounds = 1000;
    const auto t_start = std::chrono::steady_clock::now();
    const mlqmc_problem& p = ctx[0]->p;
    const int Lmax = p.n_levels - 1;
    const int R = p.n_shifts;
    const bool reuse = p.reuse != 0;
    const double inf = std::numeric_limits<double>::infinity();
    const size_t NI = static_cast<size_t>(MLQMC_MIMC_MAX_M) * 32;
    std::vector<int64_t> N(NI, 0), Nold(NI, 0);
    std::vector<double> V(NI, inf), Cst(NI, 0.0), Ybar(NI, 0.0), model(NI, 0.0);
    const size_t nsum = static_cast<size_t>(Lmax + 1) * R * 2;
    std::vector<std::vector<double>> sums(K, std::vector<double>(nsum, 0.0));
    for (int m = 0; m < K; ++m) {
        const double cyc = ctx[m]->p.mu0 + (m > 0 ? ctx[m - 1]->p.mu0 : 0);
        for (int l = 0; l <= Lmax; ++l) {
            double cells = 0.0;
            for (int t = 0; t <= l; ++t) {
                const double n = static_cast<double>(p.coarse_cells << t);
                cells += n * n;
            }
            model[m * 32 + l] = cells * cyc;
            if (opts.cost_model != 1) Cst[m * 32 + l] = model[m * 32 + l];
        }
    }

    cudaStream_t stream = nullptr;
    double* d_sums = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mlqmc_status st = MLQMC_OK;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&d_sums, nsum * K * sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        st = MLQMC_ERR_CUDA;
    if (st == MLQMC_OK && cudaMemsetAsync(d_sums, 0, nsum * K * sizeof(double), stream) != cudaSuccess)
        st = MLQMC_ERR_CUDA;

    int L = -1, rounds = 0, run_status = 0, clamped = 0;
    double Q = 0.0, varQ = inf, bias = inf, alpha = std::nan(""), gpu_s = 0.0;
    auto unsampled = [&](int Lc) {
        for (int m = 0; m < K; ++m)
            for (int t = 0; t <= Lc; ++t)
                if (std::isinf(V[m * 32 + t])) return true;
        return false;
    };
    // level differences of the largest cycle count: the mixed means summed over m
    auto level_mean = [&](int l) {
        double y = 0.0;
        for (int m = 0; m < K; ++m) y += Ybar[m * 32 + l];
        return y;
    };
    auto fit_alpha = [&](int Lc) {
        double sx = 0, sy = 0, sxx = 0, sxy = 0;
        int n = 0;
        for (int l = 1; l <= Lc; ++l) {
            const double y = std::log2(std::fabs(level_mean(l)));
            if (!std::isfinite(y)) continue;
            sx += l;
            sy += y;
            sxx += static_cast<double>(l) * l;
            sxy += l * y;
            ++n;
        }
        double a = std::nan("");
        if (n >= 2) a = -(n * sxy - sx * sy) / (n * sxx - sx * sx);
        clamped = 0;
        if (!(a > 0.0)) {
            a = 0.5;
            clamped = 1;
        }
        return a;
    };

    while (st == MLQMC_OK) {
        if (L >= 2) {
            alpha = fit_alpha(L);
            bias = std::fabs(level_mean(L)) / (std::pow(2.0, alpha) + 1.0);
            if (!(bias > eps / std::sqrt(2.0))) break;
        }
        if (L + 1 > Lmax) {
            run_status = 7;
            break;
        }
        ++L;
        for (;;) {
            varQ = inf;
            if (!unsampled(L)) {
                const MixEst e = mix_finalize(L, K, R, reuse, N, sums);
                varQ = e.varQ;
                Q = e.Q;
            }
            if (!(varQ > eps * eps / 2.0)) break;
            if (rounds >= opts.max_rounds) {
                run_status = 8;
                goto done;
            }
            // indices to double: the largest V/C (unsampled first; ties -> smallest m, then t)
            double best = -1.0;
            for (int m = 0; m < K; ++m)
                for (int t = 0; t <= L; ++t) {
                    const double ratio = std::isinf(V[m * 32 + t]) ? inf : V[m * 32 + t] / Cst[m * 32 + t];
                    if (ratio > best) best = ratio;
                }
            std::vector<int> pick;
            for (int m = 0; m < K && (opts.batched || pick.empty()); ++m)
                for (int t = 0; t <= L && (opts.batched || pick.empty()); ++t) {
                    const double ratio = std::isinf(V[m * 32 + t]) ? inf : V[m * 32 + t] / Cst[m * 32 + t];
                    const bool take = opts.batched ? (std::isinf(best) ? std::isinf(ratio) : ratio >= 0.5 * best)
                                                   : ratio == best;
                    if (take) pick.push_back(m * 32 + t);
                }
            // one mlqmc_sample_mixed call per direction that has picked indices
            for (int m = 0; m < K; ++m) {
                std::vector<mlqmc_work> work;
                double model_work = 0.0;
                for (int id : pick) {
                    if (id / 32 != m) continue;
                    const int t = id % 32;
                    N[id] = N[id] > 0 ? 2 * N[id] : 1;
                    mlqmc_work w{};
                    w.level = t;
                    w.n_begin = Nold[id];
                    w.n_end = N[id];
                    w.r_begin = 0;
                    w.r_end = R;
                    work.push_back(w);
                    model_work += model[id] * static_cast<double>((N[id] - Nold[id]) * R);
                }
                if (work.empty()) continue;
                cudaEventRecord(e0, stream);
                st = mlqmc_sample_mixed(ctx[m], m > 0 ? ctx[m - 1] : nullptr, work.data(),
                                        static_cast<int32_t>(work.size()), d_sums + nsum * m, nullptr, stream);
                cudaEventRecord(e1, stream);
                if (st != MLQMC_OK) goto done;
                if (cudaMemcpyAsync(sums[m].data(), d_sums + nsum * m, nsum * sizeof(double),
                                    cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                    cudaStreamSynchronize(stream) != cudaSuccess) {
                    st = MLQMC_ERR_CUDA;
                    goto done;
                }
                st = mlqmc_get_device_status(ctx[m], stream);
                if (st == MLQMC_OK && m > 0) st = mlqmc_get_device_status(ctx[m - 1], stream);
                if (st != MLQMC_OK) goto done;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                gpu_s += ms * 1e-3;
                for (int id : pick) {
                    if (id / 32 != m) continue;
                    Cst[id] = (opts.cost_model == 1 && model_work > 0.0) ? (ms * 1e-3) * model[id] / model_work
                                                                          : model[id];
                    Nold[id] = N[id];
                }
            }
            const MixEst e = mix_finalize(L, K, R, reuse, N, sums);
            for (int m = 0; m < K; ++m)
                for (int t = 0; t <= L; ++t) {
                    int64_t cnt = 0;
                    if (reuse) {
                        for (int i = t; i <= L; ++i) cnt += N[m * 32 + i];
                    } else {
                        cnt = N[m * 32 + t];
                    }
                    if (cnt > 0) {
                        Ybar[m * 32 + t] = e.Ybar[m * 32 + t];
                        V[m * 32 + t] = e.V[m * 32 + t];
                    }
                }
            ++rounds;
        }
    }
done:
    double bias_cycles = inf;
    if (L >= 0 && !unsampled(L)) {
        const MixEst e = mix_finalize(L, K, R, reuse, N, sums);
        Q = e.Q;
        varQ = e.varQ;
        bias_cycles = 0.0;
        for (int t = 0; t <= L; ++t) bias_cycles += std::fabs(e.Ybar[(K - 1) * 32 + t]);
    }
    std::memset(out, 0, sizeof(*out));
    out->Q = Q;
    out->varQ = varQ;
    out->bias = bias;
    out->alpha = alpha;
    out->bias_cycles = bias_cycles;
    out->L = L;
    out->K = K;
    out->rounds = rounds;
    out->run_status = run_status;
    out->alpha_clamped = clamped;
    out->gpu_seconds = gpu_s;
    for (size_t i = 0; i < NI; ++i) {
        out->N[i] = N[i];
        out->Ybar[i] = Ybar[i];
        out->Vell[i] = V[i];
        out->C[i] = Cst[i];
    }
    out->wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d_sums) cudaFree(d_sums);
    if (stream) cudaStreamDestroy(stream);
    return st;
}
