// Host-side precompute and control for the MG-MLQMC library:
//  - closed-form KL eigenpairs of the 1D exponential kernel (Sec. 5, eq. inteq),
//  - the separable 2D mode table (eq. truncatedKL),
//  - the CBC generating vector (Sec. 3.2),
//  - Algorithm 1 (Sec. 3.3) around mlqmc_sample_levels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include <cuda_runtime.h>

#include "mlqmc_internal.h"

namespace mlqmc {

// Safeguarded Newton on g(w) = (w^2 - c^2) sin w - 2 c w cos w inside the
// bracket (k pi, (k+1) pi), which holds exactly one root (the tangent form
// tan w = 2cw/(w^2-c^2) of the eigenvalue condition for the [0,1] interval).
static double kl_root(double c, int k)
{
    double lo = k * M_PI, hi = (k + 1) * M_PI;
    if (k == 0) lo = std::numeric_limits<double>::min();
    auto g = [c](double w) { return (w * w - c * c) * std::sin(w) - 2.0 * c * w * std::cos(w); };
    auto dg = [c](double w) {
        return 2.0 * w * std::sin(w) + (w * w - c * c) * std::cos(w) - 2.0 * c * std::cos(w) +
               2.0 * c * w * std::sin(w);
    };
    const bool lo_neg = g(lo) < 0.0;
    double w = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        const double gw = g(w);
        if (gw == 0.0) return w;
        if ((gw < 0.0) == lo_neg) lo = w; else hi = w;
        double step = gw / dg(w);
        double wn = w - step;
        if (!(wn > lo && wn < hi)) wn = 0.5 * (lo + hi);
        if (std::fabs(wn - w) <= 2.0 * std::numeric_limits<double>::epsilon() * w) {
            w = wn;
            break;
        }
        w = wn;
        if (hi - lo <= 4.0 * std::numeric_limits<double>::epsilon() * hi) break;
    }
    return w;
}

Eig1D kl_eigen_1d(double corr_len, int K)
{
    Eig1D e;
    const double c = 1.0 / corr_len;
    e.omega.resize(K);
    e.theta.resize(K);
    e.norm.resize(K);
    for (int k = 0; k < K; ++k) {
        const double w = kl_root(c, k);
        const double sw = std::sin(w), cw = std::cos(w);
        e.omega[k] = w;
        e.theta[k] = 2.0 * c / (w * w + c * c);
        // int_0^1 (w cos wx + c sin wx)^2 dx
        e.norm[k] = 0.5 * (w * w + c * c) + (w * w - c * c) * sw * cw / (2.0 * w) + c * sw * sw;
    }
    return e;
}

static double key40(double v)
{
    int ex = 0;
    const double m = std::frexp(v, &ex);
    return std::ldexp(std::nearbyint(std::ldexp(m, 40)), ex - 40);
}

Modes select_modes(double corr_len, double sigma, int s)
{
    Modes md;
    const Eig1D e = kl_eigen_1d(corr_len, s);
    struct Cand {
        double key, theta;
        int a, b;
    };
    std::vector<Cand> all;
    all.reserve(static_cast<size_t>(s) * s);
    const double s2 = sigma * sigma;
    for (int a = 0; a < s; ++a) {
        for (int b = 0; b < s; ++b) {
            const double t = s2 * e.theta[a] * e.theta[b];
            all.push_back({key40(t), t, a, b});
        }
    }
    auto less = [](const Cand& x, const Cand& y) {
        if (x.key != y.key) return x.key > y.key;
        if (x.a != y.a) return x.a < y.a;
        return x.b < y.b;
    };
    std::partial_sort(all.begin(), all.begin() + s, all.end(), less);
    md.a.resize(s);
    md.b.resize(s);
    md.theta.resize(s);
    int K1 = 0;
    for (int m = 0; m < s; ++m) {
        md.a[m] = all[m].a;
        md.b[m] = all[m].b;
        md.theta[m] = all[m].theta;
        K1 = std::max(K1, std::max(all[m].a, all[m].b) + 1);
    }
    md.K1 = K1;
    return md;
}

void psi_table(const Eig1D& e, double corr_len, int K1, int n, std::vector<double>& out)
{
    const double c = 1.0 / corr_len;
    out.assign(static_cast<size_t>(K1) * n, 0.0);
    for (int k = 0; k < K1; ++k) {
        const double w = e.omega[k];
        const double inv = 1.0 / std::sqrt(e.norm[k]);
        for (int i = 0; i < n; ++i) {
            const double x = (i + 0.5) / n;
            out[static_cast<size_t>(k) * n + i] = (w * std::cos(w * x) + c * std::sin(w * x)) * inv;
        }
    }
}

// ---- Algorithm 1 ----------------------------------------------------------

namespace {

struct Est {
    double Q = 0.0, varQ = std::numeric_limits<double>::infinity();
    std::vector<double> Ybar, V;
};

// eqs. Upsilon-reuse, MGMLQMC, var_of_mgmlqmc, Upsilon-reuse-bar, sample_variances
Est finalize(int L, int R, bool reuse, const int64_t* N, const std::vector<double>& sums)
{
    Est e;
    e.Ybar.assign(L + 1, 0.0);
    e.V.assign(L + 1, 0.0);
    std::vector<double> Qr(R, 0.0), U(R);
    for (int t = 0; t <= L; ++t) {
        int64_t cnt = 0;
        if (reuse) {
            for (int i = t; i <= L; ++i) cnt += N[i];
        } else {
            cnt = N[t];
        }
        double mean = 0.0;
        for (int r = 0; r < R; ++r) {
            U[r] = cnt > 0 ? sums[(static_cast<size_t>(t) * R + r) * 2] / static_cast<double>(cnt) : 0.0;
            Qr[r] += U[r];
            mean += U[r];
        }
        mean /= R;
        double v = 0.0;
        for (int r = 0; r < R; ++r) v += (U[r] - mean) * (U[r] - mean);
        e.Ybar[t] = mean;
        e.V[t] = R > 1 ? v / (static_cast<double>(R) * (R - 1)) : std::numeric_limits<double>::infinity();
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

mlqmc_status run_estimate(mlqmc_ctx* c, double eps, const mlqmc_run_opts* o, mlqmc_result* out)
{
    if (!c || !out || !(eps > 0.0)) return MLQMC_ERR_INVALID_ARG;
    mlqmc_run_opts opts{};
    if (o) opts = *o;
    if (opts.max_rounds <= 0) opts.max_rounds = 1000;
    const auto t_start = std::chrono::steady_clock::now();
    const int Lmax = c->p.n_levels - 1;
    const int R = c->p.n_shifts;
    const bool reuse = c->p.reuse != 0;
    const double inf = std::numeric_limits<double>::infinity();
    std::vector<int64_t> N(32, 0), Nold(32, 0);
    std::vector<double> V(32, inf), C(32, 0.0), Ybar(32, 0.0);
    std::vector<double> sums(static_cast<size_t>(Lmax + 1) * R * 2, 0.0);
    std::vector<double> model(32, 0.0);
    for (int l = 0; l <= Lmax; ++l)
        for (int t = 0; t <= l; ++t) {
            const double n = static_cast<double>(c->p.coarse_cells << t);
            model[l] += n * n;
        }

    cudaStream_t stream = nullptr;
    double* d_sums = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mlqmc_status st = MLQMC_OK;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&d_sums, sums.size() * sizeof(double)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = MLQMC_ERR_CUDA;
    }
    if (st == MLQMC_OK && cudaMemsetAsync(d_sums, 0, sums.size() * sizeof(double), stream) != cudaSuccess)
        st = MLQMC_ERR_CUDA;

    int L = -1, rounds = 0, run_status = 0, clamped = 0;
    double Q = 0.0, varQ = inf, bias = inf, alpha = std::nan("");
    double gpu_s = 0.0;

    auto fit_alpha = [&](int Lc) {
        double sx = 0, sy = 0, sxx = 0, sxy = 0;
        int m = 0;
        for (int l = 1; l <= Lc; ++l) {
            const double y = std::log2(std::fabs(Ybar[l]));
            if (!std::isfinite(y)) continue;
            sx += l;
            sy += y;
            sxx += static_cast<double>(l) * l;
            sxy += l * y;
            ++m;
        }
        double a = std::nan("");
        if (m >= 2) a = -(m * sxy - sx * sy) / (m * sxx - sx * sx);
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
            bias = std::fabs(Ybar[L]) / (std::pow(2.0, alpha) + 1.0);
            if (!(bias > eps / std::sqrt(2.0))) break;
        }
        if (L + 1 > Lmax) {
            run_status = 7;
            break;
        }
        ++L;
        for (;;) {
            bool unsampled = false;
            for (int l = 0; l <= L; ++l) unsampled |= std::isinf(V[l]);
            varQ = inf;
            if (!unsampled) {
                Est e = finalize(L, R, reuse, N.data(), sums);
                varQ = e.varQ;
                Q = e.Q;
            }
            if (!(varQ > eps * eps / 2.0)) break;
            if (rounds >= opts.max_rounds) {
                run_status = 8;
                goto done;
            }
            // levels to double: the largest V_l/C_l (an unsampled level wins; ties -> smallest l)
            std::vector<double> ratio(L + 1);
            double best = -1.0;
            int arg = 0;
            for (int l = 0; l <= L; ++l) {
                ratio[l] = std::isinf(V[l]) ? inf : V[l] / C[l];
                if (ratio[l] > best) {
                    best = ratio[l];
                    arg = l;
                }
            }
            std::vector<int> pick;
            if (opts.batched) {
                for (int l = 0; l <= L; ++l)
                    if ((std::isinf(best) && std::isinf(ratio[l])) || (!std::isinf(best) && ratio[l] >= 0.5 * best))
                        pick.push_back(l);
            } else {
                pick.push_back(arg);
            }
            std::vector<mlqmc_work> work;
            double model_work = 0.0;
            for (int l : pick) {
                N[l] = N[l] > 0 ? 2 * N[l] : 1;
                mlqmc_work w{};
                w.level = l;
                w.n_begin = Nold[l];
                w.n_end = N[l];
                w.r_begin = 0;
                w.r_end = R;
                work.push_back(w);
                model_work += model[l] * static_cast<double>((N[l] - Nold[l]) * R);
            }
            cudaEventRecord(e0, stream);
            st = mlqmc_sample_levels(c, work.data(), static_cast<int32_t>(work.size()), d_sums, nullptr, stream);
            cudaEventRecord(e1, stream);
            if (st != MLQMC_OK) goto done;
            st = fetch_round(c, d_sums, sums.data(), sums.size(), stream);  // sums and device status, one sync
            if (st != MLQMC_OK) goto done;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            gpu_s += ms * 1e-3;
            int top = 0;
            for (int l : pick) {
                top = std::max(top, l);
                if (opts.cost_model == 1 && model_work > 0.0)
                    C[l] = (ms * 1e-3) * model[l] / model_work;  // seconds per sample of level l
                else
                    C[l] = model[l];
            }
            Est e = finalize(L, R, reuse, N.data(), sums);
            for (int t = 0; t <= top; ++t) {
                Ybar[t] = e.Ybar[t];
                V[t] = e.V[t];
            }
            for (int l : pick) Nold[l] = N[l];
            ++rounds;
        }
    }
done:
    if (L >= 0) {
        bool unsampled = false;
        for (int l = 0; l <= L; ++l) unsampled |= std::isinf(V[l]);
        if (!unsampled) {
            Est e = finalize(L, R, reuse, N.data(), sums);
            Q = e.Q;
            varQ = e.varQ;
        }
    }
    std::memset(out, 0, sizeof(*out));
    out->Q = Q;
    out->varQ = varQ;
    out->bias = bias;
    out->alpha = alpha;
    out->L = L;
    out->rounds = rounds;
    out->run_status = run_status;
    out->alpha_clamped = clamped;
    out->gpu_seconds = gpu_s;
    for (int l = 0; l <= Lmax && l < 32; ++l) {
        out->N[l] = N[l];
        out->Ybar[l] = Ybar[l];
        out->Vell[l] = V[l];
        out->C[l] = C[l];
    }
    out->wall_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d_sums) cudaFree(d_sums);
    if (stream) cudaStreamDestroy(stream);
    return st;
}

// ---- plain MLMC (the comparison baseline: eqs. MSE, vardecomp, nopt) -------

mlqmc_status run_estimate_mlmc(mlqmc_ctx* c, double eps, const mlqmc_run_opts* o, mlqmc_result* out)
{
    if (!c || !out || !(eps > 0.0)) return MLQMC_ERR_INVALID_ARG;
    if (c->p.sampler != MLQMC_SAMPLER_MC || c->p.reuse != 0) return MLQMC_ERR_INVALID_ARG;
    mlqmc_run_opts opts{};
    if (o) opts = *o;
    if (opts.max_rounds <= 0) opts.max_rounds = 1000;
    constexpr int64_t kWarm = 32;  // first samples of a new level
    const auto t_start = std::chrono::steady_clock::now();
    const int Lmax = c->p.n_levels - 1;
    const int R = c->p.n_shifts;
    const double inf = std::numeric_limits<double>::infinity();
    std::vector<int64_t> N(32, 0), want(32, 0);
    std::vector<double> V(32, inf), C(32, 0.0), Ybar(32, 0.0), model(32, 0.0);
    std::vector<double> sums(static_cast<size_t>(Lmax + 1) * R * 2, 0.0);
    for (int l = 0; l <= Lmax; ++l)
        for (int t = 0; t <= l; ++t) {
            const double n = static_cast<double>(c->p.coarse_cells << t);
            model[l] += n * n;
        }
    cudaStream_t stream = nullptr;
    double* d_sums = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mlqmc_status st = MLQMC_OK;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&d_sums, sums.size() * sizeof(double)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(d_sums, 0, sums.size() * sizeof(double), stream) != cudaSuccess)
        st = MLQMC_ERR_CUDA;

    int L = 0, rounds = 0, run_status = 0, clamped = 0;
    double bias = inf, alpha = std::nan(""), gpu_s = 0.0;
    want[0] = kWarm;
    // eq. nopt over levels 0..L from the current V_l, C_l
    auto optimal = [&]() {
        double acc = 0.0;
        for (int l = 0; l <= L; ++l) acc += std::sqrt(V[l] * C[l]);
        for (int l = 0; l <= L; ++l) {
            const double n = std::ceil(2.0 / (eps * eps) * std::sqrt(V[l] / C[l]) * acc);
            want[l] = std::max(N[l], static_cast<int64_t>(std::min(n, 9.0e18)));
        }
    };
    while (st == MLQMC_OK) {
        std::vector<mlqmc_work> work;
        double model_work = 0.0;
        for (int l = 0; l <= L; ++l)
            if (want[l] > N[l]) {
                mlqmc_work w{};
                w.level = l;
                w.n_begin = N[l];
                w.n_end = want[l];
                w.r_begin = 0;
                w.r_end = 1;
                work.push_back(w);
                model_work += model[l] * static_cast<double>(want[l] - N[l]);
            }
        if (!work.empty()) {
            if (rounds >= opts.max_rounds) {
                run_status = 8;
                break;
            }
            cudaEventRecord(e0, stream);
            st = mlqmc_sample_levels(c, work.data(), static_cast<int32_t>(work.size()), d_sums, nullptr, stream);
            cudaEventRecord(e1, stream);
            if (st != MLQMC_OK) break;
            st = fetch_round(c, d_sums, sums.data(), sums.size(), stream);  // sums and device status, one sync
            if (st != MLQMC_OK) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            gpu_s += ms * 1e-3;
            ++rounds;
            for (const mlqmc_work& w : work) {
                const int l = w.level;
                N[l] = w.n_end;
                C[l] = (opts.cost_model == 1 && model_work > 0.0) ? (ms * 1e-3) * model[l] / model_work : model[l];
            }
            for (int l = 0; l <= L; ++l) {
                const double n = static_cast<double>(N[l]);
                const double s1 = sums[static_cast<size_t>(l) * R * 2], s2 = sums[static_cast<size_t>(l) * R * 2 + 1];
                Ybar[l] = s1 / n;
                V[l] = N[l] > 1 ? (s2 - s1 * s1 / n) / (n - 1.0) : inf;
            }
            optimal();
            continue;
        }
        // every level has its count: the bias test, else one more level
        if (L >= 2) {
            double sx = 0, sy = 0, sxx = 0, sxy = 0;
            int m = 0;
            for (int l = 1; l <= L; ++l) {
                const double y = std::log2(std::fabs(Ybar[l]));
                if (!std::isfinite(y)) continue;
                sx += l;
                sy += y;
                sxx += static_cast<double>(l) * l;
                sxy += l * y;
                ++m;
            }
            alpha = m >= 2 ? -(m * sxy - sx * sy) / (m * sxx - sx * sx) : std::nan("");
            clamped = 0;
            if (!(alpha > 0.0)) {
                alpha = 0.5;
                clamped = 1;
            }
            bias = std::fabs(Ybar[L]) / (std::pow(2.0, alpha) + 1.0);
            if (!(bias > eps / std::sqrt(2.0))) break;
        }
        if (L + 1 > Lmax) {
            run_status = 7;
            break;
        }
        ++L;
        want[L] = kWarm;
    }
    std::memset(out, 0, sizeof(*out));
    double Q = 0.0, varQ = 0.0;
    for (int l = 0; l <= L; ++l) {
        Q += Ybar[l];
        varQ += N[l] > 0 ? V[l] / static_cast<double>(N[l]) : inf;
    }
    out->Q = Q;
    out->varQ = varQ;
    out->bias = bias;
    out->alpha = alpha;
    out->L = L;
    out->rounds = rounds;
    out->run_status = run_status;
    out->alpha_clamped = clamped;
    out->gpu_seconds = gpu_s;
    for (int l = 0; l <= Lmax && l < 32; ++l) {
        out->N[l] = N[l];
        out->Ybar[l] = Ybar[l];
        out->Vell[l] = V[l];
        out->C[l] = C[l];
    }
    out->wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d_sums) cudaFree(d_sums);
    if (stream) cudaStreamDestroy(stream);
    return st;
}

}  // namespace mlqmc

// ---- C ABI: host-only entry points ---------------------------------------

extern "C" const char* mlqmc_status_string(mlqmc_status s)
{
    switch (s) {
        case MLQMC_OK: return "ok";
        case MLQMC_ERR_INVALID_ARG: return "invalid argument";
        case MLQMC_ERR_CUDA: return "CUDA runtime error";
        case MLQMC_ERR_OOM: return "out of memory";
        case MLQMC_ERR_POINTS_EXHAUSTED: return "lattice sequence exhausted (n >= 2^log2_nmax)";
        case MLQMC_ERR_NOT_CONVERGED: return "refinement did not reach refine_rtol";
        case MLQMC_ERR_TIMEOUT: return "bounded device wait timed out";
        case MLQMC_ERR_DEVICE_STATUS: return "device-side check failed";
        case MLQMC_ERR_UNSUPPORTED: return "unsupported option";
        case MLQMC_ERR_SCRATCH_LIMIT: return "problem exceeds the static scratch of the no-allocation entry point";
    }
    return "unknown status";
}

// CBC (Sec. 3.2): for each new component the criterion
// sum_k P_k (1 + gamma_j B2((k z mod N)/N)) is evaluated for every odd candidate
// z <= N/2 from a table of B2 values, candidates in parallel.
extern "C" mlqmc_status mlqmc_cbc_genvec(int32_t s, int32_t m, const double* gamma, uint32_t* z_out,
                                         double* e2_out)
{
    if (s < 1 || m < 1 || m > 24 || !gamma || !z_out) return MLQMC_ERR_INVALID_ARG;
    const int64_t N = int64_t(1) << m;
    std::vector<double> omega(N), P(N);
    for (int64_t i = 0; i < N; ++i) {
        const double x = static_cast<double>(i) / static_cast<double>(N);
        omega[i] = x * x - x + 1.0 / 6.0;
    }
    for (int64_t k = 0; k < N; ++k) P[k] = 1.0 + gamma[0] * omega[k];
    z_out[0] = 1;
    auto crit = [&]() {
        double acc = 0.0;
        for (int64_t k = 0; k < N; ++k) acc += P[k];
        return -1.0 + acc / static_cast<double>(N);
    };
    if (e2_out) e2_out[0] = crit();
    const int64_t ncand = std::max<int64_t>(1, N / 4);  // odd z in [1, N/2]
    std::vector<double> val(ncand);
    for (int j = 1; j < s; ++j) {
        const double gj = gamma[j];
#pragma omp parallel for schedule(static)
        for (int64_t ci = 0; ci < ncand; ++ci) {
            const int64_t zc = 2 * ci + 1;
            double acc = 0.0;
            int64_t idx = 0;
            for (int64_t k = 0; k < N; ++k) {
                acc += P[k] * (1.0 + gj * omega[idx]);
                idx = (idx + zc) & (N - 1);
            }
            val[ci] = acc;
        }
        int64_t best = 0;
        for (int64_t ci = 1; ci < ncand; ++ci)
            if (val[ci] < val[best]) best = ci;
        const int64_t zb = 2 * best + 1;
        z_out[j] = static_cast<uint32_t>(zb);
        int64_t idx = 0;
        for (int64_t k = 0; k < N; ++k) {
            P[k] *= 1.0 + gj * omega[idx];
            idx = (idx + zb) & (N - 1);
        }
        if (e2_out) e2_out[j] = crit();
    }
    return MLQMC_OK;
}

extern "C" mlqmc_status mlqmc_estimate(mlqmc_ctx* c, double eps, const mlqmc_run_opts* opts, mlqmc_result* out)
{
    return mlqmc::run_estimate(c, eps, opts, out);
}

extern "C" mlqmc_status mlqmc_estimate_mlmc(mlqmc_ctx* c, double eps, const mlqmc_run_opts* opts, mlqmc_result* out)
{
    return mlqmc::run_estimate_mlmc(c, eps, opts, out);
}

extern "C" mlqmc_status mlqmc_estimator_from_sums(int32_t L, int32_t R, int32_t reuse, const int64_t* N,
                                                  const double* sums, double* Q, double* varQ, double* Ybar,
                                                  double* Vell)
{
    if (L < 0 || L >= 32 || R < 1 || !N || !sums || !Q || !varQ) return MLQMC_ERR_INVALID_ARG;
    for (int t = 0; t <= L; ++t)
        if (N[t] < 0) return MLQMC_ERR_INVALID_ARG;
    const std::vector<double> s(sums, sums + static_cast<size_t>(L + 1) * R * 2);
    const mlqmc::Est e = mlqmc::finalize(L, R, reuse != 0, N, s);
    *Q = e.Q;
    *varQ = e.varQ;
    for (int t = 0; t <= L; ++t) {
        if (Ybar) Ybar[t] = e.Ybar[t];
        if (Vell) Vell[t] = e.V[t];
    }
    return MLQMC_OK;
}
