/*
 * Oracle for the multigrid multilevel (quasi-)Monte Carlo method with sample
 * recycling (Robbe, Nuyens, Vandewalle, "Recycling samples in the multigrid
 * multilevel (quasi-)Monte Carlo method", arXiv 1806.05619).
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, serial FP64 CPU
 * restatement of the method, written to be checked against the paper by eye.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline /
 * reference arm may load it. The GPU library shares no code with it.
 *
 * Every function names the passage of the paper it follows. Where the paper
 * is silent the reading used is stated in the comment (the design document
 * lists the same readings, A1..A24).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (FMA contraction is off so
 * that x86 and Arm hosts give the same bits).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_EXHAUSTED 4
#define OR_ERR_NOT_CONVERGED 5
#define OR_ERR_OOM 3

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11). */
/* Ten rounds of two 32x32->64 multiplies; the key is bumped by the Weyl      */
/* constants between rounds.                                                 */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 64 random bits for coordinate j from one Philox block (two coordinates per block). */
static uint64_t philox_u64(uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed, int j)
{
    uint32_t ctr[4] = {(uint32_t)(j >> 1), c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    if ((j & 1) == 0) return ((uint64_t)o[1] << 32) | o[0];
    return ((uint64_t)o[3] << 32) | o[2];
}

/* 53-bit midpoint map of 64 random bits into the open interval (0,1) (reading A12). */
double or_u64_to_unit(uint64_t x)
{
    return ((double)(x >> 11) + 0.5) * 0x1.0p-53;
}

/* ------------------------------------------------------------------------- */
/* Inverse standard normal CDF, Wichura's algorithm AS 241 (PPND16),          */
/* Applied Statistics 37 (1988) 477-484: rational approximations on the      */
/* central region |p-1/2| <= 0.425 and on two tail regions in r=sqrt(-ln q). */
/* The paper maps lattice points to normals through this function (Sec. 3.2) */
/* ------------------------------------------------------------------------- */
double or_ppnd16(double p)
{
    const double q = p - 0.5;
    if (fabs(q) <= 0.425) {
        const double r = 0.180625 - q * q;
        const double num =
            (((((((2.5090809287301226727e+3 * r + 3.3430575583588128105e+4) * r +
                  6.7265770927008700853e+4) * r + 4.5921953931549871457e+4) * r +
                1.3731693765509461125e+4) * r + 1.9715909503065514427e+3) * r +
              1.3314166789178437745e+2) * r + 3.3871328727963666080e+0);
        const double den =
            (((((((5.2264952788528545610e+3 * r + 2.8729085735721942674e+4) * r +
                  3.9307895800092710610e+4) * r + 2.1213794301586595867e+4) * r +
                5.3941960214247511077e+3) * r + 6.8718700749205790830e+2) * r +
              4.2313330701600911252e+1) * r + 1.0);
        return q * num / den;
    }
    double r = (q < 0.0) ? p : 1.0 - p;
    if (r <= 0.0) return (q < 0.0) ? -INFINITY : INFINITY;
    r = sqrt(-log(r));
    double val;
    if (r <= 5.0) {
        r -= 1.6;
        const double num =
            (((((((7.74545014278341407640e-4 * r + 2.27238449892691845833e-2) * r +
                  2.41780725177450611770e-1) * r + 1.27045825245236838258e+0) * r +
                3.64784832476320460504e+0) * r + 5.76949722146069140550e+0) * r +
              4.63033784615654529590e+0) * r + 1.42343711074968357734e+0);
        const double den =
            (((((((1.05075007164441684324e-9 * r + 5.47593808499534494600e-4) * r +
                  1.51986665636164571966e-2) * r + 1.48103976427480074590e-1) * r +
                6.89767334985100004550e-1) * r + 1.67638483018380384940e+0) * r +
              2.05319162663775882187e+0) * r + 1.0);
        val = num / den;
    } else {
        r -= 5.0;
        const double num =
            (((((((2.01033439929228813265e-7 * r + 2.71155556874348757815e-5) * r +
                  1.24266094738807843860e-3) * r + 2.65321895265761230930e-2) * r +
                2.96560571828504891230e-1) * r + 1.78482653991729133580e+0) * r +
              5.46378491116411436990e+0) * r + 6.65790464350110377720e+0);
        const double den =
            (((((((2.04426310338993978564e-15 * r + 1.42151175831644588870e-7) * r +
                  1.84631831751005468180e-5) * r + 7.86869131145613259100e-4) * r +
                1.48753612908506148525e-2) * r + 1.36929880922735805310e-1) * r +
              5.99832206555887937690e-1) * r + 1.0);
        val = num / den;
    }
    return (q < 0.0) ? -val : val;
}

/* ------------------------------------------------------------------------- */
/* Karhunen-Loeve eigenpairs of the 1D exponential kernel exp(-|x-x'|/lambda) */
/* on [0,1] (eq. inteq, Sec. 5, solved in closed form).                      */
/* With c = 1/lambda the k-th eigenvalue is theta_k = 2c/(w_k^2 + c^2) where */
/* w_k is the root of g(w) = (w^2 - c^2) sin w - 2 c w cos w in (k pi,       */
/* (k+1) pi), and psi_k(x) = (w_k cos w_k x + c sin w_k x)/sqrt(N_k).        */
/* ------------------------------------------------------------------------- */
static double kl_g(double w, double c)
{
    return (w * w - c * c) * sin(w) - 2.0 * c * w * cos(w);
}

int or_kl1d(double corr_len, int K, double* omega, double* theta, double* norm)
{
    if (!(corr_len > 0.0) || K <= 0) return OR_ERR_ARG;
    const double c = 1.0 / corr_len;
    for (int k = 0; k < K; ++k) {
        double lo = k * M_PI, hi = (k + 1) * M_PI;
        if (k == 0) lo = 1e-300; /* w=0 is the trivial root; g<0 just right of it */
        double glo = kl_g(lo, c);
        /* plain bisection to the last bit */
        for (int it = 0; it < 2000; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            double gm = kl_g(mid, c);
            if ((gm < 0.0) == (glo < 0.0)) {
                lo = mid;
                glo = gm;
            } else {
                hi = mid;
            }
        }
        const double w = 0.5 * (lo + hi);
        omega[k] = w;
        theta[k] = 2.0 * c / (w * w + c * c);
        norm[k] = 0.5 * (w * w + c * c) + (w * w - c * c) * sin(2.0 * w) / (4.0 * w) +
                  c * sin(w) * sin(w);
    }
    return OR_OK;
}

double or_psi1d(double w, double c, double nrm, double x)
{
    return (w * cos(w * x) + c * sin(w * x)) / sqrt(nrm);
}

/* ------------------------------------------------------------------------- */
/* 2D modes of the separable kernel: theta_ab = sigma^2 theta_a theta_b,     */
/* psi_ab(x) = psi_a(x1) psi_b(x2); keep the s largest (truncated KL,        */
/* eq. truncatedKL). Order: theta rounded to 40 mantissa bits, descending,   */
/* then a, then b (reading A19).                                             */
/* ------------------------------------------------------------------------- */
typedef struct {
    double key;
    double theta;
    int a, b;
} or_mode_t;

static double round40(double v)
{
    int e;
    double m = frexp(v, &e);
    m = nearbyint(ldexp(m, 40));
    return ldexp(m, e - 40);
}

static int mode_cmp(const void* pa, const void* pb)
{
    const or_mode_t* x = (const or_mode_t*)pa;
    const or_mode_t* y = (const or_mode_t*)pb;
    if (x->key > y->key) return -1;
    if (x->key < y->key) return 1;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return 0;
}

int or_modes(double corr_len, double sigma, int s, int* a_out, int* b_out, double* theta_out)
{
    if (s <= 0) return OR_ERR_ARG;
    const int K = s;
    double* w = malloc(sizeof(double) * K);
    double* th = malloc(sizeof(double) * K);
    double* nr = malloc(sizeof(double) * K);
    or_mode_t* all = malloc(sizeof(or_mode_t) * (size_t)K * K);
    if (!w || !th || !nr || !all) {
        free(w); free(th); free(nr); free(all);
        return OR_ERR_OOM;
    }
    or_kl1d(corr_len, K, w, th, nr);
    size_t cnt = 0;
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) {
            double t = sigma * sigma * th[a] * th[b];
            all[cnt].key = round40(t);
            all[cnt].theta = t;
            all[cnt].a = a;
            all[cnt].b = b;
            ++cnt;
        }
    qsort(all, cnt, sizeof(or_mode_t), mode_cmp);
    for (int m = 0; m < s; ++m) {
        a_out[m] = all[m].a;
        b_out[m] = all[m].b;
        theta_out[m] = all[m].theta;
    }
    free(w); free(th); free(nr); free(all);
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Rank-1 lattice sequence with random shifts (Sec. 3.2, lattice rule        */
/* t = {n z / N}, shifted points {n z/N + Delta_l^(r)}, lattice sequence of  */
/* Sec. 6 "QMC method"). Sequence order is the radical inverse phi_2(n), so  */
/* the first 2^m points are the 2^m-point rule (reading A11). Arithmetic is  */
/* integer: x = ((bitrev32(n) z mod 2^32) << 32) + S  (mod 2^64).            */
/* ------------------------------------------------------------------------- */
uint32_t or_bitrev32(uint32_t v)
{
    uint32_t r = 0;
    for (int i = 0; i < 32; ++i) {
        r = (r << 1) | (v & 1u);
        v >>= 1;
    }
    return r;
}

/* Shift of level l, shift r, coordinate j: 64 bits from Philox(seed; j/2, r, l, "SHFT"). */
uint64_t or_shift_bits(uint64_t seed, int level, int r, int j)
{
    return philox_u64((uint32_t)r, (uint32_t)level, 0x53484654u, seed, j);
}

uint64_t or_lattice_bits(uint32_t z, uint64_t n, uint64_t shift)
{
    uint32_t t = or_bitrev32((uint32_t)n) * z; /* mod 2^32 */
    return ((uint64_t)t << 32) + shift;       /* mod 2^64 */
}

/* MC coordinate j of sample n, shift (replicate) r, level l (reading A20). */
uint64_t or_mc_bits(uint64_t seed, int level, int r, uint64_t n, int j)
{
    return philox_u64((uint32_t)n, ((uint32_t)r << 8) | (uint32_t)level, 0x4D43524Eu, seed, j);
}

/* ------------------------------------------------------------------------- */
/* Problem description and derived tables.                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n_levels;    /* L+1 */
    int n0;          /* cells per side on level 0 */
    int s;           /* KL modes */
    double sigma, corr_len;
    int qoi;         /* 0: mean of the four centre cells, 1: mean of u over D */
    int mu0, nu1, nu2;
    double rtol;     /* 0: fixed cycle count; >0: each level to ||b-Au||/||b|| <= rtol */
    int max_cycles;  /* cap on correction steps beyond the first in the converged form */
    int sampler;     /* 0: Monte Carlo (Philox), 1: shifted lattice sequence */
    uint64_t seed;
    int R;           /* shifts (or MC replicates) */
    const uint32_t* z;
    int log2_nmax;
    int reuse;       /* 1: MG-ML(Q)MC, 0: ML(Q)MC */
} or_problem;

typedef struct {
    or_problem p;
    uint32_t* z;
    int* ma;
    int* mb;
    double* mtheta;
    double* w1;
    double* nrm1;
    int K1;
} or_ctx;

void or_ctx_free(or_ctx* c)
{
    if (!c) return;
    free(c->z); free(c->ma); free(c->mb); free(c->mtheta); free(c->w1); free(c->nrm1);
    free(c);
}

or_ctx* or_ctx_new(const or_problem* p)
{
    if (!p || p->n_levels < 1 || p->n0 < 2 || (p->n0 & 1) || p->s < 1 || p->R < 1) return NULL;
    or_ctx* c = calloc(1, sizeof(or_ctx));
    if (!c) return NULL;
    c->p = *p;
    c->ma = malloc(sizeof(int) * p->s);
    c->mb = malloc(sizeof(int) * p->s);
    c->mtheta = malloc(sizeof(double) * p->s);
    if (!c->ma || !c->mb || !c->mtheta) { or_ctx_free(c); return NULL; }
    if (or_modes(p->corr_len, p->sigma, p->s, c->ma, c->mb, c->mtheta) != OR_OK) {
        or_ctx_free(c);
        return NULL;
    }
    int K1 = 0;
    for (int m = 0; m < p->s; ++m) {
        if (c->ma[m] + 1 > K1) K1 = c->ma[m] + 1;
        if (c->mb[m] + 1 > K1) K1 = c->mb[m] + 1;
    }
    c->K1 = K1;
    c->w1 = malloc(sizeof(double) * K1);
    c->nrm1 = malloc(sizeof(double) * K1);
    double* th = malloc(sizeof(double) * K1);
    if (!c->w1 || !c->nrm1 || !th) { free(th); or_ctx_free(c); return NULL; }
    or_kl1d(p->corr_len, K1, c->w1, th, c->nrm1);
    free(th);
    if (p->sampler == 1) {
        if (!p->z || p->log2_nmax < 0 || p->log2_nmax > 32) { or_ctx_free(c); return NULL; }
        c->z = malloc(sizeof(uint32_t) * p->s);
        if (!c->z) { or_ctx_free(c); return NULL; }
        memcpy(c->z, p->z, sizeof(uint32_t) * p->s);
    }
    c->p.z = c->z;
    return c;
}

int or_ctx_modes(const or_ctx* c, int* a, int* b, double* theta)
{
    for (int m = 0; m < c->p.s; ++m) {
        a[m] = c->ma[m];
        b[m] = c->mb[m];
        theta[m] = c->mtheta[m];
    }
    return c->K1;
}

/* Standard normals y_{l,r}^{(n)} (Sec. 3.2: y = Phi^{-1}(t); MC: i.i.d. N(0,1)). */
int or_normals(const or_ctx* c, int level, int r, uint64_t n, double* y)
{
    const or_problem* p = &c->p;
    if (p->sampler == 1) {
        if (p->log2_nmax < 32 && n >= ((uint64_t)1 << p->log2_nmax)) return OR_ERR_EXHAUSTED;
        for (int j = 0; j < p->s; ++j) {
            uint64_t x = or_lattice_bits(c->z[j], n, or_shift_bits(p->seed, level, r, j));
            y[j] = or_ppnd16(or_u64_to_unit(x));
        }
    } else {
        if (n >= ((uint64_t)1 << 32)) return OR_ERR_EXHAUSTED;
        for (int j = 0; j < p->s; ++j)
            y[j] = or_ppnd16(or_u64_to_unit(or_mc_bits(p->seed, level, r, n, j)));
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Lognormal KL field on one level (eq. truncatedKL, a = exp(z), Sec. 5):     */
/* z(x) = sum_m y_m sqrt(theta_m) psi_m(x) evaluated at the cell centres     */
/* ((i1+1/2)h, (i2+1/2)h) of that level's own grid (reading A3).             */
/* Layout: k[i2*n + i1], i1 along x1.                                        */
/* ------------------------------------------------------------------------- */
/* Z(x) = sum_m sqrt(theta_m) y_m psi_{a_m}(x1) psi_{b_m}(x2) at the cell      */
/* centres of an n x n grid (eq. truncatedKL with the separable modes). Each  */
/* 1D factor psi_a((i + 1/2)/n) is evaluated once per coordinate and looked   */
/* up; the terms are the same products, added in mode order.                  */
static int field_sum(const or_ctx* c, int n, const double* y, double* zout)
{
    const double cc = 1.0 / c->p.corr_len;
    double* P = malloc(sizeof(double) * (size_t)c->K1 * n);  /* P[a*n + i] = psi_a((i+1/2)/n) */
    if (!P) return OR_ERR_OOM;
    for (int a = 0; a < c->K1; ++a)
        for (int i = 0; i < n; ++i) P[(size_t)a * n + i] = or_psi1d(c->w1[a], cc, c->nrm1[a], (i + 0.5) / n);
    for (int i2 = 0; i2 < n; ++i2) {
        for (int i1 = 0; i1 < n; ++i1) {
            double z = 0.0;
            for (int m = 0; m < c->p.s; ++m)
                z += y[m] * sqrt(c->mtheta[m]) * P[(size_t)c->ma[m] * n + i1] * P[(size_t)c->mb[m] * n + i2];
            zout[i2 * n + i1] = z;
        }
    }
    free(P);
    return OR_OK;
}

/* Lognormal field k = exp(Z) (Sec. 5); NaN everywhere when out of memory. */
void or_field(const or_ctx* c, int n, const double* y, double* k)
{
    if (field_sum(c, n, y, k) != OR_OK) {
        for (size_t p = 0; p < (size_t)n * n; ++p) k[p] = NAN;
        return;
    }
    for (size_t p = 0; p < (size_t)n * n; ++p) k[p] = exp(k[p]);
}

/* Gaussian part only (same sum without the exponential). */
void or_field_z(const or_ctx* c, int n, const double* y, double* zout)
{
    if (field_sum(c, n, y, zout) != OR_OK)
        for (size_t p = 0; p < (size_t)n * n; ++p) zout[p] = NAN;
}

/* ------------------------------------------------------------------------- */
/* Cell-centred finite-volume operator for -div(k grad u) = f on (0,1)^2     */
/* with u = 0 on the boundary (eq. PDE; readings A1, A2):                    */
/* (Au)_P = h^-2 [ sum_{interior Q} k_PQ (u_P - u_Q) + sum_{boundary} 2k_P u_P ] */
/* with the harmonic mean k_PQ = 2 k_P k_Q / (k_P + k_Q).                     */
/* ------------------------------------------------------------------------- */
static double hmean(double kp, double kq)
{
    return 2.0 * kp * kq / (kp + kq);
}

void or_apply_A(int n, const double* k, const double* u, double* Au)
{
    const double ih2 = (double)n * (double)n;
    for (int i2 = 0; i2 < n; ++i2)
        for (int i1 = 0; i1 < n; ++i1) {
            const int p = i2 * n + i1;
            const double kp = k[p], up = u[p];
            double acc = 0.0;
            if (i1 > 0) acc += hmean(kp, k[p - 1]) * (up - u[p - 1]); else acc += 2.0 * kp * up;
            if (i1 < n - 1) acc += hmean(kp, k[p + 1]) * (up - u[p + 1]); else acc += 2.0 * kp * up;
            if (i2 > 0) acc += hmean(kp, k[p - n]) * (up - u[p - n]); else acc += 2.0 * kp * up;
            if (i2 < n - 1) acc += hmean(kp, k[p + n]) * (up - u[p + n]); else acc += 2.0 * kp * up;
            Au[p] = ih2 * acc;
        }
}

/* One Gauss-Seidel relaxation of the cells of one colour (red: i1+i2 even). */
static void gs_colour(int n, const double* k, const double* b, double* u, int colour)
{
    const double h2 = 1.0 / ((double)n * (double)n);
    for (int i2 = 0; i2 < n; ++i2)
        for (int i1 = 0; i1 < n; ++i1) {
            if (((i1 + i2) & 1) != colour) continue;
            const int p = i2 * n + i1;
            const double kp = k[p];
            double diag = 0.0, off = 0.0, kf;
            if (i1 > 0) { kf = hmean(kp, k[p - 1]); diag += kf; off += kf * u[p - 1]; } else diag += 2.0 * kp;
            if (i1 < n - 1) { kf = hmean(kp, k[p + 1]); diag += kf; off += kf * u[p + 1]; } else diag += 2.0 * kp;
            if (i2 > 0) { kf = hmean(kp, k[p - n]); diag += kf; off += kf * u[p - n]; } else diag += 2.0 * kp;
            if (i2 < n - 1) { kf = hmean(kp, k[p + n]); diag += kf; off += kf * u[p + n]; } else diag += 2.0 * kp;
            u[p] = (h2 * b[p] + off) / diag;
        }
}

/* Restriction: coarse value = mean of the four children (reading A4). */
static void restrict_mean(int nc, const double* fine, double* coarse)
{
    const int nf = 2 * nc;
    for (int I2 = 0; I2 < nc; ++I2)
        for (int I1 = 0; I1 < nc; ++I1) {
            const int f = (2 * I2) * nf + 2 * I1;
            coarse[I2 * nc + I1] = 0.25 * (fine[f] + fine[f + 1] + fine[f + nf] + fine[f + nf + 1]);
        }
}

/* Coarse value with odd reflection across the Dirichlet boundary (reading A4). */
static double coarse_ghost(int nc, const double* e, int I1, int I2)
{
    double sign = 1.0;
    if (I1 < 0) { I1 = 0; sign = -sign; }
    if (I1 >= nc) { I1 = nc - 1; sign = -sign; }
    if (I2 < 0) { I2 = 0; sign = -sign; }
    if (I2 >= nc) { I2 = nc - 1; sign = -sign; }
    return sign * e[I2 * nc + I1];
}

/* Bilinear cell-centred prolongation, weights 9/16, 3/16, 3/16, 1/16; adds into fine. */
static void prolong_add(int nc, const double* e, double* fine)
{
    const int nf = 2 * nc;
    for (int i2 = 0; i2 < nf; ++i2)
        for (int i1 = 0; i1 < nf; ++i1) {
            const int I1 = i1 >> 1, I2 = i2 >> 1;
            const int s1 = (i1 & 1) ? 1 : -1, s2 = (i2 & 1) ? 1 : -1;
            const double v = 9.0 * coarse_ghost(nc, e, I1, I2) +
                             3.0 * coarse_ghost(nc, e, I1 + s1, I2) +
                             3.0 * coarse_ghost(nc, e, I1, I2 + s2) +
                             1.0 * coarse_ghost(nc, e, I1 + s1, I2 + s2);
            fine[i2 * nf + i1] += v / 16.0;
        }
}

/* The prolongation above on its own (tests): fine (2nc x 2nc) += P e. */
void or_prolong_add(int nc, const double* e, double* fine)
{
    prolong_add(nc, e, fine);
}

/* Dense Cholesky of the level-0 matrix (reading A5: exact coarsest solve). */
static int chol_factor(int n, const double* k, double* Lm)
{
    const int N = n * n;
    double* e = calloc(N, sizeof(double));
    double* col = malloc(sizeof(double) * N);
    if (!e || !col) { free(e); free(col); return OR_ERR_OOM; }
    /* assemble column by column: A e_q */
    for (int q = 0; q < N; ++q) {
        e[q] = 1.0;
        or_apply_A(n, k, e, col);
        for (int p = 0; p < N; ++p) Lm[p * N + q] = col[p];
        e[q] = 0.0;
    }
    free(e); free(col);
    for (int j = 0; j < N; ++j) {
        double d = Lm[j * N + j];
        for (int t = 0; t < j; ++t) d -= Lm[j * N + t] * Lm[j * N + t];
        if (!(d > 0.0)) return OR_ERR_ARG;
        d = sqrt(d);
        Lm[j * N + j] = d;
        for (int i = j + 1; i < N; ++i) {
            double v = Lm[i * N + j];
            for (int t = 0; t < j; ++t) v -= Lm[i * N + t] * Lm[j * N + t];
            Lm[i * N + j] = v / d;
        }
    }
    return OR_OK;
}

static void chol_solve(int N, const double* Lm, const double* b, double* x)
{
    for (int i = 0; i < N; ++i) {
        double v = b[i];
        for (int t = 0; t < i; ++t) v -= Lm[i * N + t] * x[t];
        x[i] = v / Lm[i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {
        double v = x[i];
        for (int t = i + 1; t < N; ++t) v -= Lm[t * N + i] * x[t];
        x[i] = v / Lm[i * N + i];
    }
}

/* ------------------------------------------------------------------------- */
/* Full multigrid (Sec. 4, Fig. FMG).                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    int L;          /* finest level of this solve */
    int n0, nu1, nu2;
    double** k;     /* per level coefficient */
    double** b;     /* per level right-hand side of the current cycle */
    double** u;     /* per level iterate */
    double** tmp;   /* per level scratch */
    double* chol;   /* level-0 factor */
    int* log;       /* optional visit log */
    int log_len, log_cap;
} or_mg;

static int nlev(const or_mg* g, int t) { return g->n0 << t; }

static void mg_log(or_mg* g, int t)
{
    if (g->log && g->log_len < g->log_cap) g->log[g->log_len] = t;
    g->log_len++;
}

/* Correction scheme of Sec. 4 (steps 1-6) applied recursively: a V-cycle. */
static void vcycle(or_mg* g, int t, double* u, const double* b)
{
    mg_log(g, t);
    const int n = nlev(g, t);
    if (t == 0) {
        chol_solve(n * n, g->chol, b, u);
        return;
    }
    for (int s = 0; s < g->nu1; ++s) {
        gs_colour(n, g->k[t], b, u, 0);
        gs_colour(n, g->k[t], b, u, 1);
    }
    double* r = g->tmp[t];
    or_apply_A(n, g->k[t], u, r);
    for (int p = 0; p < n * n; ++p) r[p] = b[p] - r[p];
    const int nc = n / 2;
    double* bc = g->b[t - 1];
    double* ec = g->u[t - 1];
    restrict_mean(nc, r, bc);
    for (int p = 0; p < nc * nc; ++p) ec[p] = 0.0;
    vcycle(g, t - 1, ec, bc);
    prolong_add(nc, ec, u);
    for (int s = 0; s < g->nu2; ++s) {
        gs_colour(n, g->k[t], b, u, 1);
        gs_colour(n, g->k[t], b, u, 0);
    }
    mg_log(g, t);
}

static double qoi_value(int qoi, int n, const double* u)
{
    if (qoi == 1) {
        double s = 0.0;
        for (int p = 0; p < n * n; ++p) s += u[p];
        return s / ((double)n * (double)n);
    }
    const int m = n / 2;
    return 0.25 * (u[(m - 1) * n + (m - 1)] + u[(m - 1) * n + m] + u[m * n + (m - 1)] + u[m * n + m]);
}

/*
 * FMG for one sample whose finest level is L. Fields k[t] must be filled for
 * t = 0..L. The right-hand side is f on the finest grid restricted down the
 * hierarchy (the descent of Fig. FMG); then level 0 is solved exactly and each
 * level t = 1..L starts from the prolongated solution of level t-1 and runs mu0
 * V-cycles (and, in the converged form, further V-cycles until the relative
 * residual is below rtol). F_t is taken from the solution that ends each level
 * (the encircled nodes of Fig. FMG).
 * usol (optional): per-level copies of the final solutions, concatenated.
 */
static int fmg_solve(const or_ctx* c, or_mg* g, const double* rhs, double* F, double* usol,
                     int* cycles_out)
{
    const or_problem* p = &c->p;
    const int L = g->L;
    int status = OR_OK;
    double** bl = calloc(L + 1, sizeof(double*));
    double** ul = calloc(L + 1, sizeof(double*));
    if (!bl || !ul) { free(bl); free(ul); return OR_ERR_OOM; }
    for (int t = 0; t <= L; ++t) {
        const size_t n = (size_t)nlev(g, t);
        bl[t] = malloc(sizeof(double) * n * n);
        ul[t] = calloc(n * n, sizeof(double));
        if (!bl[t] || !ul[t]) { status = OR_ERR_OOM; goto done; }
    }
    /* descent of Fig. FMG: f on the finest grid (f = 1 unless given), restricted down */
    {
        const size_t n = (size_t)nlev(g, L);
        for (size_t q = 0; q < n * n; ++q) bl[L][q] = rhs ? rhs[q] : 1.0;
        for (int t = L; t >= 0; --t) {
            mg_log(g, t);
            if (t > 0) restrict_mean(nlev(g, t - 1), bl[t], bl[t - 1]);
        }
    }
    status = chol_factor(g->n0, g->k[0], g->chol);
    if (status != OR_OK) goto done;
    /* level 0: exact solve (the first encircled node) */
    chol_solve(g->n0 * g->n0, g->chol, bl[0], ul[0]);
    F[0] = qoi_value(p->qoi, g->n0, ul[0]);
    size_t off = 0;
    if (usol) memcpy(usol, ul[0], sizeof(double) * g->n0 * g->n0);
    off = (size_t)g->n0 * g->n0;
    for (int t = 1; t <= L; ++t) {
        const int n = nlev(g, t);
        prolong_add(n / 2, ul[t - 1], ul[t]); /* FMG interpolation: u_t = P u_{t-1} */
        int cyc = 0;
        if (p->rtol > 0.0) {
            /* converged form (reading A21): defect correction. r = b - A u, mu0
             * V-cycles on A e = r from e = 0, u += e, until ||r|| <= rtol ||b||;
             * the first step equals mu0 V-cycles on u. */
            const size_t nn = (size_t)n * n;
            double* r = malloc(sizeof(double) * nn);
            double* e = malloc(sizeof(double) * nn);
            for (int it = 0;; ++it) {
                or_apply_A(n, g->k[t], ul[t], r);
                double rr = 0.0, bb = 0.0;
                for (size_t q = 0; q < nn; ++q) {
                    r[q] = bl[t][q] - r[q];
                    rr += r[q] * r[q];
                    bb += bl[t][q] * bl[t][q];
                }
                if (it > 0 && sqrt(rr) <= p->rtol * sqrt(bb)) break;
                if (it > p->max_cycles) { status = OR_ERR_NOT_CONVERGED; break; }
                for (size_t q = 0; q < nn; ++q) e[q] = 0.0;
                for (int q = 0; q < p->mu0; ++q) {
                    vcycle(g, t, e, r);
                    ++cyc;
                }
                for (size_t q = 0; q < nn; ++q) ul[t][q] += e[q];
            }
            free(r);
            free(e);
        } else {
            for (int q = 0; q < p->mu0; ++q) {
                vcycle(g, t, ul[t], bl[t]);
                ++cyc;
            }
        }
        if (cycles_out) cycles_out[t] = cyc;
        F[t] = qoi_value(p->qoi, n, ul[t]);
        if (usol) memcpy(usol + off, ul[t], sizeof(double) * n * n);
        off += (size_t)n * n;
        if (status != OR_OK) break;
    }
done:
    for (int t = 0; t <= L; ++t) { free(bl[t]); free(ul[t]); }
    free(bl);
    free(ul);
    return status;
}

static or_mg* mg_new(int n0, int L, int nu1, int nu2)
{
    or_mg* g = calloc(1, sizeof(or_mg));
    g->L = L; g->n0 = n0; g->nu1 = nu1; g->nu2 = nu2;
    g->k = calloc(L + 1, sizeof(double*));
    g->b = calloc(L + 1, sizeof(double*));
    g->u = calloc(L + 1, sizeof(double*));
    g->tmp = calloc(L + 1, sizeof(double*));
    for (int t = 0; t <= L; ++t) {
        const size_t n = (size_t)(n0 << t);
        g->k[t] = calloc(n * n, sizeof(double));
        g->b[t] = calloc(n * n, sizeof(double));
        g->u[t] = calloc(n * n, sizeof(double));
        g->tmp[t] = calloc(n * n, sizeof(double));
    }
    g->chol = calloc((size_t)n0 * n0 * n0 * n0, sizeof(double));
    return g;
}

static void mg_free(or_mg* g)
{
    if (!g) return;
    for (int t = 0; t <= g->L; ++t) { free(g->k[t]); free(g->b[t]); free(g->u[t]); free(g->tmp[t]); }
    free(g->k); free(g->b); free(g->u); free(g->tmp); free(g->chol);
    free(g);
}

/*
 * One sample: normals, fields on every level t <= L, FMG, F_0..F_L
 * (SampleAndSolve body of Algorithm 1).
 * usol: optional, concatenated solutions of levels 0..L.
 * log/log_cap: optional visit log (Fig. FMG); returns the log length in *log_len.
 */
int or_sample(const or_ctx* c, int L, int r, uint64_t n, double* F, double* usol,
              int* log, int log_cap, int* log_len, int* cycles)
{
    const or_problem* p = &c->p;
    if (L < 0 || L >= p->n_levels) return OR_ERR_ARG;
    double* y = malloc(sizeof(double) * p->s);
    int st = or_normals(c, L, r, n, y);
    if (st != OR_OK) { free(y); return st; }
    or_mg* g = mg_new(p->n0, L, p->nu1, p->nu2);
    g->log = log; g->log_cap = log_cap; g->log_len = 0;
    for (int t = 0; t <= L; ++t) or_field(c, p->n0 << t, y, g->k[t]);
    st = fmg_solve(c, g, NULL, F, usol, cycles);
    if (log_len) *log_len = g->log_len;
    mg_free(g);
    free(y);
    return st;
}

/* FMG on explicitly given coefficient fields (tests: manufactured and direct-solve checks).
 * k_all: concatenated k of levels 0..L; rhs: finest-level right-hand side (NULL: f = 1). */
int or_fmg_fields(const or_ctx* c, int L, const double* k_all, const double* rhs, double* F,
                  double* usol, int* cycles)
{
    const or_problem* p = &c->p;
    or_mg* g = mg_new(p->n0, L, p->nu1, p->nu2);
    size_t off = 0;
    for (int t = 0; t <= L; ++t) {
        const size_t n = (size_t)(p->n0 << t);
        memcpy(g->k[t], k_all + off, sizeof(double) * n * n);
        off += n * n;
    }
    int st = fmg_solve(c, g, rhs, F, usol, cycles);
    mg_free(g);
    return st;
}

/* One V-cycle on level t of given fields from a given iterate (contraction tests). */
int or_vcycle_fields(const or_ctx* c, int t, const double* k_all, const double* b, double* u)
{
    const or_problem* p = &c->p;
    or_mg* g = mg_new(p->n0, t, p->nu1, p->nu2);
    size_t off = 0;
    for (int q = 0; q <= t; ++q) {
        const size_t n = (size_t)(p->n0 << q);
        memcpy(g->k[q], k_all + off, sizeof(double) * n * n);
        off += n * n;
    }
    int st = chol_factor(p->n0, g->k[0], g->chol);
    if (st == OR_OK) vcycle(g, t, u, b);
    mg_free(g);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Estimator sums (eq. MLMC / eq. MGMLMC, with shifts: eq. Upsilon-reuse).   */
/* sums[(t*R + r)*2 + 0] += dF_t, [..+1] += dF_t^2 for every sample of level */
/* k >= t (reuse) or k == t (no reuse), dF_t = F_t - F_{t-1}, F_{-1} = 0.     */
/* A work item is (level, n_begin, n_end, r_begin, r_end).                   */
/* F_out (optional): per sample, in work order (item, r, n), n_levels values */
/* (F_0..F_level, rest zero).                                                */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t level;
    int32_t pad;
    int64_t n_begin, n_end;
    int32_t r_begin, r_end;
} or_work;

int or_sample_levels(const or_ctx* c, const or_work* w, int n_work, double* sums, double* F_out)
{
    const or_problem* p = &c->p;
    double* F = malloc(sizeof(double) * p->n_levels);
    size_t idx = 0;
    int st = OR_OK;
    for (int it = 0; it < n_work && st == OR_OK; ++it) {
        const int L = w[it].level;
        for (int r = w[it].r_begin; r < w[it].r_end && st == OR_OK; ++r) {
            for (int64_t n = w[it].n_begin; n < w[it].n_end; ++n) {
                st = or_sample(c, L, r, (uint64_t)n, F, NULL, NULL, 0, NULL, NULL);
                if (st != OR_OK) break;
                for (int t = 0; t <= L; ++t) {
                    if (!p->reuse && t != L) continue;
                    const double d = F[t] - (t > 0 ? F[t - 1] : 0.0);
                    sums[((size_t)t * p->R + r) * 2 + 0] += d;
                    sums[((size_t)t * p->R + r) * 2 + 1] += d * d;
                }
                if (F_out) {
                    for (int t = 0; t < p->n_levels; ++t)
                        F_out[idx * p->n_levels + t] = (t <= L) ? F[t] : 0.0;
                }
                ++idx;
            }
        }
    }
    free(F);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Estimates from the sums (eqs. Upsilon-reuse, MGMLQMC, var_of_mgmlqmc,     */
/* Upsilon-reuse-bar, sample_variances). N[l] = samples whose FMG ends at    */
/* level l (reading A9). Levels 0..L are used.                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    double Q, varQ, bias, alpha;
    int L, rounds, status, alpha_clamped;
    double Ybar[32], Vell[32], C[32];
    int64_t N[32];
} or_result;

void or_finalize(int L, int R, int reuse, const int64_t* N, const double* sums,
                 double* Ups /* [L+1][R] */, double* Ybar, double* Vell, double* Q, double* varQ)
{
    double* Qr = calloc(R, sizeof(double));
    for (int t = 0; t <= L; ++t) {
        int64_t cnt = 0;
        if (reuse) { for (int i = t; i <= L; ++i) cnt += N[i]; }
        else cnt = N[t];
        double mean = 0.0;
        for (int r = 0; r < R; ++r) {
            const double y = cnt > 0 ? sums[((size_t)t * R + r) * 2] / (double)cnt : 0.0;
            Ups[t * R + r] = y;
            Qr[r] += y;
            mean += y;
        }
        mean /= R;
        Ybar[t] = mean;
        double v = 0.0;
        for (int r = 0; r < R; ++r) v += (Ups[t * R + r] - mean) * (Ups[t * R + r] - mean);
        Vell[t] = R > 1 ? v / ((double)R * (R - 1)) : INFINITY;
    }
    double qm = 0.0;
    for (int r = 0; r < R; ++r) qm += Qr[r];
    qm /= R;
    double v = 0.0;
    for (int r = 0; r < R; ++r) v += (Qr[r] - qm) * (Qr[r] - qm);
    *Q = qm;
    *varQ = R > 1 ? v / ((double)R * (R - 1)) : INFINITY;
    free(Qr);
}

/* alpha from a least-squares fit of log2|Ybar_l| on l = 1..L (reading A15). */
static double fit_alpha(int L, const double* Ybar, int* clamped)
{
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    int m = 0;
    for (int l = 1; l <= L; ++l) {
        const double y = log2(fabs(Ybar[l]));
        if (!isfinite(y)) continue;
        sx += l; sy += y; sxx += (double)l * l; sxy += l * y;
        ++m;
    }
    double alpha = NAN;
    if (m >= 2) {
        const double slope = (m * sxy - sx * sy) / (m * sxx - sx * sx);
        alpha = -slope;
    }
    *clamped = 0;
    if (!(alpha > 0.0)) { alpha = 0.5; *clamped = 1; }
    return alpha;
}

/*
 * Algorithm 1 (MG-MLQMC(eps)), in its exact one-level-per-iteration form.
 * cost_mode 0: C_l = sum_{t<=l} n_t^2, the cell count of the FMG hierarchy
 * (reading A17, parity mode). Level L may not exceed n_levels-1: reaching it
 * with the bias test still failing ends the run with status 7 (flagged).
 * An unsampled level makes the variance estimate +infinity (reading A24).
 */
int or_estimate(const or_ctx* c, double eps, int max_rounds, or_result* res)
{
    const or_problem* p = &c->p;
    const int Lmax = p->n_levels - 1;
    const int R = p->R;
    int64_t N[32] = {0}, Nold[32] = {0};
    double V[32], C[32], Ybar[32];
    double* sums = calloc((size_t)(Lmax + 1) * R * 2, sizeof(double));
    double* Ups = calloc((size_t)(Lmax + 1) * R, sizeof(double));
    for (int l = 0; l <= Lmax; ++l) { V[l] = INFINITY; C[l] = 0.0; Ybar[l] = 0.0; }
    int L = -1, rounds = 0, st = OR_OK;
    double Q = 0.0, varQ = INFINITY, bias = INFINITY, alpha = NAN;
    int clamped = 0;
    for (;;) {
        if (L >= 2) {
            alpha = fit_alpha(L, Ybar, &clamped);
            bias = fabs(Ybar[L]) / (pow(2.0, alpha) + 1.0);
            if (!(bias > eps / sqrt(2.0))) break;
        }
        if (L + 1 > Lmax) { st = 7; break; }
        L = L + 1;
        for (;;) {
            int unsampled = 0;
            for (int l = 0; l <= L; ++l) if (isinf(V[l])) unsampled = 1;
            double vq = INFINITY;
            if (!unsampled) {
                double Yb[32], Vl[32];
                or_finalize(L, R, p->reuse, N, sums, Ups, Yb, Vl, &Q, &vq);
            }
            varQ = vq;
            if (!(varQ > eps * eps / 2.0)) break;
            if (rounds >= max_rounds) { st = 8; goto out; }
            /* level with the largest V_l / C_l; an infinite ratio wins, ties -> smallest l */
            int best = 0;
            double bestv = -1.0;
            for (int l = 0; l <= L; ++l) {
                const double ratio = isinf(V[l]) ? INFINITY : V[l] / C[l];
                if (ratio > bestv) { bestv = ratio; best = l; }
            }
            const int l = best;
            N[l] = N[l] > 0 ? 2 * N[l] : 1;
            /* SampleAndSolve(l) */
            or_work w;
            w.level = l; w.pad = 0; w.n_begin = Nold[l]; w.n_end = N[l];
            w.r_begin = 0; w.r_end = R;
            st = or_sample_levels(c, &w, 1, sums, NULL);
            if (st != OR_OK) goto out;
            double cl = 0.0;
            for (int t = 0; t <= l; ++t) cl += (double)(p->n0 << t) * (double)(p->n0 << t);
            C[l] = cl;
            {
                double Yb[32], Vl[32], q, vqq;
                /* the counts of levels t <= l include every level up to L */
                or_finalize(L, R, p->reuse, N, sums, Ups, Yb, Vl, &q, &vqq);
                for (int t = 0; t <= l; ++t) { Ybar[t] = Yb[t]; V[t] = Vl[t]; }
            }
            Nold[l] = N[l];
            ++rounds;
        }
    }
out:
    if (L >= 0) {
        double Yb[32], Vl[32];
        int unsampled = 0;
        for (int l = 0; l <= L; ++l) if (isinf(V[l])) unsampled = 1;
        if (!unsampled) or_finalize(L, R, p->reuse, N, sums, Ups, Yb, Vl, &Q, &varQ);
    }
    res->Q = Q; res->varQ = varQ; res->bias = bias; res->alpha = alpha;
    res->L = L; res->rounds = rounds; res->status = st; res->alpha_clamped = clamped;
    for (int l = 0; l < 32; ++l) {
        res->Ybar[l] = l <= Lmax ? Ybar[l] : 0.0;
        res->Vell[l] = l <= Lmax ? V[l] : 0.0;
        res->C[l] = l <= Lmax ? C[l] : 0.0;
        res->N[l] = l <= Lmax ? N[l] : 0;
    }
    free(sums); free(Ups);
    return (st == 7) ? OR_OK : st;
}

/* ------------------------------------------------------------------------- */
/* Plain MLMC, the comparison baseline (Sec. 2): independent MC samples per  */
/* level, no recycling, one replicate (r = 0). MSE split (eq. MSE): variance */
/* sum V_l/N_l <= eps^2/2 (eq. vardecomp) through the counts of eq. nopt,    */
/* bias <= eps/sqrt(2) by the test of Algorithm 1 (readings A14, A15).       */
/* Reading A28: levels are added one at a time from L = 0, a new level first */
/* takes 32 samples; after each round every level below its eq. nopt count  */
/* is topped up (one round); when none is short the bias test (L >= 2)      */
/* stops the run or adds a level. V_l: sample variance (ddof 1) of          */
/* F_l - F_{l-1}; C_l: the cell count of the FMG hierarchy (reading A17).    */
/* ------------------------------------------------------------------------- */

/* eq. nopt: N_l = ceil(2/eps^2 sqrt(V_l/C_l) sum_{t<=L} sqrt(V_t C_t)). */
void or_mlmc_nopt(int L, const double* V, const double* C, double eps, double* N_out)
{
    double acc = 0.0;
    for (int t = 0; t <= L; ++t) acc += sqrt(V[t] * C[t]);
    for (int l = 0; l <= L; ++l) N_out[l] = ceil(2.0 / (eps * eps) * sqrt(V[l] / C[l]) * acc);
}

int or_estimate_mlmc(const or_ctx* c, double eps, int max_rounds, or_result* res)
{
    const or_problem* p = &c->p;
    if (p->sampler != 0 || p->reuse != 0 || !(eps > 0.0)) return OR_ERR_ARG;
    const int Lmax = p->n_levels - 1;
    const int R = p->R;
    int64_t N[32] = {0}, want[32] = {0};
    double V[32], C[32], Ybar[32], Nopt[32];
    double* sums = calloc((size_t)(Lmax + 1) * R * 2, sizeof(double));
    for (int l = 0; l <= Lmax; ++l) {
        V[l] = INFINITY;
        Ybar[l] = 0.0;
        C[l] = 0.0;
        for (int t = 0; t <= l; ++t) C[l] += (double)(p->n0 << t) * (double)(p->n0 << t);
    }
    int L = 0, rounds = 0, st = OR_OK, clamped = 0;
    double bias = INFINITY, alpha = NAN;
    want[0] = 32;
    for (;;) {
        int short_any = 0;
        for (int l = 0; l <= L; ++l) if (want[l] > N[l]) short_any = 1;
        if (short_any) {
            if (rounds >= max_rounds) { st = 8; break; }
            for (int l = 0; l <= L; ++l) {
                if (want[l] <= N[l]) continue;
                or_work w;
                w.level = l; w.pad = 0; w.n_begin = N[l]; w.n_end = want[l]; w.r_begin = 0; w.r_end = 1;
                st = or_sample_levels(c, &w, 1, sums, NULL);
                if (st != OR_OK) goto out;
                N[l] = want[l];
            }
            ++rounds;
            for (int l = 0; l <= L; ++l) {
                const double n = (double)N[l];
                const double s1 = sums[(size_t)l * R * 2], s2 = sums[(size_t)l * R * 2 + 1];
                Ybar[l] = s1 / n;
                V[l] = N[l] > 1 ? (s2 - s1 * s1 / n) / (n - 1.0) : INFINITY;
            }
            or_mlmc_nopt(L, V, C, eps, Nopt);
            for (int l = 0; l <= L; ++l) {
                const int64_t n = (int64_t)(Nopt[l] < 9.0e18 ? Nopt[l] : 9.0e18);
                want[l] = n > N[l] ? n : N[l];
            }
            continue;
        }
        if (L >= 2) {
            alpha = fit_alpha(L, Ybar, &clamped);
            bias = fabs(Ybar[L]) / (pow(2.0, alpha) + 1.0);
            if (!(bias > eps / sqrt(2.0))) break;
        }
        if (L + 1 > Lmax) { st = 7; break; }
        L = L + 1;
        want[L] = 32;
    }
out:
    {
        double Q = 0.0, varQ = 0.0;
        for (int l = 0; l <= L; ++l) {
            Q += Ybar[l];
            varQ += N[l] > 0 ? V[l] / (double)N[l] : INFINITY;
        }
        res->Q = Q; res->varQ = varQ;
    }
    res->bias = bias; res->alpha = alpha;
    res->L = L; res->rounds = rounds; res->status = st; res->alpha_clamped = clamped;
    for (int l = 0; l < 32; ++l) {
        res->Ybar[l] = l <= Lmax ? Ybar[l] : 0.0;
        res->Vell[l] = l <= Lmax ? V[l] : 0.0;
        res->C[l] = l <= Lmax ? C[l] : 0.0;
        res->N[l] = l <= Lmax ? N[l] : 0;
    }
    free(sums);
    return (st == 7 || st == 8) ? OR_OK : st;
}

/* ------------------------------------------------------------------------- */
/* Component-by-component construction of the generating vector (Sec. 3.2   */
/* cites Nuyens-Cools; reading A13). Criterion: shift-averaged worst-case    */
/* error in the unanchored weighted Sobolev space with product weights:      */
/*   e^2 = -1 + (1/N) sum_k prod_j (1 + gamma_j B2({k z_j / N})),            */
/* B2(x) = x^2 - x + 1/6. z_1 = 1; each next z_j is the odd z <= N/2 with    */
/* the smallest criterion (ties: smallest z). Naive O(s N^2) form.           */
/* e2_out[j] = criterion after j+1 components.                               */
/* ------------------------------------------------------------------------- */
static double bern2(double x) { return x * x - x + 1.0 / 6.0; }

int or_cbc(int s, int m, const double* gamma, uint32_t* z, double* e2_out)
{
    if (s < 1 || m < 1 || m > 24) return OR_ERR_ARG;
    const int64_t N = (int64_t)1 << m;
    double* P = malloc(sizeof(double) * N);
    if (!P) return OR_ERR_OOM;
    z[0] = 1;
    for (int64_t k = 0; k < N; ++k)
        P[k] = 1.0 + gamma[0] * bern2((double)(k % N) / (double)N);
    {
        double acc = 0.0;
        for (int64_t k = 0; k < N; ++k) acc += P[k];
        e2_out[0] = -1.0 + acc / (double)N;
    }
    for (int j = 1; j < s; ++j) {
        double best = INFINITY;
        int64_t bestz = 1;
        for (int64_t cand = 1; cand <= N / 2; cand += 2) {
            double acc = 0.0;
            for (int64_t k = 0; k < N; ++k) {
                const double x = (double)((k * cand) % N) / (double)N;
                acc += P[k] * (1.0 + gamma[j] * bern2(x));
            }
            if (acc < best) { best = acc; bestz = cand; }
        }
        z[j] = (uint32_t)bestz;
        for (int64_t k = 0; k < N; ++k)
            P[k] *= 1.0 + gamma[j] * bern2((double)((k * bestz) % N) / (double)N);
        double acc = 0.0;
        for (int64_t k = 0; k < N; ++k) acc += P[k];
        e2_out[j] = -1.0 + acc / (double)N;
    }
    free(P);
    return OR_OK;
}

/* Criterion of a given vector (same definition), for tests. */
double or_cbc_criterion(int s, int m, const double* gamma, const uint32_t* z)
{
    const int64_t N = (int64_t)1 << m;
    double acc = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        double prod = 1.0;
        for (int j = 0; j < s; ++j)
            prod *= 1.0 + gamma[j] * bern2((double)((k * (int64_t)z[j]) % N) / (double)N);
        acc += prod;
    }
    return -1.0 + acc / (double)N;
}
