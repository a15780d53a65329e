// Tiled red-black Gauss-Seidel smoother for the FP32 V-cycles (Sec. 4), fed
// by the TMA.
//
// Persistent CTAs of 256 threads walk the tiles of one level (TILE x TILE
// cells of one sample each, tiles of a sample consecutive so that their
// halos meet in L2). For each tile the TMA brings, as 3D tiled copies out of
// the sample pools, the tile plus a 4-cell halo of u, b, the x faces and the
// y faces (zeros outside the domain, which is the Dirichlet ghost value), and
// for the fused coarse-grid correction the coarse solution around it. Two
// buffers: while one tile is smoothed in shared memory the next one is in
// flight. On the staged tile, half sweep p (p = 0 .. 2 NS - 1) updates its
// colour on the tile grown by 2 NS - 1 - p cells, so after the last one the
// tile itself holds exactly NS sweeps (temporal blocking); the result goes to
// u2 (ping-pong: the halos of neighbouring tiles must see the old values).
// The last pre-smoothing launch of a level can also form the residual of its
// tile and its 2 x 2 restriction (the right-hand side of the next coarser
// level), so that no separate pass re-reads u, b and the faces.
#include "rbgs_tma.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "ptx_async.cuh"

using namespace mlqmc_dev;
using namespace mlqmc_ptx;

namespace {

constexpr int kH = 4;  // staged halo (keeps x - kH a multiple of 4 floats: 16-byte TMA coordinates)
constexpr int kThreads = 256;

struct Maps {
    CUtensorMap u, kx, ky, b, e;
};

constexpr int round32(int v) { return (v + 31) / 32 * 32; }  // 128-byte aligned sub-buffers

// RR (pre-smoothing with the restricted residual): u is staged with one more
// cell of halo (UOY = 1 more row above and below; UOX = 4 more columns on
// each side, so that the copy's x origin stays on a 16-byte boundary), the
// half sweeps grow one cell further, and the tile plus a one-cell ring end
// with exactly NS sweeps: the residual of every tile cell follows.
template <int TILE, bool POST, bool RR = false>
struct TGeom {
    static constexpr int SU = TILE + 2 * kH;       // staged cells per side (b, faces; u without RR)
    static constexpr int XW = SU + 4;              // staged x faces per row (box width, 16-byte multiple)
    static constexpr int EC = TILE / 2 + 2 * kH;   // staged coarse cells per side
    static constexpr int UOX = RR ? 4 : 0, UOY = RR ? 1 : 0;
    static constexpr int UP = SU + 2 * UOX;        // staged u: row pitch
    static constexpr int UR = SU + 2 * UOY;        // staged u: rows
    static constexpr int oU = 0;
    static constexpr int oB = oU + round32(UP * UR);
    static constexpr int oKX = oB + round32(SU * SU);
    static constexpr int oKY = oKX + round32(SU * XW);
    static constexpr int oE = oKY + round32((SU + 1) * SU);
    static constexpr int buf = oE + (POST ? round32(EC * EC) : 0);  // floats per buffer
    static constexpr size_t bytes = 128 + 2 * sizeof(float) * static_cast<size_t>(buf);
    static constexpr int ctas_per_sm = POST ? 3 : 4;  // as many as fit the 228 KB of shared memory
    static_assert(!(POST && RR), "the correction is fused into post-smoothing, the residual into pre-smoothing");
    static_assert((SU * 4) % 16 == 0 && (XW * 4) % 16 == 0 && (EC * 4) % 16 == 0 && (UP * 4) % 16 == 0,
                  "TMA boxes: 16-byte rows");
};

template <int TILE, int NS, bool POST, bool RR = false>
__global__ void __launch_bounds__(kThreads, TGeom<TILE, POST, RR>::ctas_per_sm)
    kb_rbgs_tma(const __grid_constant__ Maps maps, FmgArgs A, int t, int B, int ones, int first, int zin)
{
    using Gm = TGeom<TILE, POST, RR>;
    constexpr int SU = Gm::SU, XW = Gm::XW, EC = Gm::EC;
    constexpr int UP = Gm::UP, UOX = Gm::UOX, UOY = Gm::UOY;
    constexpr int HN = 2 * NS;          // half sweeps
    constexpr int GR = RR ? 1 : 0;      // extra growth: the ring around the tile ends fully swept
    constexpr int NRING = RR ? 2 : 1;   // ring cells per thread and half sweep (at most 288 with RR)
    static_assert(HN <= kH && HN + GR <= kH + UOY, "halo");
    // staged u index of the cell at (sy, sx) of the b/face frame (origin x0 - kH, y0 - kH)
    auto uix = [](int sy, int sx) { return (sy + UOY) * UP + sx + UOX; };
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
    float* bufs = reinterpret_cast<float*>(smraw + 128);

    const int n = A.lv[t].n;
    const int tx_n = n / TILE;
    const int per = tx_n * tx_n;
    const int total = B * per;
    const float h2 = 1.0f / (static_cast<float>(n) * static_cast<float>(n));
    // zin (pre-smoothing of a correction, never with POST): u is zero on entry,
    // so its tile is cleared in shared memory instead of copied
    const uint32_t tx_bytes =
        4u * ((zin ? 0 : UP * Gm::UR) + XW * SU + (SU + 1) * SU + (ones ? 0 : SU * SU) + (POST ? EC * EC : 0));

    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue = [&](int tile, int slot) {
        const int i = tile / per;
        const int tr = tile - i * per;
        const int y0 = (tr / tx_n) * TILE, x0 = (tr % tx_n) * TILE;
        float* S = bufs + slot * Gm::buf;
        uint64_t* bar = &full[slot];
        mbar_arrive_tx(bar, tx_bytes);
        if (!zin) tensor_load_3d(S + Gm::oU, &maps.u, bar, x0 - kH - UOX, y0 - kH - UOY, i);
        tensor_load_3d(S + Gm::oKX, &maps.kx, bar, x0 - kH, y0 - kH, i);
        tensor_load_3d(S + Gm::oKY, &maps.ky, bar, x0 - kH, y0 - kH, i);
        if (!ones) tensor_load_3d(S + Gm::oB, &maps.b, bar, x0 - kH, y0 - kH, i);
        if (POST) tensor_load_3d(S + Gm::oE, &maps.e, bar, x0 / 2 - kH, y0 / 2 - kH, i);
    };

    // Work of half sweep ph (growth g = HN - 1 - ph) on the staged tile:
    // - the tile's own 32 rows x 16 cells of the colour, two per thread: warp
    //   w takes row pairs w and w + 8, lanes 0-15 the upper row and 16-31 the
    //   lower one, so every shared access of a warp hits 32 distinct banks;
    // - the ring of the grown region around the tile (64 g + 2 g^2 cells, at
    //   most one per thread): the 2g full rows above and below ((16 + g) cells
    //   each, by cell index m) and g cells at the ends of each tile row (by
    //   index k: the left strip's cells first). Packed per thread: bit 15 =
    //   end-of-row cell, bits 8-14 staged row, bits 0-7 m or k; -1: none.
    static_assert(TILE == 32 && kThreads == 256, "two tile cells per thread and half sweep");
    int ring[HN][NRING];
#pragma unroll
    for (int ph = 0; ph < HN; ++ph) {
        const int g = HN - 1 - ph + GR;
        const int full = 2 * g * (TILE / 2 + g);
#pragma unroll
        for (int q = 0; q < NRING; ++q) {
            const int r = threadIdx.x + q * kThreads;
            int pk = -1;
            if (r < full) {
                const int rr = r / (TILE / 2 + g), m = r - rr * (TILE / 2 + g);
                const int sy = rr < g ? kH - g + rr : kH + TILE + rr - g;
                pk = (sy << 8) | m;
            } else if (r < full + TILE * g) {
                const int rr = (r - full) / g, k = r - full - rr * g;
                pk = 0x8000 | ((kH + rr) << 8) | k;
            }
            ring[ph][q] = g > 0 ? pk : -1;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    bool live = true;
    int issued = 0;  // tiles issued by this CTA (thread 0's count)
    if (threadIdx.x == 0 && static_cast<int>(blockIdx.x) < total) {
        issue(blockIdx.x, 0);
        issued = 1;
    }
    int it = 0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
        const int slot = it & 1;
        const int next = tile + gridDim.x;
        if (threadIdx.x == 0 && next < total) {
            issue(next, slot ^ 1);  // the other buffer was released by the barrier ending the last iteration
            ++issued;
        }
        if (live) live = mbar_wait(&full[slot], (it >> 1) & 1, A.status, kStatusTimeout);
        const int i = tile / per;
        const int tr = tile - i * per;
        const int y0 = (tr / tx_n) * TILE, x0 = (tr % tx_n) * TILE;
        // uniform per CTA: a skipped tile skips every barrier below together
        if (!(A.active && !A.active[i])) {
            float* S = bufs + slot * Gm::buf;
            float* su = S + Gm::oU;
            if (zin) {
                for (int q = threadIdx.x; q < UP * Gm::UR; q += kThreads) su[q] = 0.0f;
                __syncthreads();
            }
            const float* sb = S + Gm::oB;
            const float* skx = S + Gm::oKX;
            const float* sky = S + Gm::oKY;
            if constexpr (POST) {
                // coarse-grid correction on every staged cell of the domain, one
                // 2 x 2 block of fine cells (one coarse parent) per thread: the
                // parent's 3 x 3 coarse neighbourhood, a neighbour outside the
                // coarse grid replaced by minus the parent's row or column
                // (odd reflection; the corner then by the product of the two
                // signs), gives each fine cell the arithmetic of prolong_cell
                const float* se = S + Gm::oE;
                const int nc = n >> 1;
                constexpr int SB = SU / 2;  // staged blocks per side (x0 - kH, y0 - kH even)
                for (int q = threadIdx.x; q < SB * SB; q += kThreads) {
                    const int by = q / SB, bx = q - (q / SB) * SB;
                    const int I2 = (y0 - kH) / 2 + by, I1 = (x0 - kH) / 2 + bx;
                    if (I2 < 0 || I2 >= nc || I1 < 0 || I1 >= nc) continue;
                    const int ey = I2 - (y0 / 2 - kH), ex = I1 - (x0 / 2 - kH);  // in the staged coarse box
                    const bool lo1 = I1 == 0, hi1 = I1 == nc - 1, lo2 = I2 == 0, hi2 = I2 == nc - 1;
                    float E[3][3];
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx) {
                            const bool ry = (dy < 0 && lo2) || (dy > 0 && hi2);
                            const bool rx = (dx < 0 && lo1) || (dx > 0 && hi1);
                            const float v = se[(ey + (ry ? 0 : dy)) * EC + ex + (rx ? 0 : dx)];
                            E[dy + 1][dx + 1] = (ry != rx) ? -v : v;
                        }
                    }
                    float* f = su + uix(2 * by, 2 * bx);
#pragma unroll
                    for (int fy = 0; fy < 2; ++fy) {
#pragma unroll
                        for (int fx = 0; fx < 2; ++fx) {
                            const int dy = 2 * fy, dx = 2 * fx;  // -1 -> 0, +1 -> 2 in E
                            f[fy * UP + fx] +=
                                fmaf(0.5625f, E[1][1], fmaf(0.1875f, E[1][dx] + E[dy][1], 0.0625f * E[dy][dx]));
                        }
                    }
                }
                __syncthreads();
            }
            // tiles whose grown regions stay inside the domain skip the per-cell test
            const bool interior =
                x0 >= HN + GR && y0 >= HN + GR && x0 + TILE + HN + GR <= n && y0 + TILE + HN + GR <= n;
            // one red-black update of staged cell (sy, sx)
            auto update = [&](int sy, int sx) {
                const int c0 = sy * SU + sx;
                const int cu = uix(sy, sx);
                const float* kr = skx + sy * XW;
                const float w = kr[sx], e = kr[sx + 1];
                const float nn = sky[c0], so = sky[c0 + SU];
                float acc = h2 * (ones ? 1.0f : sb[c0]);
                acc += w * su[cu - 1];
                acc += e * su[cu + 1];
                acc += nn * su[cu - UP];
                acc += so * su[cu + UP];
                su[cu] = __fdividef(acc, w + e + nn + so);  // hardware reciprocal: within 2 ulp
            };
            // the thread's own tile cells (two rows, both colours): their faces,
            // h^2 b and diagonal stay in registers across the half sweeps, so an
            // update reads only the four neighbouring u from shared memory (same
            // operands, same order as `update`)
            float cw[2][2], ce[2][2], cn[2][2], cso[2][2], cb[2][2], cd[2][2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int sy = kH + 2 * (warp + 8 * j) + (lane >> 4);
                // lanes 16-31 hold the next row (every row pitch is even): they load
                // their other column first, so each load of the warp hits 32 banks
                const bool swap = (lane >> 4) != 0;
                float vw[2], ve[2], vn[2], vs[2], vb[2];
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int sx = kH + 2 * (lane & 15) + (pp ^ (lane >> 4));
                    const int c0 = sy * SU + sx;
                    const float* kr = skx + sy * XW;
                    vw[pp] = kr[sx];
                    ve[pp] = kr[sx + 1];
                    vn[pp] = sky[c0];
                    vs[pp] = sky[c0 + SU];
                    vb[pp] = ones ? 1.0f : sb[c0];
                }
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int q = p ^ 1;
                    cw[j][p] = swap ? vw[q] : vw[p];
                    ce[j][p] = swap ? ve[q] : ve[p];
                    cn[j][p] = swap ? vn[q] : vn[p];
                    cso[j][p] = swap ? vs[q] : vs[p];
                    cb[j][p] = h2 * (swap ? vb[q] : vb[p]);
                    cd[j][p] = cw[j][p] + ce[j][p] + cn[j][p] + cso[j][p];
                }
            }
#pragma unroll
            for (int ph = 0; ph < HN; ++ph) {
                const int colour = (first + ph) & 1;
                const int g = HN - 1 - ph + GR;  // growth of the updated region beyond the tile
                // colour cells: (gx + gy) & 1 == colour, with x0 - kH and y0 - kH even
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int sy = kH + 2 * (warp + 8 * j) + (lane >> 4);
                    const int p = (colour + sy) & 1;
                    const int cu = uix(sy, kH + 2 * (lane & 15) + p);
                    float acc = p ? cb[j][1] : cb[j][0];
                    acc += (p ? cw[j][1] : cw[j][0]) * su[cu - 1];
                    acc += (p ? ce[j][1] : ce[j][0]) * su[cu + 1];
                    acc += (p ? cn[j][1] : cn[j][0]) * su[cu - UP];
                    acc += (p ? cso[j][1] : cso[j][0]) * su[cu + UP];
                    su[cu] = __fdividef(acc, p ? cd[j][1] : cd[j][0]);
                }
#pragma unroll
                for (int q = 0; q < NRING; ++q) {
                    const int pk = ring[ph][q];
                    if (pk >= 0) {
                        const int sy = (pk >> 8) & 127;
                        const int p = (colour + g + sy) & 1;
                        int m = pk & 255;
                        if (pk & 0x8000) m = m < ((g - p + 1) >> 1) ? m : m + TILE / 2;  // left strip, then right
                        const int sx = kH - g + 2 * m + p;
                        const int gy = y0 - kH + sy, gx = x0 - kH + sx;
                        if (interior || (gy >= 0 && gy < n && gx >= 0 && gx < n)) update(sy, sx);
                    }
                }
                __syncthreads();
            }
            if constexpr (RR) {
                // residual b - A u (flux form, u = 0 across the boundary, where the
                // face holds 2 k) of the thread's four tile cells, from their faces
                // in registers; the 2 x 2 mean of each coarse cell's children (its
                // two rows are lanes l and l + 16) is the right-hand side of level
                // t - 1. Lanes 16-31 take their other column first (32 banks).
                const float ih2 = static_cast<float>(n) * static_cast<float>(n);
                const bool swap = (lane >> 4) != 0;
                float* bco = at<float>(A.lv[t - 1].bc, i);
                const int nc = n >> 1;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int sy = kH + 2 * (warp + 8 * j) + (lane >> 4);
                    float rs = 0.0f;
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const int p = pp ^ (lane >> 4);
                        const int cu = uix(sy, kH + 2 * (lane & 15) + p);
                        const int q = pp ^ 1;
                        const float w = swap ? cw[j][q] : cw[j][pp], e = swap ? ce[j][q] : ce[j][pp];
                        const float nn = swap ? cn[j][q] : cn[j][pp], so = swap ? cso[j][q] : cso[j][pp];
                        const float bb = swap ? cb[j][q] : cb[j][pp];
                        const float up = su[cu];
                        float acc = w * (up - su[cu - 1]);
                        acc += e * (up - su[cu + 1]);
                        acc += nn * (up - su[cu - UP]);
                        acc += so * (up - su[cu + UP]);
                        rs += (bb - acc) * ih2;
                    }
                    const float tot = rs + __shfl_xor_sync(0xffffffffu, rs, 16);
                    if (lane < 16) bco[static_cast<size_t>(y0 / 2 + warp + 8 * j) * nc + x0 / 2 + lane] = 0.25f * tot;
                }
            }
            float* uo = at<float>(A.lv[t].u2, i);
            constexpr int TV = TILE / 4;
            static_assert((UP * 4) % 16 == 0 && ((kH + UOX) * 4) % 16 == 0, "16-byte aligned staged rows");
            for (int q = threadIdx.x; q < TILE * TV; q += kThreads) {
                const int ry = q / TV, v = q - (q / TV) * TV;
                *reinterpret_cast<float4*>(uo + static_cast<size_t>(y0 + ry) * n + x0 + 4 * v) =
                    *reinterpret_cast<const float4*>(su + uix(ry + kH, kH + 4 * v));
            }
        }
        // this buffer is refilled by the TMA next iteration: order the generic accesses first
        fence_proxy_async();
        __syncthreads();
    }
    if (threadIdx.x == 0 && !live) {
        // a wait gave up: let the tiles still in flight land before the CTA leaves
        const uint64_t t0 = now_ns();
        for (int k = issued - 2 < 0 ? 0 : issued - 2; k < issued; ++k)
            while (!mbar_test(&full[k & 1], (k >> 1) & 1) && now_ns() - t0 < 1000000000ull) {
            }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// FP32 array of per-sample blocks: x extent w (row pitch `pitch` floats), h rows, B samples.
bool encode_3d(CUtensorMap* map, const ArrDesc& a, uint64_t w, uint64_t pitch, uint64_t h, uint64_t B, uint32_t bw,
               uint32_t bh)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || !a.base) return false;
    const cuuint64_t dims[3] = {w, h, B};
    const cuuint64_t strides[2] = {pitch * sizeof(float), static_cast<cuuint64_t>(a.stride)};
    const cuuint32_t box[3] = {bw, bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TILE, int NS, bool POST, bool RR = false>
bool attr()
{
    return cudaFuncSetAttribute(kb_rbgs_tma<TILE, NS, POST, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TGeom<TILE, POST, RR>::bytes)) == cudaSuccess;
}

template <int TILE>
bool attrs()
{
    return attr<TILE, 1, false>() && attr<TILE, 1, true>() && attr<TILE, 2, false>() && attr<TILE, 2, true>() &&
           attr<TILE, 1, false, true>() && attr<TILE, 2, false, true>();
}

template <int TILE, int NS, bool POST, bool RR = false>
void run(const Maps& m, const FmgArgs& A, int t, int B, int tiles, int ones, int first, int zin, int sm_count,
         cudaStream_t st)
{
    using Gm = TGeom<TILE, POST, RR>;
    const int cap = Gm::ctas_per_sm * sm_count;
    kb_rbgs_tma<TILE, NS, POST, RR>
        <<<tiles < cap ? tiles : cap, kThreads, Gm::bytes, st>>>(m, A, t, B, ones, first, zin);
}

template <int TILE>
bool go(const FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool post, int zin, bool rr,
        int sm_count, cudaStream_t st)
{
    using Gm = TGeom<TILE, true>;
    using Gr = TGeom<TILE, false, true>;
    const LevelDesc& L = A.lv[t];
    Maps m;
    std::memset(&m, 0, sizeof(m));
    const uint64_t un = static_cast<uint64_t>(n), ub = static_cast<uint64_t>(B);
    bool ok = (rr ? encode_3d(&m.u, L.u, un, un, un, ub, Gr::UP, Gr::UR)
                  : encode_3d(&m.u, L.u, un, un, un, ub, Gm::SU, Gm::SU)) &&
              encode_3d(&m.kx, L.kx, un + 4, static_cast<uint64_t>(kx_pitch(n)), un, ub, Gm::XW, Gm::SU) &&
              encode_3d(&m.ky, L.ky, un, un, un + 1, ub, Gm::SU, Gm::SU + 1) &&
              (ones || encode_3d(&m.b, L.bc, un, un, un, ub, Gm::SU, Gm::SU)) &&
              (!post || encode_3d(&m.e, A.lv[t - 1].u, un / 2, un / 2, un / 2, ub, Gm::EC, Gm::EC));
    if (!ok) return false;
    const int tiles = B * (n / TILE) * (n / TILE);
    if (ns == 2) {
        if (post) run<TILE, 2, true>(m, A, t, B, tiles, ones, first, 0, sm_count, st);
        else if (rr) run<TILE, 2, false, true>(m, A, t, B, tiles, ones, first, zin, sm_count, st);
        else run<TILE, 2, false>(m, A, t, B, tiles, ones, first, zin, sm_count, st);
    } else {
        if (post) run<TILE, 1, true>(m, A, t, B, tiles, ones, first, 0, sm_count, st);
        else if (rr) run<TILE, 1, false, true>(m, A, t, B, tiles, ones, first, zin, sm_count, st);
        else run<TILE, 1, false>(m, A, t, B, tiles, ones, first, zin, sm_count, st);
    }
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace

namespace mlqmc_tma {

bool supported(int n)
{
    return n >= 64 && n % 32 == 0;  // every TMA box within the tensor's extent
}

bool prepare()
{
    return encode_fn() != nullptr && attrs<32>();
}

bool launch(const FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool post, bool zin, bool rr,
            int sm_count, cudaStream_t st)
{
    if (B <= 0) return true;
    if (!supported(n) || t < 1 || A.lv[t].n != n || (ns != 1 && ns != 2) || (zin && post) || (rr && post))
        return false;
    return go<32>(A, t, n, B, ns, ones, first, post, zin ? 1 : 0, rr, sm_count, st);
}

}  // namespace mlqmc_tma
