// Tiled red-black Gauss-Seidel smoother for the FP32 V-cycles (Sec. 4), fed
// by the TMA.
//
// Persistent CTAs walk the tiles of one level (TX x TY cells of one sample
// each, TX * TY / 4 threads; tiles of a sample consecutive so that their
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
constexpr int kSmemPerSM = 233472;  // 228 KB of shared memory per SM, 1 KB of it reserved per CTA

struct Maps {
    CUtensorMap u, kx, ky, b, e;
};

constexpr int round32(int v) { return (v + 31) / 32 * 32; }  // 128-byte aligned sub-buffers

// RR (pre-smoothing with the restricted residual): u is staged with one more
// cell of halo (UOY = 1 more row above and below; UOX = 4 more columns on
// each side, so that the copy's x origin stays on a 16-byte boundary), the
// half sweeps grow one cell further, and the tile plus a one-cell ring end
// with exactly NS sweeps: the residual of every tile cell follows.
template <int TX, int TY, bool POST, bool RR = false>
struct TGeom {
    static constexpr int SX = TX + 2 * kH;         // staged cells per row (b, faces; u without RR)
    static constexpr int SY = TY + 2 * kH;         // staged rows
    static constexpr int XW = SX + 4;              // staged x faces per row (box width, 16-byte multiple)
    static constexpr int ECX = TX / 2 + 2 * kH;    // staged coarse cells per row
    static constexpr int ECY = TY / 2 + 2 * kH;    // staged coarse rows
    static constexpr int UOX = RR ? 4 : 0, UOY = RR ? 1 : 0;
    static constexpr int UP = SX + 2 * UOX;        // staged u: row pitch
    static constexpr int UR = SY + 2 * UOY;        // staged u: rows
    static constexpr int oU = 0;
    static constexpr int oB = oU + round32(UP * UR);
    static constexpr int oKX = oB + round32(SX * SY);
    static constexpr int oKY = oKX + round32(XW * SY);
    static constexpr int oE = oKY + round32((SY + 1) * SX);
    static constexpr int buf = oE + (POST ? round32(ECX * ECY) : 0);  // floats per buffer
    static constexpr size_t bytes = 128 + 2 * sizeof(float) * static_cast<size_t>(buf);
    static constexpr int threads = TX * TY / 4;    // four tile cells per thread
    static constexpr int by_smem = static_cast<int>(kSmemPerSM / (bytes + 1024));
    static constexpr int ctas_per_sm = by_smem < 2048 / threads ? by_smem : 2048 / threads;
    static_assert(!(POST && RR), "the correction is fused into post-smoothing, the residual into pre-smoothing");
    static_assert((SX * 4) % 16 == 0 && (XW * 4) % 16 == 0 && (ECX * 4) % 16 == 0 && (UP * 4) % 16 == 0,
                  "TMA boxes: 16-byte rows");
    static_assert(TX % 32 == 0 && (TY / 2) % (threads / 32 / (TX / 32)) == 0 && TY == 4 * (threads / 32 / (TX / 32)),
                  "each warp: a 32-column half-tile row pair, two row pairs per thread");
};

template <int TX, int TY, int NS, bool POST, bool RR = false>
__global__ void __launch_bounds__(TGeom<TX, TY, POST, RR>::threads, TGeom<TX, TY, POST, RR>::ctas_per_sm)
    kb_rbgs_tma(const __grid_constant__ Maps maps, FmgArgs A, int t, int B, int ones, int first, int zin)
{
    using Gm = TGeom<TX, TY, POST, RR>;
    constexpr int SX = Gm::SX, XW = Gm::XW, ECX = Gm::ECX;
    constexpr int UP = Gm::UP, UOX = Gm::UOX, UOY = Gm::UOY;
    constexpr int kThreads = Gm::threads;
    constexpr int HN = 2 * NS;          // half sweeps
    constexpr int GR = RR ? 1 : 0;      // extra growth: the ring around the tile ends fully swept
    constexpr int GMAX = HN - 1 + GR;   // largest growth
    constexpr int NRING = (2 * GMAX * (TX / 2 + GMAX) + TY * GMAX + kThreads - 1) / kThreads;  // ring cells per thread
    constexpr int CH = TX / 32;                  // 32-column halves of the tile
    constexpr int WR = kThreads / 32 / CH;       // warps per half: row pairs rp, rp + WR
    static_assert(HN <= kH && HN + GR <= kH + UOY, "halo");
    // staged u index of the cell at (sy, sx) of the b/face frame (origin x0 - kH, y0 - kH)
    auto uix = [](int sy, int sx) { return (sy + UOY) * UP + sx + UOX; };
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
    float* bufs = reinterpret_cast<float*>(smraw + 128);

    const int n = A.lv[t].n;
    const int txn = n / TX, tyn = n / TY;
    const int per = txn * tyn;
    const int total = B * per;
    const float h2 = 1.0f / (static_cast<float>(n) * static_cast<float>(n));
    // zin (pre-smoothing of a correction, never with POST): u is zero on entry,
    // so its tile is cleared in shared memory instead of copied
    const uint32_t tx_bytes =
        4u * ((zin ? 0 : UP * Gm::UR) + XW * Gm::SY + (Gm::SY + 1) * SX + (ones ? 0 : SX * Gm::SY) +
              (POST ? ECX * Gm::ECY : 0));

    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue = [&](int tile, int slot) {
        const int i = tile / per;
        const int tr = tile - i * per;
        const int y0 = (tr / txn) * TY, x0 = (tr % txn) * TX;
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
    // - the tile's own TY rows x TX / 2 cells of the colour, two per thread:
    //   warp w takes the 32-column half ch = w / WR of the tile and the row
    //   pairs rp and rp + WR (rp = w % WR), lanes 0-15 the upper row of a
    //   pair and 16-31 the lower one, so every shared access of a warp hits
    //   32 distinct banks;
    // - the ring of the grown region around the tile (2 g (TX / 2 + g) + TY g
    //   cells, NRING per thread): the 2g full rows above and below (TX / 2 + g
    //   cells each, by cell index m) and g cells at the ends of each tile row
    //   (by index k: the left strip's cells first). Packed per thread: bit 15
    //   = end-of-row cell, bits 8-14 staged row, bits 0-7 m or k; -1: none.
    int ring[HN][NRING];
#pragma unroll
    for (int ph = 0; ph < HN; ++ph) {
        const int g = HN - 1 - ph + GR;
        const int full = 2 * g * (TX / 2 + g);
#pragma unroll
        for (int q = 0; q < NRING; ++q) {
            const int r = threadIdx.x + q * kThreads;
            int pk = -1;
            if (r < full) {
                const int rr = r / (TX / 2 + g), m = r - rr * (TX / 2 + g);
                const int sy = rr < g ? kH - g + rr : kH + TY + rr - g;
                pk = (sy << 8) | m;
            } else if (r < full + TY * g) {
                const int rr = (r - full) / g, k = r - full - rr * g;
                pk = 0x8000 | ((kH + rr) << 8) | k;
            }
            ring[ph][q] = g > 0 ? pk : -1;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = warp / WR, rp = warp - (warp / WR) * WR;

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
        const int y0 = (tr / txn) * TY, x0 = (tr % txn) * TX;
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
                constexpr int SBX = SX / 2, SBY = Gm::SY / 2;  // staged blocks (x0 - kH, y0 - kH even)
                for (int q = threadIdx.x; q < SBX * SBY; q += kThreads) {
                    const int by = q / SBX, bx = q - (q / SBX) * SBX;
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
                            const float v = se[(ey + (ry ? 0 : dy)) * ECX + ex + (rx ? 0 : dx)];
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
                x0 >= HN + GR && y0 >= HN + GR && x0 + TX + HN + GR <= n && y0 + TY + HN + GR <= n;
            // one red-black update of staged cell (sy, sx)
            auto update = [&](int sy, int sx) {
                const int c0 = sy * SX + sx;
                const int cu = uix(sy, sx);
                const float* kr = skx + sy * XW;
                const float w = kr[sx], e = kr[sx + 1];
                const float nn = sky[c0], so = sky[c0 + SX];
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
                const int sy = kH + 2 * (rp + WR * j) + (lane >> 4);
                // lanes 16-31 hold the next row (every row pitch is even): they load
                // their other column first, so each load of the warp hits 32 banks
                const bool swap = (lane >> 4) != 0;
                float vw[2], ve[2], vn[2], vs[2], vb[2];
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int sx = kH + 32 * ch + 2 * (lane & 15) + (pp ^ (lane >> 4));
                    const int c0 = sy * SX + sx;
                    const float* kr = skx + sy * XW;
                    vw[pp] = kr[sx];
                    ve[pp] = kr[sx + 1];
                    vn[pp] = sky[c0];
                    vs[pp] = sky[c0 + SX];
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
                    const int sy = kH + 2 * (rp + WR * j) + (lane >> 4);
                    const int p = (colour + sy) & 1;
                    const int cu = uix(sy, kH + 32 * ch + 2 * (lane & 15) + p);
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
                        if (pk & 0x8000) m = m < ((g - p + 1) >> 1) ? m : m + TX / 2;  // left strip, then right
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
                    const int sy = kH + 2 * (rp + WR * j) + (lane >> 4);
                    float rs = 0.0f;
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const int p = pp ^ (lane >> 4);
                        const int cu = uix(sy, kH + 32 * ch + 2 * (lane & 15) + p);
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
                    if (lane < 16)
                        bco[static_cast<size_t>(y0 / 2 + rp + WR * j) * nc + x0 / 2 + 16 * ch + lane] = 0.25f * tot;
                }
            }
            float* uo = at<float>(A.lv[t].u2, i);
            constexpr int TV = TX / 4;
            static_assert((UP * 4) % 16 == 0 && ((kH + UOX) * 4) % 16 == 0, "16-byte aligned staged rows");
            for (int q = threadIdx.x; q < TY * TV; q += kThreads) {
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

template <int TX, int TY, int NS, bool POST, bool RR = false>
bool attr()
{
    return cudaFuncSetAttribute(kb_rbgs_tma<TX, TY, NS, POST, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TGeom<TX, TY, POST, RR>::bytes)) == cudaSuccess;
}

// Tile shapes: pre-smoothing (with or without the restricted residual) in
// 64 x 32 tiles of 512 threads where the side allows (less halo and ring per
// cell, half the barriers per cell), else 32 x 32; post-smoothing with the
// fused correction in 32 x 32 tiles of 256 threads (its extra registers).
bool attrs()
{
    return attr<32, 32, 1, false>() && attr<32, 32, 1, true>() && attr<32, 32, 2, false>() &&
           attr<32, 32, 2, true>() && attr<32, 32, 1, false, true>() && attr<32, 32, 2, false, true>() &&
           attr<64, 32, 1, false>() && attr<64, 32, 2, false>() && attr<64, 32, 1, false, true>() &&
           attr<64, 32, 2, false, true>();
}

template <int TX, int TY, int NS, bool POST, bool RR>
bool run(const FmgArgs& A, int t, int n, int B, int ones, int first, int zin, int sm_count, cudaStream_t st)
{
    using Gm = TGeom<TX, TY, POST, RR>;
    const LevelDesc& L = A.lv[t];
    Maps m;
    std::memset(&m, 0, sizeof(m));
    const uint64_t un = static_cast<uint64_t>(n), ub = static_cast<uint64_t>(B);
    const bool ok = encode_3d(&m.u, L.u, un, un, un, ub, Gm::UP, Gm::UR) &&
                    encode_3d(&m.kx, L.kx, un + 4, static_cast<uint64_t>(kx_pitch(n)), un, ub, Gm::XW, Gm::SY) &&
                    encode_3d(&m.ky, L.ky, un, un, un + 1, ub, Gm::SX, Gm::SY + 1) &&
                    (ones || encode_3d(&m.b, L.bc, un, un, un, ub, Gm::SX, Gm::SY)) &&
                    (!POST || encode_3d(&m.e, A.lv[t - 1].u, un / 2, un / 2, un / 2, ub, Gm::ECX, Gm::ECY));
    if (!ok) return false;
    const int tiles = B * (n / TX) * (n / TY);
    const int cap = Gm::ctas_per_sm * sm_count;
    kb_rbgs_tma<TX, TY, NS, POST, RR>
        <<<tiles < cap ? tiles : cap, Gm::threads, Gm::bytes, st>>>(m, A, t, B, ones, first, zin);
    return cudaGetLastError() == cudaSuccess;
}

template <int NS>
bool go(const FmgArgs& A, int t, int n, int B, int ones, int first, bool post, int zin, bool rr, int sm_count,
        cudaStream_t st)
{
    if (post) return run<32, 32, NS, true, false>(A, t, n, B, ones, first, 0, sm_count, st);
    if (n % 64 == 0 && n >= 128) {  // every box (up to 80 columns) within the level's extent
        if (rr) return run<64, 32, NS, false, true>(A, t, n, B, ones, first, zin, sm_count, st);
        return run<64, 32, NS, false, false>(A, t, n, B, ones, first, zin, sm_count, st);
    }
    if (rr) return run<32, 32, NS, false, true>(A, t, n, B, ones, first, zin, sm_count, st);
    return run<32, 32, NS, false, false>(A, t, n, B, ones, first, zin, sm_count, st);
}

}  // namespace

namespace mlqmc_tma {

bool supported(int n)
{
    return n >= 64 && n % 32 == 0;  // every TMA box within the tensor's extent
}

bool prepare()
{
    return encode_fn() != nullptr && attrs();
}

bool launch(const FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool post, bool zin, bool rr,
            int sm_count, cudaStream_t st)
{
    if (B <= 0) return true;
    if (!supported(n) || t < 1 || A.lv[t].n != n || (ns != 1 && ns != 2) || (zin && post) || (rr && post))
        return false;
    return ns == 2 ? go<2>(A, t, n, B, ones, first, post, zin ? 1 : 0, rr, sm_count, st)
                   : go<1>(A, t, n, B, ones, first, post, zin ? 1 : 0, rr, sm_count, st);
}

}  // namespace mlqmc_tma
