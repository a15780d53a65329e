// Tiled red-black Gauss-Seidel smoother for the FP32 V-cycles (Sec. 4), fed
// by the TMA.
//
// Persistent CTAs walk the tiles of one level (TX x TY cells of one sample
// each; tiles of a sample consecutive so that their halos meet in L2). For
// each tile the TMA brings, as 3D tiled copies out of the sample pools, the
// "frame" -- the tile plus kH = 4 cells on every side -- of b, the x faces and
// the y faces, u on the frame plus one more cell around it (zeros outside the
// domain, which is the Dirichlet ghost value), and for the fused coarse-grid
// correction the coarse solution around it. Two buffers: while one tile is
// smoothed the next one is in flight.
//
// Every thread owns a 4 x 2 block of the frame and keeps its u, faces, h^2 b
// and reciprocal diagonal in registers. Half sweep p (p = 0 .. 2 NS - 1)
// updates the colour's cells of the whole frame: a cell's update reads its
// two in-block neighbours from registers, the rows above and below the block
// with one 16-byte shared load each and its left or right neighbour from the
// next lane (a warp shuffle; shared memory where that lane holds another
// row). Frame cells at distance d from the tile are exact after half sweep p
// while d <= kH - p (their neighbours one cell further out were exact one half
// sweep earlier, and the extra ring of u is exact before the first one), so
// after the last half sweep the tile and one ring around it hold exactly NS
// sweeps (temporal blocking); values further out are discarded. Cells
// outside the domain have a zero reciprocal diagonal and right-hand side, so
// they stay at zero. The result goes to u2 (ping-pong: the halos of
// neighbouring tiles must see the old values). The last pre-smoothing launch
// of a level can also form the residual of its tile and its 2 x 2 restriction
// (the right-hand side of the next coarser level), so that no separate pass
// re-reads u, b and the faces.
#include "rbgs_tma.h"

#include <cstdint>
#include <cstring>

#include "ptx_async.cuh"
#include "tma_encode.h"

using namespace mlqmc_dev;
using namespace mlqmc_ptx;

namespace {

constexpr int kH = 4;  // staged frame around the tile (keeps x - kH a multiple of 4 floats: 16-byte TMA coordinates)
constexpr int kSmemPerSM = 233472;  // 228 KB of shared memory per SM, 1 KB of it reserved per CTA
constexpr unsigned kFull = 0xffffffffu;

struct Maps {
    CUtensorMap u, kx, ky, b, e;
};

constexpr int round32(int v) { return (v + 31) / 32 * 32; }  // 128-byte aligned sub-buffers

template <int V>
struct Colour {
    static constexpr int value = V;
};

template <bool V>
struct Flag {
    static constexpr bool value = V;
};

// Coordinates (sample i, tile row ty, tile column tx) of a CTA's tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...: split once, then advanced by
// gridDim.x with carries instead of two divisions per tile.
struct TileWalk {
    int txn, tyn, gi, gty, gtx;
    __device__ TileWalk(int txn_, int tyn_) : txn(txn_), tyn(tyn_) { split(gridDim.x, gi, gty, gtx); }
    __device__ void split(int tile, int& i, int& ty, int& tx) const
    {
        const int per = txn * tyn;
        i = tile / per;
        const int tr = tile - i * per;
        ty = tr / txn;
        tx = tr - ty * txn;
    }
    __device__ void advance(int& i, int& ty, int& tx) const
    {
        tx += gtx;
        if (tx >= txn) {
            tx -= txn;
            ++ty;
        }
        ty += gty;
        if (ty >= tyn) {
            ty -= tyn;
            ++i;
        }
        i += gi;
    }
};

template <int TX, int TY, bool POST>
struct TGeom {
    static constexpr int SX = TX + 2 * kH;         // frame cells per row (b, faces)
    static constexpr int SY = TY + 2 * kH;         // frame rows
    static constexpr int XW = SX + 4;              // staged x faces per row (box width, 16-byte multiple)
    static constexpr int ECX = TX / 2 + 2 * kH;    // staged coarse cells per row
    static constexpr int ECY = TY / 2 + 2 * kH;    // staged coarse rows
    static constexpr int UP = SX + 8;              // staged u: row pitch (4 more columns on each side)
    static constexpr int UR = SY + 2;              // staged u: rows (one more above and below)
    static constexpr int BX = SX / 4, BY = SY / 2;  // 4 x 2 blocks of the frame, one per thread
    static constexpr int NB = BX * BY;
    static constexpr int threads = round32(NB);
    static constexpr int oU = 0;
    static constexpr int oB = oU + round32(UP * UR);
    static constexpr int oKX = oB + round32(SX * SY);
    static constexpr int oKY = oKX + round32(XW * SY);
    static constexpr int oE = oKY + round32((SY + 1) * SX);
    static constexpr int buf = oE + (POST ? round32(ECX * ECY) : 0);  // floats per buffer
    static constexpr size_t bytes = 128 + 2 * sizeof(float) * static_cast<size_t>(buf);
    static constexpr int by_smem = static_cast<int>(kSmemPerSM / (bytes + 1024));
    static constexpr int ctas_per_sm = by_smem < 2048 / threads ? by_smem : 2048 / threads;
    static_assert((SX * 4) % 16 == 0 && (XW * 4) % 16 == 0 && (ECX * 4) % 16 == 0 && (UP * 4) % 16 == 0,
                  "TMA boxes: 16-byte rows");
    static_assert(TX % 32 == 0 && TY % 2 == 0 && kH % 4 == 0, "whole blocks on the tile and the frame");
    static_assert(ctas_per_sm >= 1, "shared memory");
};

template <int TX, int TY, int NS, bool POST, bool RR>
__global__ void __launch_bounds__(TGeom<TX, TY, POST>::threads, TGeom<TX, TY, POST>::ctas_per_sm)
    kb_rbgs_tma(const __grid_constant__ Maps maps, FmgArgs A, int t, int B, int ones, int first, int zin)
{
    using Gm = TGeom<TX, TY, POST>;
    constexpr int SX = Gm::SX, SY = Gm::SY, XW = Gm::XW, ECX = Gm::ECX, UP = Gm::UP, BX = Gm::BX;
    constexpr int kThreads = Gm::threads;
    constexpr int HN = 2 * NS;  // half sweeps
    static_assert(HN <= kH, "the tile and one ring around it end exact");
    static_assert(!(POST && RR), "the correction is fused into post-smoothing, the residual into pre-smoothing");
    // staged u index of the frame cell (sy, sx) (frame origin x0 - kH, y0 - kH)
    auto uix = [](int sy, int sx) { return (sy + 1) * UP + sx + 4; };
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
        4u * ((zin ? 0 : UP * Gm::UR) + XW * SY + (SY + 1) * SX + (ones ? 0 : SX * SY) + (POST ? ECX * Gm::ECY : 0));

    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue = [&](int i, int ty, int tx, int slot) {
        const int y0 = ty * TY, x0 = tx * TX;
        float* S = bufs + slot * Gm::buf;
        uint64_t* bar = &full[slot];
        mbar_arrive_tx(bar, tx_bytes);
        if (!zin) tensor_load_3d(S + Gm::oU, &maps.u, bar, x0 - kH - 4, y0 - kH - 1, i);
        tensor_load_3d(S + Gm::oKX, &maps.kx, bar, x0 - kH, y0 - kH, i);
        tensor_load_3d(S + Gm::oKY, &maps.ky, bar, x0 - kH, y0 - kH, i);
        if (!ones) tensor_load_3d(S + Gm::oB, &maps.b, bar, x0 - kH, y0 - kH, i);
        if (POST) tensor_load_3d(S + Gm::oE, &maps.e, bar, x0 / 2 - kH, y0 / 2 - kH, i);
    };

    // the thread's block: frame rows sy0, sy0 + 1, columns sx0 .. sx0 + 3
    const int lane = threadIdx.x & 31;
    const bool owner = static_cast<int>(threadIdx.x) < Gm::NB;
    const int br = threadIdx.x / BX, bc = threadIdx.x - (threadIdx.x / BX) * BX;
    const int sy0 = 2 * br, sx0 = 4 * bc;
    const bool core = owner && br >= kH / 2 && br < kH / 2 + TY / 2 && bc >= kH / 4 && bc < kH / 4 + TX / 4;
    // side neighbours come from the next lane unless that lane holds another
    // frame row (or is in another warp): then from shared memory
    const bool lsm = owner && (lane == 0 || bc == 0);
    const bool rsm = owner && (lane == 31 || bc == BX - 1);

    const TileWalk walk(txn, tyn);
    int ci, cty, ctx;  // this tile
    walk.split(blockIdx.x, ci, cty, ctx);
    int ni = ci, nty = cty, ntx = ctx;  // the next one
    bool live = true;
    int issued = 0;  // tiles issued by this CTA (thread 0's count)
    if (threadIdx.x == 0 && static_cast<int>(blockIdx.x) < total) {
        issue(ci, cty, ctx, 0);
        issued = 1;
    }
    int it = 0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
        const int slot = it & 1;
        const int next = tile + gridDim.x;
        walk.advance(ni, nty, ntx);
        if (threadIdx.x == 0 && next < total) {
            issue(ni, nty, ntx, slot ^ 1);  // the other buffer was released by the barrier ending the last iteration
            ++issued;
        }
        if (live) live = mbar_wait(&full[slot], (it >> 1) & 1, A.status, kStatusTimeout);
        const int i = ci;
        const int y0 = cty * TY, x0 = ctx * TX;
        ci = ni, cty = nty, ctx = ntx;
        // uniform per CTA: a skipped tile skips every barrier below together
        if (!(A.active && !A.active[i])) {
            float* S = bufs + slot * Gm::buf;
            float* su = S + Gm::oU;
            if (zin) {
                float4* s4 = reinterpret_cast<float4*>(su);
                for (int q = threadIdx.x; q < UP * Gm::UR / 4; q += kThreads) s4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                __syncthreads();
            }
            const float* sb = S + Gm::oB;
            const float* skx = S + Gm::oKX;
            const float* sky = S + Gm::oKY;

            // the block in registers: u, x faces (w of cell k = fx[r][k], e =
            // fx[r][k + 1]), y faces (north fy[r][k], south fy[r + 1][k]), h^2 b
            // and the reciprocal diagonal; both zero outside the domain
            float uu[2][4], fx[2][5], fy[3][4], cb[2][4], id[2][4];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
#pragma unroll
                for (int k = 0; k < 4; ++k) uu[r][k] = fx[r][k] = fy[r][k] = cb[r][k] = id[r][k] = 0.0f;
                fx[r][4] = 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) fy[2][k] = 0.0f;
            if (owner) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float4 v = *reinterpret_cast<const float4*>(su + uix(sy0 + r, sx0));
                    uu[r][0] = v.x, uu[r][1] = v.y, uu[r][2] = v.z, uu[r][3] = v.w;
                    const float4 kv = *reinterpret_cast<const float4*>(skx + (sy0 + r) * XW + sx0);
                    fx[r][0] = kv.x, fx[r][1] = kv.y, fx[r][2] = kv.z, fx[r][3] = kv.w;
                    fx[r][4] = skx[(sy0 + r) * XW + sx0 + 4];
                }
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float4 yv = *reinterpret_cast<const float4*>(sky + (sy0 + j) * SX + sx0);
                    fy[j][0] = yv.x, fy[j][1] = yv.y, fy[j][2] = yv.z, fy[j][3] = yv.w;
                }
                float bv[2][4];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    bv[r][0] = bv[r][1] = bv[r][2] = bv[r][3] = 1.0f;
                    if (!ones) {
                        const float4 v = *reinterpret_cast<const float4*>(sb + (sy0 + r) * SX + sx0);
                        bv[r][0] = v.x, bv[r][1] = v.y, bv[r][2] = v.z, bv[r][3] = v.w;
                    }
                }
                auto diag = [&](auto all_in) {
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int gy = y0 - kH + sy0 + r;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int gx = x0 - kH + sx0 + k;
                            const bool in = decltype(all_in)::value || (gy >= 0 && gy < n && gx >= 0 && gx < n);
                            const float d = fx[r][k] + fx[r][k + 1] + fy[r][k] + fy[r + 1][k];
                            id[r][k] = in ? __fdividef(1.0f, d) : 0.0f;
                            cb[r][k] = in ? h2 * bv[r][k] : 0.0f;
                        }
                    }
                };
                if (x0 >= kH && x0 + TX + kH <= n && y0 >= kH && y0 + TY + kH <= n) diag(Flag<true>());
                else diag(Flag<false>());
            }
            if constexpr (POST) {
                // coarse-grid correction of the block's cells in the domain: each
                // coarse parent's 3 x 3 neighbourhood, a neighbour outside the
                // coarse grid replaced by minus the parent's row or column (odd
                // reflection; the corner then by the product of the two signs)
                const float* se = S + Gm::oE;
                const int nc = n >> 1;
                const int I2 = (y0 - kH) / 2 + br, I1b = (x0 - kH) / 2 + 2 * bc;
                if (owner && I2 >= 0 && I2 < nc) {
                    // coarse rows I2 - 1 .. I2 + 1, columns I1b - 1 .. I1b + 2 of the staged box
                    const float* sc = se + (br + 1) * ECX + 2 * bc + 1;
                    float C[3][4];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) C[a][b] = sc[a * ECX + b];
                    const bool lo2 = I2 == 0, hi2 = I2 == nc - 1;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const int I1 = I1b + kk;
                        if (I1 < 0 || I1 >= nc) continue;
                        const bool lo1 = I1 == 0, hi1 = I1 == nc - 1;
                        float E[3][3];
#pragma unroll
                        for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
                            for (int dx = -1; dx <= 1; ++dx) {
                                const bool ry = (dy < 0 && lo2) || (dy > 0 && hi2);
                                const bool rx = (dx < 0 && lo1) || (dx > 0 && hi1);
                                const float a = rx ? C[1 + dy][kk + 1] : C[1 + dy][kk + 1 + dx];
                                const float b = rx ? C[1][kk + 1] : C[1][kk + 1 + dx];
                                const float v = ry ? b : a;
                                E[dy + 1][dx + 1] = (ry != rx) ? -v : v;
                            }
                        }
#pragma unroll
                        for (int fy2 = 0; fy2 < 2; ++fy2) {
#pragma unroll
                            for (int fx2 = 0; fx2 < 2; ++fx2) {
                                const int dy = 2 * fy2, dx = 2 * fx2;  // -1 -> 0, +1 -> 2 in E
                                uu[fy2][2 * kk + fx2] +=
                                    fmaf(0.5625f, E[1][1], fmaf(0.1875f, E[1][dx] + E[dy][1], 0.0625f * E[dy][dx]));
                            }
                        }
                    }
                }
                if (owner) {
#pragma unroll
                    for (int r = 0; r < 2; ++r)
                        *reinterpret_cast<float4*>(su + uix(sy0 + r, sx0)) =
                            make_float4(uu[r][0], uu[r][1], uu[r][2], uu[r][3]);
                }
                __syncthreads();
            }

            // one update: neighbours west, east, north, south (operand order of
            // the other smoothers' update)
            auto upd = [&](int r, int k, float uw, float ue, float un, float us) {
                float acc = cb[r][k];
                acc += fx[r][k] * uw;
                acc += fx[r][k + 1] * ue;
                acc += fy[r][k] * un;
                acc += fy[r + 1][k] * us;
                uu[r][k] = acc * id[r][k];
            };
            // half sweep of colour C: cells (sx + sy) % 2 == C, i.e. k = C, C + 2
            // in row 0 of the block and k = 1 - C, 3 - C in row 1
            auto half = [&](auto colour) {
                constexpr int C = decltype(colour)::value;
                float ab[4] = {0.f, 0.f, 0.f, 0.f}, bl[4] = {0.f, 0.f, 0.f, 0.f};
                if (owner) {
                    const float4 a = *reinterpret_cast<const float4*>(su + uix(sy0 - 1, sx0));
                    const float4 b = *reinterpret_cast<const float4*>(su + uix(sy0 + 2, sx0));
                    ab[0] = a.x, ab[1] = a.y, ab[2] = a.z, ab[3] = a.w;
                    bl[0] = b.x, bl[1] = b.y, bl[2] = b.z, bl[3] = b.w;
                }
                if constexpr (C == 0) {
                    // row 0 needs the west neighbour of k = 0, row 1 the east one of k = 3
                    float l0 = __shfl_up_sync(kFull, uu[0][3], 1);
                    float r1 = __shfl_down_sync(kFull, uu[1][0], 1);
                    if (lsm) l0 = su[uix(sy0, sx0 - 1)];
                    if (rsm) r1 = su[uix(sy0 + 1, sx0 + 4)];
                    upd(0, 0, l0, uu[0][1], ab[0], uu[1][0]);
                    upd(0, 2, uu[0][1], uu[0][3], ab[2], uu[1][2]);
                    upd(1, 1, uu[1][0], uu[1][2], uu[0][1], bl[1]);
                    upd(1, 3, uu[1][2], r1, uu[0][3], bl[3]);
                } else {
                    float r0 = __shfl_down_sync(kFull, uu[0][0], 1);
                    float l1 = __shfl_up_sync(kFull, uu[1][3], 1);
                    if (rsm) r0 = su[uix(sy0, sx0 + 4)];
                    if (lsm) l1 = su[uix(sy0 + 1, sx0 - 1)];
                    upd(0, 1, uu[0][0], uu[0][2], ab[1], uu[1][1]);
                    upd(0, 3, uu[0][2], r0, ab[3], uu[1][3]);
                    upd(1, 0, l1, uu[1][1], uu[0][0], bl[0]);
                    upd(1, 2, uu[1][1], uu[1][3], uu[0][2], bl[2]);
                }
                // the other colour's values in these rows are rewritten unchanged,
                // so readers of them in this half sweep see the same value
                if (owner) {
#pragma unroll
                    for (int r = 0; r < 2; ++r)
                        *reinterpret_cast<float4*>(su + uix(sy0 + r, sx0)) =
                            make_float4(uu[r][0], uu[r][1], uu[r][2], uu[r][3]);
                }
                __syncthreads();
            };
#pragma unroll
            for (int ph = 0; ph < HN; ++ph) {
                if ((first + ph) & 1) half(Colour<1>());
                else half(Colour<0>());
            }
            if constexpr (RR) {
                // residual b - A u (flux form, u = 0 across the boundary, where the
                // face holds 2 k) and its 2 x 2 restriction (the right-hand side of
                // level t - 1). The colour of the last half sweep has a zero
                // residual (its update solved each of its equations with the other
                // colour fixed), so only the other colour's cells are formed: in
                // row r of the block the cells k with (k + r) % 2 != L, L the last
                // colour; each coarse cell has one of them in each of its rows.
                auto restrict_rr = [&](auto last) {
                    constexpr int L = decltype(last)::value;
                    float ab[4] = {0.f, 0.f, 0.f, 0.f}, bl[4] = {0.f, 0.f, 0.f, 0.f};
                    if (owner) {
                        const float4 a = *reinterpret_cast<const float4*>(su + uix(sy0 - 1, sx0));
                        const float4 b = *reinterpret_cast<const float4*>(su + uix(sy0 + 2, sx0));
                        ab[0] = a.x, ab[1] = a.y, ab[2] = a.z, ab[3] = a.w;
                        bl[0] = b.x, bl[1] = b.y, bl[2] = b.z, bl[3] = b.w;
                    }
                    // row 0 forms k = 1 - L, 3 - L (the west neighbour of k = 0 when
                    // L = 1), row 1 forms k = L, L + 2 (the east one of k = 3 when L = 1)
                    float s0, s1;
                    if constexpr (L == 1) {
                        s0 = __shfl_up_sync(kFull, uu[0][3], 1);
                        s1 = __shfl_down_sync(kFull, uu[1][0], 1);
                        if (lsm) s0 = su[uix(sy0, sx0 - 1)];
                        if (rsm) s1 = su[uix(sy0 + 1, sx0 + 4)];
                    } else {
                        s0 = __shfl_down_sync(kFull, uu[0][0], 1);
                        s1 = __shfl_up_sync(kFull, uu[1][3], 1);
                        if (rsm) s0 = su[uix(sy0, sx0 + 4)];
                        if (lsm) s1 = su[uix(sy0 + 1, sx0 - 1)];
                    }
                    if (core) {
                        const float ih2 = static_cast<float>(n) * static_cast<float>(n);
                        float res[2][2];  // [row][coarse cell]
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                const int k = 2 * kk + ((r + L + 1) & 1);
                                const float sd = r == 0 ? s0 : s1;
                                const float up = uu[r][k];
                                const float uw = k == 0 ? sd : uu[r][k > 0 ? k - 1 : 0];
                                const float ue = k == 3 ? sd : uu[r][k < 3 ? k + 1 : 3];
                                const float un = r == 0 ? ab[k] : uu[0][k];
                                const float us = r == 1 ? bl[k] : uu[1][k];
                                float acc = fx[r][k] * (up - uw);
                                acc += fx[r][k + 1] * (up - ue);
                                acc += fy[r][k] * (up - un);
                                acc += fy[r + 1][k] * (up - us);
                                res[r][kk] = (cb[r][k] - acc) * ih2;
                            }
                        }
                        const int nc = n >> 1;
                        float* bco = at<float>(A.lv[t - 1].bc, i);
                        const float2 o = make_float2(0.25f * (res[0][0] + res[1][0]), 0.25f * (res[0][1] + res[1][1]));
                        *reinterpret_cast<float2*>(bco + static_cast<size_t>((y0 - kH) / 2 + br) * nc + (x0 - kH) / 2 +
                                                   2 * bc) = o;
                    }
                };
                if ((first + HN - 1) & 1) restrict_rr(Colour<1>());
                else restrict_rr(Colour<0>());
            }
            if (core) {
                float* uo = at<float>(A.lv[t].u2, i);
#pragma unroll
                for (int r = 0; r < 2; ++r)
                    *reinterpret_cast<float4*>(uo + static_cast<size_t>(y0 - kH + sy0 + r) * n + x0 - kH + sx0) =
                        make_float4(uu[r][0], uu[r][1], uu[r][2], uu[r][3]);
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

// Band form for sides of 128 and more: tiles of 56 x TY cells (the last tile
// of a row shifted left to end at the domain's edge, so that it overlaps its
// neighbour; both compute the shared cells from the same inputs in the same
// order and write identical values), whose 64-column frame is one warp wide.
// Warp w owns frame rows 4 w .. 4 w + 3, lane l columns 2 l, 2 l + 1: a cell's
// left and right neighbours come from the same thread or a warp shuffle, its
// vertical ones from the same thread except in a band's first and last row,
// which are exchanged through shared memory. The frame edge's outer
// neighbours (the extra ring of u) are read from shared memory in the first
// half sweep only: later half sweeps only need them for cells that are no
// longer exact.
template <int TY, bool POST>
struct BGeom {
    static constexpr int TX = 56;
    static constexpr int SX = TX + 2 * kH;         // 64 frame columns: 32 lanes x 2
    static constexpr int SY = TY + 2 * kH;
    static constexpr int XW = SX + 4;
    static constexpr int ECX = TX / 2 + 2 * kH;
    static constexpr int ECY = TY / 2 + 2 * kH;
    static constexpr int UP = SX + 8;
    static constexpr int UR = SY + 2;
    static constexpr int bands = SY / 4;
    static constexpr int threads = 32 * bands;
    static constexpr int oU = 0;
    static constexpr int oB = oU + round32(UP * UR);
    static constexpr int oKX = oB + round32(SX * SY);
    static constexpr int oKY = oKX + round32(XW * SY);
    static constexpr int oE = oKY + round32((SY + 1) * SX);
    static constexpr int buf = oE + (POST ? round32(ECX * ECY) : 0);
    static constexpr size_t bytes = 128 + 2 * sizeof(float) * static_cast<size_t>(buf);
    static constexpr int by_smem = static_cast<int>(kSmemPerSM / (bytes + 1024));
    static constexpr int ctas_per_sm = by_smem < 2048 / threads ? by_smem : 2048 / threads;
    static_assert(SX == 64 && SY % 4 == 0 && TY % 4 == 0, "one warp per 4-row band of a 64-column frame");
    static_assert((SX * 4) % 16 == 0 && (XW * 4) % 16 == 0 && (ECX * 4) % 16 == 0 && (UP * 4) % 16 == 0,
                  "TMA boxes: 16-byte rows");
    static_assert(ctas_per_sm >= 1, "shared memory");
};

template <int TY, int NS, bool POST, bool RR>
__global__ void __launch_bounds__(BGeom<TY, POST>::threads, BGeom<TY, POST>::ctas_per_sm)
    kb_rbgs_tma_band(const __grid_constant__ Maps maps, FmgArgs A, int t, int B, int ones, int first, int zin)
{
    using Gm = BGeom<TY, POST>;
    constexpr int TX = Gm::TX, SX = Gm::SX, SY = Gm::SY, XW = Gm::XW, ECX = Gm::ECX, UP = Gm::UP;
    constexpr int kThreads = Gm::threads;
    constexpr int HN = 2 * NS;
    static_assert(HN <= kH, "the tile and one ring around it end exact");
    static_assert(!(POST && RR), "the correction is fused into post-smoothing, the residual into pre-smoothing");
    auto uix = [](int sy, int sx) { return (sy + 1) * UP + sx + 4; };
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
    float* bufs = reinterpret_cast<float*>(smraw + 128);

    const int n = A.lv[t].n;
    const int txn = (n + TX - 1) / TX, tyn = n / TY;
    const int per = txn * tyn;
    const int total = B * per;
    const float h2 = 1.0f / (static_cast<float>(n) * static_cast<float>(n));
    const uint32_t tx_bytes =
        4u * ((zin ? 0 : UP * Gm::UR) + XW * SY + (SY + 1) * SX + (ones ? 0 : SX * SY) + (POST ? ECX * Gm::ECY : 0));

    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
    }
    __syncthreads();

    // the last tile of a row ends at the domain's edge
    auto x_of = [&](int tx) { return tx * TX < n - TX ? tx * TX : n - TX; };
    auto issue = [&](int i, int ty, int tx, int slot) {
        const int x0 = x_of(tx), y0 = ty * TY;
        float* S = bufs + slot * Gm::buf;
        uint64_t* bar = &full[slot];
        mbar_arrive_tx(bar, tx_bytes);
        if (!zin) tensor_load_3d(S + Gm::oU, &maps.u, bar, x0 - kH - 4, y0 - kH - 1, i);
        tensor_load_3d(S + Gm::oKX, &maps.kx, bar, x0 - kH, y0 - kH, i);
        tensor_load_3d(S + Gm::oKY, &maps.ky, bar, x0 - kH, y0 - kH, i);
        if (!ones) tensor_load_3d(S + Gm::oB, &maps.b, bar, x0 - kH, y0 - kH, i);
        if (POST) tensor_load_3d(S + Gm::oE, &maps.e, bar, x0 / 2 - kH, y0 / 2 - kH, i);
    };

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int sy0 = 4 * w, sx0 = 2 * lane;
    const bool core = w >= kH / 4 && w < kH / 4 + TY / 4 && lane >= kH / 2 && lane < kH / 2 + TX / 2;

    const TileWalk walk(txn, tyn);
    int ci, cty, ctx;
    walk.split(blockIdx.x, ci, cty, ctx);
    int ni = ci, nty = cty, ntx = ctx;
    bool live = true;
    int issued = 0;
    if (threadIdx.x == 0 && static_cast<int>(blockIdx.x) < total) {
        issue(ci, cty, ctx, 0);
        issued = 1;
    }
    int it = 0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
        const int slot = it & 1;
        const int next = tile + gridDim.x;
        walk.advance(ni, nty, ntx);
        if (threadIdx.x == 0 && next < total) {
            issue(ni, nty, ntx, slot ^ 1);
            ++issued;
        }
        if (live) live = mbar_wait(&full[slot], (it >> 1) & 1, A.status, kStatusTimeout);
        const int i = ci, x0 = x_of(ctx), y0 = cty * TY;
        ci = ni, cty = nty, ctx = ntx;
        if (!(A.active && !A.active[i])) {
            float* S = bufs + slot * Gm::buf;
            float* su = S + Gm::oU;
            if (zin) {
                float4* s4 = reinterpret_cast<float4*>(su);
                for (int q = threadIdx.x; q < UP * Gm::UR / 4; q += kThreads) s4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                __syncthreads();
            }
            const float* sb = S + Gm::oB;
            const float* skx = S + Gm::oKX;
            const float* sky = S + Gm::oKY;

            // the thread's 2 x 4 cells: u, x faces (w of column j = fx[r][j], e =
            // fx[r][j + 1]), y faces (north fy[r][j], south fy[r + 1][j]), h^2 b
            // and the reciprocal diagonal, both zero outside the domain
            float uu[4][2], fx[4][3], fy[5][2], cb[4][2], id[4][2];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float2 v = *reinterpret_cast<const float2*>(su + uix(sy0 + r, sx0));
                uu[r][0] = v.x, uu[r][1] = v.y;
                const float2 kv = *reinterpret_cast<const float2*>(skx + (sy0 + r) * XW + sx0);
                fx[r][0] = kv.x, fx[r][1] = kv.y;
                fx[r][2] = __shfl_down_sync(kFull, kv.x, 1);
                if (lane == 31) fx[r][2] = skx[(sy0 + r) * XW + SX];
            }
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const float2 v = *reinterpret_cast<const float2*>(sky + (sy0 + j) * SX + sx0);
                fy[j][0] = v.x, fy[j][1] = v.y;
            }
            float bv[4][2];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                bv[r][0] = bv[r][1] = 1.0f;
                if (!ones) {
                    const float2 v = *reinterpret_cast<const float2*>(sb + (sy0 + r) * SX + sx0);
                    bv[r][0] = v.x, bv[r][1] = v.y;
                }
            }
            // cells outside the domain get a zero reciprocal diagonal, so that
            // they stay 0 (their h^2 b is finite: the TMA's zero fill, or 1);
            // the column and row tests only where the tile's frame leaves the
            // domain on that axis (tile-uniform)
            auto diag = [&](auto cols_in, auto rows_in) {
                constexpr bool CA = decltype(cols_in)::value, RA = decltype(rows_in)::value;
                const int gy0 = y0 - kH + sy0, gx0 = x0 - kH + sx0;
                bool ci[2], ri[4];
#pragma unroll
                for (int j = 0; j < 2; ++j) ci[j] = CA || static_cast<unsigned>(gx0 + j) < static_cast<unsigned>(n);
#pragma unroll
                for (int r = 0; r < 4; ++r) ri[r] = RA || static_cast<unsigned>(gy0 + r) < static_cast<unsigned>(n);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const float d = fx[r][j] + fx[r][j + 1] + fy[r][j] + fy[r + 1][j];
                        const float q = __fdividef(1.0f, d);
                        id[r][j] = (CA || ci[j]) && (RA || ri[r]) ? q : 0.0f;
                        cb[r][j] = h2 * bv[r][j];
                    }
                }
            };
            {
                const bool ax = x0 >= kH && x0 + TX + kH <= n, ay = y0 >= kH && y0 + TY + kH <= n;
                if (ax && ay) diag(Flag<true>(), Flag<true>());
                else if (ay) diag(Flag<false>(), Flag<true>());
                else if (ax) diag(Flag<true>(), Flag<false>());
                else diag(Flag<false>(), Flag<false>());
            }
            if constexpr (POST) {
                // coarse-grid correction (odd reflection at the coarse boundary, as
                // in the square-block form): the thread's two columns share the
                // coarse column I1, its rows 0-1 and 2-3 the coarse rows I2a, I2a + 1
                const float* se = S + Gm::oE;
                const int nc = n >> 1;
                const int I1 = (x0 - kH) / 2 + lane, I2a = (y0 - kH) / 2 + 2 * w;
                // away from the coarse boundary (every parent and its neighbours
                // inside the coarse grid) no reflection is needed
                const bool inx = x0 >= 6 && x0 + TX + 6 <= n, iny = y0 >= 6 && y0 + TY + 6 <= n;
                auto correct = [&](auto reflect_x, auto reflect_y) {
                    constexpr bool RX = decltype(reflect_x)::value, RY = decltype(reflect_y)::value;
                    if (RX && (I1 < 0 || I1 >= nc)) return;
                    const float* sc = se + (2 * w + 1) * ECX + lane + 1;  // coarse (I2a - 1, I1 - 1)
                    float C[4][3];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) C[a][b] = sc[a * ECX + b];
                    // the odd reflection written into the coarse block: a ghost
                    // column is minus the boundary column beside it, then a ghost
                    // row minus the row beside it (so a ghost corner is plus the
                    // boundary cell); row a holds coarse row I2a - 1 + a
                    if constexpr (RX) {
                        if (I1 == 0) {
#pragma unroll
                            for (int a = 0; a < 4; ++a) C[a][0] = -C[a][1];
                        }
                        if (I1 == nc - 1) {
#pragma unroll
                            for (int a = 0; a < 4; ++a) C[a][2] = -C[a][1];
                        }
                    }
                    if constexpr (RY) {
#pragma unroll
                        for (int a = 2; a >= 0; --a)
                            if (I2a - 1 + a < 0) {
#pragma unroll
                                for (int b = 0; b < 3; ++b) C[a][b] = -C[a + 1][b];
                            }
#pragma unroll
                        for (int a = 1; a < 4; ++a)
                            if (I2a - 1 + a >= nc) {
#pragma unroll
                                for (int b = 0; b < 3; ++b) C[a][b] = -C[a - 1][b];
                            }
                    }
#pragma unroll
                    for (int pr = 0; pr < 2; ++pr) {
                        const int I2 = I2a + pr;
                        if (RY && (I2 < 0 || I2 >= nc)) continue;
#pragma unroll
                        for (int fy2 = 0; fy2 < 2; ++fy2) {
#pragma unroll
                            for (int fx2 = 0; fx2 < 2; ++fx2) {
                                const int dy = 2 * fy2, dx = 2 * fx2;  // E[i][j] = C[pr + i][j]
                                uu[2 * pr + fy2][fx2] +=
                                    fmaf(0.5625f, C[pr + 1][1],
                                         fmaf(0.1875f, C[pr + 1][dx] + C[pr + dy][1], 0.0625f * C[pr + dy][dx]));
                            }
                        }
                    }
                };
                if (inx && iny) correct(Flag<false>(), Flag<false>());
                else if (iny) correct(Flag<true>(), Flag<false>());
                else if (inx) correct(Flag<false>(), Flag<true>());
                else correct(Flag<true>(), Flag<true>());
                *reinterpret_cast<float2*>(su + uix(sy0, sx0)) = make_float2(uu[0][0], uu[0][1]);
                *reinterpret_cast<float2*>(su + uix(sy0 + 3, sx0)) = make_float2(uu[3][0], uu[3][1]);
                __syncthreads();
            }

            auto upd = [&](int r, int j, float uw, float ue, float un, float us) {
                float acc = cb[r][j];
                acc += fx[r][j] * uw;
                acc += fx[r][j + 1] * ue;
                acc += fy[r][j] * un;
                acc += fy[r + 1][j] * us;
                uu[r][j] = acc * id[r][j];
            };
            // half sweep of colour C: in row r of the band the cell of column
            // j = (C + r) % 2; edge: read the frame's outer ring (first half sweep)
            auto half = [&](auto colour, bool edge) {
                constexpr int C = decltype(colour)::value;
                float side[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (((C + r) & 1) == 0) {
                        side[r] = __shfl_up_sync(kFull, uu[r][1], 1);  // west neighbour of column 0
                        if (edge && lane == 0) side[r] = su[uix(sy0 + r, -1)];
                    } else {
                        side[r] = __shfl_down_sync(kFull, uu[r][0], 1);  // east neighbour of column 1
                        if (edge && lane == 31) side[r] = su[uix(sy0 + r, SX)];
                    }
                }
                const float above = su[uix(sy0 - 1, sx0 + C)];
                const float below = su[uix(sy0 + 4, sx0 + 1 - C)];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int j = (C + r) & 1;
                    const float uw = j == 0 ? side[r] : uu[r][0];
                    const float ue = j == 0 ? uu[r][1] : side[r];
                    const float un = r == 0 ? above : uu[r > 0 ? r - 1 : 0][j];
                    const float us = r == 3 ? below : uu[r < 3 ? r + 1 : 3][j];
                    upd(r, j, uw, ue, un, us);
                }
                *reinterpret_cast<float2*>(su + uix(sy0, sx0)) = make_float2(uu[0][0], uu[0][1]);
                *reinterpret_cast<float2*>(su + uix(sy0 + 3, sx0)) = make_float2(uu[3][0], uu[3][1]);
                __syncthreads();
            };
#pragma unroll
            for (int ph = 0; ph < HN; ++ph) {
                if ((first + ph) & 1) half(Colour<1>(), ph == 0);
                else half(Colour<0>(), ph == 0);
            }
            if constexpr (RR) {
                // residual b - A u (flux form, u = 0 across the boundary, where the
                // face holds 2 k) and its 2 x 2 restriction (the right-hand side of
                // level t - 1). The colour of the last half sweep has a zero
                // residual (its update solved each of its equations with the other
                // colour fixed), so only the other colour's cells are formed: in
                // row r the cell of column (L + 1 + r) % 2, L the last colour.
                auto restrict_rr = [&](auto last) {
                    constexpr int L = decltype(last)::value;
                    float side[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        side[r] = ((L + 1 + r) & 1) == 0 ? __shfl_up_sync(kFull, uu[r][1], 1)
                                                         : __shfl_down_sync(kFull, uu[r][0], 1);
                    const float above = su[uix(sy0 - 1, sx0 + ((L + 1) & 1))];
                    const float below = su[uix(sy0 + 4, sx0 + (L & 1))];
                    if (core) {
                        const float ih2 = static_cast<float>(n) * static_cast<float>(n);
                        float res[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int j = (L + 1 + r) & 1;
                            const float up = uu[r][j];
                            const float uw = j == 0 ? side[r] : uu[r][0];
                            const float ue = j == 0 ? uu[r][1] : side[r];
                            const float un = r == 0 ? above : uu[r > 0 ? r - 1 : 0][j];
                            const float us = r == 3 ? below : uu[r < 3 ? r + 1 : 3][j];
                            float acc = fx[r][j] * (up - uw);
                            acc += fx[r][j + 1] * (up - ue);
                            acc += fy[r][j] * (up - un);
                            acc += fy[r + 1][j] * (up - us);
                            res[r] = (cb[r][j] - acc) * ih2;
                        }
                        const int nc = n >> 1;
                        float* bco = at<float>(A.lv[t - 1].bc, i);
#pragma unroll
                        for (int pr = 0; pr < 2; ++pr)
                            bco[static_cast<size_t>((y0 - kH) / 2 + 2 * w + pr) * nc + (x0 - kH) / 2 + lane] =
                                0.25f * (res[2 * pr] + res[2 * pr + 1]);
                    }
                };
                if ((first + HN - 1) & 1) restrict_rr(Colour<1>());
                else restrict_rr(Colour<0>());
            }
            if (core) {
                float* uo = at<float>(A.lv[t].u2, i);
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    *reinterpret_cast<float2*>(uo + static_cast<size_t>(y0 - kH + sy0 + r) * n + x0 - kH + sx0) =
                        make_float2(uu[r][0], uu[r][1]);
            }
        }
        fence_proxy_async();
        __syncthreads();
    }
    if (threadIdx.x == 0 && !live) {
        const uint64_t t0 = now_ns();
        for (int k = issued - 2 < 0 ? 0 : issued - 2; k < issued; ++k)
            while (!mbar_test(&full[k & 1], (k >> 1) & 1) && now_ns() - t0 < 1000000000ull) {
            }
    }
}

using mlqmc_tmap::encode_3d;
using mlqmc_tmap::encode_fn;

template <int TX, int TY, int NS, bool POST, bool RR = false>
bool attr()
{
    return cudaFuncSetAttribute(kb_rbgs_tma<TX, TY, NS, POST, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TGeom<TX, TY, POST>::bytes)) == cudaSuccess;
}

template <int TY, int NS, bool POST, bool RR = false>
bool battr()
{
    return cudaFuncSetAttribute(kb_rbgs_tma_band<TY, NS, POST, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(BGeom<TY, POST>::bytes)) == cudaSuccess;
}

// Square-block form (32 x 32 tiles, 224 threads) for sides below 128; band
// form (56 x 32 tiles, 320 threads) from 128 on.
bool attrs()
{
    return attr<32, 32, 1, false>() && attr<32, 32, 1, true>() && attr<32, 32, 2, false>() &&
           attr<32, 32, 2, true>() && attr<32, 32, 1, false, true>() && attr<32, 32, 2, false, true>() &&
           battr<32, 1, false>() && battr<32, 1, true>() && battr<32, 2, false>() && battr<32, 2, true>() &&
           battr<32, 1, false, true>() && battr<32, 2, false, true>();
}

// Persistent grid for `per` tiles per sample. A CTA takes every grid-th tile,
// so it visits per / gcd(grid, per) tile positions in turn; when that cycle
// is short (the capacity a multiple of a large part of `per`, e.g. 304 CTAs
// for the 608 tiles of a 1024 x 1024 level) the CTAs holding edge tiles
// (domain tests, reflections, the shifted last tile) hold them in every
// sample and set the launch's length. Then the largest count up to the
// capacity that shares no factor with `per` is taken instead.
int grid_of(int tiles, int per, int cap)
{
    if (tiles <= cap) return tiles;
    auto gcd = [](int a, int b) {
        while (b) {
            const int r = a % b;
            a = b;
            b = r;
        }
        return a;
    };
    if (per / gcd(cap, per) >= 8) return cap;
    for (int g = cap; g > cap - 32 && g > 0; --g)
        if (gcd(g, per) == 1) return g;
    return cap;
}

template <int TX, int TY, int NS, bool POST, bool RR>
bool run(const FmgArgs& A, int t, int n, int B, int ones, int first, int zin, int sm_count, cudaStream_t st)
{
    using Gm = TGeom<TX, TY, POST>;
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
    const int per = (n / TX) * (n / TY);
    kb_rbgs_tma<TX, TY, NS, POST, RR><<<grid_of(B * per, per, Gm::ctas_per_sm * sm_count), Gm::threads, Gm::bytes,
                                        st>>>(m, A, t, B, ones, first, zin);
    return cudaGetLastError() == cudaSuccess;
}

template <int TY, int NS, bool POST, bool RR>
bool run_band(const FmgArgs& A, int t, int n, int B, int ones, int first, int zin, int sm_count, cudaStream_t st)
{
    using Gm = BGeom<TY, POST>;
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
    const int per = ((n + Gm::TX - 1) / Gm::TX) * (n / TY);
    kb_rbgs_tma_band<TY, NS, POST, RR><<<grid_of(B * per, per, Gm::ctas_per_sm * sm_count), Gm::threads, Gm::bytes,
                                         st>>>(m, A, t, B, ones, first, zin);
    return cudaGetLastError() == cudaSuccess;
}

template <int NS>
bool go(const FmgArgs& A, int t, int n, int B, int ones, int first, bool post, int zin, bool rr, int sm_count,
        cudaStream_t st)
{
    if (n >= 128) {  // every box (up to 72 columns) within the level's extent
        if (post) return run_band<32, NS, true, false>(A, t, n, B, ones, first, 0, sm_count, st);
        if (rr) return run_band<32, NS, false, true>(A, t, n, B, ones, first, zin, sm_count, st);
        return run_band<32, NS, false, false>(A, t, n, B, ones, first, zin, sm_count, st);
    }
    if (post) return run<32, 32, NS, true, false>(A, t, n, B, ones, first, 0, sm_count, st);
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
