// FMG interpolation of a level and its first refinement residual (mixed
// forms, Sec. 4 with the FP64 refinement around the FP32 V-cycles), fed by
// the TMA.
//
// Persistent CTAs walk 64 x 32 fine tiles (32 x 16 coarse parents) of one
// level, tiles of a sample consecutive. For each tile one thread issues three
// 3D tensor copies into one of two shared-memory buffers while the other is
// used: the coarse parents with one more coarse cell around them (four more
// columns on each side, so that the copy's x origin stays on a 16-byte
// boundary), the tile's x faces and its y faces. Each thread then takes two
// parents, i.e. two 2 x 2 quads of fine cells: the quad and its ring of eight
// fine neighbours interpolate from the 3 x 3 coarse block around the parent
// (odd reflection across the coarse boundary: a fine cell's out-of-range
// coarse neighbour is minus the value in its parent's own row or column), and
// each quad cell's residual 1 - A u64 is formed from FP32 error-free pairs
// (resid_f32x2) and rounded once to FP32; u64 gets the widened interpolant
// (interp32: the FP32 interpolant goes to the level's field array instead,
// for the fixed-cycle forms whose refinement update reads it only as FP32).
// The operations are those of the grid-stride form, value for value, so the
// two give the same bits; this one reads every input once per tile from
// shared memory instead of global memory.
#include "resid_tma.h"

#include <cstdint>
#include <cstring>

#include "ptx_async.cuh"
#include "tma_encode.h"

using namespace mlqmc_dev;
using namespace mlqmc_ptx;

namespace {

constexpr int kCX = 32, kCY = 16;             // coarse parents per tile
constexpr int kFX = 2 * kCX, kFY = 2 * kCY;   // fine cells per tile
constexpr int kEW = kCX + 8, kEH = kCY + 2;   // staged coarse box (x from the tile's first parent - 4, y - 1)
constexpr int kXW = kFX + 4;                  // staged x faces per fine row (65 used)
constexpr int kThreads = 256;                 // two parents per thread
constexpr int kSmemPerSM = 233472;

constexpr int round32(int v) { return (v + 31) / 32 * 32; }
constexpr int oE = 0;
constexpr int oKX = oE + round32(kEW * kEH);
constexpr int oKY = oKX + round32(kXW * kFY);
constexpr int kBuf = oKY + round32(kFX * (kFY + 1));  // floats per buffer
constexpr size_t kBytes = 128 + 2 * sizeof(float) * static_cast<size_t>(kBuf);
constexpr int kCtasPerSM = 4;  // 64 registers per thread
static_assert(kCtasPerSM * (kBytes + 1024) <= static_cast<size_t>(kSmemPerSM), "shared memory");
static_assert(kCX * kCY == 2 * kThreads && kCX == 32, "a warp takes one row of 32 parents");
static_assert((kEW * 4) % 16 == 0 && (kXW * 4) % 16 == 0 && (kFX * 4) % 16 == 0, "TMA boxes: 16-byte rows");

struct Maps {
    CUtensorMap e, kx, ky;
};

template <bool V>
struct Edge {
    static constexpr bool value = V;
};

__global__ void __launch_bounds__(kThreads, kCtasPerSM)
    kb_prolong_resid_tma(const __grid_constant__ Maps maps, FmgArgs A, int t, int B, int interp32)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
    float* bufs = reinterpret_cast<float*>(smraw + 128);

    const int n = A.lv[t].n, nc = n >> 1;
    const int txn = nc / kCX, tyn = nc / kCY;
    const int per = txn * tyn;
    const int total = B * per;
    const float ih2 = static_cast<float>(n) * static_cast<float>(n);
    constexpr uint32_t kTx = 4u * (kEW * kEH + kXW * kFY + kFX * (kFY + 1));

    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue = [&](int i, int ty, int tx, int slot) {
        const int I1 = tx * kCX, I2 = ty * kCY;
        float* S = bufs + slot * kBuf;
        uint64_t* bar = &full[slot];
        mbar_arrive_tx(bar, kTx);
        tensor_load_3d(S + oE, &maps.e, bar, I1 - 4, I2 - 1, i);
        tensor_load_3d(S + oKX, &maps.kx, bar, 2 * I1, 2 * I2, i);
        tensor_load_3d(S + oKY, &maps.ky, bar, 2 * I1, 2 * I2, i);
    };
    // (sample, tile row, tile column) of the CTA's tiles blockIdx.x,
    // blockIdx.x + gridDim.x, ...: split once, then stepped with carries
    auto split = [&](int tile, int& i, int& ty, int& tx) {
        i = tile / per;
        const int tr = tile - i * per;
        ty = tr / txn;
        tx = tr - ty * txn;
    };
    int gi, gty, gtx;
    split(static_cast<int>(gridDim.x), gi, gty, gtx);
    auto advance = [&](int& i, int& ty, int& tx) {
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
    };
    int ci, cty, ctx;
    split(static_cast<int>(blockIdx.x), ci, cty, ctx);
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
        advance(ni, nty, ntx);
        if (threadIdx.x == 0 && next < total) {
            issue(ni, nty, ntx, slot ^ 1);  // the other buffer was released by the barrier ending the last iteration
            ++issued;
        }
        if (live) live = mbar_wait(&full[slot], (it >> 1) & 1, A.status, kStatusTimeout);
        const int i = ci, I1_0 = ctx * kCX, I2_0 = cty * kCY;
        ci = ni, cty = nty, ctx = ntx;
        if (!(A.active && !A.active[i])) {  // uniform per CTA
            const float* S = bufs + slot * kBuf;
            const float* se = S + oE;
            const float* skx = S + oKX;
            const float* sky = S + oKY;
            const Lv<float> L = view<float>(A, t, i);
            // the tile's parents all lie inside the coarse grid; the reflection
            // and the zero cells outside the fine grid only on an axis where
            // the tile reaches the coarse boundary (uniform per CTA)
            const bool ex = I1_0 == 0 || I1_0 + kCX >= nc, ey = I2_0 == 0 || I2_0 + kCY >= nc;
            auto quads = [&](auto edge_x, auto edge_y) {
                constexpr bool EX = decltype(edge_x)::value, EY = decltype(edge_y)::value;
#pragma unroll 1
                for (int k = 0; k < 2; ++k) {
                    const int q = static_cast<int>(threadIdx.x) + k * kThreads;
                    const int cx = q & (kCX - 1), cy = q / kCX;
                    const int I1 = I1_0 + cx, I2 = I2_0 + cy;
                    // the quad's faces (staged fine row 2 cy + qy, column 2 cx)
                    float2 kx01[2], kyn[2], kys[2];
                    float kx2[2];
#pragma unroll
                    for (int qy = 0; qy < 2; ++qy) {
                        const int r = 2 * cy + qy, c = 2 * cx;
                        kx01[qy] = *reinterpret_cast<const float2*>(skx + r * kXW + c);
                        kx2[qy] = skx[r * kXW + c + 2];
                        kyn[qy] = *reinterpret_cast<const float2*>(sky + r * kFX + c);
                        kys[qy] = *reinterpret_cast<const float2*>(sky + (r + 1) * kFX + c);
                    }
                    float E[3][3];  // E[dy + 1][dx + 1]; parent at staged (cy + 1, cx + 4)
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx) E[dy + 1][dx + 1] = se[(cy + 1 + dy) * kEW + cx + 4 + dx];
                    // odd reflection across the coarse boundary, written into the
                    // block: a ghost column is minus the parent's column, then a
                    // ghost row minus the parent's row (a ghost corner: plus the parent)
                    if constexpr (EX) {
                        if (I1 == 0) {
#pragma unroll
                            for (int a = 0; a < 3; ++a) E[a][0] = -E[a][1];
                        }
                        if (I1 == nc - 1) {
#pragma unroll
                            for (int a = 0; a < 3; ++a) E[a][2] = -E[a][1];
                        }
                    }
                    if constexpr (EY) {
                        if (I2 == 0) {
#pragma unroll
                            for (int b = 0; b < 3; ++b) E[0][b] = -E[1][b];
                        }
                        if (I2 == nc - 1) {
#pragma unroll
                            for (int b = 0; b < 3; ++b) E[2][b] = -E[1][b];
                        }
                    }
                    // fine cells 2I + f, f = -1..2 per axis (the four ring corners unused):
                    // parent offset (f - 1) / 2 rounded down, coarse neighbour towards the
                    // cell's side (+1 for odd f, -1 for even f); cells outside the grid are 0
                    float U[4][4];
#pragma unroll
                    for (int fy = -1; fy <= 2; ++fy)
#pragma unroll
                        for (int fx = -1; fx <= 2; ++fx) {
                            const bool ring_x = fx < 0 || fx > 1, ring_y = fy < 0 || fy > 1;
                            if (ring_x && ring_y) {
                                U[fy + 1][fx + 1] = 0.0f;
                                continue;
                            }
                            const int px = fx < 0 ? -1 : (fx > 1 ? 1 : 0), py = fy < 0 ? -1 : (fy > 1 ? 1 : 0);
                            const int sx = (fx & 1) ? 1 : -1, sy = (fy & 1) ? 1 : -1;
                            const float a = E[py + 1][px + 1];
                            const float bx = E[py + 1][px + sx + 1];
                            const float cyv = E[py + sy + 1][px + 1];
                            const float d = E[py + sy + 1][px + sx + 1];
                            U[fy + 1][fx + 1] = fmaf(0.5625f, a, fmaf(0.1875f, bx + cyv, 0.0625f * d));
                        }
                    // ring cells outside the fine grid are 0 (fine cell 2 I + f, f = -1 or 2)
                    if constexpr (EX) {
                        if (I1 == 0) U[1][0] = U[2][0] = 0.0f;
                        if (I1 == nc - 1) U[1][3] = U[2][3] = 0.0f;
                    }
                    if constexpr (EY) {
                        if (I2 == 0) U[0][1] = U[0][2] = 0.0f;
                        if (I2 == nc - 1) U[3][1] = U[3][2] = 0.0f;
                    }
#pragma unroll
                    for (int qy = 0; qy < 2; ++qy) {
                        const int i1 = 2 * I1, i2 = 2 * I2 + qy;
                        const int p = i2 * n + i1;
                        float r[2];
#pragma unroll
                        for (int qx = 0; qx < 2; ++qx) {
                            const float up = U[qy + 1][qx + 1];
                            const float uv[4] = {U[qy + 1][qx], U[qy + 1][qx + 2], U[qy][qx + 1], U[qy + 2][qx + 1]};
                            const float kv[4] = {qx ? kx01[qy].y : kx01[qy].x, qx ? kx2[qy] : kx01[qy].y,
                                                 qx ? kyn[qy].y : kyn[qy].x, qx ? kys[qy].y : kys[qy].x};
                            r[qx] = resid_f32x2(kv, up, uv, ih2);
                        }
                        if (interp32)  // the interpolant in FP32, in the level's field array (no longer read)
                            *reinterpret_cast<float2*>(L.k + p) = make_float2(U[qy + 1][1], U[qy + 1][2]);
                        else
                            *reinterpret_cast<double2*>(L.u64 + p) =
                                make_double2(widen(U[qy + 1][1]), widen(U[qy + 1][2]));
                        *reinterpret_cast<float2*>(L.bc + p) = make_float2(r[0], r[1]);
                    }
                }
            };
            if (!ex && !ey) quads(Edge<false>(), Edge<false>());
            else if (!ey) quads(Edge<true>(), Edge<false>());
            else if (!ex) quads(Edge<false>(), Edge<true>());
            else quads(Edge<true>(), Edge<true>());
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

}  // namespace

namespace mlqmc_resid {

bool supported(int n)
{
    return n >= 128 && n % 64 == 0;  // whole tiles; the coarse box (40 wide) within the coarse extent
}

bool prepare()
{
    return mlqmc_tmap::encode_fn() != nullptr &&
           cudaFuncSetAttribute(kb_prolong_resid_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kBytes)) == cudaSuccess;
}

bool launch(const FmgArgs& A, int t, int n, int B, bool interp32, int sm_count, cudaStream_t st)
{
    if (B <= 0) return true;
    if (!supported(n) || t < 1 || A.lv[t].n != n) return false;
    const LevelDesc& L = A.lv[t];
    Maps m;
    std::memset(&m, 0, sizeof(m));
    const uint64_t un = static_cast<uint64_t>(n), uc = un / 2, ub = static_cast<uint64_t>(B);
    const bool ok = mlqmc_tmap::encode_3d(&m.e, A.lv[t - 1].u, uc, uc, uc, ub, kEW, kEH) &&
                    mlqmc_tmap::encode_3d(&m.kx, L.kx, un + 4, static_cast<uint64_t>(kx_pitch(n)), un, ub, kXW, kFY) &&
                    mlqmc_tmap::encode_3d(&m.ky, L.ky, un, un, un + 1, ub, kFX, kFY + 1);
    if (!ok) return false;
    const int tiles = B * (n / kFX) * (n / kFY);
    const int cap = kCtasPerSM * sm_count;
    kb_prolong_resid_tma<<<tiles < cap ? tiles : cap, kThreads, kBytes, st>>>(m, A, t, B, interp32 ? 1 : 0);
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace mlqmc_resid
