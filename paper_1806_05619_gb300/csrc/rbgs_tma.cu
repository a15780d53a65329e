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

template <int TILE>
struct TGeom {
    static constexpr int SU = TILE + 2 * kH;       // staged cells per side
    static constexpr int XW = SU + 4;              // staged x faces per row (box width, 16-byte multiple)
    static constexpr int EC = TILE / 2 + 2 * kH;   // staged coarse cells per side
    static constexpr int oU = 0;
    static constexpr int oB = oU + round32(SU * SU);
    static constexpr int oKX = oB + round32(SU * SU);
    static constexpr int oKY = oKX + round32(SU * XW);
    static constexpr int oE = oKY + round32((SU + 1) * SU);
    static constexpr int buf = oE + round32(EC * EC);  // floats per buffer
    static constexpr size_t bytes = 128 + 2 * sizeof(float) * static_cast<size_t>(buf);
    static_assert((SU * 4) % 16 == 0 && (XW * 4) % 16 == 0 && (EC * 4) % 16 == 0, "TMA boxes: 16-byte rows");
};

template <int TILE, int NS, bool POST>
__global__ void __launch_bounds__(kThreads, 3)
    kb_rbgs_tma(const __grid_constant__ Maps maps, FmgArgs A, int t, int B, int ones, int first)
{
    using Gm = TGeom<TILE>;
    constexpr int SU = Gm::SU, XW = Gm::XW, EC = Gm::EC;
    constexpr int HN = 2 * NS;  // halo the NS sweeps consume
    static_assert(HN <= kH, "halo");
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
    float* bufs = reinterpret_cast<float*>(smraw + 128);

    const int n = A.lv[t].n;
    const int tx_n = n / TILE;
    const int per = tx_n * tx_n;
    const int total = B * per;
    const float h2 = 1.0f / (static_cast<float>(n) * static_cast<float>(n));
    const uint32_t tx_bytes = 4u * (SU * SU + XW * SU + (SU + 1) * SU + (ones ? 0 : SU * SU) + (POST ? EC * EC : 0));

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
        tensor_load_3d(S + Gm::oU, &maps.u, bar, x0 - kH, y0 - kH, i);
        tensor_load_3d(S + Gm::oKX, &maps.kx, bar, x0 - kH, y0 - kH, i);
        tensor_load_3d(S + Gm::oKY, &maps.ky, bar, x0 - kH, y0 - kH, i);
        if (!ones) tensor_load_3d(S + Gm::oB, &maps.b, bar, x0 - kH, y0 - kH, i);
        if (POST) tensor_load_3d(S + Gm::oE, &maps.e, bar, x0 / 2 - kH, y0 / 2 - kH, i);
    };

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
            const float* sb = S + Gm::oB;
            const float* skx = S + Gm::oKX;
            const float* sky = S + Gm::oKY;
            if constexpr (POST) {
                // coarse-grid correction on every staged cell of the domain (as prolong_cell)
                const float* se = S + Gm::oE;
                const int nc = n >> 1;
                const int ex0 = x0 / 2 - kH, ey0 = y0 / 2 - kH;
                for (int q = threadIdx.x; q < SU * SU; q += kThreads) {
                    const int gy = y0 - kH + q / SU, gx = x0 - kH + q % SU;
                    if (gy < 0 || gy >= n || gx < 0 || gx >= n) continue;
                    const int I1 = gx >> 1, I2 = gy >> 1;
                    const int J1 = (gx & 1) ? I1 + 1 : I1 - 1;
                    const int J2 = (gy & 1) ? I2 + 1 : I2 - 1;
                    const bool o1 = J1 < 0 || J1 >= nc, o2 = J2 < 0 || J2 >= nc;
                    const int K1 = o1 ? I1 : J1, K2 = o2 ? I2 : J2;
                    const float a = se[(I2 - ey0) * EC + I1 - ex0];
                    const float b0 = se[(I2 - ey0) * EC + K1 - ex0];
                    const float c0 = se[(K2 - ey0) * EC + I1 - ex0];
                    const float d0 = se[(K2 - ey0) * EC + K1 - ex0];
                    const float bb = o1 ? -b0 : b0;
                    const float cc = o2 ? -c0 : c0;
                    const float dd = (o1 != o2) ? -d0 : d0;
                    su[q] += fmaf(0.5625f, a, fmaf(0.1875f, bb + cc, 0.0625f * dd));
                }
                __syncthreads();
            }
            // tiles whose grown regions stay inside the domain skip the per-cell test
            const bool interior = x0 >= HN && y0 >= HN && x0 + TILE + HN <= n && y0 + TILE + HN <= n;
#pragma unroll
            for (int ph = 0; ph < HN; ++ph) {
                const int colour = (first + ph) & 1;
                const int g = HN - 1 - ph;  // growth of the updated region beyond the tile
                const int side = TILE + 2 * g;
                const int half = side / 2;
                for (int q = threadIdx.x; q < side * half; q += kThreads) {
                    const int ry = q / half;
                    const int gy = y0 - g + ry;
                    const int rx = 2 * (q - ry * half) + ((gy + x0 - g + colour) & 1);
                    const int gx = x0 - g + rx;
                    if (!interior && (gy < 0 || gy >= n || gx < 0 || gx >= n)) continue;
                    const int sy = gy - y0 + kH, sx = gx - x0 + kH;
                    const int c0 = sy * SU + sx;
                    const float* kr = skx + sy * XW;
                    const float w = kr[sx], e = kr[sx + 1];
                    const float nn = sky[sy * SU + sx], so = sky[(sy + 1) * SU + sx];
                    float acc = h2 * (ones ? 1.0f : sb[c0]);
                    acc += w * su[c0 - 1];
                    acc += e * su[c0 + 1];
                    acc += nn * su[c0 - SU];
                    acc += so * su[c0 + SU];
                    su[c0] = __fdividef(acc, w + e + nn + so);  // hardware reciprocal: within 2 ulp
                }
                __syncthreads();
            }
            float* uo = at<float>(A.lv[t].u2, i);
            constexpr int TV = TILE / 4;
            for (int q = threadIdx.x; q < TILE * TV; q += kThreads) {
                const int ry = q / TV, v = q - (q / TV) * TV;
                const float* src = su + (ry + kH) * SU + kH + 4 * v;
                *reinterpret_cast<float4*>(uo + static_cast<size_t>(y0 + ry) * n + x0 + 4 * v) =
                    make_float4(src[0], src[1], src[2], src[3]);
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

template <int TILE, int NS, bool POST>
bool attr()
{
    return cudaFuncSetAttribute(kb_rbgs_tma<TILE, NS, POST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(TGeom<TILE>::bytes)) == cudaSuccess;
}

template <int TILE>
bool attrs()
{
    return attr<TILE, 1, false>() && attr<TILE, 1, true>() && attr<TILE, 2, false>() && attr<TILE, 2, true>();
}

template <int TILE>
bool go(const FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool post, int max_ctas, cudaStream_t st)
{
    using Gm = TGeom<TILE>;
    const LevelDesc& L = A.lv[t];
    Maps m;
    std::memset(&m, 0, sizeof(m));
    const uint64_t un = static_cast<uint64_t>(n), ub = static_cast<uint64_t>(B);
    bool ok = encode_3d(&m.u, L.u, un, un, un, ub, Gm::SU, Gm::SU) &&
              encode_3d(&m.kx, L.kx, un + 4, static_cast<uint64_t>(kx_pitch(n)), un, ub, Gm::XW, Gm::SU) &&
              encode_3d(&m.ky, L.ky, un, un, un + 1, ub, Gm::SU, Gm::SU + 1) &&
              (ones || encode_3d(&m.b, L.bc, un, un, un, ub, Gm::SU, Gm::SU)) &&
              (!post || encode_3d(&m.e, A.lv[t - 1].u, un / 2, un / 2, un / 2, ub, Gm::EC, Gm::EC));
    if (!ok) return false;
    const int tiles = B * (n / TILE) * (n / TILE);
    const int grid = tiles < max_ctas ? tiles : max_ctas;
    if (ns == 2) {
        if (post) kb_rbgs_tma<TILE, 2, true><<<grid, kThreads, Gm::bytes, st>>>(m, A, t, B, ones, first);
        else kb_rbgs_tma<TILE, 2, false><<<grid, kThreads, Gm::bytes, st>>>(m, A, t, B, ones, first);
    } else {
        if (post) kb_rbgs_tma<TILE, 1, true><<<grid, kThreads, Gm::bytes, st>>>(m, A, t, B, ones, first);
        else kb_rbgs_tma<TILE, 1, false><<<grid, kThreads, Gm::bytes, st>>>(m, A, t, B, ones, first);
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

bool launch(const FmgArgs& A, int t, int n, int B, int ns, int ones, int first, bool post, int sm_count,
            cudaStream_t st)
{
    if (B <= 0) return true;
    if (!supported(n) || t < 1 || A.lv[t].n != n || (ns != 1 && ns != 2)) return false;
    return go<32>(A, t, n, B, ns, ones, first, post, 3 * sm_count, st);
}

}  // namespace mlqmc_tma
