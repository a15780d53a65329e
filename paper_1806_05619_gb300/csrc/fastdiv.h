// Division of 32-bit unsigned integers by a divisor fixed for a whole launch,
// by a multiply-high, an add and two shifts instead of the division
// instruction sequence: the method of Granlund and Montgomery, "Division by
// invariant integers using multiplication" (PLDI 1994), Sec. 4, Fig. 4.1,
// exact for every 32-bit dividend. The multiplier is formed once on the host
// and travels in the level descriptor of the kernels' arguments.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define MLQMC_HD __host__ __device__
#else
#define MLQMC_HD
#endif

namespace mlqmc_dev {

struct FastDiv {
    uint32_t m = 1;    // m' = floor(2^32 (2^l - d) / d) + 1, l = ceil(log2 d)
    uint32_t sh1 = 0;  // min(l, 1)
    uint32_t sh2 = 0;  // max(l - 1, 0)

    FastDiv() = default;
    // d >= 1
    explicit FastDiv(uint32_t d)
    {
        uint32_t l = 0;
        while (l < 32 && (uint64_t{1} << l) < d) ++l;
        m = static_cast<uint32_t>(((uint64_t{1} << 32) * ((uint64_t{1} << l) - d)) / d + 1);
        sh1 = l < 1 ? l : 1;
        sh2 = l > 1 ? l - 1 : 0;
    }

    MLQMC_HD uint32_t div(uint32_t x) const
    {
#if defined(__CUDA_ARCH__)
        const uint32_t t = __umulhi(m, x);
#else
        const uint32_t t = static_cast<uint32_t>((static_cast<uint64_t>(m) * x) >> 32);
#endif
        return (t + ((x - t) >> sh1)) >> sh2;
    }
};

}  // namespace mlqmc_dev
