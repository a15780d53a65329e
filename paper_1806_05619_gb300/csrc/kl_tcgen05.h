// Host interface of the tensor-core KL synthesis (kl_tcgen05.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace mlqmc_kl {

// Opaque storage for the two TMA descriptors of one level (CUtensorMap is 128 bytes, 64-byte aligned).
struct alignas(64) TensorMaps {
    unsigned char psi[128];
    unsigned char c[128];     // C operand in boxes of 256 sample rows
    unsigned char c128[128];  // the same in boxes of 128 sample rows
};

// Operand form: TF32 (one rounding per operand) or split BF16 (three products).
enum class Variant { TF32, BF16X3 };

int kpad_for(int s);                    // s padded to whole 32-element blocks (TF32)
int kdim_for(Variant v, int s);         // K of the GEMM: kpad_for(s), or 3 x (s padded to 64) for BF16X3
size_t row_bytes(Variant v, int s);     // bytes of one operand row (a whole number of 128-byte K blocks)
int tile_samples();                     // samples per CTA tile (the widest; launch takes 128 or 256)

// Psi of one level (n x n cells, row-major p = i2*n + i1; kdim_for(v, s) columns) from the FP64 1D tables.
bool build_psi(Variant v, const double* d_psi1d, int n, int s, const int* d_ma, const int* d_mb, void* d_out,
               cudaStream_t st);

// Psi of one level from dense FP64 modes (M cells x s, cell-major), same operand layout.
bool build_psi_dense(Variant v, const double* d_modes, int64_t M, int s, void* d_out, cudaStream_t st);

// C rows i < count: sqrt(theta_m) y_m of the sample whose normals are row canon[i] of Y (canon NULL: row i).
bool build_c(Variant v, const double* d_Y, const int* d_canon, int count, int s, const double* d_sqrt_theta,
             void* d_out, cudaStream_t st);

bool make_maps(Variant v, const void* d_psi, int M, const void* d_c, int rows_c, int s, TensorMaps* maps);
bool prepare_kernel();

// k[b * kstride + p] = exp(sum_m Psi[p][m] C[b][m]) for p < M (M a multiple of 128), b < B,
// in tiles of 128 cells x nt samples (nt 128 or 256).
bool launch(Variant v, const TensorMaps& maps, int M, int B, int s, float* d_k, size_t kstride, int* d_err,
            cudaStream_t st, int nt = 256);

}  // namespace mlqmc_kl
