// Tensor-core (tcgen05) macromodel GEMM, BF16/FP16 inputs, FP32 accumulation.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>

namespace mm {

int tc_tile_m();
int tc_tile_n();
int tc_tile_k();
size_t tc_smem_bytes();
// Offset of the imaginary half in the K dimension of both operands (Nh rounded up to 8).
int tc_k_split(int Nh);
// CTAs per cluster along M (1, the default: no multicast; 2: B slices multicast to both).
void tc_set_cluster(int cm);
cudaError_t tc_gemm_init();
// u, v (complex64) = [M; D] x for the elements of one type.  A: packed real
// operator (Mp x Kp, 16-bit, K-major); Bt: scratch for the packed right-hand
// side (capacity bt_cap elements); err: device flag set if a wait expired.
cudaError_t tc_macro_gemm(bool bf16, const uint16_t* A, int Mp, int Kp, int Nh, const int32_t* elems, int nel,
                          int nrhs, const int64_t* off, const float2* x, uint16_t* Bt, size_t bt_cap, float2* u,
                          float2* v, int* err, cudaStream_t st);

}  // namespace mm
