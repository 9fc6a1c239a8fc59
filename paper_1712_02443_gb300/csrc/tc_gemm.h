// Tensor-core (tcgen05) macromodel GEMM, BF16/FP16 inputs, FP32 accumulation.
#pragma once

#include <cuda.h>
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
// Testing hook: ms > 0 makes the following GEMMs issue no products and give up
// every wait after ms milliseconds (the error flag is set); 0 restores them.
void tc_set_stall(int ms);
int tc_stall_ms();
// 2-D tiled tensor map (128-byte swizzle, zero fill outside) over a row-major
// matrix of `rows` rows of `inner` elements, rows ld_bytes apart; box of
// box_inner x box_rows elements.  False if the encoder is unavailable or refuses.
bool tc_encode_2d(CUtensorMap* m, CUtensorMapDataType dtype, const void* base, uint64_t inner, uint64_t rows,
                  uint64_t ld_bytes, uint32_t box_inner, uint32_t box_rows);
cudaError_t tc_gemm_init();
// u, v (complex64) = [M; D] x for the elements of one type.  A: packed real
// operator (Mp x Kp, 16-bit, K-major); Bt: scratch for the packed right-hand
// side (capacity bt_cap elements); err: device flag set if a wait expired.
cudaError_t tc_macro_gemm(bool bf16, const uint16_t* A, int Mp, int Kp, int Nh, const int32_t* elems, int nel,
                          int nrhs, const int64_t* off, const float2* x, uint16_t* Bt, size_t bt_cap, float2* u,
                          float2* v, int* err, cudaStream_t st);

}  // namespace mm
