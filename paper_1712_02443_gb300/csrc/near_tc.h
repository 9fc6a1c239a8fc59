// Block near field on tensor cores (TF32 with a three-product split, FP32
// accumulation): v -= G_NF u over the translation-invariant blocks.
#pragma once

#include <cuda_runtime.h>

#include "device.h"

namespace mm {

// Kernel shapes: 0 = 32 complex columns per tile (MMA N 64, three stages),
// 1 = 64 complex columns per tile (MMA N 128, two stages).
constexpr int kNearTcShapes = 2;

// Function attributes and the device address of the kernel's error flag
// (a.near_err), once per array (the array's device current).
cudaError_t near_tc_init(DevArray& a);
// v -= G_NF u: the tensor-core products of all blocks into the partial-sum
// buffer P (a.nfg_prows x nrhs complex), then the per-element reduction into v.
cudaError_t near_tc_launch(int shape, const DevArray& a, const DevPrec<float>& p, int nrhs, const float2* u,
                           float2* v, float2* P, cudaStream_t st);
// TF32 hi / lo parts (round to nearest even) of a complex entry given in FP64.
void near_tc_split(double re, double im, float* hi, float* lo);

}  // namespace mm
