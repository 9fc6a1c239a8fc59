// Block near field on tensor cores (TF32 with a three-product split, FP32
// accumulation): v -= G_NF u over the translation-invariant blocks.
#pragma once

#include <cuda_runtime.h>

#include "device.h"

namespace mm {

// Kernel shapes: 0 = 32 complex columns per tile (MMA N 64, four stages),
// 1 = 64 complex columns per tile (MMA N 128, three stages); both with columns
// = (element pair, right-hand side) and partial sums.  2, 3 = the direct form
// (columns = right-hand sides of one element, 32 or 64 per tile, accumulated
// over the element's pairs and subtracted from v in place); it needs an even
// right-hand-side count and 16-byte aligned u and v (near_tc_direct_ok).  4 =
// the direct form with 64 right-hand sides and two stages (153 KB of shared
// memory instead of 222 KB: an FFT block fits beside it on an SM).
constexpr int kNearTcShapes = 5;

// Function attributes and the device address of the kernel's error flag
// (a.near_err), once per array (the array's device current).
cudaError_t near_tc_init(DevArray& a);
// v -= G_NF u: shapes 0, 1: the tensor-core products of all blocks into the
// partial-sum buffer P (a.nfg_prows x nrhs complex), then the per-element
// reduction into v; shapes 2, 3: into v directly (P unused).
bool near_tc_direct_ok(const DevArray& a, int nrhs, const void* u, const void* v);
// ks (1 or 2, shapes 0 and 1): each unit's k tiles split over ks units, whose
// partial sums go to ks planes of P (P then holds ks a.nfg_prows x nrhs).
cudaError_t near_tc_launch(int shape, const DevArray& a, const DevPrec<float>& p, int nrhs, const float2* u,
                           float2* v, float2* P, int ks, cudaStream_t st);
// TF32 hi / lo parts (round to nearest even) of a complex entry given in FP64.
void near_tc_split(double re, double im, float* hi, float* lo);

}  // namespace mm
