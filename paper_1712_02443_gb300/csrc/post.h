// Post-processing: element currents and far field (device side).
#pragma once

#include "device.h"
#include "solver.h"

namespace mm {

cudaError_t elem_gemm(const void* W, int M, int K, const int32_t* elems, int nel, int nrhs, const int64_t* in_off,
                      const void* in, const int64_t* out_off, void* out, cudaStream_t st);
cudaError_t farfield(const DevArray& a, const int32_t* elem_of, const double* const* geo, int nrhs, const void* J,
                     int64_t ndir, const double* th, const double* ph, double k0, double eta0, const QuadRule& q,
                     void* F, cudaStream_t st);

}  // namespace mm
