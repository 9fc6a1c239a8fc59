// Driven elements (delta-gap feeds) and the ground-plane excitation (device side).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace mm {

// out[(off[e] + n) nrhs + j] (+)= w[n] V[e nrhs + j] for the nel elements elems[]
// of one type (w: M complex128 entries; V: per element nrhs complex128 volts).
cudaError_t feed_axpy(const void* w, int M, const int32_t* elems, int nel, int nrhs, const int64_t* off,
                      const void* V, void* out, bool accumulate, cudaStream_t st);
// V[i nrhs + j] += c[j] V2[i nrhs + j], i < n (complex64 when single, else complex128).
cudaError_t rhs_combine(bool single, int64_t n, int nrhs, const double* c, const void* V2, void* V, cudaStream_t st);

}  // namespace mm
