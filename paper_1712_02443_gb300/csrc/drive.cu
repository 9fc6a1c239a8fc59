// Driven elements and ground-plane excitation: small element-wise kernels.
//
// Delta-gap feed (Sec. VI, driven helix elements): the feed enters the
// scatterer's equation, so each driven element adds J_f V to its scatterer
// currents and its equivalent current J^_f V = T J_f V radiates into the
// exterior problem (excitation V^ - G J^_f).  feed_axpy scatters those
// per-type vectors times each element's volts into element-major vectors.
// Ground plane by image theory: the excitation of the incident wave plus its
// image is the sum of two plane-wave excitations, combined by rhs_combine.
#include "drive.h"

namespace mm {

namespace {

__global__ void __launch_bounds__(256) k_feed_axpy(const double2* __restrict__ w, int M,
                                                   const int32_t* __restrict__ elems, int nrhs,
                                                   const int64_t* __restrict__ off, const double2* __restrict__ V,
                                                   double2* __restrict__ out, int accumulate) {
  const int e = elems[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)M * nrhs) return;
  const int n = (int)(i / nrhs), j = (int)(i - (int64_t)n * nrhs);
  const double2 a = w[n], v = V[(int64_t)e * nrhs + j];
  double2 r = make_double2(fma(a.x, v.x, -a.y * v.y), fma(a.x, v.y, a.y * v.x));
  double2* d = out + (off[e] + n) * nrhs + j;
  if (accumulate) {
    r.x += d->x;
    r.y += d->y;
  }
  *d = r;
}

template <typename C>
__global__ void __launch_bounds__(256) k_rhs_combine(int64_t n, int nrhs, const double* __restrict__ c,
                                                     const C* __restrict__ V2, C* __restrict__ V) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  const int j = (int)(i % nrhs);
  const double cr = c[2 * j], ci = c[2 * j + 1];
  const C b = V2[i];
  C a = V[i];
  a.x += (decltype(a.x))(cr * b.x - ci * b.y);
  a.y += (decltype(a.y))(cr * b.y + ci * b.x);
  V[i] = a;
}

}  // namespace

cudaError_t feed_axpy(const void* w, int M, const int32_t* elems, int nel, int nrhs, const int64_t* off,
                      const void* V, void* out, bool accumulate, cudaStream_t st) {
  if (nel <= 0 || M <= 0) return cudaSuccess;
  const int64_t items = (int64_t)M * nrhs;
  for (int e0 = 0; e0 < nel; e0 += 65535) {
    const int ne = nel - e0 < 65535 ? nel - e0 : 65535;
    dim3 g((unsigned)((items + 255) / 256), (unsigned)ne);
    k_feed_axpy<<<g, 256, 0, st>>>(static_cast<const double2*>(w), M, elems + e0, nrhs, off,
                                   static_cast<const double2*>(V), static_cast<double2*>(out), accumulate ? 1 : 0);
  }
  return cudaGetLastError();
}

cudaError_t rhs_combine(bool single, int64_t n, int nrhs, const double* c, const void* V2, void* V, cudaStream_t st) {
  const int64_t items = n * nrhs;
  if (items <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((items + 255) / 256);
  if (single)
    k_rhs_combine<float2><<<blocks, 256, 0, st>>>(n, nrhs, c, static_cast<const float2*>(V2), static_cast<float2*>(V));
  else
    k_rhs_combine<double2><<<blocks, 256, 0, st>>>(n, nrhs, c, static_cast<const double2*>(V2),
                                                   static_cast<double2*>(V));
  return cudaGetLastError();
}

}  // namespace mm
