// Hot-path kernels of the macromodel + AIM matrix-vector product (eq. (MV_product1)):
//
//   y = D x - (G_FF + G_NF) T A^-1 B x,
//   G_FF = sum_psi I_psi H_psi P_psi        (Sec. V, steps (i)-(iii))
//
//  k_macro_gemm   u = M_t x_e and v = D_t x_e for every element of type t (stacked
//                 [M_t; D_t], one GEMM per type, shared by identical elements, Sec. III);
//                 k_macro_gemm3 is its FP64 form with three real products per term
//  k_project      step (i): grid currents (psi = x, y, z) and charges (phi) on each
//                 element's stencil box, gathered per box node from per-type lists,
//                 added into the grids with atomics (neighbouring boxes overlap)
//  k_fft_fwd_planes / k_fft_conv_lines / k_fft_inv_planes
//                 step (ii): zero-padded 3D FFT convolution with the Green's
//                 spectrum; direct DFT along the short z axis, warp FFTs along y and
//                 x (in registers for complex64 lines of 32 R points, Stockham
//                 mixed-radix stages in shared memory otherwise), the spectrum
//                 multiply fused between the forward and inverse x transforms
//  k_interp       step (iii): interpolation with I = P^T, psi-sum with c_A, c_phi,
//                 and y = v - y_ff
//  k_near_blocks  v -= G_NF u as translation-invariant dense blocks (the default)
//  k_spmv_near*   the same as CSR rows (warp per row; k_spmv_near_3m is the FP64
//                 form with three real products per non-zero)
//  matvec         the schedule: A1 on the caller's stream, then the near field on
//                 the array's low-priority stream beside A2-A4 on its high-priority
//                 stream, joined back into the caller's stream
//  *_ff, <FFTag>, <NearFF>
//                 the complex128 product in float-float arithmetic (ffops.cuh):
//                 k_split_f6, k_macro_gemm_ff, k_project_ff, the FFT stages on
//                 CF values, k_interp_ff, k_near_blocks<NearFF>
//
// Layouts: vectors element-major with RHS innermost; grids [4 nrhs][Nx][Ny][Nz]
// (batch b = psi * nrhs + j); partial spectra [b][x][ky][kz]; Green's spectrum
// [ky][kz][kx].
#include <cstdio>
#include <functional>

#include "device.h"
#include "ffops.cuh"
#include "near_tc.h"
#include "tc_gemm.h"

namespace mm {

template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  T c;
  c.x = a.x * b.x - a.y * b.y;
  c.y = a.x * b.y + a.y * b.x;
  return c;
}
// acc += a b as four fused multiply-adds (the plain expression compiles to six
// operations: a product, two FMAs and a separate add per component)
__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename T> __device__ __forceinline__ void cmac(T& acc, const T& a, const T& b) {
  acc.x = fmx(a.x, b.x, acc.x);
  acc.x = fmx(-a.y, b.y, acc.x);
  acc.y = fmx(a.x, b.y, acc.y);
  acc.y = fmx(a.y, b.x, acc.y);
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) {
  T c;
  c.x = a.x + b.x;
  c.y = a.y + b.y;
  return c;
}
template <typename T> __device__ __forceinline__ T csub(T a, T b) {
  T c;
  c.x = a.x - b.x;
  c.y = a.y - b.y;
  return c;
}
template <typename T, typename R> __device__ __forceinline__ T cscale(T a, R s) {
  T c;
  c.x = a.x * s;
  c.y = a.y * s;
  return c;
}
template <typename T> __device__ __forceinline__ T czero() {
  T c;
  c.x = 0;
  c.y = 0;
  return c;
}

// Block-wide staging copy: store(i, load(i)) for i < n, with U loads per
// thread issued before their stores.  (Written as one loop, each load would
// wait on the shared-memory store of the previous one: one memory latency per
// element and thread.)
template <int U, typename T, typename Load, typename Store>
__device__ __forceinline__ void staged_copy(int n, Load load, Store store) {
  for (int i0 = threadIdx.x; i0 < n; i0 += U * blockDim.x) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      if (i < n) v[u] = load(i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      if (i < n) store(i, v[u]);
    }
  }
}


// q = i / d, r = i % d for 0 <= i < 2^22 by a float reciprocal and one
// correction step (an integer division costs tens of instructions)
struct SmallDiv {
  int d;
  float rd;
  __device__ explicit SmallDiv(int d_) : d(d_), rd(1.0f / (float)d_) {}
  __device__ __forceinline__ void operator()(int i, int& q, int& r) const {
    q = __float2int_rz((float)i * rd);
    r = i - q * d;
    if (r >= d) {
      r -= d;
      ++q;
    } else if (r < 0) {
      r += d;
      --q;
    }
  }
};

FftPlan make_plan(int L) {
  FftPlan p;
  p.L = L;
  int n = L;
  for (int r : {4, 2, 3, 5, 7, 11})
    while (n % r == 0 && p.nst < 16) {
      p.rad[p.nst++] = r;
      n /= r;
    }
  if (n != 1) p.nst = -1;
  return p;
}

// ---------------------------------------------------------------- A1: macromodel GEMM
// C (2Nh x ncols) = W (2Nh x Nh) X (Nh x ncols); column c = j * nrhs + rhs of element elems[j].
// Rows [0, Nh) go to u = M x, rows [Nh, 2Nh) to v = D x.  BM x BN tile per CTA of
// 256 threads (each a TM x TN block of outputs), BK-deep k slices staged in
// shared memory; the next slice is loaded into registers while the current one
// is multiplied (the product is latency-bound at these sizes).
template <typename R, int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_macro_gemm(const typename V2<R>::T* __restrict__ W, int Nh, int rows,
                                                    const int32_t* __restrict__ elems, int ncols, int nrhs,
                                                    const int64_t* __restrict__ off,
                                                    const typename V2<R>::T* __restrict__ x,
                                                    typename V2<R>::T* __restrict__ u,
                                                    typename V2<R>::T* __restrict__ v) {
  typedef typename V2<R>::T C;
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LA = BM * BK / 256, LB = BN * BK / 256;   // elements each thread stages per slice
  __shared__ C As[BK][BM + 1];
  __shared__ C Bs[BK][BN + 1];
  __shared__ int64_t colbase[BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
  const int M2 = rows;   // 2 Nh for the stacked [M; D]; Nh for a single operator (u only)
  for (int c = tid; c < BN; c += 256) {
    const int gc = col0 + c;
    colbase[c] = gc < ncols ? off[elems[gc / nrhs]] * nrhs + gc % nrhs : -1;
  }
  C acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = czero<C>();
  __syncthreads();
  C ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      const int r = e / BK, kk = e % BK;
      const int gr = row0 + r, gk = k0 + kk;
      ra[q] = (gr < M2 && gk < Nh) ? W[(int64_t)gr * Nh + gk] : czero<C>();
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      const int kk = e % BK, c = e / BK;   // lanes run along k: one element's vector is contiguous
      const int gk = k0 + kk;
      const int64_t cb = colbase[c];
      rb[q] = (cb >= 0 && gk < Nh) ? x[cb + (int64_t)gk * nrhs] : czero<C>();
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      As[e % BK][e / BK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      Bs[e % BK][e / BK] = rb[q];
    }
  };
  load(0);
  store();
  __syncthreads();
  for (int k0 = 0; k0 < Nh; k0 += BK) {
    const bool more = k0 + BK < Nh;
    if (more) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          cmac(acc[i][j], a[i], b[j]);
        }
    }
    __syncthreads();
    if (more) {
      store();
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gr = row0 + ty * TM + i;
    if (gr >= M2) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = tx * TN + j;
      const int64_t cb = colbase[c];
      if (cb < 0) continue;
      if (gr < Nh)
        u[cb + (int64_t)gr * nrhs] = acc[i][j];
      else
        v[cb + (int64_t)(gr - Nh) * nrhs] = acc[i][j];
    }
  }
}

// FP64 form of the macromodel GEMM with three real products per complex term
// (Gauss): with w = a + ib, x = c + id, t1 = a c, t2 = b d, t3 = (a + b)(c + d),
// w x = (t1 - t2) + i (t3 - t1 - t2).  The three sums run as three real
// accumulations (three FMAs per term instead of four); a + b is stored with the
// matrix (W3: Re, Im, Re + Im per entry), c + d is formed when x is staged.  The
// GEMM is bound by GB300's FP64 rate, so the FMA count sets its time.
struct D3 {
  double r, i, s;
};
template <int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_macro_gemm3(const double* __restrict__ W3, int Nh, int rows,
                                                     const int32_t* __restrict__ elems, int ncols, int nrhs,
                                                     const int64_t* __restrict__ off, const double2* __restrict__ x,
                                                     double2* __restrict__ u, double2* __restrict__ v,
                                                     double* __restrict__ us) {
  // us (optional): Re u + Im u, the summed operand of the three-product near field
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LA = BM * BK / 256, LB = BN * BK / 256;
  __shared__ D3 As[BK][BM + 1];
  __shared__ D3 Bs[BK][BN + 1];
  __shared__ int64_t colbase[BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
  for (int c = tid; c < BN; c += 256) {
    const int gc = col0 + c;
    colbase[c] = gc < ncols ? off[elems[gc / nrhs]] * nrhs + gc % nrhs : -1;
  }
  double t1[TM][TN], t2[TM][TN], t3[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) t1[i][j] = t2[i][j] = t3[i][j] = 0.0;
  __syncthreads();
  D3 ra[LA];
  double2 rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      const int r = e / BK, kk = e % BK;
      const int gr = row0 + r, gk = k0 + kk;
      if (gr < rows && gk < Nh) {
        const double* w = W3 + 3 * ((int64_t)gr * Nh + gk);
        ra[q] = D3{w[0], w[1], w[2]};
      } else {
        ra[q] = D3{0, 0, 0};
      }
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      const int kk = e % BK, c = e / BK;
      const int gk = k0 + kk;
      const int64_t cb = colbase[c];
      rb[q] = (cb >= 0 && gk < Nh) ? x[cb + (int64_t)gk * nrhs] : make_double2(0, 0);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      As[e % BK][e / BK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      Bs[e % BK][e / BK] = D3{rb[q].x, rb[q].y, rb[q].x + rb[q].y};
    }
  };
  load(0);
  store();
  __syncthreads();
  for (int k0 = 0; k0 < Nh; k0 += BK) {
    const bool more = k0 + BK < Nh;
    if (more) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      D3 a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          t1[i][j] = __fma_rn(a[i].r, b[j].r, t1[i][j]);
          t2[i][j] = __fma_rn(a[i].i, b[j].i, t2[i][j]);
          t3[i][j] = __fma_rn(a[i].s, b[j].s, t3[i][j]);
        }
    }
    __syncthreads();
    if (more) {
      store();
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gr = row0 + ty * TM + i;
    if (gr >= rows) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t cb = colbase[tx * TN + j];
      if (cb < 0) continue;
      const double2 o = make_double2(t1[i][j] - t2[i][j], t3[i][j] - t1[i][j] - t2[i][j]);
      if (gr < Nh) {
        u[cb + (int64_t)gr * nrhs] = o;
        if (us != nullptr) us[cb + (int64_t)gr * nrhs] = o.x + o.y;
      } else {
        v[cb + (int64_t)(gr - Nh) * nrhs] = o;
      }
    }
  }
}

// x (complex128) -> F6: each of re, im, re + im as a float pair (the
// float-float GEMM's right-hand operand, split once per product)
__global__ void k_split_f6(const double2* __restrict__ x, int64_t n, F6* __restrict__ x6) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 z = x[i];
    f6_store(x6 + i, f6_from(z.x, z.y));
  }
}

// The complex128 macromodel GEMM in float-float arithmetic (the three-product
// form of k_macro_gemm3, each real product and sum carried as a float pair):
// W6 and x6 hold re, im and re + im split into hi + lo floats.  Writes u and v
// in FP64 and, when u6 is given, u split again for the float-float near
// field.  About 2^-44 relative error on the sums of |w x|, against 2^-53 for
// FP64; the FP32 pipe runs it several times faster than GB300's FP64 pipe.
template <int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_macro_gemm_ff(const F6* __restrict__ W6, int Nh, int rows,
                                                       const int32_t* __restrict__ elems, int ncols, int nrhs,
                                                       const int64_t* __restrict__ off, const F6* __restrict__ x6,
                                                       double2* __restrict__ u, double2* __restrict__ v,
                                                       F6* __restrict__ u6, double* __restrict__ us) {
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LA = BM * BK / 256, LB = BN * BK / 256;
  __shared__ F6 As[BK][BM + 1];
  __shared__ F6 Bs[BK][BN + 1];
  __shared__ int64_t colbase[BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
  for (int c = tid; c < BN; c += 256) {
    const int gc = col0 + c;
    colbase[c] = gc < ncols ? off[elems[gc / nrhs]] * nrhs + gc % nrhs : -1;
  }
  FF3 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = ff3_zero();
  __syncthreads();
  F6 ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      const int r = e / BK, kk = e % BK;
      const int gr = row0 + r, gk = k0 + kk;
      ra[q] = (gr < rows && gk < Nh) ? f6_load(W6 + (int64_t)gr * Nh + gk) : f6_zero();
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      const int kk = e % BK, c = e / BK;
      const int gk = k0 + kk;
      const int64_t cb = colbase[c];
      rb[q] = (cb >= 0 && gk < Nh) ? f6_load(x6 + cb + (int64_t)gk * nrhs) : f6_zero();
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + 256 * q;
      As[e % BK][e / BK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + 256 * q;
      Bs[e % BK][e / BK] = rb[q];
    }
  };
  load(0);
  store();
  __syncthreads();
  for (int k0 = 0; k0 < Nh; k0 += BK) {
    const bool more = k0 + BK < Nh;
    if (more) load(k0 + BK);
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      F6 a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) ff3_mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
    if (more) {
      store();
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gr = row0 + ty * TM + i;
    if (gr >= rows) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t cb = colbase[tx * TN + j];
      if (cb < 0) continue;
      FF re, im;
      ff3_result(acc[i][j], re, im);
      const double2 o = make_double2(ff_to_double(re), ff_to_double(im));
      if (gr < Nh) {
        const int64_t idx = cb + (int64_t)gr * nrhs;
        u[idx] = o;
        if (u6 != nullptr) {
          const FF sm = ff_add(re, im);
          f6_store(u6 + idx, F6{re.s, im.s, sm.s, re.c, im.c, sm.c});
        }
        if (us != nullptr) us[idx] = o.x + o.y;
      } else {
        v[cb + (int64_t)(gr - Nh) * nrhs] = o;
      }
    }
  }
}

// ---------------------------------------------------------------- A2: projection (step i)
// One CTA per element.  Each thread owns nodes of the element's stencil box and
// gathers the (basis, stencil node) contributions listed for that node (lists
// precomputed per type), so there are no shared-memory atomics; the box is
// then added into the global grids (neighbouring boxes overlap: atomics).
template <typename C> __device__ __forceinline__ void atomic_add_c(C* p, C v);
template <> __device__ __forceinline__ void atomic_add_c<float2>(float2* p, float2 v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void atomic_add_c<double2>(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

template <typename R> struct W4;
template <> struct W4<float> {
  typedef float4 T;
  static __device__ __forceinline__ float4 load(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
};
template <> struct W4<double> {
  struct T { double x, y, z, w; };
  static __device__ __forceinline__ T load(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return T{a.x, a.y, b.x, b.y};
  }
};

template <typename R, int RC>
__global__ void __launch_bounds__(RC == 1 ? 512 : 256, RC == 1 && sizeof(R) == 8 ? 1 : 2) k_project(const int32_t* __restrict__ elems, int Nh, int bx, int by, int bz,
                                                 const int32_t* __restrict__ inv_ptr,
                                                 const int32_t* __restrict__ inv_ent, const R* __restrict__ Pi,
                                                 const int64_t* __restrict__ off, const int32_t* __restrict__ boxorg,
                                                 int nrhs, const typename V2<R>::T* __restrict__ u, int Nx, int Ny,
                                                 int Nz, typename V2<R>::T* __restrict__ grid,
                                                 typename V2<R>::T* __restrict__ boxbuf, int nodes_max) {
  typedef typename V2<R>::T C;
  extern __shared__ unsigned char smem_raw[];
  C* us = reinterpret_cast<C*>(smem_raw);  // [n][c] element's u for this RHS chunk
  const int e = elems[blockIdx.x];
  const int nodes = bx * by * bz;
  const int64_t o = off[e];
  const int gx0 = boxorg[3 * e], gy0 = boxorg[3 * e + 1], gz0 = boxorg[3 * e + 2];
  const int64_t gstride = (int64_t)Nx * Ny * Nz;
  for (int c0 = 0; c0 < nrhs; c0 += RC) {
    const int cn = min(RC, nrhs - c0);
    staged_copy<4, C>(
        Nh * RC,
        [&](int i) {
          const int n = i / RC, c = i % RC;
          return c < cn ? u[(o + n) * nrhs + c0 + c] : czero<C>();
        },
        [&](int i, C v) { us[i] = v; });
    __syncthreads();
    // T consecutive lanes share a node (T = 1, 2 or 4 when the block has the
    // threads): each takes every T-th group of four entries, then they add up
    // by shuffles within their group
    // (one right-hand side only: with several, the per-node accumulators are
    // many and the shuffles cost more than the split saves)
    const int T = RC > 1 ? 1 : ((int)blockDim.x >= 4 * nodes ? 4 : ((int)blockDim.x >= 2 * nodes ? 2 : 1));
    const int sub = threadIdx.x % T;
    const unsigned gmask = ((1u << T) - 1u) << ((threadIdx.x % 32) & ~(T - 1));
    for (int node = threadIdx.x / T; node < nodes; node += blockDim.x / T) {
      C acc[4][RC];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[q][c] = czero<C>();
      const int q0 = inv_ptr[node], q1 = inv_ptr[node + 1];
      if (q0 == q1) continue;
      for (int q = q0 + 4 * sub; q < q1; q += 4 * T) {
        int ent[4];
        typename W4<R>::T w[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) ent[t] = q + t < q1 ? __ldg(inv_ent + q + t) : -1;
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (ent[t] >= 0) w[t] = W4<R>::load(Pi + ((int64_t)(ent[t] >> 16) * Nh + (ent[t] & 0xffff)) * 4);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (ent[t] < 0) continue;
          const int n = ent[t] & 0xffff;
#pragma unroll
          for (int c = 0; c < RC; ++c) {
            const C uv = us[n * RC + c];
            acc[0][c].x += w[t].x * uv.x; acc[0][c].y += w[t].x * uv.y;
            acc[1][c].x += w[t].y * uv.x; acc[1][c].y += w[t].y * uv.y;
            acc[2][c].x += w[t].z * uv.x; acc[2][c].y += w[t].z * uv.y;
            acc[3][c].x += w[t].w * uv.x; acc[3][c].y += w[t].w * uv.y;
          }
        }
      }
      for (int o = 1; o < T; o <<= 1)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int c = 0; c < RC; ++c) {
            acc[q][c].x += __shfl_xor_sync(gmask, acc[q][c].x, o);
            acc[q][c].y += __shfl_xor_sync(gmask, acc[q][c].y, o);
          }
      if (sub != 0) continue;
      const int lz = node % bz, ly = (node / bz) % by, lx = node / (by * bz);
      const int64_t gidx = ((int64_t)(gx0 + lx) * Ny + (gy0 + ly)) * Nz + (gz0 + lz);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < RC; ++c)
          if (c < cn) {
            if (boxbuf)   // two-pass form: the element's own box, plain stores
              boxbuf[(((int64_t)e * 4 + q) * nrhs + c0 + c) * nodes_max + node] = acc[q][c];
            else
              atomic_add_c(grid + ((int64_t)q * nrhs + c0 + c) * gstride + gidx, acc[q][c]);
          }
    }
    __syncthreads();
  }
}

// Projection of the float-float complex128 product: the schedule of
// k_project for one right-hand side at a time (T lanes per box node, shuffles),
// u from the GEMM's F6 split (re, im as float pairs in shared memory), the
// weights as float pairs Pf[(s Nh + n) 2 + {0: hi, 1: lo}] (x, y, z, phi), every
// node's four complex sums in float-float, added into the FP64 grid.
__global__ void __launch_bounds__(512, 2) k_project_ff(const int32_t* __restrict__ elems, int Nh, int bx, int by,
                                                       int bz, const int32_t* __restrict__ inv_ptr,
                                                       const int32_t* __restrict__ inv_ent,
                                                       const float4* __restrict__ Pf,
                                                       const int64_t* __restrict__ off,
                                                       const int32_t* __restrict__ boxorg, int nrhs,
                                                       const F6* __restrict__ u6, int Nx, int Ny, int Nz,
                                                       double2* __restrict__ grid) {
  extern __shared__ float4 us4[];   // [n]: (re hi, im hi, re lo, im lo)
  const int e = elems[blockIdx.x];
  const int nodes = bx * by * bz;
  const int64_t o = off[e];
  const int gx0 = boxorg[3 * e], gy0 = boxorg[3 * e + 1], gz0 = boxorg[3 * e + 2];
  const int64_t gstride = (int64_t)Nx * Ny * Nz;
  const int T = (int)blockDim.x >= 4 * nodes ? 4 : ((int)blockDim.x >= 2 * nodes ? 2 : 1);
  const int sub = threadIdx.x % T;
  const unsigned gmask = ((1u << T) - 1u) << ((threadIdx.x % 32) & ~(T - 1));
  for (int c = 0; c < nrhs; ++c) {
    for (int n = threadIdx.x; n < Nh; n += blockDim.x) {
      const F6 f = f6_load(u6 + (o + n) * nrhs + c);
      us4[n] = make_float4(f.rh, f.ih, f.rl, f.il);
    }
    __syncthreads();
    for (int node = threadIdx.x / T; node < nodes; node += blockDim.x / T) {
      const int q0 = inv_ptr[node], q1 = inv_ptr[node + 1];
      if (q0 == q1) continue;
      FF acc[4][2];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q][0] = acc[q][1] = ff_zero();
      for (int q = q0 + sub; q < q1; q += T) {
        const int ent = __ldg(inv_ent + q);
        const int n = ent & 0xffff, sn = ent >> 16;
        const float4 wh = __ldg(Pf + ((int64_t)sn * Nh + n) * 2), wl = __ldg(Pf + ((int64_t)sn * Nh + n) * 2 + 1);
        const float4 uv = us4[n];
        ff_mac(acc[0][0], wh.x, wl.x, uv.x, uv.z);
        ff_mac(acc[0][1], wh.x, wl.x, uv.y, uv.w);
        ff_mac(acc[1][0], wh.y, wl.y, uv.x, uv.z);
        ff_mac(acc[1][1], wh.y, wl.y, uv.y, uv.w);
        ff_mac(acc[2][0], wh.z, wl.z, uv.x, uv.z);
        ff_mac(acc[2][1], wh.z, wl.z, uv.y, uv.w);
        ff_mac(acc[3][0], wh.w, wl.w, uv.x, uv.z);
        ff_mac(acc[3][1], wh.w, wl.w, uv.y, uv.w);
      }
      for (int o2 = 1; o2 < T; o2 <<= 1)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const FF other{__shfl_xor_sync(gmask, acc[q][r].s, o2), __shfl_xor_sync(gmask, acc[q][r].c, o2)};
            acc[q][r] = ff_add(acc[q][r], other);
          }
      if (sub != 0) continue;
      const int lz = node % bz, ly = (node / bz) % by, lx = node / (by * bz);
      const int64_t gidx = ((int64_t)(gx0 + lx) * Ny + (gy0 + ly)) * Nz + (gz0 + lz);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double2* g = grid + ((int64_t)q * nrhs + c) * gstride + gidx;
        atomicAdd(&g->x, ff_to_double(acc[q][0]));
        atomicAdd(&g->y, ff_to_double(acc[q][1]));
      }
    }
    __syncthreads();
  }
}

// Second pass of the two-pass projection: every grid point (plane b = psi
// nrhs + c, node g) sums the boxes of the elements whose stencil box covers g
// (per node the list of (element, local node), gptr / gent, fixed at set-up);
// no atomics, and every point is written (the grid needs no clearing).
template <typename C>
__global__ void __launch_bounds__(256) k_grid_gather(int64_t ng, int B, const int32_t* __restrict__ gptr,
                                                     const int64_t* __restrict__ gent, const C* __restrict__ boxbuf,
                                                     int nodes_max, int nrhs, C* __restrict__ grid) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ng * B) return;
  const int64_t g = t % ng, b = t / ng;
  C acc = czero<C>();
  for (int k = gptr[g]; k < gptr[g + 1]; ++k) {
    const int64_t ent = gent[k];   // element * nodes_max + local node
    const int64_t e = ent / nodes_max, ln = ent - e * nodes_max;
    const C v = boxbuf[((e * 4) * nrhs + b) * nodes_max + ln];
    acc.x += v.x;
    acc.y += v.y;
  }
  grid[t] = acc;
}

// Projection of one right-hand side from the same tables (complex64), read
// from global memory (L1 / L2): one CTA per element, u of its bases staged in
// shared memory; a warp takes eight box nodes, four lanes per node striding
// its entries (weight and basis index loaded together, four entries per step:
// no dependent loads), folded by two shuffle levels; lane g of a node adds
// component g into the grid.
__global__ void __launch_bounds__(512) k_project_g1(const int32_t* __restrict__ elems, int Nh, int bx, int by, int bz,
                                                    const int32_t* __restrict__ inv_ptr,
                                                    const unsigned char* __restrict__ tab, int E,
                                                    const int64_t* __restrict__ off,
                                                    const int32_t* __restrict__ boxorg, const float2* __restrict__ u,
                                                    int Nx, int Ny, int Nz, float2* __restrict__ grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* us = reinterpret_cast<float2*>(smem_raw);
  int* ip = reinterpret_cast<int*>(us + Nh);   // the box nodes' list starts (nodes + 1), staged with u
  const float4* tw = reinterpret_cast<const float4*>(tab);
  const uint16_t* tn = reinterpret_cast<const uint16_t*>(tab + 16 * (size_t)E);
  const int e = elems[blockIdx.x];
  const int64_t o = off[e];
  const int nodes = bx * by * bz;
  const int64_t gstride = (int64_t)Nx * Ny * Nz;
  const int64_t gbase = ((int64_t)boxorg[3 * e] * Ny + boxorg[3 * e + 1]) * Nz + boxorg[3 * e + 2];
  for (int n = threadIdx.x; n < Nh; n += blockDim.x) us[n] = u[o + n];
  for (int n = threadIdx.x; n <= nodes; n += blockDim.x) ip[n] = __ldg(inv_ptr + n);
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  const int j = lane / 4, g = lane % 4;
  for (int node0 = 8 * warp; node0 < nodes; node0 += 8 * nw) {
    const int node = node0 + j;
    float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f, ax2 = 0.f, ay2 = 0.f, ax3 = 0.f, ay3 = 0.f;
    auto mac = [&](const float4 w, const float2 uv) {
      ax0 = fmaf(w.x, uv.x, ax0); ay0 = fmaf(w.x, uv.y, ay0);
      ax1 = fmaf(w.y, uv.x, ax1); ay1 = fmaf(w.y, uv.y, ay1);
      ax2 = fmaf(w.z, uv.x, ax2); ay2 = fmaf(w.z, uv.y, ay2);
      ax3 = fmaf(w.w, uv.x, ax3); ay3 = fmaf(w.w, uv.y, ay3);
    };
    if (node < nodes) {
      const int q1 = ip[node + 1];
      int q = ip[node] + g;
      for (; q + 12 < q1; q += 16) {
        const float4 w0 = __ldg(tw + q), w1 = __ldg(tw + q + 4), w2 = __ldg(tw + q + 8), w3 = __ldg(tw + q + 12);
        const int n0 = __ldg(tn + q), n1 = __ldg(tn + q + 4), n2 = __ldg(tn + q + 8), n3 = __ldg(tn + q + 12);
        mac(w0, us[n0]);
        mac(w1, us[n1]);
        mac(w2, us[n2]);
        mac(w3, us[n3]);
      }
      for (; q < q1; q += 4) mac(__ldg(tw + q), us[__ldg(tn + q)]);
    }
#pragma unroll
    for (int o2 = 1; o2 < 4; o2 <<= 1) {
      ax0 += __shfl_xor_sync(0xffffffffu, ax0, o2); ay0 += __shfl_xor_sync(0xffffffffu, ay0, o2);
      ax1 += __shfl_xor_sync(0xffffffffu, ax1, o2); ay1 += __shfl_xor_sync(0xffffffffu, ay1, o2);
      ax2 += __shfl_xor_sync(0xffffffffu, ax2, o2); ay2 += __shfl_xor_sync(0xffffffffu, ay2, o2);
      ax3 += __shfl_xor_sync(0xffffffffu, ax3, o2); ay3 += __shfl_xor_sync(0xffffffffu, ay3, o2);
    }
    if (node < nodes) {
      const int lz = node % bz, ly = (node / bz) % by, lx = node / (by * bz);
      const float sx = g == 0 ? ax0 : g == 1 ? ax1 : g == 2 ? ax2 : ax3;
      const float sy = g == 0 ? ay0 : g == 1 ? ay1 : g == 2 ? ay2 : ay3;
      atomicAdd(grid + (int64_t)g * gstride + gbase + ((int64_t)lx * Ny + ly) * Nz + lz, make_float2(sx, sy));
    }
  }
}

// Projection of many right-hand sides from shared-memory tables (complex64):
// one launch for all types; each CTA takes a contiguous range of the elements
// listed type by type, and copies a type's inverse stencil lists (weights and
// basis indices in box-node order, DevPrec::prj_tab) into shared memory when
// its walk enters that type.  Per element and chunk of CH
// right-hand sides, u of the element's bases is staged; a warp takes a box
// node, its lanes = CH right-hand sides x 32 / CH groups that stride the node's
// entries (all table and u reads from shared memory, conflict-free), folded by
// shuffles; the box (4 components x CH x nodes) passes through shared memory
// and is added into the grids with atomics along consecutive nodes.
__host__ __device__ inline size_t prj_tab_bytes(int E) { return 16 * (size_t)E + ((size_t)2 * E + 15) / 16 * 16; }
__host__ __device__ inline size_t prj_us_offset(int E, int nodes) {
  return (prj_tab_bytes(E) + 4 * (size_t)(2 * nodes + 1) + 15) / 16 * 16;
}
constexpr size_t kPrjSmemMax = 220 * 1024;        // shared memory the table-driven projection may take
constexpr size_t kInterpRhsSmemMax = 200 * 1024;  // ... and the right-hand-side-lane interpolation
constexpr size_t kInterpTabSmemMax = 220 * 1024;  // ... and the table-driven interpolation
template <int CH>
__host__ __device__ inline size_t prj_smem_bytes(int E, int nodes, int Nh) {
  return prj_us_offset(E, nodes) + 8 * (size_t)CH * ((size_t)Nh + 4 * (size_t)nodes);
}

template <int CH>
__global__ void __launch_bounds__(512, 1) k_project_tab(const PrjTypeDev* __restrict__ types, int64_t total,
                                                        const int64_t* __restrict__ off,
                                                        const int32_t* __restrict__ boxorg, int nrhs,
                                                        const float2* __restrict__ u, int Nx, int Ny, int Nz,
                                                        float2* __restrict__ grid) {
  static_assert(CH >= 1 && CH <= 8 && 32 % CH == 0, "lanes: CH right-hand sides x at least four entry groups");
  constexpr int G = 32 / CH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  const int c = lane % CH, g = lane / CH;
  const int64_t gstride = (int64_t)Nx * Ny * Nz;
  // this CTA's contiguous range of the elements (all types, in type order)
  const int64_t i0 = (int64_t)blockIdx.x * total / gridDim.x, i1 = (int64_t)(blockIdx.x + 1) * total / gridDim.x;
  int t = -1;   // type whose tables are in shared memory
  int64_t tb = 0, te = 0;
  int E = 0, Nh = 0, nodes = 0;
  const int32_t* elems = nullptr;
  const float4* sw = nullptr;
  const uint16_t* sn = nullptr;
  int* sptr = nullptr;
  int* goff = nullptr;
  float2* us = nullptr;
  float2* box = nullptr;
  // right-hand-side chunks outermost: the CTAs move through the chunks together,
  // so the grid planes being added to (4 CH of them) stay in L2; the element
  // range is walked forwards and backwards in turn, so that one chunk ends on
  // the type the next begins with
  int pass = 0;
  for (int c0 = 0; c0 < nrhs; c0 += CH, ++pass) {
    for (int64_t k = 0; k < i1 - i0; ++k) {
      const int64_t gi = (pass & 1) ? i1 - 1 - k : i0 + k;
      if (gi < tb || gi >= te) {
        // another type: its tables into shared memory (every thread takes this branch)
        t = 0;
        tb = 0;
        te = types[0].ne;
        while (gi >= te) {
          ++t;
          tb = te;
          te += types[t].ne;
        }
        const PrjTypeDev ty = types[t];
        E = ty.E;
        Nh = ty.Nh;
        nodes = ty.bx * ty.by * ty.bz;
        elems = ty.elems;
        sw = reinterpret_cast<const float4*>(smem_raw);
        sn = reinterpret_cast<const uint16_t*>(smem_raw + 16 * (size_t)E);
        sptr = reinterpret_cast<int*>(smem_raw + prj_tab_bytes(E));
        goff = sptr + nodes + 1;
        us = reinterpret_cast<float2*>(smem_raw + prj_us_offset(E, nodes));
        box = us + (size_t)Nh * CH;
        __syncthreads();   // the previous type's tables are no longer read
        const int n16 = (int)(prj_tab_bytes(E) / 16);
        for (int i = threadIdx.x; i < n16; i += blockDim.x)
          reinterpret_cast<float4*>(smem_raw)[i] = __ldg(reinterpret_cast<const float4*>(ty.tab) + i);
        for (int i = threadIdx.x; i <= nodes; i += blockDim.x) sptr[i] = ty.inv_ptr[i];
        for (int i = threadIdx.x; i < nodes; i += blockDim.x) {
          const int lz = i % ty.bz, ly = (i / ty.bz) % ty.by, lx = i / (ty.by * ty.bz);
          goff[i] = (lx * Ny + ly) * Nz + lz;
        }
      }
      const SmallDiv dnodes(nodes);
      const int e = elems[gi - tb];
      const int64_t o = off[e];
      const int64_t gbase = ((int64_t)boxorg[3 * e] * Ny + boxorg[3 * e + 1]) * Nz + boxorg[3 * e + 2];
      for (int i = threadIdx.x; i < Nh * CH; i += blockDim.x) {
        const int n = i / CH, cc = i % CH;
        us[i] = c0 + cc < nrhs ? u[(o + n) * nrhs + c0 + cc] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      for (int node = warp; node < nodes; node += nw) {
        float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f, ax2 = 0.f, ay2 = 0.f, ax3 = 0.f, ay3 = 0.f;
        auto mac = [&](const float4 w, const float2 uv) {
          ax0 = fmaf(w.x, uv.x, ax0); ay0 = fmaf(w.x, uv.y, ay0);
          ax1 = fmaf(w.y, uv.x, ax1); ay1 = fmaf(w.y, uv.y, ay1);
          ax2 = fmaf(w.z, uv.x, ax2); ay2 = fmaf(w.z, uv.y, ay2);
          ax3 = fmaf(w.w, uv.x, ax3); ay3 = fmaf(w.w, uv.y, ay3);
        };
        const int q1 = sptr[node + 1];
        int q = sptr[node] + g;
        // four entries per step: their table and u reads are issued together
        for (; q + 3 * G < q1; q += 4 * G) {
          const float4 w0 = sw[q], w1 = sw[q + G], w2 = sw[q + 2 * G], w3 = sw[q + 3 * G];
          const int n0 = sn[q], n1 = sn[q + G], n2 = sn[q + 2 * G], n3 = sn[q + 3 * G];
          const float2 u0 = us[n0 * CH + c], u1 = us[n1 * CH + c], u2 = us[n2 * CH + c], u3 = us[n3 * CH + c];
          mac(w0, u0);
          mac(w1, u1);
          mac(w2, u2);
          mac(w3, u3);
        }
        for (; q < q1; q += G) mac(sw[q], us[(int)sn[q] * CH + c]);
#pragma unroll
        for (int o2 = CH; o2 < 32; o2 <<= 1) {
          ax0 += __shfl_xor_sync(0xffffffffu, ax0, o2); ay0 += __shfl_xor_sync(0xffffffffu, ay0, o2);
          ax1 += __shfl_xor_sync(0xffffffffu, ax1, o2); ay1 += __shfl_xor_sync(0xffffffffu, ay1, o2);
          ax2 += __shfl_xor_sync(0xffffffffu, ax2, o2); ay2 += __shfl_xor_sync(0xffffffffu, ay2, o2);
          ax3 += __shfl_xor_sync(0xffffffffu, ax3, o2); ay3 += __shfl_xor_sync(0xffffffffu, ay3, o2);
        }
        // every lane now holds the four sums of its right-hand side; group g
        // (g < 4) stores component g
        if (g < 4) {
          const float sx = g == 0 ? ax0 : g == 1 ? ax1 : g == 2 ? ax2 : ax3;
          const float sy = g == 0 ? ay0 : g == 1 ? ay1 : g == 2 ? ay2 : ay3;
          box[(g * CH + c) * nodes + node] = make_float2(sx, sy);
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < 4 * CH * nodes; i += blockDim.x) {
        int pc, node;
        dnodes(i, pc, node);
        const int q = pc / CH, cc = pc % CH;
        if (c0 + cc < nrhs) atomicAdd(grid + ((int64_t)q * nrhs + c0 + cc) * gstride + gbase + goff[node], box[i]);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- A3: FFT convolution (step ii)
// CTAs per SM asked of the compiler for the FFT stages: three for complex64,
// one for FP64, two for float-float (its radix-11 and radix-7 butterflies
// spill rather than hold the SM to one CTA)
template <typename R> struct FftOcc { static constexpr int kMinBlocks = sizeof(R) == 4 ? 3 : 1; };
template <> struct FftOcc<FFTag> { static constexpr int kMinBlocks = 2; };
// Grid values in and out of the FFT stages: the same type, or FP64 grids
// around the float-float stages (split on the way in, summed on the way out).
template <typename C, typename G> __device__ __forceinline__ C grid_in(const G& g) { return g; }
template <> __device__ __forceinline__ CF grid_in<CF, double2>(const double2& g) {
  return CF{ffv_from(g.x), ffv_from(g.y)};
}
template <typename G, typename C> __device__ __forceinline__ G grid_out(const C& c) { return c; }
template <> __device__ __forceinline__ double2 grid_out<double2, CF>(const CF& c) {
  return make_double2(ffv_to_double(c.x), ffv_to_double(c.y));
}

// Line buffers in shared memory hold element i at PAD(i) = i + i/16, which
// breaks the bank conflicts of the strided Stockham stores.
__device__ __forceinline__ int PAD(int i) { return i + (i >> 4); }
__host__ __device__ inline int padded_len(int L) { return L + (L >> 4) + 1; }


template <typename C, int RADIX, bool INV>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ a, C* __restrict__ b, int L, int Ns,
                                               const C* __restrict__ tw, int lane, int nlanes) {
  const int nb = L / RADIX;
  const int st = nb / Ns;
  const int stR = nb;
  // j / Ns and j % Ns by a float reciprocal and one correction step (exact for
  // j < 2^22; an integer division would cost tens of instructions per butterfly)
  const float rNs = 1.0f / (float)Ns;
  C wr[RADIX];   // roots of unity of order RADIX (conjugated for the inverse)
#pragma unroll
  for (int m = 0; m < RADIX; ++m) {
    wr[m] = tw[m * stR];
    if (INV) wr[m].y = -wr[m].y;
  }
  for (int j = lane; j < nb; j += nlanes) {
    int g = __float2int_rz((float)j * rNs);
    int k = j - g * Ns;
    if (k >= Ns) {
      k -= Ns;
      ++g;
    } else if (k < 0) {
      k += Ns;
      --g;
    }
    C v[RADIX];
#pragma unroll
    for (int q = 0; q < RADIX; ++q) v[q] = a[PAD(j + q * nb)];
    if (k != 0) {
#pragma unroll
      for (int q = 1; q < RADIX; ++q) {
        C w = tw[q * k * st];
        if (INV) w.y = -w.y;
        v[q] = cmul(v[q], w);
      }
    }
    const int base = g * Ns * RADIX + k;
    if constexpr (RADIX == 2) {
      b[PAD(base)] = cadd(v[0], v[1]);
      b[PAD(base + Ns)] = csub(v[0], v[1]);
    } else if constexpr (RADIX == 4) {
      const C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]), b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
      C jb1;   // -i*b1 forward, +i*b1 inverse
      if (INV) { jb1.x = -b1.y; jb1.y = b1.x; } else { jb1.x = b1.y; jb1.y = -b1.x; }
      b[PAD(base)] = cadd(a0, b0);
      b[PAD(base + Ns)] = cadd(a1, jb1);
      b[PAD(base + 2 * Ns)] = csub(a0, b0);
      b[PAD(base + 3 * Ns)] = csub(a1, jb1);
    } else if constexpr (RADIX % 2 == 0) {
#pragma unroll
      for (int p = 0; p < RADIX; ++p) {
        C acc = v[0];
#pragma unroll
        for (int q = 1; q < RADIX; ++q) acc = cadd(acc, cmul(v[q], wr[(p * q) % RADIX]));
        b[PAD(base + p * Ns)] = acc;
      }
    } else {
      // odd radix R: inputs q and R - q meet the roots e^(-/+ i theta) with
      // theta = 2 pi p q / R, so with t_q = v_q + v_(R-q), d_q = v_q - v_(R-q)
      // output p is A_p - i B_p and output R - p is A_p + i B_p (forward),
      // A_p = v_0 + sum_q cos(theta) t_q, B_p = sum_q sin(theta) d_q: real
      // multiply-adds over half the inputs instead of complex ones over all
      typedef decltype(v[0].x) Rr;
      constexpr int H = (RADIX - 1) / 2;
      C t[H], d[H];
      C s0 = v[0];
#pragma unroll
      for (int q = 1; q <= H; ++q) {
        t[q - 1] = cadd(v[q], v[RADIX - q]);
        d[q - 1] = csub(v[q], v[RADIX - q]);
        s0 = cadd(s0, t[q - 1]);
      }
      b[PAD(base)] = s0;
#pragma unroll
      for (int p = 1; p <= H; ++p) {
        C A = v[0], B = czero<C>();
#pragma unroll
        for (int q = 1; q <= H; ++q) {
          const int m = (p * q) % RADIX;
          const Rr cs = wr[m].x, sn = INV ? wr[m].y : -wr[m].y;   // cos, sin of 2 pi m / R
          A.x = fmx(cs, t[q - 1].x, A.x);
          A.y = fmx(cs, t[q - 1].y, A.y);
          B.x = fmx(sn, d[q - 1].x, B.x);
          B.y = fmx(sn, d[q - 1].y, B.y);
        }
        C o1, o2;   // forward: o1 = A - i B (output p), o2 = A + i B (output R - p)
        if (INV) {
          o1.x = A.x - B.y; o1.y = A.y + B.x;
          o2.x = A.x + B.y; o2.y = A.y - B.x;
        } else {
          o1.x = A.x + B.y; o1.y = A.y - B.x;
          o2.x = A.x - B.y; o2.y = A.y + B.x;
        }
        b[PAD(base + p * Ns)] = o1;
        b[PAD(base + (RADIX - p) * Ns)] = o2;
      }
    }
  }
}

// Warp-level Stockham FFT of one line held in shared memory (buffers a, b of
// length L); returns the buffer that holds the result.

// Warp FFT of a line of L = 32 RR points kept in registers (complex64 lines).
// With n = n1 + 32 n2 and k = k2 + RR k1 (n1, k1 < 32; n2, k2 < RR):
//   X[k2 + RR k1] = sum_n1 W_32^(n1 k1) [W_L^(n1 k2) sum_n2 x[n1 + 32 n2] W_RR^(n2 k2)],
// so lane n1 takes the RR-point DFT of its own points, multiplies by W_L^(n1 k2),
// and the 32-point DFTs over n1 run across the lanes as five radix-2
// decimation-in-frequency butterflies through shuffles, which leave lane l with
// k1 = bit-reverse(l).  tw holds W_L^i = exp(-2 pi i / L) (conjugated for the
// inverse); W_RR^m = tw[32 m] and W_32^m = tw[RR m].  The RR-point DFT pairs
// inputs q and RR - q (real cos / sin multiply-adds, as in the odd-radix
// Stockham stage).  a and dst may be the same buffer: every lane has read its
// points before the first shuffle, and writes after the last one.
template <typename C, int RR, bool INV>
__device__ __forceinline__ void warp_fft_reg(const C* a, C* dst, const C* __restrict__ tw, int lane) {
  typedef decltype(a[0].x) Rr;
  C y[RR];
  {
    C x[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) x[r] = a[PAD(lane + 32 * r)];
    if constexpr (RR == 1) {
      y[0] = x[0];
    } else {
      constexpr int H = (RR - 1) / 2;
      C t[H > 0 ? H : 1], d[H > 0 ? H : 1];
      C s0 = x[0];
#pragma unroll
      for (int q = 1; q <= H; ++q) {
        t[q - 1] = cadd(x[q], x[RR - q]);
        d[q - 1] = csub(x[q], x[RR - q]);
        s0 = cadd(s0, t[q - 1]);
      }
      if constexpr (RR % 2 == 0) s0 = cadd(s0, x[RR / 2]);
      y[0] = s0;
#pragma unroll
      for (int p = 1; 2 * p <= RR; ++p) {
        C A = x[0], B = czero<C>();
#pragma unroll
        for (int q = 1; q <= H; ++q) {
          const C w = tw[32 * ((p * q) % RR)];
          const Rr cs = w.x, sn = -w.y;   // cos, sin of 2 pi m / RR
          A.x = fmx(cs, t[q - 1].x, A.x);
          A.y = fmx(cs, t[q - 1].y, A.y);
          B.x = fmx(sn, d[q - 1].x, B.x);
          B.y = fmx(sn, d[q - 1].y, B.y);
        }
        if constexpr (RR % 2 == 0) {
          if (p & 1) A = csub(A, x[RR / 2]);
          else A = cadd(A, x[RR / 2]);
        }
        if (2 * p == RR) {
          y[p] = A;   // sin(pi q) = 0
        } else {
          C o1, o2;   // forward: A - i B (output p), A + i B (output RR - p)
          if (INV) {
            o1.x = A.x - B.y; o1.y = A.y + B.x;
            o2.x = A.x + B.y; o2.y = A.y - B.x;
          } else {
            o1.x = A.x + B.y; o1.y = A.y - B.x;
            o2.x = A.x - B.y; o2.y = A.y + B.x;
          }
          y[p] = o1;
          y[RR - p] = o2;
        }
      }
    }
  }
#pragma unroll
  for (int k2 = 1; k2 < RR; ++k2) {
    C w = tw[lane * k2];
    if (INV) w.y = -w.y;
    y[k2] = cmul(y[k2], w);
  }
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
    C w = tw[RR * (lane & (h - 1)) * (16 / h)];   // W_(2h)^j, j = lane mod h
    if (INV) w.y = -w.y;
    if (!up) {
      w.x = 1;
      w.y = 0;
    }
    // sum (lower lane) or difference (upper lane) of the pair as one signed
    // multiply-add per component: s y + o with s = +1 or -1
    const Rr sg = up ? Rr(-1) : Rr(1);
#pragma unroll
    for (int k2 = 0; k2 < RR; ++k2) {
      C o;
      o.x = __shfl_xor_sync(0xffffffffu, y[k2].x, h);
      o.y = __shfl_xor_sync(0xffffffffu, y[k2].y, h);
      C sd;
      sd.x = fmx(sg, y[k2].x, o.x);
      sd.y = fmx(sg, y[k2].y, o.y);
      y[k2] = h == 1 ? sd : cmul(sd, w);
    }
  }
  __syncwarp();
  const int k1 = (int)(__brev((unsigned)lane) >> 27);
#pragma unroll
  for (int k2 = 0; k2 < RR; ++k2) dst[PAD(k2 + RR * k1)] = y[k2];
  __syncwarp();
}

template <typename C, bool INV>
__device__ C* warp_fft(C* a, C* b, const FftPlan& P, const C* tw, int lane) {
  if constexpr (sizeof(C) == 8) {
    // complex64 lines of 32 RR points (RR <= 16) in registers; the result goes
    // where the Stockham stages would leave it (a after an even stage count)
    if ((P.L & 31) == 0 && P.L <= 32 * kRegFftMax && P.nst > 0) {
      C* dst = (P.nst % 2 == 0) ? a : b;
      switch (P.L >> 5) {
        case 1: warp_fft_reg<C, 1, INV>(a, dst, tw, lane); break;
        case 2: warp_fft_reg<C, 2, INV>(a, dst, tw, lane); break;
        case 3: warp_fft_reg<C, 3, INV>(a, dst, tw, lane); break;
        case 4: warp_fft_reg<C, 4, INV>(a, dst, tw, lane); break;
        case 5: warp_fft_reg<C, 5, INV>(a, dst, tw, lane); break;
        case 6: warp_fft_reg<C, 6, INV>(a, dst, tw, lane); break;
        case 7: warp_fft_reg<C, 7, INV>(a, dst, tw, lane); break;
        case 8: warp_fft_reg<C, 8, INV>(a, dst, tw, lane); break;
        case 9: warp_fft_reg<C, 9, INV>(a, dst, tw, lane); break;
        case 10: warp_fft_reg<C, 10, INV>(a, dst, tw, lane); break;
        case 11: warp_fft_reg<C, 11, INV>(a, dst, tw, lane); break;
        default: warp_fft_reg<C, 12, INV>(a, dst, tw, lane); break;
      }
      return dst;
    }
  }
  int Ns = 1;
  for (int s = 0; s < P.nst; ++s) {
    const int r = P.rad[s];
    switch (r) {
      case 8: stockham_stage<C, 8, INV>(a, b, P.L, Ns, tw, lane, 32); break;
      case 4: stockham_stage<C, 4, INV>(a, b, P.L, Ns, tw, lane, 32); break;
      case 2: stockham_stage<C, 2, INV>(a, b, P.L, Ns, tw, lane, 32); break;
      case 3: stockham_stage<C, 3, INV>(a, b, P.L, Ns, tw, lane, 32); break;
      case 5: stockham_stage<C, 5, INV>(a, b, P.L, Ns, tw, lane, 32); break;
      case 7: stockham_stage<C, 7, INV>(a, b, P.L, Ns, tw, lane, 32); break;
      default: stockham_stage<C, 11, INV>(a, b, P.L, Ns, tw, lane, 32); break;
    }
    __syncwarp();
    C* t = a;
    a = b;
    b = t;
    Ns *= r;
  }
  return a;
}

// Forward: z DFT (direct, Nz -> Pz) then y FFT (Ny -> Py) of plane (b, x).
template <typename R>
__global__ void __launch_bounds__(256, FftOcc<R>::kMinBlocks) k_fft_fwd_planes(const typename GridT<R>::T* __restrict__ grid, int Nx, int Ny,
                                                        int Nz, FftPlan py, int Pz,
                                                        const typename V2<R>::T* __restrict__ twy,
                                                        const typename V2<R>::T* __restrict__ twz,
                                                        typename V2<R>::T* __restrict__ spec) {
  typedef typename V2<R>::T C;
  extern __shared__ unsigned char smem_raw[];
  const int Py = py.L;
  C* ty = reinterpret_cast<C*>(smem_raw);
  C* tz = ty + Py;
  const int LpY = padded_len(Py);
  C* b0 = tz + Pz;            // [kz][PAD(y)]
  C* b1 = b0 + Pz * LpY;      // [kz][PAD(y)]
  const int x = blockIdx.x, b = blockIdx.y;
  for (int i = threadIdx.x; i < Py; i += blockDim.x) ty[i] = twy[i];
  for (int i = threadIdx.x; i < Pz; i += blockDim.x) tz[i] = twz[i];
  const typename GridT<R>::T* src = grid + ((int64_t)b * Nx + x) * Ny * Nz;
  staged_copy<8, C>(Ny * Nz, [&](int i) { return grid_in<C>(src[i]); }, [&](int i, C v) { b1[i] = v; });   // staging [y][z]
  __syncthreads();
  // z DFT: a thread per y line, the root index kz z mod Pz kept incrementally
  for (int y = threadIdx.x; y < Py; y += blockDim.x) {
    const C* xr = b1 + y * Nz;
    for (int kz = 0; kz < Pz; ++kz) {
      C acc = czero<C>();
      if (y < Ny) {
        int m = 0;
        for (int z = 0; z < Nz; ++z) {
          cmac(acc, xr[z], tz[m]);
          m += kz;
          if (m >= Pz) m -= Pz;
        }
      }
      b0[kz * LpY + PAD(y)] = acc;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  C* res = nullptr;
  for (int kz = warp; kz < Pz; kz += nw) res = warp_fft<C, false>(b0 + kz * LpY, b1 + kz * LpY, py, ty, lane);
  __syncthreads();
  const bool in_b0 = (py.nst % 2) == 0;
  (void)res;
  const C* out = in_b0 ? b0 : b1;
  C* dst = spec + ((int64_t)b * Nx + x) * Py * Pz;
  const SmallDiv divz(Pz);
  for (int i = threadIdx.x; i < Py * Pz; i += blockDim.x) {
    int ky, kz;
    divz(i, ky, kz);
    dst[i] = out[kz * LpY + PAD(ky)];
  }
}

// x FFT (Nx -> Px), multiply by the Green's spectrum, inverse x FFT (keep Nx),
// for the Pz lines of one (b, ky); warp per line.
template <typename R>
__global__ void __launch_bounds__(256, FftOcc<R>::kMinBlocks) k_fft_conv_lines(typename V2<R>::T* __restrict__ spec, int Nx, int Py,
                                                        int Pz, FftPlan px, const typename V2<R>::T* __restrict__ twx,
                                                        const typename V2<R>::T* __restrict__ Ghat) {
  typedef typename V2<R>::T C;
  extern __shared__ unsigned char smem_raw[];
  const int Px = px.L;
  C* tx = reinterpret_cast<C*>(smem_raw);
  const int LpX = padded_len(Px);
  C* b0 = tx + Px;            // [kz][PAD(x)]
  C* b1 = b0 + Pz * LpX;
  const int ky = blockIdx.x, b = blockIdx.y;
  for (int i = threadIdx.x; i < Px; i += blockDim.x) tx[i] = twx[i];
  C* base = spec + (int64_t)b * Nx * Py * Pz + (int64_t)ky * Pz;
  const SmallDiv divz(Pz);
  staged_copy<8, C>(
      Pz * Px,
      [&](int i) {
        int x, kz;
        divz(i, x, kz);
        return (x < Nx) ? base[(int64_t)x * Py * Pz + kz] : czero<C>();
      },
      [&](int i, C v) {
        int x, kz;
        divz(i, x, kz);
        b0[kz * LpX + PAD(x)] = v;
      });
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int kz = warp; kz < Pz; kz += nw) {
    C* a = b0 + kz * LpX;
    C* c = b1 + kz * LpX;
    C* r = warp_fft<C, false>(a, c, px, tx, lane);
    const C* g = Ghat + ((int64_t)ky * Pz + kz) * Px;
    for (int i = lane; i < Px; i += 32) r[PAD(i)] = cmul(r[PAD(i)], g[i]);
    __syncwarp();
    C* other = (r == a) ? c : a;
    warp_fft<C, true>(r, other, px, tx, lane);
  }
  __syncthreads();
  // after 2 nst stages the result is back in the buffer that held the input
  const C* out = b0;
  for (int i = threadIdx.x; i < Pz * Nx; i += blockDim.x) {
    int x, kz;
    divz(i, x, kz);
    base[(int64_t)x * Py * Pz + kz] = out[kz * LpX + PAD(x)];
  }
}

// Inverse: y FFT (keep Ny) then z DFT (keep Nz) of plane (b, x).
template <typename R>
__global__ void __launch_bounds__(256, FftOcc<R>::kMinBlocks) k_fft_inv_planes(const typename V2<R>::T* __restrict__ spec, int Nx, int Ny,
                                                        int Nz, FftPlan py, int Pz,
                                                        const typename V2<R>::T* __restrict__ twy,
                                                        const typename V2<R>::T* __restrict__ twz,
                                                        typename GridT<R>::T* __restrict__ grid) {
  typedef typename V2<R>::T C;
  extern __shared__ unsigned char smem_raw[];
  const int Py = py.L;
  C* ty = reinterpret_cast<C*>(smem_raw);
  C* tz = ty + Py;
  const int LpY = padded_len(Py);
  C* b0 = tz + Pz;
  C* b1 = b0 + Pz * LpY;
  const int x = blockIdx.x, b = blockIdx.y;
  for (int i = threadIdx.x; i < Py; i += blockDim.x) ty[i] = twy[i];
  for (int i = threadIdx.x; i < Pz; i += blockDim.x) tz[i] = twz[i];
  const C* src = spec + ((int64_t)b * Nx + x) * Py * Pz;
  const SmallDiv divz(Pz);
  staged_copy<8, C>(
      Py * Pz, [&](int i) { return src[i]; },
      [&](int i, C v) {
        int ky, kz;
        divz(i, ky, kz);
        b0[kz * LpY + PAD(ky)] = v;
      });
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int kz = warp; kz < Pz; kz += nw) warp_fft<C, true>(b0 + kz * LpY, b1 + kz * LpY, py, ty, lane);
  __syncthreads();
  const C* res = (py.nst % 2 == 0) ? b0 : b1;
  typename GridT<R>::T* dst = grid + ((int64_t)b * Nx + x) * Ny * Nz;
  // inverse z DFT (first Nz outputs): a thread per y line
  for (int y = threadIdx.x; y < Ny; y += blockDim.x) {
    for (int z = 0; z < Nz; ++z) {
      C acc = czero<C>();
      int m = 0;
      for (int kz = 0; kz < Pz; ++kz) {
        C w = tz[m];
        w.y = -w.y;
        cmac(acc, res[kz * LpY + PAD(y)], w);
        m += z;
        if (m >= Pz) m -= Pz;
      }
      dst[y * Nz + z] = grid_out<typename GridT<R>::T>(acc);
    }
  }
}

// ---------------------------------------------------------------- A4: interpolation (step iii)
// y = v - [c_A sum_{xyz} Pi.Phi + c_phi Pi_phi.Phi_phi]; one CTA per element.
template <typename R, int CR>
__global__ void __launch_bounds__(CR == 1 ? (sizeof(R) == 4 ? 576 : 512) : 256, CR == 1 && sizeof(R) == 8 ? 1 : 2) k_interp(const int32_t* __restrict__ elems, int Nh, int S, int n1, int o1lo,
                                                int bx, int by, int bz, const int32_t* __restrict__ anc,
                                                const R* __restrict__ Pi, const int64_t* __restrict__ off,
                                                const int32_t* __restrict__ boxorg, int nrhs, int rc,
                                                const typename V2<R>::T* __restrict__ grid, int Nx, int Ny, int Nz,
                                                R cAr, R cAi, R cPr, R cPi,
                                                const typename V2<R>::T* __restrict__ v,
                                                typename V2<R>::T* __restrict__ y) {
  typedef typename V2<R>::T C;
  extern __shared__ unsigned char smem_raw[];
  C* box = reinterpret_cast<C*>(smem_raw);  // [psi][c][node]
  const int e = elems[blockIdx.x];
  const int nodes = bx * by * bz;
  const int64_t o = off[e];
  const int gx0 = boxorg[3 * e], gy0 = boxorg[3 * e + 1], gz0 = boxorg[3 * e + 2];
  const int64_t gstride = (int64_t)Nx * Ny * Nz;
  C cA, cP;
  cA.x = cAr; cA.y = cAi; cP.x = cPr; cP.y = cPi;
  // stencil point s -> box-node offset (ix by + iy) bz + iz, once per CTA
  int* soff = reinterpret_cast<int*>(box + 4 * rc * nodes);
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const int ix = s % n1, iy = (s / n1) % n1, iz = s / (n1 * n1);
    soff[s] = (ix * by + iy) * bz + iz;
  }
  const SmallDiv dnodes(nodes), dbyz(by * bz), dbz(bz);
  for (int c0 = 0; c0 < nrhs; c0 += rc) {
    const int cn = min(rc, nrhs - c0);
    const SmallDiv dcn(cn);
    staged_copy<8, C>(
        4 * cn * nodes,
        [&](int i) {
          int pc, node, psi, c, lx, r, ly, lz;
          dnodes(i, pc, node);
          dcn(pc, psi, c);
          dbyz(node, lx, r);
          dbz(r, ly, lz);
          const int64_t b = (int64_t)psi * nrhs + c0 + c;
          return grid[b * gstride + ((int64_t)(gx0 + lx) * Ny + (gy0 + ly)) * Nz + (gz0 + lz)];
        },
        [&](int i, C v) { box[i] = v; });
    __syncthreads();
    if constexpr (CR == 1) {
      // item = (basis n, right-hand side c); T consecutive lanes share an item
      // (T = 1, 2 or 4 when the block has the threads), each taking every
      // T-th stencil point, and add up by shuffles within their group
      const int items = Nh * cn;
      const int T = (int)blockDim.x >= 4 * items ? 4 : ((int)blockDim.x >= 2 * items ? 2 : 1);
      const int sub = threadIdx.x % T;
      const unsigned gmask = ((1u << T) - 1u) << ((threadIdx.x % 32) & ~(T - 1));
      for (int p = threadIdx.x / T; p < items; p += blockDim.x / T) {
        int n, c;
        dcn(p, n, c);
        C sA = czero<C>(), sP = czero<C>();
        const int nb = ((anc[3 * n] + o1lo) * by + (anc[3 * n + 1] + o1lo)) * bz + (anc[3 * n + 2] + o1lo);
        const C* bx0 = box + c * nodes + nb;
        for (int s = sub; s < S; s += T) {
          const int node = soff[s];
          const typename W4<R>::T w = W4<R>::load(Pi + ((int64_t)s * Nh + n) * 4);
          const C f0 = bx0[(0 * cn) * nodes + node];
          const C f1 = bx0[(1 * cn) * nodes + node];
          const C f2 = bx0[(2 * cn) * nodes + node];
          const C f3 = bx0[(3 * cn) * nodes + node];
          sA.x = fmx(w.x, f0.x, fmx(w.y, f1.x, fmx(w.z, f2.x, sA.x)));
          sA.y = fmx(w.x, f0.y, fmx(w.y, f1.y, fmx(w.z, f2.y, sA.y)));
          sP.x = fmx(w.w, f3.x, sP.x);
          sP.y = fmx(w.w, f3.y, sP.y);
        }
        for (int off2 = 1; off2 < T; off2 <<= 1) {
          sA.x += __shfl_xor_sync(gmask, sA.x, off2);
          sA.y += __shfl_xor_sync(gmask, sA.y, off2);
          sP.x += __shfl_xor_sync(gmask, sP.x, off2);
          sP.y += __shfl_xor_sync(gmask, sP.y, off2);
        }
        if (sub != 0) continue;
        const C yff = cadd(cmul(cA, sA), cmul(cP, sP));
        const int64_t idx = (o + n) * nrhs + c0 + c;
        y[idx] = csub(v[idx], yff);
      }
      __syncthreads();
      continue;
    }
    // item = (basis n, chunk of CR right-hand sides); consecutive threads take
    // consecutive bases (contiguous weights); each stencil weight and node index
    // is loaded once for the whole chunk
    const int nch = (cn + CR - 1) / CR;
    for (int p = threadIdx.x; p < Nh * nch; p += blockDim.x) {
      const int n = p % Nh, cb = (p / Nh) * CR;
      C sA[CR], sP[CR];
#pragma unroll
      for (int c = 0; c < CR; ++c) {
        sA[c] = czero<C>();
        sP[c] = czero<C>();
      }
      const int nb = ((anc[3 * n] + o1lo) * by + (anc[3 * n + 1] + o1lo)) * bz + (anc[3 * n + 2] + o1lo);
      for (int s = 0; s < S; ++s) {
        const int node = nb + soff[s];
        const typename W4<R>::T w = W4<R>::load(Pi + ((int64_t)s * Nh + n) * 4);
        const C* b0 = box + cb * nodes + node;
#pragma unroll
        for (int c = 0; c < CR; ++c) {
          if (cb + c < cn) {
            const C f0 = b0[(0 * cn + c) * nodes];
            const C f1 = b0[(1 * cn + c) * nodes];
            const C f2 = b0[(2 * cn + c) * nodes];
            const C f3 = b0[(3 * cn + c) * nodes];
            sA[c].x += w.x * f0.x + w.y * f1.x + w.z * f2.x;
            sA[c].y += w.x * f0.y + w.y * f1.y + w.z * f2.y;
            sP[c].x += w.w * f3.x;
            sP[c].y += w.w * f3.y;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < CR; ++c) {
        if (cb + c < cn) {
          const C yff = cadd(cmul(cA, sA[c]), cmul(cP, sP[c]));
          const int64_t idx = (o + n) * nrhs + c0 + cb + c;
          y[idx] = csub(v[idx], yff);
        }
      }
    }
    __syncthreads();
  }
}


// Interpolation of the float-float complex128 product: the schedule of
// k_interp for one right-hand side at a time (T lanes per basis), the element's
// box of FP64 potentials split into CF in shared memory, the weights as float
// pairs (Pf, as for the projection), the two sums per basis in float-float;
// y = v - (c_A sA + c_phi sP) in FP64.
__global__ void __launch_bounds__(576, 1) k_interp_ff(const int32_t* __restrict__ elems, int Nh, int S, int n1,
                                                      int o1lo, int bx, int by, int bz,
                                                      const int32_t* __restrict__ anc, const float4* __restrict__ Pf,
                                                      const int64_t* __restrict__ off,
                                                      const int32_t* __restrict__ boxorg, int nrhs,
                                                      const double2* __restrict__ grid, int Nx, int Ny, int Nz,
                                                      double cAr, double cAi, double cPr, double cPi,
                                                      const double2* __restrict__ v, double2* __restrict__ y) {
  extern __shared__ unsigned char smem_raw[];
  CF* box = reinterpret_cast<CF*>(smem_raw);   // [psi][node]
  const int e = elems[blockIdx.x];
  const int nodes = bx * by * bz;
  const int64_t o = off[e];
  const int gx0 = boxorg[3 * e], gy0 = boxorg[3 * e + 1], gz0 = boxorg[3 * e + 2];
  const int64_t gstride = (int64_t)Nx * Ny * Nz;
  int* soff = reinterpret_cast<int*>(box + 4 * nodes);
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const int ix = s % n1, iy = (s / n1) % n1, iz = s / (n1 * n1);
    soff[s] = (ix * by + iy) * bz + iz;
  }
  const int T = (int)blockDim.x >= 4 * Nh ? 4 : ((int)blockDim.x >= 2 * Nh ? 2 : 1);
  const int sub = threadIdx.x % T;
  const unsigned gmask = ((1u << T) - 1u) << ((threadIdx.x % 32) & ~(T - 1));
  const SmallDiv dnodes(nodes), dbyz(by * bz), dbz(bz);
  for (int c = 0; c < nrhs; ++c) {
    staged_copy<8, CF>(
        4 * nodes,
        [&](int i) {
          int psi, node, lx, r, ly, lz;
          dnodes(i, psi, node);
          dbyz(node, lx, r);
          dbz(r, ly, lz);
          return grid_in<CF>(grid[((int64_t)psi * nrhs + c) * gstride +
                                  ((int64_t)(gx0 + lx) * Ny + (gy0 + ly)) * Nz + (gz0 + lz)]);
        },
        [&](int i, CF val) { box[i] = val; });
    __syncthreads();
    for (int n = threadIdx.x / T; n < Nh; n += blockDim.x / T) {
      FF sAr = ff_zero(), sAi = ff_zero(), sPr = ff_zero(), sPi = ff_zero();
      const int nb = ((anc[3 * n] + o1lo) * by + (anc[3 * n + 1] + o1lo)) * bz + (anc[3 * n + 2] + o1lo);
      for (int s = sub; s < S; s += T) {
        const int node = nb + soff[s];
        const float4 wh = __ldg(Pf + ((int64_t)s * Nh + n) * 2), wl = __ldg(Pf + ((int64_t)s * Nh + n) * 2 + 1);
        const CF f0 = box[node], f1 = box[nodes + node], f2 = box[2 * nodes + node], f3 = box[3 * nodes + node];
        ff_mac(sAr, wh.x, wl.x, f0.x.h, f0.x.l);
        ff_mac(sAi, wh.x, wl.x, f0.y.h, f0.y.l);
        ff_mac(sAr, wh.y, wl.y, f1.x.h, f1.x.l);
        ff_mac(sAi, wh.y, wl.y, f1.y.h, f1.y.l);
        ff_mac(sAr, wh.z, wl.z, f2.x.h, f2.x.l);
        ff_mac(sAi, wh.z, wl.z, f2.y.h, f2.y.l);
        ff_mac(sPr, wh.w, wl.w, f3.x.h, f3.x.l);
        ff_mac(sPi, wh.w, wl.w, f3.y.h, f3.y.l);
      }
      for (int o2 = 1; o2 < T; o2 <<= 1) {
        sAr = ff_add(sAr, FF{__shfl_xor_sync(gmask, sAr.s, o2), __shfl_xor_sync(gmask, sAr.c, o2)});
        sAi = ff_add(sAi, FF{__shfl_xor_sync(gmask, sAi.s, o2), __shfl_xor_sync(gmask, sAi.c, o2)});
        sPr = ff_add(sPr, FF{__shfl_xor_sync(gmask, sPr.s, o2), __shfl_xor_sync(gmask, sPr.c, o2)});
        sPi = ff_add(sPi, FF{__shfl_xor_sync(gmask, sPi.s, o2), __shfl_xor_sync(gmask, sPi.c, o2)});
      }
      if (sub != 0) continue;
      const double ar = ff_to_double(sAr), ai = ff_to_double(sAi), pr = ff_to_double(sPr), pi = ff_to_double(sPi);
      const double yr = cAr * ar - cAi * ai + cPr * pr - cPi * pi;
      const double yi = cAr * ai + cAi * ar + cPr * pi + cPi * pr;
      const int64_t idx = (o + n) * nrhs + c;
      const double2 vv = v[idx];
      y[idx] = make_double2(vv.x - yr, vv.y - yi);
    }
    __syncthreads();
  }
}

// Interpolation of many right-hand sides from shared-memory tables (complex64):
// one launch for all types, each CTA a contiguous range of the elements listed
// type by type (walked forwards and backwards in turn, right-hand-side chunks
// outermost so that the grid planes being read stay in L2).  On entering a
// type its weights Pi ([s][n] float4) and the bases' first box nodes are
// copied into shared memory; per element and chunk of CH right-hand sides the
// box of grid potentials is staged as [psi][node][CH + 1]; a warp takes four
// bases at a time, lanes = CH right-hand sides x 4 bases, and walks the S
// stencil points with every read from shared memory.  y = v - (c_A sum_xyz +
// c_phi sum_phi).
__host__ __device__ inline size_t itp_box_offset(int S, int Nh, int nodes) {
  return ((size_t)16 * S * Nh + 4 * ((size_t)Nh + S + nodes) + 15) / 16 * 16;
}
template <int CH>
__host__ __device__ inline size_t itp_smem_bytes(int S, int Nh, int nodes) {
  return itp_box_offset(S, Nh, nodes) + (size_t)8 * 4 * nodes * (CH + 1);
}
size_t interp_tab_smem(int S, int Nh, int nodes) { return itp_smem_bytes<8>(S, Nh, nodes); }

template <int CH>
__global__ void __launch_bounds__(512, 1) k_interp_tab(const ItpTypeDev* __restrict__ types, int64_t total, int S,
                                                       int n1, int o1lo, const int64_t* __restrict__ off,
                                                       const int32_t* __restrict__ boxorg, int nrhs,
                                                       const float2* __restrict__ grid, int Nx, int Ny, int Nz,
                                                       float cAr, float cAi, float cPr, float cPi,
                                                       const float2* __restrict__ v, float2* __restrict__ y) {
  static_assert(CH == 8, "lanes: 8 right-hand sides x 4 bases");
  constexpr int LD = CH + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  const int c = lane % CH, g = lane / CH;
  const int64_t gstride = (int64_t)Nx * Ny * Nz;
  const int64_t i0 = (int64_t)blockIdx.x * total / gridDim.x, i1 = (int64_t)(blockIdx.x + 1) * total / gridDim.x;
  float2 cA, cP;
  cA.x = cAr; cA.y = cAi; cP.x = cPr; cP.y = cPi;
  int t = -1;
  int64_t tb = 0, te = 0;
  int Nh = 0, nodes = 0, by = 1, bz = 1;
  const int32_t* elems = nullptr;
  const float4* sPi = reinterpret_cast<const float4*>(smem_raw);
  int* nbt = nullptr;
  int* soff = nullptr;
  int* goff = nullptr;
  float2* box = nullptr;
  int pass = 0;
  for (int c0 = 0; c0 < nrhs; c0 += CH, ++pass) {
    for (int64_t k = 0; k < i1 - i0; ++k) {
      const int64_t gi = (pass & 1) ? i1 - 1 - k : i0 + k;
      if (gi < tb || gi >= te) {
        t = 0;
        tb = 0;
        te = types[0].ne;
        while (gi >= te) {
          ++t;
          tb = te;
          te += types[t].ne;
        }
        const ItpTypeDev ty = types[t];
        Nh = ty.Nh;
        by = ty.by;
        bz = ty.bz;
        nodes = ty.bx * by * bz;
        elems = ty.elems;
        nbt = reinterpret_cast<int*>(smem_raw + (size_t)16 * S * Nh);
        soff = nbt + Nh;
        goff = soff + S;
        box = reinterpret_cast<float2*>(smem_raw + itp_box_offset(S, Nh, nodes));
        __syncthreads();   // the previous type's tables are no longer read
        for (int i = threadIdx.x; i < S * Nh; i += blockDim.x)
          reinterpret_cast<float4*>(smem_raw)[i] = __ldg(reinterpret_cast<const float4*>(ty.Pi) + i);
        for (int n = threadIdx.x; n < Nh; n += blockDim.x)
          nbt[n] = ((ty.anc[3 * n] + o1lo) * by + (ty.anc[3 * n + 1] + o1lo)) * bz + (ty.anc[3 * n + 2] + o1lo);
        for (int sp = threadIdx.x; sp < S; sp += blockDim.x) {
          const int ix = sp % n1, iy = (sp / n1) % n1, iz = sp / (n1 * n1);
          soff[sp] = (ix * by + iy) * bz + iz;
        }
        for (int i = threadIdx.x; i < nodes; i += blockDim.x) {
          const int lz = i % bz, ly = (i / bz) % by, lx = i / (by * bz);
          goff[i] = (lx * Ny + ly) * Nz + lz;
        }
        __syncthreads();
      }
      const SmallDiv dnodes(nodes);
      const int e = elems[gi - tb];
      const int64_t o = off[e];
      const int64_t gbase = ((int64_t)boxorg[3 * e] * Ny + boxorg[3 * e + 1]) * Nz + boxorg[3 * e + 2];
      // stage: consecutive threads take consecutive nodes of one (psi, c) plane
      for (int i = threadIdx.x; i < 4 * CH * nodes; i += blockDim.x) {
        int pc, node;
        dnodes(i, pc, node);
        const int q = pc / CH, cc = pc % CH;
        float2 val = make_float2(0.f, 0.f);
        if (c0 + cc < nrhs) val = grid[((int64_t)q * nrhs + c0 + cc) * gstride + gbase + goff[node]];
        box[((size_t)q * nodes + node) * LD + cc] = val;
      }
      __syncthreads();
      for (int n0 = 4 * warp; n0 < Nh; n0 += 4 * nw) {
        const int n = n0 + g;
        if (n < Nh) {
          const int nb = nbt[n];
          // v of this output is loaded first, so that its latency passes during the sums
          const bool live = c0 + c < nrhs;
          const int64_t idx = (o + n) * nrhs + c0 + c;
          const float2 vv = live ? v[idx] : make_float2(0.f, 0.f);
          float2 sA = make_float2(0.f, 0.f), sP = make_float2(0.f, 0.f);
#pragma unroll 3
          for (int sp = 0; sp < S; ++sp) {
            const float4 w = sPi[sp * Nh + n];
            const float2* b = box + (size_t)(nb + soff[sp]) * LD + c;
            const float2 f0 = b[0], f1 = b[(size_t)nodes * LD], f2 = b[(size_t)2 * nodes * LD],
                         f3 = b[(size_t)3 * nodes * LD];
            sA.x = fmaf(w.x, f0.x, fmaf(w.y, f1.x, fmaf(w.z, f2.x, sA.x)));
            sA.y = fmaf(w.x, f0.y, fmaf(w.y, f1.y, fmaf(w.z, f2.y, sA.y)));
            sP.x = fmaf(w.w, f3.x, sP.x);
            sP.y = fmaf(w.w, f3.y, sP.y);
          }
          if (live) y[idx] = csub(vv, cadd(cmul(cA, sA), cmul(cP, sP)));
        }
      }
      __syncthreads();
    }
  }
}

// Interpolation of many right-hand sides (complex64), lanes over right-hand
// sides: one CTA per element; per chunk of CH right-hand sides the element's box
// of grid potentials is staged as [psi][node][c] (c fastest, node stride CH + 1
// so that the staging stores of consecutive nodes spread over the banks); a
// warp takes four bases at a time, its lanes = CH right-hand sides x 4 bases,
// and walks the S stencil points: one weight load per point for CH columns,
// four conflict-free box loads.  y = v - (c_A sum_xyz + c_phi sum_phi).
template <int CH>
__global__ void __launch_bounds__(256) k_interp_rhs(const int32_t* __restrict__ elems, int Nh, int S, int n1, int o1lo,
                                                    int bx, int by, int bz, const int32_t* __restrict__ anc,
                                                    const float* __restrict__ Pi, const int64_t* __restrict__ off,
                                                    const int32_t* __restrict__ boxorg, int nrhs,
                                                    const float2* __restrict__ grid, int Nx, int Ny, int Nz, float cAr,
                                                    float cAi, float cPr, float cPi, const float2* __restrict__ v,
                                                    float2* __restrict__ y) {
  static_assert(CH == 8, "lanes: 8 right-hand sides x 4 bases");
  constexpr int LD = CH + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nodes = bx * by * bz;
  float2* box = reinterpret_cast<float2*>(smem_raw);                   // [psi][node][LD]
  int* soff = reinterpret_cast<int*>(box + (size_t)4 * nodes * LD);    // S
  int* goff = soff + S;                                                 // nodes
  const int e = elems[blockIdx.x];
  const int64_t o = off[e];
  const int64_t gbase = ((int64_t)boxorg[3 * e] * Ny + boxorg[3 * e + 1]) * Nz + boxorg[3 * e + 2];
  const int64_t gstride = (int64_t)Nx * Ny * Nz;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const int ix = s % n1, iy = (s / n1) % n1, iz = s / (n1 * n1);
    soff[s] = (ix * by + iy) * bz + iz;
  }
  for (int i = threadIdx.x; i < nodes; i += blockDim.x) {
    const int lz = i % bz, ly = (i / bz) % by, lx = i / (by * bz);
    goff[i] = (lx * Ny + ly) * Nz + lz;
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  const int c = lane % CH, g = lane / CH;
  const SmallDiv dnodes(nodes);
  float2 cA, cP;
  cA.x = cAr; cA.y = cAi; cP.x = cPr; cP.y = cPi;
  for (int c0 = 0; c0 < nrhs; c0 += CH) {
    __syncthreads();   // tables written; the previous chunk's box no longer read
    // stage: consecutive threads take consecutive nodes of one (psi, c) plane
    for (int i = threadIdx.x; i < 4 * CH * nodes; i += blockDim.x) {
      int pc, node;
      dnodes(i, pc, node);
      const int q = pc / CH, cc = pc % CH;
      float2 val = make_float2(0.f, 0.f);
      if (c0 + cc < nrhs) val = grid[((int64_t)q * nrhs + c0 + cc) * gstride + gbase + goff[node]];
      box[((size_t)q * nodes + node) * LD + cc] = val;
    }
    __syncthreads();
    for (int n0 = 4 * warp; n0 < Nh; n0 += 4 * nw) {
      const int n = n0 + g;
      if (n >= Nh) continue;
      const int nb = ((anc[3 * n] + o1lo) * by + (anc[3 * n + 1] + o1lo)) * bz + (anc[3 * n + 2] + o1lo);
      float2 sA = make_float2(0.f, 0.f), sP = make_float2(0.f, 0.f);
#pragma unroll 3
      for (int s = 0; s < S; ++s) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(Pi) + ((int64_t)s * Nh + n));
        const float2* b = box + (size_t)(nb + soff[s]) * LD + c;
        const float2 f0 = b[0], f1 = b[(size_t)nodes * LD], f2 = b[(size_t)2 * nodes * LD],
                     f3 = b[(size_t)3 * nodes * LD];
        sA.x = fmaf(w.x, f0.x, fmaf(w.y, f1.x, fmaf(w.z, f2.x, sA.x)));
        sA.y = fmaf(w.x, f0.y, fmaf(w.y, f1.y, fmaf(w.z, f2.y, sA.y)));
        sP.x = fmaf(w.w, f3.x, sP.x);
        sP.y = fmaf(w.w, f3.y, sP.y);
      }
      if (c0 + c < nrhs) {
        const float2 yff = cadd(cmul(cA, sA), cmul(cP, sP));
        const int64_t idx = (o + n) * nrhs + c0 + c;
        y[idx] = csub(v[idx], yff);
      }
    }
  }
}
// ---------------------------------------------------------------- A5: near field
// y[row] -= sum_k val[k] u[col[k]].  Rows are padded to multiples of 4 entries
// (zero values), so a lane reads 4 columns with one 16-byte load and 4 values
// with 16-byte loads.  Single RHS: warp per row.
template <typename R>
__global__ void __launch_bounds__(256) k_spmv_near1(int64_t N, const int64_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col,
                                                    const typename V2<R>::T* __restrict__ val,
                                                    const typename V2<R>::T* __restrict__ u,
                                                    typename V2<R>::T* __restrict__ y) {
  typedef typename V2<R>::T C;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= N) return;
  const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
  C s0 = czero<C>(), s1 = czero<C>();   // two accumulators: shorter FMA chains
  for (int64_t p = p0 + 4 * lane; p < p1; p += 128) {
    const int4 c4 = __ldg(reinterpret_cast<const int4*>(col + p));
    C v[4];
    if (sizeof(R) == 4) {
      const float4 a01 = __ldg(reinterpret_cast<const float4*>(val + p));
      const float4 a23 = __ldg(reinterpret_cast<const float4*>(val + p + 2));
      v[0].x = a01.x; v[0].y = a01.y; v[1].x = a01.z; v[1].y = a01.w;
      v[2].x = a23.x; v[2].y = a23.y; v[3].x = a23.z; v[3].y = a23.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = val[p + q];
    }
    const C b0 = u[c4.x], b1 = u[c4.y], b2 = u[c4.z], b3 = u[c4.w];
    cmac(s0, v[0], b0);
    cmac(s1, v[1], b1);
    cmac(s0, v[2], b2);
    cmac(s1, v[3], b3);
  }
  R ar = s0.x + s1.x, ai = s0.y + s1.y;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, s);
    ai += __shfl_xor_sync(0xffffffffu, ai, s);
  }
  if (lane == 0) {
    C o = y[row];
    o.x -= ar;
    o.y -= ai;
    y[row] = o;
  }
}

// FP64 near field with three real products per term (values stored as Re,
// Im, Re + Im; us = Re u + Im u from the GEMM, or formed here when absent):
// sums t1 = sum Re a Re u, t2 = sum Im a Im u, t3 = sum (Re a + Im a)(Re u + Im u),
// and y -= (t1 - t2) + i (t3 - t1 - t2).  Bound by GB300's FP64 rate: three FMAs
// per non-zero instead of four.
template <int RC>
__global__ void __launch_bounds__(256) k_spmv_near_3m(int64_t N, const int64_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ val3, int nrhs,
                                                      const double2* __restrict__ u, const double* __restrict__ us,
                                                      double2* __restrict__ y) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= N) return;
  const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
  for (int c0 = 0; c0 < nrhs; c0 += RC) {
    double t1[RC], t2[RC], t3[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) t1[c] = t2[c] = t3[c] = 0.0;
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const double ar = val3[3 * p], ai = val3[3 * p + 1], as = val3[3 * p + 2];
      const int64_t cidx = (int64_t)col[p] * nrhs + c0;
#pragma unroll
      for (int c = 0; c < RC; ++c)
        if (c0 + c < nrhs) {
          const double2 b = u[cidx + c];
          const double bs = us != nullptr ? us[cidx + c] : b.x + b.y;
          t1[c] = __fma_rn(ar, b.x, t1[c]);
          t2[c] = __fma_rn(ai, b.y, t2[c]);
          t3[c] = __fma_rn(as, bs, t3[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < RC; ++c) {
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        t1[c] += __shfl_xor_sync(0xffffffffu, t1[c], s);
        t2[c] += __shfl_xor_sync(0xffffffffu, t2[c], s);
        t3[c] += __shfl_xor_sync(0xffffffffu, t3[c], s);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < RC; ++c)
        if (c0 + c < nrhs) {
          const int64_t idx = row * nrhs + c0 + c;
          double2 o = y[idx];
          o.x -= t1[c] - t2[c];
          o.y -= t3[c] - t1[c] - t2[c];
          y[idx] = o;
        }
    }
  }
}

// Several RHS: warp per row, RHS columns in passes of RC.
template <typename R, int RC>
__global__ void __launch_bounds__(256) k_spmv_near(int64_t N, const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col,
                                                   const typename V2<R>::T* __restrict__ val, int nrhs,
                                                   const typename V2<R>::T* __restrict__ u,
                                                   typename V2<R>::T* __restrict__ y) {
  typedef typename V2<R>::T C;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= N) return;
  const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
  for (int c0 = 0; c0 < nrhs; c0 += RC) {
    C acc[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[c] = czero<C>();
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const C a = val[p];
      const int64_t cidx = (int64_t)col[p] * nrhs + c0;
#pragma unroll
      for (int c = 0; c < RC; ++c)
        if (c0 + c < nrhs) {
          const C b = u[cidx + c];
          cmac(acc[c], a, b);
        }
    }
#pragma unroll
    for (int c = 0; c < RC; ++c) {
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, s);
        acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, s);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < RC; ++c)
        if (c0 + c < nrhs) {
          const int64_t idx = row * nrhs + c0 + c;
          y[idx] = csub(y[idx], acc[c]);
        }
    }
  }
}

// y_a -= B_q u_b over all element pairs (a, b) and their distinct near-field
// blocks q, in one launch.  B_q is dense (rows of a's type, columns of b's);
// only its 16-column k tiles that hold a non-zero in the CTA's 64-row tile are
// visited; each type's bases are stored in anchor order (perm: sorted position
// -> basis), which gathers the near pairs into fewer tiles.  The GEMM's
// columns are (pair, right-hand side), n = p nrhs + c, so one right-hand side
// still fills the tiles.  Tiles are numbered group by
// group (group = the pairs of one block: row tiles x column tiles); a CTA
// finds its group by a prefix over the group sizes, staged in shared memory
// 128 groups at a time.  A row element has up to one pair per lattice offset,
// so its outputs receive several block products: they are accumulated with
// atomic adds (summation order not fixed).  The CTA's set-up loads are issued
// in as few dependent rounds as possible (the CTAs do only a few k tiles each).
// Arithmetic of the block near field: plain complex (R = float or double), or
// float-float (NearFF: F6 operands, three Gauss sums per output, FP64 output).
template <typename R> struct NearPlain {
  typedef typename V2<R>::T V;   // staged operand entry (block value, u)
  typedef typename V2<R>::T A;   // accumulator of one output
  typedef typename V2<R>::T Y;   // output element
  // CTAs per SM asked of the compiler: the shape's count for complex64, one for FP64
  static constexpr int min_blocks(int mb) { return sizeof(R) == 4 ? mb : 1; }
  static constexpr int kUnrollK = 16;   // the whole k tile
  static __device__ __forceinline__ V vzero() { return czero<V>(); }
  static __device__ __forceinline__ A azero() { return czero<A>(); }
  static __device__ __forceinline__ V load(const V* p) { return *p; }
  static __device__ __forceinline__ void mac(A& acc, const V& a, const V& b) { cmac(acc, a, b); }
  static __device__ __forceinline__ void sub(Y* dst, const A& acc) {
    R* d = reinterpret_cast<R*>(dst);
    atomicAdd(d, -acc.x);
    atomicAdd(d + 1, -acc.y);
  }
};
struct NearFF {
  typedef F6 V;
  typedef FF3 A;
  typedef double2 Y;
  static constexpr int min_blocks(int mb) { return mb; }
  // two k steps per loop body: the unrolled float-float tile is some 5,000
  // instructions, which the instruction cache does not hold
  static constexpr int kUnrollK = 2;
  static __device__ __forceinline__ V vzero() { return f6_zero(); }
  static __device__ __forceinline__ A azero() { return ff3_zero(); }
  static __device__ __forceinline__ V load(const V* p) { return f6_load(p); }
  static __device__ __forceinline__ void mac(A& acc, const V& a, const V& b) { ff3_mac(acc, a, b); }
  static __device__ __forceinline__ void sub(Y* dst, const A& acc) {
    FF re, im;
    ff3_result(acc, re, im);
    atomicAdd(&dst->x, -ff_to_double(re));
    atomicAdd(&dst->y, -ff_to_double(im));
  }
};

template <typename Ar, int TN, int MB, int TM>
__global__ void __launch_bounds__(16 * (TN / 4), Ar::min_blocks(MB)) k_near_blocks(
    const NearGroupDev* __restrict__ groups, int ngroups, const longlong2* __restrict__ poff,
    const typename Ar::V* __restrict__ vals, const int64_t* __restrict__ boff, const int32_t* __restrict__ bnb,
    int nmt, const int32_t* __restrict__ tptr, const int32_t* __restrict__ tlist, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ bpa, const int32_t* __restrict__ bpb, int nrhs,
    int ksplit, const typename Ar::V* __restrict__ u, typename Ar::Y* __restrict__ y) {
  typedef typename Ar::V C;
  // TM rows (64 or 32) x TN columns per CTA, MR x 4 complex outputs per thread
  constexpr int TK = 16, TX = TN / 4, NT = 16 * TX, MR = TM / 16;
  __shared__ C As[TK][TM + 1];
  __shared__ C Bs[TK][TN + 1];
  __shared__ int64_t cin[TN], cout[TN];   // u / y index of row 0 of each column, -1 past the end
  __shared__ int64_t s_nt[NT];            // tiles of up to NT groups (prefix search)
  __shared__ int s_g, s_mt;
  __shared__ int64_t s_ct, s_t;
  __shared__ NearGroupDev s_gr;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const int part = blockIdx.y;   // which of the ksplit shares of the row tile's k tiles
  if (tid == 0) {
    s_g = ngroups;
    s_t = blockIdx.x;
  }
  for (int g0 = 0; g0 < ngroups; g0 += NT) {
    __syncthreads();
    if (s_g < ngroups) break;   // found in an earlier chunk
    const int g = g0 + tid;
    if (g < ngroups) {
      const NearGroupDev gg = groups[g];
      s_nt[tid] = ((gg.npairs * nrhs + TN - 1) / TN) * ((gg.Na + TM - 1) / TM);
    }
    __syncthreads();
    if (tid == 0) {
      int64_t t = s_t;
      for (int q = 0; q < NT && g0 + q < ngroups; ++q) {
        if (t < s_nt[q]) {
          const NearGroupDev gg = groups[g0 + q];
          const int64_t nct = (gg.npairs * nrhs + TN - 1) / TN;
          s_gr = gg;
          s_g = g0 + q;
          s_mt = (int)(t / nct);
          s_ct = t % nct;
          break;
        }
        t -= s_nt[q];
      }
      s_t = t;
    }
  }
  __syncthreads();
  if (s_g >= ngroups) return;
  const NearGroupDev gr = s_gr;
  const int mt = s_mt, q = gr.q, Na = gr.Na;
  // one round of loads that depend only on the block and the tile
  const int Nb = bnb[q];
  const C* Bq = vals + boff[q];
  const int32_t* pa = perm + bpa[q];   // the block's rows and columns are in anchor order
  const int32_t* pb = perm + bpb[q];
  const int ea = tptr[q * nmt + mt], eb = tptr[q * nmt + mt + 1];
  const int m0 = mt * TM;
  const int64_t ncol = gr.npairs * nrhs, n0 = s_ct * TN;
  for (int cc = tid; cc < TN; cc += NT) {
    const int64_t n = n0 + cc;
    if (n < ncol) {
      const int64_t pp = n / nrhs;
      const int c = (int)(n - pp * nrhs);
      const longlong2 pr = poff[gr.first_pair + pp];   // (row element, column element) unknown offsets
      cin[cc] = pr.y * nrhs + c;
      cout[cc] = pr.x * nrhs + c;
    } else {
      cin[cc] = -1;
      cout[cc] = -1;
    }
  }
  typename Ar::A acc[MR][4];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Ar::azero();
  __syncthreads();
  const bool kfast = nrhs < 16;   // few right-hand sides: a column's rows are the contiguous run
  const int e0 = ea + (int)((int64_t)(eb - ea) * part / ksplit), e1 = ea + (int)((int64_t)(eb - ea) * (part + 1) / ksplit);
  if (e0 == e1) return;   // nothing in this share
  // the next k tile is loaded into registers while the current one is used
  constexpr int NA = TM * TK / NT, NB = TK * TN / NT;
  C ra[NA], rb[NB];
  auto fetch = [&](int e) {
    const int k0 = tlist[e] * TK;
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      const int idx = tid + r * NT, m = idx / TK, kk = idx % TK;
      ra[r] = (m0 + m < Na && k0 + kk < Nb) ? Ar::load(Bq + (int64_t)(m0 + m) * Nb + k0 + kk) : Ar::vzero();
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const int idx = tid + r * NT;
      const int kk = kfast ? idx % TK : idx / TN, cc = kfast ? idx / TK : idx % TN;
      const int64_t ci = cin[cc];
      rb[r] = (ci >= 0 && k0 + kk < Nb) ? Ar::load(u + ci + (int64_t)pb[k0 + kk] * nrhs) : Ar::vzero();
    }
  };
  if (e0 < e1) fetch(e0);
  for (int e = e0; e < e1; ++e) {
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      const int idx = tid + r * NT;
      As[idx % TK][idx / TK] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const int idx = tid + r * NT;
      const int kk = kfast ? idx % TK : idx / TN, cc = kfast ? idx / TK : idx % TN;
      Bs[kk][cc] = rb[r];
    }
    __syncthreads();
    if (e + 1 < e1) fetch(e + 1);
#pragma unroll Ar::kUnrollK
    for (int kk = 0; kk < TK; ++kk) {
      C a[MR], b[4];
#pragma unroll
      for (int i = 0; i < MR; ++i) a[i] = As[kk][ty * MR + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          Ar::mac(acc[i][j], a[i], b[j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t co = cout[tx * 4 + j];
    if (co < 0) continue;
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int m = m0 + ty * MR + i;
      if (m < Na) Ar::sub(y + co + (int64_t)pa[m] * nrhs, acc[i][j]);
    }
  }
}

template <typename R, int TN, int MB, int TM = 64>
static void near_blocks_launch(const DevArray& a, const DevPrec<R>& p, int nrhs, const typename V2<R>::T* u,
                               typename V2<R>::T* y, cudaStream_t st, int& nl, int ksplit) {
  int64_t tiles = 0;
  for (const auto& g : a.nfg) tiles += ((g.npairs * nrhs + TN - 1) / TN) * ((g.Na + TM - 1) / TM);
  if (tiles == 0) return;
  // ksplit > 1 splits each row tile's k tiles over several CTAs (the outputs are
  // accumulated atomically anyway): more CTAs when the output tiles are few
  k_near_blocks<NearPlain<R>, TN, MB, TM><<<dim3((unsigned)tiles, (unsigned)ksplit), 16 * (TN / 4), 0, st>>>(
      reinterpret_cast<const NearGroupDev*>(a.nfg_dev), (int)a.nfg.size(), a.nfg_poff,
      static_cast<const typename V2<R>::T*>(p.nfb_val), a.nfb_off, a.nfb_nb, TM == 64 ? a.nfb_nmt : a.nfb_nmt32,
      TM == 64 ? a.nfb_tptr : a.nfb_tptr32, TM == 64 ? a.nfb_tlist : a.nfb_tlist32,
      a.nfb_perm, a.nfb_pa, a.nfb_pb, nrhs, ksplit, u, y);
  ++nl;
}

// The block near field of the float-float complex128 product: 32 x 32 tiles,
// one CTA per tile (the F6 operands and three Gauss sums per output hold about
// 150 registers per thread), outputs added to v in FP64.
template <int TN, int MB, int TM>
static void near_ff_shape(const DevArray& a, const DevPrec<double>& pd, int nrhs, const F6* u6, double2* y,
                          cudaStream_t st) {
  int64_t tiles = 0;
  for (const auto& g : a.nfg) tiles += ((g.npairs * nrhs + TN - 1) / TN) * ((g.Na + TM - 1) / TM);
  if (tiles == 0) return;
  k_near_blocks<NearFF, TN, MB, TM><<<dim3((unsigned)tiles, 1u), 16 * (TN / 4), 0, st>>>(
      reinterpret_cast<const NearGroupDev*>(a.nfg_dev), (int)a.nfg.size(), a.nfg_poff,
      static_cast<const F6*>(pd.ff_nfb), a.nfb_off, a.nfb_nb, TM == 64 ? a.nfb_nmt : a.nfb_nmt32,
      TM == 64 ? a.nfb_tptr : a.nfb_tptr32, TM == 64 ? a.nfb_tlist : a.nfb_tlist32, a.nfb_perm, a.nfb_pa, a.nfb_pb,
      nrhs, 1, u6, y);
}
static void near_blocks_ff_launch(const DevArray& a, const DevPrec<double>& pd, int nrhs, const F6* u6, double2* y,
                                  cudaStream_t st, int& nl) {
  switch (a.ff_near_shape) {
    case 1: near_ff_shape<32, 3, 32>(a, pd, nrhs, u6, y, st); break;
    case 2: near_ff_shape<64, 1, 32>(a, pd, nrhs, u6, y, st); break;
    case 3: near_ff_shape<16, 1, 32>(a, pd, nrhs, u6, y, st); break;
    default: near_ff_shape<32, 1, 32>(a, pd, nrhs, u6, y, st); break;
  }
  ++nl;
}

// Kernel shapes of the block near field (64-row tiles unless named): 0 =
// 32-column tiles (four CTAs per SM), 1 = 32-column tiles compiled for five CTAs
// per SM (fewer registers, more warps to hide the loads), 2 = 64-column tiles
// (two CTAs per SM), 3 = 32 x 32 tiles (eight CTAs per SM), 4 = 32 x 64 tiles
// (four CTAs per SM).  32-row tiles skip more zero k tiles of the sparse blocks
// (about 1.9 times the non-zero work instead of 2.3 at 16x16).  The CTA counts
// per SM apply to complex64; the FP64 forms keep their registers.
// Shapes 5 and 6 are the tensor-core form (near_tc.cu: 32 or 64 complex
// columns per tile, partial sums; k split 2 for up to 8 right-hand sides), 7-9
// its direct form (32 or 64 right-hand sides per tile, an even count of them),
// complex64 only.
template <typename R>
static bool near_shape_ok(int shape, const DevArray& a, const DevPrec<R>& p, int nrhs, const void* u, const void* v,
                          const void* np) {
  if (shape < 5) return true;
  if (sizeof(R) != 4 || p.nfb_tc == nullptr) return false;
  if (shape < 7) return np != nullptr;
  return nrhs >= 16 && near_tc_direct_ok(a, nrhs, u, v);
}

template <typename R>
static void near_shape_launch(int shape, const DevArray& a, const DevPrec<R>& p, int nrhs,
                              const typename V2<R>::T* u, typename V2<R>::T* y, cudaStream_t st, int& nl, int ks,
                              void* np, int np_parts = 1) {
  if (shape >= 5) {
    if constexpr (sizeof(R) == 4) {
      if (near_shape_ok<R>(shape, a, p, nrhs, u, y, np)) {
        near_tc_launch(shape - 5, a, p, nrhs, u, y, static_cast<float2*>(np), std::min(ks, np_parts), st);
        nl += shape >= 7 ? 1 : 2;
        return;
      }
    }
    shape = 0;
    ks = 1;
  }
  if (shape == 4)
    near_blocks_launch<R, 64, 4, 32>(a, p, nrhs, u, y, st, nl, ks);
  else if (shape == 3)
    near_blocks_launch<R, 32, 8, 32>(a, p, nrhs, u, y, st, nl, ks);
  else if (shape == 2)
    near_blocks_launch<R, 64, 2>(a, p, nrhs, u, y, st, nl, ks);
  else if (shape == 1)
    near_blocks_launch<R, 32, 5>(a, p, nrhs, u, y, st, nl, ks);
  else
    near_blocks_launch<R, 32, 4>(a, p, nrhs, u, y, st, nl, ks);
}

// Size rule of the block near field (products that may not time shapes, and
// the fallback when timing fails): tensor cores when their blocks exist (the
// direct form from 64 right-hand sides), else 64 x 64 tiles for many columns,
// 64 x 32 tiles with a k split of 4 for few.
template <typename R>
static std::pair<int, int> near_size_rule(const DevArray& a, const DevPrec<R>& p, int nrhs, const void* u,
                                          const void* v, void* np) {
  int64_t cols = 0;
  for (const auto& g : a.nfg) cols += g.npairs * nrhs;
  std::pair<int, int> best = {cols >= (int64_t)64 * 4 * 152 ? 2 : 0, cols >= (int64_t)64 * 4 * 152 ? 1 : 4};
  if (near_shape_ok<R>(5, a, p, nrhs, u, v, np)) best = {cols >= (int64_t)64 * 4 * 152 ? 6 : 5, 1};
  if (nrhs >= 64 && near_shape_ok<R>(8, a, p, nrhs, u, v, np)) best = {8, 1};
  return best;
}

// (The FFT kernels' complex64 forms are bounded to 3 CTAs per SM, which they
// reach without spilling; the transforms are latency-bound.)
// ---------------------------------------------------------------- launchers
template <typename R>
size_t fft_smem_bytes(const DevArray& a, int which) {
  const size_t cs = sizeof(typename V2<R>::T);
  const int Py = a.fft[1], Pz = a.fft[2], Px = a.fft[0];
  if (which == 0) return cs * ((size_t)Py + Pz + 2 * (size_t)Pz * padded_len(Py));
  return cs * ((size_t)Px + 2 * (size_t)Pz * padded_len(Px));
}

static int box_rc(const DevArray& a, int t, int nrhs, size_t csize, size_t limit) {
  const size_t nodes = (size_t)a.box[3 * t] * a.box[3 * t + 1] * a.box[3 * t + 2];
  int rc = nrhs;
  while (rc > 1 && 4 * rc * nodes * csize > limit) rc = (rc + 1) / 2;
  return rc;
}

cudaError_t kernels_init(DevArray& a) {
  const int lim = 200 * 1024;
  cudaError_t e;
#define MM_ATTR(K)                                                                \
  e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
  if (e != cudaSuccess) return e;
  MM_ATTR(k_fft_fwd_planes<float>) MM_ATTR(k_fft_fwd_planes<double>)
  MM_ATTR(k_fft_conv_lines<float>) MM_ATTR(k_fft_conv_lines<double>)
  MM_ATTR(k_fft_inv_planes<float>) MM_ATTR(k_fft_inv_planes<double>)
  MM_ATTR(k_fft_fwd_planes<FFTag>) MM_ATTR(k_fft_conv_lines<FFTag>) MM_ATTR(k_fft_inv_planes<FFTag>)
  MM_ATTR(k_project_ff) MM_ATTR(k_interp_ff)
  MM_ATTR((k_project<float, 1>)) MM_ATTR((k_project<double, 1>)) MM_ATTR((k_project<float, 4>))
  MM_ATTR((k_project<double, 4>))
  MM_ATTR((k_interp<float, 1>)) MM_ATTR((k_interp<double, 1>)) MM_ATTR((k_interp<float, 8>))
  MM_ATTR((k_interp<double, 8>))
#undef MM_ATTR
  e = cudaFuncSetAttribute(k_project_tab<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrjSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_interp_rhs<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInterpRhsSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_interp_tab<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInterpTabSmemMax);
  if (e != cudaSuccess) return e;
  e = tc_gemm_init();
  if (e != cudaSuccess) return e;
  return near_tc_init(a);
}

// Launch schedules of the projection and the interpolation (the grid-stage
// tuner's choices).  Projection, one right-hand side: variant v < 3 gives 4 >> v
// lanes per stencil-box node (4, 2, 1; CTAs of up to 512 threads), variant 3
// (complex64) reads the type's stencil tables (k_project_g1); several:
// variant 0 stages four right-hand sides per pass (RC = 4), variant 1 one,
// variant 2 (eight or more, when the array has a box buffer) is the two-pass
// form: each element writes its box, then every grid point sums the boxes
// covering it (no atomics); variant 3 (complex64, eight or more, when the
// type's tables fit in shared memory) is the table-driven form k_project_tab,
// eight right-hand sides per pass.
// Interpolation, one right-hand side: 4 >> v lanes per basis; eight or more:
// variant 0 takes eight right-hand sides per thread (CR = 8), variant 1 one,
// variant 2 (complex64) puts eight right-hand sides on the lanes of a warp
// (k_interp_rhs), variant 3 (complex64, where the weights fit) does the same
// from shared-memory weights in one launch for all types (k_interp_tab).
size_t project_tab_smem(int E, int nodes, int Nh) { return prj_smem_bytes<8>(E, nodes, Nh); }

// The table-driven projection applies when every type's tables, u chunk and
// box fit in shared memory (complex64, eight or more right-hand sides).
template <typename R>
static bool project_tab_all(const DevArray& a, const DevPrec<R>& p, int nrhs) {
  (void)a;
  return sizeof(R) == 4 && nrhs >= 8 && p.prj_types != nullptr && p.prj_smem <= kPrjSmemMax && p.prj_total > 0;
}

template <typename R>
static void project_launch(int var, const DevArray& a, const DevPrec<R>& p, int nrhs, const typename V2<R>::T* u,
                           typename V2<R>::T* grid, void* boxbuf, cudaStream_t cs, int& nl) {
  typedef typename V2<R>::T C;
  const int Nx = a.grid[0], Ny = a.grid[1], Nz = a.grid[2];
  if constexpr (sizeof(R) == 4) {
    if (var == 3 && project_tab_all(a, p, nrhs)) {
      int dev = 0, sms = 148;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int ctas = (int)std::min<int64_t>(p.prj_total, sms);
      k_project_tab<8><<<ctas, 512, p.prj_smem, cs>>>(p.prj_types, p.prj_total, a.off, a.boxorg, nrhs, u, Nx, Ny,
                                                     Nz, grid);
      ++nl;
      return;
    }
  }
  for (int64_t t = 0; t < a.n_types; ++t) {
    if (a.n_of_type[t] == 0) continue;
    const int Nh = (int)a.Nh[t];
    const int bx = a.box[3 * t], by = a.box[3 * t + 1], bz = a.box[3 * t + 2];
    const int pnodes = bx * by * bz;
    if constexpr (sizeof(R) == 4) {
      if (var == 3 && nrhs == 1 && (size_t)t < p.prj_tab.size()) {
        // 16 warps of 8 nodes per round; u and the list starts in shared memory
        k_project_g1<<<(unsigned)a.n_of_type[t], 512, sizeof(float2) * Nh + sizeof(int) * (pnodes + 1), cs>>>(
            a.elems[t], Nh, bx, by, bz, a.inv_ptr[t], static_cast<const unsigned char*>(p.prj_tab[t]), a.inv_len[t],
            a.off, a.boxorg, reinterpret_cast<const float2*>(u), Nx, Ny, Nz, reinterpret_cast<float2*>(grid));
        ++nl;
        continue;
      }
    }
    if (nrhs == 1 || var == 1) {
      // T lanes per node with T nodes <= 512 (two CTAs fit on an SM: one wave)
      int pT = nrhs == 1 ? (4 >> var) : 1;
      while (pT > 1 && pT * pnodes > 512) pT >>= 1;
      const int pthreads = std::min(512, (pT * pnodes + 31) / 32 * 32);
      k_project<R, 1><<<(unsigned)a.n_of_type[t], std::max(256, pthreads), sizeof(C) * Nh, cs>>>(
          a.elems[t], Nh, bx, by, bz, a.inv_ptr[t], a.inv_ent[t], p.Pi[t], a.off, a.boxorg, nrhs, u, Nx, Ny, Nz, grid,
          nullptr, 0);
    } else {
      k_project<R, 4><<<(unsigned)a.n_of_type[t], 256, sizeof(C) * Nh * 4, cs>>>(
          a.elems[t], Nh, bx, by, bz, a.inv_ptr[t], a.inv_ent[t], p.Pi[t], a.off, a.boxorg, nrhs, u, Nx, Ny, Nz, grid,
          var == 2 && boxbuf != nullptr ? static_cast<C*>(boxbuf) : nullptr, a.box_nodes_max);
    }
    ++nl;
  }
  if (var == 2 && nrhs > 1) {
    const int64_t ng = (int64_t)Nx * Ny * Nz, items = ng * 4 * nrhs;
    k_grid_gather<C><<<(unsigned)((items + 255) / 256), 256, 0, cs>>>(ng, 4 * nrhs, a.gptr, a.gent,
                                                                      static_cast<const C*>(boxbuf),
                                                                      a.box_nodes_max, nrhs, grid);
    ++nl;
  }
}

// the table-driven interpolation: complex64, eight or more right-hand sides,
// every type's weights and box within the shared-memory limit
template <typename R>
static bool interp_tab_ok(const DevPrec<R>& p, int nrhs) {
  return sizeof(R) == 4 && nrhs >= 8 && p.itp_types != nullptr && p.itp_smem <= kInterpTabSmemMax &&
         p.prj_total > 0;
}

// shared memory of k_interp_rhs<8> for type t: the box [psi][node][9], the
// stencil offsets and the node offsets
static size_t interp_rhs_smem(const DevArray& a, int t) {
  const size_t nodes = (size_t)a.box[3 * t] * a.box[3 * t + 1] * a.box[3 * t + 2];
  return 8 * 4 * nodes * 9 + 4 * (size_t)a.S + 4 * nodes;
}

// The float-float projection and interpolation, per type (T lanes per box node
// or basis as in the FP64 schedules).
static void project_ff_launch(const DevArray& a, const DevPrec<double>& pd, int nrhs, const F6* u6, double2* grid,
                              cudaStream_t cs, int& nl) {
  for (int64_t t = 0; t < a.n_types; ++t) {
    if (a.n_of_type[t] == 0) continue;
    const int Nh = (int)a.Nh[t];
    const int bx = a.box[3 * t], by = a.box[3 * t + 1], bz = a.box[3 * t + 2];
    const int pnodes = bx * by * bz;
    int pT = 4;
    while (pT > 1 && pT * pnodes > 512) pT >>= 1;
    const int threads = std::max(256, std::min(512, (pT * pnodes + 31) / 32 * 32));
    k_project_ff<<<(unsigned)a.n_of_type[t], threads, sizeof(float4) * Nh, cs>>>(
        a.elems[t], Nh, bx, by, bz, a.inv_ptr[t], a.inv_ent[t], static_cast<const float4*>(pd.ff_Pi[t]), a.off,
        a.boxorg, nrhs, u6, a.grid[0], a.grid[1], a.grid[2], grid);
    ++nl;
  }
}
static void interp_ff_launch(const DevArray& a, const DevPrec<double>& pd, int nrhs, const double2* grid,
                             const double2* v, double2* y, cudaStream_t cs, int& nl) {
  for (int64_t t = 0; t < a.n_types; ++t) {
    if (a.n_of_type[t] == 0) continue;
    const int Nh = (int)a.Nh[t];
    const size_t nodes = (size_t)a.box[3 * t] * a.box[3 * t + 1] * a.box[3 * t + 2];
    int iT = 4;
    while (iT > 1 && iT * Nh > 576) iT >>= 1;
    const int threads = std::max(64, std::min(576, (iT * Nh + 31) / 32 * 32));
    k_interp_ff<<<(unsigned)a.n_of_type[t], threads, sizeof(CF) * 4 * nodes + sizeof(int) * (size_t)a.S, cs>>>(
        a.elems[t], Nh, a.S, a.n1, a.o1lo, a.box[3 * t], a.box[3 * t + 1], a.box[3 * t + 2], a.anc[t],
        static_cast<const float4*>(pd.ff_Pi[t]), a.off, a.boxorg, nrhs, grid, a.grid[0], a.grid[1], a.grid[2],
        a.cA[0], a.cA[1], a.cphi[0], a.cphi[1], v, y);
    ++nl;
  }
}

template <typename R>
static void interp_launch(int var, const DevArray& a, const DevPrec<R>& p, int nrhs, const typename V2<R>::T* grid,
                          const typename V2<R>::T* v, typename V2<R>::T* y, cudaStream_t cs, int& nl) {
  typedef typename V2<R>::T C;
  const int Nx = a.grid[0], Ny = a.grid[1], Nz = a.grid[2];
  if constexpr (sizeof(R) == 4) {
    if (var == 3 && interp_tab_ok(p, nrhs)) {
      int dev = 0, sms = 148;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int ctas = (int)std::min<int64_t>(p.prj_total, sms);
      k_interp_tab<8><<<ctas, 512, p.itp_smem, cs>>>(p.itp_types, p.prj_total, a.S, a.n1, a.o1lo, a.off, a.boxorg,
                                                    nrhs, grid, Nx, Ny, Nz, (float)a.cA[0], (float)a.cA[1],
                                                    (float)a.cphi[0], (float)a.cphi[1], v, y);
      ++nl;
      return;
    }
  }
  const size_t slim = 96 * 1024;
  for (int64_t t = 0; t < a.n_types; ++t) {
    if (a.n_of_type[t] == 0) continue;
    const int rc = box_rc(a, (int)t, nrhs, sizeof(C), slim);
    const size_t nodes = (size_t)a.box[3 * t] * a.box[3 * t + 1] * a.box[3 * t + 2];
    const size_t sm = 4 * rc * nodes * sizeof(C) + sizeof(int) * (size_t)a.S;   // box + stencil offsets
    // T lanes per basis with T N^_t <= 576 (512 for FP64): two CTAs per SM
    const int icap = sizeof(R) == 4 ? 576 : 512;
    int iT = 4 >> (nrhs == 1 ? var : 0);
    while (iT > 1 && iT * a.Nh[t] > icap) iT >>= 1;
    const int ithreads = std::min(icap, (int)((iT * a.Nh[t] + 31) / 32 * 32));
    if constexpr (sizeof(R) == 4) {
      if (var == 2 && nrhs >= 8 && interp_rhs_smem(a, (int)t) <= kInterpRhsSmemMax) {
        k_interp_rhs<8><<<(unsigned)a.n_of_type[t], 256, interp_rhs_smem(a, (int)t), cs>>>(
            a.elems[t], (int)a.Nh[t], a.S, a.n1, a.o1lo, a.box[3 * t], a.box[3 * t + 1], a.box[3 * t + 2], a.anc[t],
            p.Pi[t], a.off, a.boxorg, nrhs, grid, Nx, Ny, Nz, (float)a.cA[0], (float)a.cA[1], (float)a.cphi[0],
            (float)a.cphi[1], v, y);
        ++nl;
        continue;
      }
    }
    if (rc >= 8 && var != 1)
      k_interp<R, 8><<<(unsigned)a.n_of_type[t], 256, sm, cs>>>(
          a.elems[t], (int)a.Nh[t], a.S, a.n1, a.o1lo, a.box[3 * t], a.box[3 * t + 1], a.box[3 * t + 2], a.anc[t],
          p.Pi[t], a.off, a.boxorg, nrhs, rc, grid, Nx, Ny, Nz, (R)a.cA[0], (R)a.cA[1], (R)a.cphi[0], (R)a.cphi[1], v,
          y);
    else
      k_interp<R, 1><<<(unsigned)a.n_of_type[t], nrhs == 1 ? std::max(256, ithreads) : 256, sm, cs>>>(
          a.elems[t], (int)a.Nh[t], a.S, a.n1, a.o1lo, a.box[3 * t], a.box[3 * t + 1], a.box[3 * t + 2], a.anc[t],
          p.Pi[t], a.off, a.boxorg, nrhs, rc, grid, Nx, Ny, Nz, (R)a.cA[0], (R)a.cA[1], (R)a.cphi[0], (R)a.cphi[1], v,
          y);
    ++nl;
  }
}

// Grid-stage tuner: on an array's first product for a right-hand-side count and
// precision, each projection and each interpolation variant is timed with CUDA
// events (one warm-up and one timed launch, into the product's own grid and
// into the idle spectrum buffer as y); the fastest of each is kept, with the
// times, for the array.  Without a large enough spectrum buffer variant 0 is used.
template <typename R>
static std::pair<int, int> grid_autotune(DevArray& a, const DevPrec<R>& p, int nrhs, Work& w, cudaStream_t st) {
  typedef typename V2<R>::T C;
  const int np = 4, ni = nrhs == 1 ? 3 : 4;
  std::pair<int, int> best = {0, 0};
  const size_t spec_elems = (size_t)4 * nrhs * a.grid[0] * a.fft[1] * a.fft[2];
  if (spec_elems < (size_t)a.N * nrhs) return best;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return best;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return best;
  }
  std::vector<float> tp(np, -1.f), ti(ni, -1.f);
  C* grid = static_cast<C*>(w.grid);
  const C* u = static_cast<const C*>(w.u);
  const C* v = static_cast<const C*>(w.v);
  C* yscr = static_cast<C*>(w.spec);
  auto timeit = [&](const std::function<void()>& run) -> float {
    run();
    cudaEventRecord(e0, st);
    run();
    cudaEventRecord(e1, st);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = -1.f;
    return ms;
  };
  for (int var = 0; var < np; ++var) {
    int nl = 0;
    // variants a product could not run are not timed (the two-pass form without
    // a box buffer, the table form where a type's tables do not fit)
    if (nrhs > 1 && ((var == 2 && w.boxbuf == nullptr) || (var == 3 && !project_tab_all(a, p, nrhs)))) continue;
    if (nrhs == 1 && var == 3 && (sizeof(R) != 4 || (int64_t)p.prj_tab.size() != a.n_types)) continue;
    tp[var] = timeit([&] { project_launch<R>(var, a, p, nrhs, u, grid, w.boxbuf, st, nl); });
    if (tp[var] >= 0 && (tp[best.first] < 0 || tp[var] < tp[best.first])) best.first = var;
  }
  for (int var = 0; var < ni; ++var) {
    int nl = 0;
    if (nrhs > 1 && var == 2 && (sizeof(R) != 4 || nrhs < 8)) continue;   // the right-hand-side-lane form: complex64, 8+
    if (nrhs > 1 && var == 3 && !interp_tab_ok(p, nrhs)) continue;
    ti[var] = timeit([&] { interp_launch<R>(var, a, p, nrhs, grid, v, yscr, st, nl); });
    if (ti[var] >= 0 && (ti[best.second] < 0 || ti[var] < ti[best.second])) best.second = var;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GridTune g;
  g.project = best.first;
  g.interp = best.second;
  g.project_ms = tp;
  g.interp_ms = ti;
  a.grid_tune[std::make_pair(nrhs, (int)sizeof(R))] = g;
  return best;
}

// Near-field tuner, on the first product of an array with a given
// right-hand-side count and precision.  (1) The CUDA-core (shape, k split)
// pairs are timed alone (one warm-up and one timed launch, CUDA events, into
// the idle spectrum buffer); complex128 keeps the fastest.  (2) Complex64: that
// pair and every tensor-core shape are timed over whole products (one warm-up
// and one timed product): the near field runs beside the far-field chain, and
// what it takes from the chain's SMs counts as much as its own time (16x16,
// 1 RHS: the tensor-core shape 5 is slower alone than CUDA-core shape 0 with a
// k split of 2 but gives 325 instead of 300 solves/s).  With 16 or more
// right-hand sides and the tensor-core direct form available, step (1) is
// skipped (those shapes are 4-5x slower there).  The choice is kept for the
// array; the products write y, which the caller's product then overwrites.
template <typename R>
static cudaError_t near_tune_products(DevArray& a, DevPrec<R>& p, Work& w, int nrhs, const void* x, void* y,
                                      cudaStream_t st, int gemm_mode, bool pre, unsigned flags) {
  typedef typename V2<R>::T C;
  const auto key = std::make_pair(nrhs, (int)sizeof(R));
  const C* u = static_cast<const C*>((flags & kMvUInput) ? x : w.u);
  C* scratch = static_cast<C*>(w.spec);
  const size_t scratch_elems = (size_t)4 * nrhs * a.grid[0] * a.fft[1] * a.fft[2];
  std::pair<int, int> best = near_size_rule<R>(a, p, nrhs, u, w.v, w.np);
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  auto elapsed = [&](float& ms) -> cudaError_t {
    cudaError_t r = cudaEventSynchronize(e1);
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
    return r;
  };
  const bool skip_cuda_cores = nrhs >= 16 && near_shape_ok<R>(7, a, p, nrhs, u, w.v, w.np);
  std::vector<std::pair<int, int>> cand;
  if (!skip_cuda_cores && scratch != nullptr && scratch_elems >= (size_t)a.N * nrhs) {
    float best_ms = 1e30f;
    std::pair<int, int> bs = best;
    for (int tn = 0; tn < 5 && e == cudaSuccess; ++tn)
      for (int ks : {1, 2, 4}) {
        int nl = 0;
        near_shape_launch<R>(tn, a, p, nrhs, u, scratch, st, nl, ks, w.np);
        e = cudaEventRecord(e0, st);
        near_shape_launch<R>(tn, a, p, nrhs, u, scratch, st, nl, ks, w.np);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        float ms = 0;
        if (e == cudaSuccess) e = elapsed(ms);
        if (e != cudaSuccess) break;
        if (ms < best_ms) {
          best_ms = ms;
          bs = {tn, ks};
        }
      }
    best = bs;
    cand.push_back(bs);
  }
  if (sizeof(R) == 4 && e == cudaSuccess) {
    for (int tn = 5; tn < kNearShapes; ++tn)
      if (near_shape_ok<R>(tn, a, p, nrhs, u, w.v, w.np)) {
        cand.push_back({tn, 1});
        if (tn < 7 && w.np_parts >= 2) cand.push_back({tn, 2});   // k tiles split over two units
      }
    if (cand.size() > 1) {
      float best_ms = 1e30f;
      for (const auto& c : cand) {
        a.near_tune[key] = c;
        e = matvec<R>(a, p, w, nrhs, x, y, st, gemm_mode, pre, flags | kMvNoProfile);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = matvec<R>(a, p, w, nrhs, x, y, st, gemm_mode, pre, flags | kMvNoProfile);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        float ms = 0;
        if (e == cudaSuccess) e = elapsed(ms);
        if (e != cudaSuccess) break;
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
    } else if (cand.size() == 1) {
      best = cand[0];
    }
  }
  a.near_tune[key] = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

template <typename R>
cudaError_t matvec(DevArray& a, DevPrec<R>& p, Work& w, int nrhs, const void* xv, void* yv, cudaStream_t st,
                   int gemm_mode, bool pre, unsigned flags) {
  typedef typename V2<R>::T C;
  {
    // first product of this width and precision with block near field: tune it over whole products
    const bool csr0 = a.nnz > 0 && (a.near_mode == 2 || sizeof(R) == 8);
    const bool blocks0 = a.nfb_entries > 0 && p.nfb_val != nullptr && !csr0;
    if (blocks0 && !(flags & (kMvNoTune | kMvFF)) && a.near_force_shape < 0 &&
        a.near_tune.find(std::make_pair(nrhs, (int)sizeof(R))) == a.near_tune.end()) {
      const cudaError_t te = near_tune_products<R>(a, p, w, nrhs, xv, yv, st, gemm_mode, pre, flags);
      if (te != cudaSuccess) return te;
    }
  }
  const C* x = static_cast<const C*>(xv);
  C* y = static_cast<C*>(yv);
  C* u = static_cast<C*>(w.u);
  C* v = static_cast<C*>(w.v);
  C* grid = static_cast<C*>(w.grid);
  C* spec = static_cast<C*>(w.spec);
  const int Nx = a.grid[0], Ny = a.grid[1], Nz = a.grid[2];
  const int Px = a.fft[0], Py = a.fft[1], Pz = a.fft[2];
  const int B = 4 * nrhs;
  const size_t gbytes = sizeof(C) * (size_t)B * Nx * Ny * Nz;
  // launch schedules of the projection and the interpolation (tuned once per
  // right-hand-side count and precision; the size rule's variant 0 otherwise)
  std::pair<int, int> gv = {0, 0};
  {
    const auto gk = std::make_pair(nrhs, (int)sizeof(R));
    const auto gt = a.grid_tune.find(gk);
    if (a.grid_force_p >= 0)
      gv = {a.grid_force_p, a.grid_force_i};
    else if (gt != a.grid_tune.end())
      gv = {gt->second.project, gt->second.interp};
    else if (!(flags & (kMvNoTune | kMvFF)) && a.tune_grid)
      gv = grid_autotune<R>(a, p, nrhs, w, st);
    if (sizeof(R) == 8 && (flags & kMvFF)) gv = {0, 0};   // the float-float stages have one schedule
  }
  // the two-pass projection writes every grid point; the atomic forms add into a cleared grid
  const bool two_pass = gv.first == 2 && w.boxbuf != nullptr && nrhs > 1;
  cudaError_t e = two_pass ? cudaSuccess : cudaMemsetAsync(grid, 0, gbytes, st);
  if (e != cudaSuccess) return e;
  Profiler off;   // stays disabled: records nothing, creates no events
  Profiler& pr = (flags & kMvNoProfile) ? off : a.prof;
  const int sb = sizeof(R) == 8 ? 8 : 0;   // profiler slot base of this precision
  // A1: u = M x, v = D x, per type (with kMvUInput, u = x and v = 0 instead:
  // the product is then y = -G x, the coupling operator alone)
  // float-float contractions: complex128 only, with the F6 operands uploaded
  const DevPrec<double>& ffd = a.pd;
  const bool ff = sizeof(R) == 8 && (flags & kMvFF) != 0;
  if (ff && (!ffd.ff_ready || w.x6 == nullptr || w.u6 == nullptr || pre)) return cudaErrorInvalidValue;
  const bool ff_near_u6 = ff && a.nfb_entries > 0 && ffd.ff_nfb != nullptr && a.near_mode != 2;
  pr.begin(sb + 0, st);
  int nl = 0;
  const bool u_input = (flags & kMvUInput) != 0;
  if (u_input) {
    u = const_cast<C*>(x);
    e = cudaMemsetAsync(v, 0, sizeof(C) * (size_t)a.N * nrhs, st);
    if (e != cudaSuccess) return e;
  }
  if (ff) {
    // the float-float GEMM's right-hand operand (or, without the GEMM, the near field's)
    const int64_t n = a.N * nrhs;
    k_split_f6<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(
        reinterpret_cast<const double2*>(x), n, static_cast<F6*>(u_input ? w.u6 : w.x6));
    ++nl;
  }
  if (u_input) {
    // no macromodel stage
  } else if (sizeof(R) == 4 && gemm_mode != 0) {
    for (int64_t t = 0; t < a.n_types; ++t) {
      if (a.n_of_type[t] == 0) continue;
      const void* At = (pre ? p.AtcP : p.Atc)[gemm_mode - 1][t];
      cudaError_t e2 = tc_macro_gemm(gemm_mode == 1, static_cast<const uint16_t*>(At), p.Mp[t],
                                     p.Kp[t], (int)a.Nh[t], a.elems[t], (int)a.n_of_type[t], nrhs, a.off,
                                     reinterpret_cast<const float2*>(x), static_cast<uint16_t*>(w.bt), w.bt_cap,
                                     reinterpret_cast<float2*>(u), reinterpret_cast<float2*>(v), w.err, st);
      if (e2 != cudaSuccess) return e2;
      nl += 2;
    }
  }
  for (int64_t t = 0; t < a.n_types && !u_input && !(sizeof(R) == 4 && gemm_mode != 0); ++t) {
    if (a.n_of_type[t] == 0) continue;
    const int Nh = (int)a.Nh[t];
    const int ncols = (int)(a.n_of_type[t] * nrhs);
    const int64_t big = (int64_t)((2 * Nh + 63) / 64) * ((ncols + 63) / 64);
    constexpr int BKs = sizeof(R) == 4 ? 32 : 16;
    const C* Wt = static_cast<const C*>((pre ? p.WP : p.W)[t]);
    if constexpr (sizeof(R) == 8) {
      if (ff) {
        const F6* W6 = static_cast<const F6*>(ffd.ffW[t]);
        const F6* x6 = static_cast<const F6*>(w.x6);
        double2* ud = reinterpret_cast<double2*>(u);
        double2* vd = reinterpret_cast<double2*>(v);
        F6* u6 = static_cast<F6*>(w.u6);   // the projection's and the block near field's operand
        double* us = ff_near_u6 ? nullptr : w.us;
        if (a.ff_gemm_shape == 1) {
          dim3 g((2 * Nh + 15) / 16, (ncols + 31) / 32);
          k_macro_gemm_ff<16, 32, 16><<<g, 256, 0, st>>>(W6, Nh, 2 * Nh, a.elems[t], ncols, nrhs, a.off, x6, ud, vd,
                                                         u6, us);
        } else if (a.ff_gemm_shape == 2) {
          dim3 g((2 * Nh + 31) / 32, (ncols + 63) / 64);
          k_macro_gemm_ff<32, 64, 16><<<g, 256, 0, st>>>(W6, Nh, 2 * Nh, a.elems[t], ncols, nrhs, a.off, x6, ud, vd,
                                                         u6, us);
        } else {
          dim3 g((2 * Nh + 31) / 32, (ncols + 31) / 32);
          k_macro_gemm_ff<32, 32, 16><<<g, 256, 0, st>>>(W6, Nh, 2 * Nh, a.elems[t], ncols, nrhs, a.off, x6, ud, vd,
                                                         u6, us);
        }
        ++nl;
        continue;
      }
      const auto& W3v = pre ? p.WP3 : p.W3;
      if ((size_t)t < W3v.size() && W3v[t] != nullptr) {
        dim3 g((2 * Nh + 31) / 32, (ncols + 31) / 32);
        k_macro_gemm3<32, 32, 16><<<g, 256, 0, st>>>(static_cast<const double*>(W3v[t]), Nh, 2 * Nh, a.elems[t],
                                                     ncols, nrhs, a.off, reinterpret_cast<const double2*>(x),
                                                     reinterpret_cast<double2*>(u), reinterpret_cast<double2*>(v),
                                                     w.us);
        ++nl;
        continue;
      }
    }
    if (big >= 2 * 152) {
      dim3 g((2 * Nh + 63) / 64, (ncols + 63) / 64);
      k_macro_gemm<R, 64, 64, 16><<<g, 256, 0, st>>>(Wt, Nh, 2 * Nh, a.elems[t], ncols, nrhs, a.off, x, u, v);
    } else {
      dim3 g((2 * Nh + 31) / 32, (ncols + 31) / 32);
      k_macro_gemm<R, 32, 32, BKs><<<g, 256, 0, st>>>(Wt, Nh, 2 * Nh, a.elems[t], ncols, nrhs, a.off, x, u, v);
    }
    ++nl;
  }
  pr.end(st, nl);
  // A5: v -= G_NF u (the interpolation then writes y = v - far field), as
  // dense blocks (columns = pairs x right-hand sides), or as CSR rows when the
  // array asked for them (DevArray::near_mode); complex128 products take CSR
  // rows when assembled (FP64 arithmetic on the dense blocks costs more than
  // streaming the CSR from HBM).  It only needs u, so it runs on the array's
  // second stream beside A2-A3 and joins before A4.
  // float-float products take the block near field whenever the blocks exist
  const bool ff_near = ff && a.nfb_entries > 0 && ffd.ff_nfb != nullptr && a.near_mode != 2;
  const bool csr = !ff_near && a.nnz > 0 && (a.near_mode == 2 || sizeof(R) == 8);
  const bool nf_blocks = !ff_near && a.nfb_entries > 0 && p.nfb_val != nullptr && !csr;
  const bool nf = ff_near || nf_blocks || a.nnz > 0;
  int tn = 0, ks = 1;   // kernel shape (near_shape_launch), k split
  if (nf_blocks) {
    // first product with this shape: tune on st while the spectra are idle
    const auto key = std::make_pair(nrhs, (int)sizeof(R));
    auto it = a.near_tune.find(key);
    if (it == a.near_tune.end() && a.near_force_shape >= 0)
      it = a.near_tune.emplace(key, std::make_pair(a.near_force_shape, a.near_force_ks)).first;
    if (it != a.near_tune.end()) {
      tn = it->second.first;
      ks = it->second.second;
    } else {
      // size rule, not remembered (kMvNoTune, or timing failed): a later tuned
      // product may still time the shapes
      const auto rule = near_size_rule<R>(a, p, nrhs, u, v, w.np);
      tn = rule.first;
      ks = rule.second;
    }
    if (a.near_force_shape >= 0) {
      tn = a.near_force_shape;
      ks = a.near_force_ks;
    }
  }
  // ns: the near field's stream; cs: the far-field chain's, of higher priority
  // so that the block scheduler serves the chain first and the near field
  // fills the SMs it leaves idle
  cudaStream_t ns = st, cs = st;
  if (nf && a.side != nullptr) {
    e = cudaEventRecord(a.ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(a.side, a.ev_fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(a.chain, a.ev_fork, 0);
    if (e != cudaSuccess) return e;
    ns = a.side;
    cs = a.chain;
  }
  // A2: projection
  pr.begin(sb + 1, cs);
  nl = 0;
  if (ff)
    project_ff_launch(a, ffd, nrhs, static_cast<const F6*>(w.u6), reinterpret_cast<double2*>(grid), cs, nl);
  else
    project_launch<R>(gv.first == 2 && !w.boxbuf ? 0 : gv.first, a, p, nrhs, u, grid, w.boxbuf, cs, nl);
  pr.end(cs, nl);
  // A5 on its stream, launched after the projection so that the chain's first
  // kernel is dispatched ahead of it
  if (ff_near) {
    pr.begin(sb + 6, ns);
    nl = 0;
    near_blocks_ff_launch(a, ffd, nrhs, static_cast<const F6*>(w.u6), reinterpret_cast<double2*>(v), ns, nl);
    pr.end(ns, nl);
  } else if (nf_blocks) {
    pr.begin(sb + 6, ns);
    nl = 0;
    near_shape_launch<R>(tn, a, p, nrhs, u, v, ns, nl, ks, w.np, w.np_parts);
    pr.end(ns, nl);
  } else if (a.nnz > 0) {
    pr.begin(sb + 6, ns);
    const unsigned blocks = (unsigned)((a.N + 7) / 8);
    if constexpr (sizeof(R) == 8) {
      const double* val3 = static_cast<const double*>(p.val);
      const double* us = u_input ? nullptr : w.us;   // Re u + Im u, written by the GEMM
      const double2* ud = reinterpret_cast<const double2*>(u);
      double2* vd = reinterpret_cast<double2*>(v);
      if (nrhs == 1)
        k_spmv_near_3m<1><<<blocks, 256, 0, ns>>>(a.N, a.rowptr, a.col, val3, nrhs, ud, us, vd);
      else if (nrhs <= 4)
        k_spmv_near_3m<4><<<blocks, 256, 0, ns>>>(a.N, a.rowptr, a.col, val3, nrhs, ud, us, vd);
      else
        k_spmv_near_3m<8><<<blocks, 256, 0, ns>>>(a.N, a.rowptr, a.col, val3, nrhs, ud, us, vd);
    } else if (nrhs == 1)
      k_spmv_near1<R><<<blocks, 256, 0, ns>>>(a.N, a.rowptr, a.col, static_cast<const C*>(p.val), u, v);
    else if (nrhs <= 4)
      k_spmv_near<R, 4><<<blocks, 256, 0, ns>>>(a.N, a.rowptr, a.col, static_cast<const C*>(p.val), nrhs, u, v);
    else
      k_spmv_near<R, 8><<<blocks, 256, 0, ns>>>(a.N, a.rowptr, a.col, static_cast<const C*>(p.val), nrhs, u, v);
    pr.end(ns, 1);
  }
  if (ns != st) {
    e = cudaEventRecord(a.ev_join, ns);
    if (e != cudaSuccess) return e;
  }
  // A3: FFT convolution
  pr.begin(sb + 2, cs);
  if (ff) {
    // float-float stages (CF spectra in the FP64 spectrum buffer, same size)
    CF* fspec = reinterpret_cast<CF*>(spec);
    double2* dgrid = reinterpret_cast<double2*>(grid);
    k_fft_fwd_planes<FFTag><<<dim3(Nx, B), 256, fft_smem_bytes<FFTag>(a, 0), cs>>>(
        dgrid, Nx, Ny, Nz, a.py, Pz, static_cast<const CF*>(ffd.ff_twy), static_cast<const CF*>(ffd.ff_twz), fspec);
    pr.end(cs, 1);
    pr.begin(sb + 3, cs);
    k_fft_conv_lines<FFTag><<<dim3(Py, B), 32 * std::min(Pz, 8), fft_smem_bytes<FFTag>(a, 1), cs>>>(
        fspec, Nx, Py, Pz, a.px, static_cast<const CF*>(ffd.ff_twx), static_cast<const CF*>(ffd.ff_Ghat));
    pr.end(cs, 1);
    pr.begin(sb + 4, cs);
    k_fft_inv_planes<FFTag><<<dim3(Nx, B), 256, fft_smem_bytes<FFTag>(a, 0), cs>>>(
        fspec, Nx, Ny, Nz, a.py, Pz, static_cast<const CF*>(ffd.ff_twy), static_cast<const CF*>(ffd.ff_twz), dgrid);
    pr.end(cs, 1);
  } else {
    k_fft_fwd_planes<R><<<dim3(Nx, B), 256, fft_smem_bytes<R>(a, 0), cs>>>(
        grid, Nx, Ny, Nz, a.py, Pz, static_cast<const C*>(p.twy), static_cast<const C*>(p.twz), spec);
    pr.end(cs, 1);
    pr.begin(sb + 3, cs);
    k_fft_conv_lines<R><<<dim3(Py, B), 32 * std::min(Pz, 8), fft_smem_bytes<R>(a, 1), cs>>>(
        spec, Nx, Py, Pz, a.px, static_cast<const C*>(p.twx), static_cast<const C*>(p.Ghat));
    pr.end(cs, 1);
    pr.begin(sb + 4, cs);
    k_fft_inv_planes<R><<<dim3(Nx, B), 256, fft_smem_bytes<R>(a, 0), cs>>>(
        spec, Nx, Ny, Nz, a.py, Pz, static_cast<const C*>(p.twy), static_cast<const C*>(p.twz), grid);
    pr.end(cs, 1);
  }
  (void)Px;
  if (ns != st) {
    e = cudaStreamWaitEvent(cs, a.ev_join, 0);
    if (e != cudaSuccess) return e;
  }
  // A4: interpolation, y = v - y_ff
  pr.begin(sb + 5, cs);
  nl = 0;
  if (ff)
    interp_ff_launch(a, ffd, nrhs, reinterpret_cast<const double2*>(grid), reinterpret_cast<const double2*>(v),
                     reinterpret_cast<double2*>(y), cs, nl);
  else
    interp_launch<R>(gv.second, a, p, nrhs, grid, v, y, cs, nl);
  pr.end(cs, nl);
  if (cs != st) {
    e = cudaEventRecord(a.ev_done, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, a.ev_done, 0);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t precond_apply(DevArray& a, DevPrec<R>& p, int nrhs, const void* xv, void* yv, cudaStream_t st) {
  typedef typename V2<R>::T C;
  const C* x = static_cast<const C*>(xv);
  C* y = static_cast<C*>(yv);
  a.prof.begin(sizeof(R) == 8 ? 8 : 0, st);   // counted with the macromodel stage
  int nl = 0;
  for (int64_t t = 0; t < a.n_types; ++t) {
    if (a.n_of_type[t] == 0) continue;
    const int Nh = (int)a.Nh[t];
    const int ncols = (int)(a.n_of_type[t] * nrhs);
    constexpr int BKs = sizeof(R) == 4 ? 32 : 16;
    if ((int64_t)((Nh + 63) / 64) * ((ncols + 63) / 64) >= 2 * 152) {
      dim3 g((Nh + 63) / 64, (ncols + 63) / 64);
      k_macro_gemm<R, 64, 64, 16><<<g, 256, 0, st>>>(static_cast<const C*>(p.PJ[t]), Nh, Nh, a.elems[t], ncols,
                                                     nrhs, a.off, x, y, nullptr);
    } else {
      dim3 g((Nh + 31) / 32, (ncols + 31) / 32);
      k_macro_gemm<R, 32, 32, BKs><<<g, 256, 0, st>>>(static_cast<const C*>(p.PJ[t]), Nh, Nh, a.elems[t], ncols,
                                                      nrhs, a.off, x, y, nullptr);
    }
    ++nl;
  }
  a.prof.end(st, nl);
  return cudaGetLastError();
}

template cudaError_t precond_apply<float>(DevArray&, DevPrec<float>&, int, const void*, void*, cudaStream_t);
template cudaError_t precond_apply<double>(DevArray&, DevPrec<double>&, int, const void*, void*, cudaStream_t);
template cudaError_t matvec<float>(DevArray&, DevPrec<float>&, Work&, int, const void*, void*, cudaStream_t, int,
                                   bool, unsigned);
template cudaError_t matvec<double>(DevArray&, DevPrec<double>&, Work&, int, const void*, void*, cudaStream_t, int,
                                    bool, unsigned);
template size_t fft_smem_bytes<float>(const DevArray&, int);
template size_t fft_smem_bytes<double>(const DevArray&, int);
template size_t fft_smem_bytes<FFTag>(const DevArray&, int);

}  // namespace mm
