// GMRES (Sec. V; Saad and Schultz 1986) for the final system (eq. (finalsystem)),
// with Arnoldi (classical Gram-Schmidt, one pass, a selective second pass, or
// two passes) in FP64 or, for the inner solves of refinement, on a float-float
// Krylov basis, FP64 Givens rotations, independent columns for several
// right-hand sides, and iterative refinement around a complex64 inner operator
// (residuals through the complex128 operator).  Also the plane-wave excitation
// kernels (Sec. IV, eq. (V1)).
#include <cooperative_groups.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "ffops.cuh"
#include "solver.h"

namespace cg = cooperative_groups;

namespace mm {

typedef double2 Z;

__device__ __forceinline__ Z zmul(Z a, Z b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ Z zconjmul(Z a, Z b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__global__ void k_to_c64(const Z* __restrict__ s, float2* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = make_float2((float)s[i].x, (float)s[i].y);
}
__global__ void k_to_c128(const float2* __restrict__ s, Z* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = make_double2((double)s[i].x, (double)s[i].y);
}

// partial[(i * r + j) * nblk + blk] = sum over this block's rows of conj(V_i[n, j]) w[n, j]
__global__ void k_dot_partial(const Z* __restrict__ V, int64_t vstride, const Z* __restrict__ w, int64_t N, int r,
                              int nblk, double* __restrict__ partial) {
  const int i = blockIdx.y, j = blockIdx.z, blk = blockIdx.x;
  const Z* vi = V + (int64_t)i * vstride;
  const int64_t chunk = (N + nblk - 1) / nblk;
  const int64_t n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
  double sr = 0, si = 0;
  for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    Z p = zconjmul(vi[n * r + j], w[n * r + j]);
    sr += p.x;
    si += p.y;
  }
  __shared__ double s_r[256], s_i[256];
  s_r[threadIdx.x] = sr;
  s_i[threadIdx.x] = si;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s_r[threadIdx.x] += s_r[threadIdx.x + s];
      s_i[threadIdx.x] += s_i[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int64_t o = ((int64_t)i * r + j) * nblk + blk;
    partial[2 * o] = s_r[0];
    partial[2 * o + 1] = s_i[0];
  }
}

// out[i * r + j] = sum_blk partial (fixed order: deterministic)
// A warp per output: lane-strided sums of the block partials, then a butterfly
// (a serial FP64 chain over the blocks costs far more at GB300's FP64 rate).
__global__ void k_dot_final(const double* __restrict__ partial, int nvec, int r, int nblk, Z* __restrict__ out) {
  const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (t >= nvec * r) return;
  double sr = 0, si = 0;
  for (int b = lane; b < nblk; b += 32) {
    sr += partial[2 * ((int64_t)t * nblk + b)];
    si += partial[2 * ((int64_t)t * nblk + b) + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) out[t] = make_double2(sr, si);
}

// acc += conj(v) w and a -= v h with four FP64 fused multiply-adds each (the
// FP64 pipe bounds the Arnoldi step on GB300: the zmul-then-add form takes six).
__device__ __forceinline__ void zconj_fma(const Z v, const Z w, Z& acc) {
  acc.x = fma(v.x, w.x, acc.x);
  acc.x = fma(v.y, w.y, acc.x);
  acc.y = fma(v.x, w.y, acc.y);
  acc.y = fma(-v.y, w.x, acc.y);
}
__device__ __forceinline__ void zsub_mul(const Z v, const Z h, Z& a) {
  a.x = fma(-v.x, h.x, a.x);
  a.x = fma(v.y, h.y, a.x);
  a.y = fma(-v.x, h.y, a.y);
  a.y = fma(-v.y, h.x, a.y);
}
__device__ __forceinline__ void zadd_mul(const Z v, const Z h, Z& a) {
  a.x = fma(v.x, h.x, a.x);
  a.x = fma(-v.y, h.y, a.x);
  a.y = fma(v.x, h.y, a.y);
  a.y = fma(v.y, h.x, a.y);
}

// w[n, j] -= sum_{i < nvec} V_i[n, j] h[i * r + j]
__global__ void k_orth_update(const Z* __restrict__ V, int64_t vstride, const Z* __restrict__ h, int nvec, int64_t N,
                              int r, Z* __restrict__ w) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % r);
    Z acc = w[t];
    for (int i = 0; i < nvec; ++i) zsub_mul(V[(int64_t)i * vstride + t], h[i * r + j], acc);
    w[t] = acc;
  }
}

// dst[n, j] = active[j] ? src[n, j] * scale[j] : 0
__global__ void k_scale_cols(const Z* __restrict__ src, const double* __restrict__ scale,
                             const int32_t* __restrict__ active, int64_t N, int r, Z* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % r);
    Z v = src[t];
    double s = active[j] ? scale[j] : 0.0;
    dst[t] = make_double2(v.x * s, v.y * s);
  }
}

// x[n, j] += sum_i V_i[n, j] y[i * r + j]
__global__ void k_add_basis(const Z* __restrict__ V, int64_t vstride, const Z* __restrict__ y, int nvec, int64_t N,
                            int r, Z* __restrict__ x) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % r);
    Z acc = x[t];
    for (int i = 0; i < nvec; ++i) zadd_mul(V[(int64_t)i * vstride + t], y[i * r + j], acc);
    x[t] = acc;
  }
}

// d = a - b
__global__ void k_sub(const Z* a, const Z* b, int64_t n, Z* d) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    d[t] = make_double2(a[t].x - b[t].x, a[t].y - b[t].y);
}
// x += d
__global__ void k_add(const Z* __restrict__ d, int64_t n, Z* __restrict__ x) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    x[t] = make_double2(x[t].x + d[t].x, x[t].y + d[t].y);
}


// ---------------------------------------------------------------- device-side GMRES cycle
// State of one GMRES cycle for r independent columns, all in device memory.
// The Arnoldi index k lives on the device so every iteration issues the same
// kernels; the host only watches a mapped flag one iteration behind.
struct GmresDev {
  int* k;          // completed Arnoldi steps in this cycle (index of the next basis vector)
  int* active;     // r
  int* kdone;      // r
  double* tol;     // r  absolute residual targets
  double* res;     // r  residual estimates
  double* scale;   // r  1/||w|| for the next basis vector (0 when inactive)
  Z* g;            // (m+1) r
  Z* cs;           // m r
  Z* sn;           // m r
  Z* H;            // r (m+1) m, column j, Arnoldi column k: H[(j m + k)(m+1) + i]
  Z* y;            // m r
  int* flag;       // mapped host memory: [0] any column active, [1] k, [2] max kdone
  double* hres;    // mapped host memory: max over active columns of res / tol after the
                   // step (-1: not reported), for the host's convergence forecast
  Z* hcol;         // (m+1) r: the step's Hessenberg column h + h2 (cooperative step)
  double* hn2;     // r: the step's ||w||^2 (cooperative step)
  int m, r;
  int orth;        // 1 one Gram-Schmidt pass, 2 selective second pass, 3 two passes
};

static_assert(sizeof(GmresDev) <= 160, "GmresDev must fit Solver::gdev_");

// V[k] = w * scale (per column); out = V[k] converted to the operator precision.
template <typename T>
__global__ void k_fetch(Z* __restrict__ V, int64_t vs, const Z* __restrict__ w, GmresDev gd, int64_t n,
                        T* __restrict__ out) {
  const int k = *gd.k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % gd.r);
    const double sc = gd.scale[j];
    const Z v = make_double2(w[t].x * sc, w[t].y * sc);
    V[(int64_t)k * vs + t] = v;
    T o;
    o.x = v.x;
    o.y = v.y;
    out[t] = o;
  }
}

__device__ __forceinline__ Z warp_sum(Z v) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, s);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, s);
  }
  return v;
}

// Partial dot products of w with V_0..V_k over one block of rows:
// P[(i r + j) nblk + blk].  `sh` holds (m+1) x nwarps partial sums.  Four basis
// vectors per pass keep several loads in flight.
__device__ void block_dots(const Z* __restrict__ V, int64_t vs, const Z* __restrict__ w, int k, int64_t n0,
                           int64_t n1, int r, int j, int blk, int nblk, Z* sh, Z* __restrict__ P) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int i0 = 0; i0 <= k; i0 += 4) {
    Z acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_double2(0, 0);
    for (int64_t nn = n0 + threadIdx.x; nn < n1; nn += blockDim.x) {
      const int64_t t = nn * r + j;
      const Z wt = w[t];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i0 + q <= k) zconj_fma(V[(int64_t)(i0 + q) * vs + t], wt, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const Z a = warp_sum(acc[q]);
      if (lane == 0 && i0 + q <= k) sh[(i0 + q) * nw + warp] = a;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    Z acc = make_double2(0, 0);
    for (int q = 0; q < nw; ++q) {
      acc.x += sh[i * nw + q].x;
      acc.y += sh[i * nw + q].y;
    }
    P[((int64_t)i * r + j) * nblk + blk] = acc;
  }
}

// dst[i r + j] = sum over blocks of P for i <= k and all columns: a warp per (i, j).
__device__ void reduce_all_partials(const Z* __restrict__ P, int k, int r, int nblk, Z* dst) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int p = warp; p < (k + 1) * r; p += nw) {
    const int i = p / r, j = p % r;
    const Z* src = P + ((int64_t)i * r + j) * nblk;
    Z acc = make_double2(0, 0);
    for (int b = lane; b < nblk; b += 32) {
      acc.x += src[b].x;
      acc.y += src[b].y;
    }
    acc = warp_sum(acc);
    if (lane == 0) dst[i * r + j] = acc;
  }
  __syncthreads();
}

// CGS pass 1: partial <V_i, w>, i <= k.  Grid (nblk, r).
__global__ void k_cgs_dots(const Z* __restrict__ V, int64_t vs, const Z* __restrict__ w, GmresDev gd, int64_t N,
                           int nblk, Z* __restrict__ P1) {
  extern __shared__ Z sh[];
  const int k = *gd.k, j = blockIdx.y, blk = blockIdx.x;
  const int64_t chunk = (N + nblk - 1) / nblk, n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
  block_dots(V, vs, w, k, n0, n1, gd.r, j, blk, nblk, sh, P1);
}

// Sum of the partials of column j for i <= k into hs[i] (shared memory).
__device__ void reduce_partials(const Z* __restrict__ P, int k, int r, int j, int nblk, Z* hs) {
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    Z acc = make_double2(0, 0);
    for (int b = 0; b < nblk; ++b) {
      const Z v = P[((int64_t)i * r + j) * nblk + b];
      acc.x += v.x;
      acc.y += v.y;
    }
    hs[i] = acc;
  }
  __syncthreads();
}

// w -= sum_i V_i h_i over this block's rows, then partial <V_i, w> (CGS pass 2 dots).
__global__ void k_cgs_update_dots(const Z* __restrict__ V, int64_t vs, GmresDev gd, const Z* __restrict__ P1,
                                  Z* __restrict__ w, int64_t N, int nblk, Z* __restrict__ P2) {
  extern __shared__ Z sh[];
  const int k = *gd.k, j = blockIdx.y, blk = blockIdx.x, r = gd.r;
  Z* hs = sh;                      // m+1
  Z* ws = sh + (gd.m + 1);         // (m+1) x nwarps
  reduce_partials(P1, k, r, j, nblk, hs);
  const int64_t chunk = (N + nblk - 1) / nblk, n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
  for (int64_t nn = n0 + threadIdx.x; nn < n1; nn += blockDim.x) {
    const int64_t t = nn * r + j;
    Z a = w[t];
    for (int i = 0; i <= k; ++i) {
      zsub_mul(V[(int64_t)i * vs + t], hs[i], a);
    }
    w[t] = a;
  }
  __syncthreads();
  if (gd.orth == 1) {   // one pass: the second-pass coefficients are zero
    for (int i = threadIdx.x; i <= k; i += blockDim.x) P2[((int64_t)i * r + j) * nblk + blk] = make_double2(0, 0);
    return;
  }
  block_dots(V, vs, w, k, n0, n1, r, j, blk, nblk, ws, P2);
}

// w -= sum_i V_i h2_i, then partial ||w||^2: PN[j nblk + blk].
__global__ void k_cgs_update_norm(const Z* __restrict__ V, int64_t vs, GmresDev gd, const Z* __restrict__ P2,
                                  Z* __restrict__ w, int64_t N, int nblk, double* __restrict__ PN) {
  extern __shared__ Z sh[];
  const int k = *gd.k, j = blockIdx.y, blk = blockIdx.x, r = gd.r;
  reduce_partials(P2, k, r, j, nblk, sh);
  const int64_t chunk = (N + nblk - 1) / nblk, n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
  double acc = 0;
  for (int64_t nn = n0 + threadIdx.x; nn < n1; nn += blockDim.x) {
    const int64_t t = nn * r + j;
    Z a = w[t];
    for (int i = 0; i <= k; ++i) {
      zsub_mul(V[(int64_t)i * vs + t], sh[i], a);
    }
    w[t] = a;
    acc = fma(a.x, a.x, fma(a.y, a.y, acc));
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  __shared__ double red[32];
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t2 = 0;
    for (int q = 0; q < (int)blockDim.x / 32; ++q) t2 += red[q];
    PN[(int64_t)j * nblk + blk] = t2;
  }
}

// Partial ||w_j||^2 over a block of rows.  Grid (nblk, r).
__global__ void k_norm_partial(const Z* __restrict__ w, int64_t N, int r, int nblk, double* __restrict__ PN) {
  const int j = blockIdx.y, blk = blockIdx.x;
  const int64_t chunk = (N + nblk - 1) / nblk, n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
  double acc = 0;
  for (int64_t nn = n0 + threadIdx.x; nn < n1; nn += blockDim.x) {
    const Z a = w[nn * r + j];
    acc = fma(a.x, a.x, fma(a.y, a.y, acc));
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  __shared__ double red[32];
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t2 = 0;
    for (int q = 0; q < (int)blockDim.x / 32; ++q) t2 += red[q];
    PN[(int64_t)j * nblk + blk] = t2;
  }
}

// Cycle start: beta_j = ||r0_j||, g = (beta, 0, ...), active = beta > tol, scale = 1/beta.
__global__ void k_cycle_init(GmresDev gd, const double* __restrict__ PN, int nblk) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < (gd.m + 1) * gd.r; i += blockDim.x) gd.g[i] = make_double2(0, 0);
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int j = warp; j < gd.r; j += nw) {   // a warp per column
    double s2 = 0;
    for (int b = lane; b < nblk; b += 32) s2 += PN[(int64_t)j * nblk + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane != 0) continue;
    const double beta = sqrt(fmax(0.0, s2));
    gd.g[j] = make_double2(beta, 0);
    gd.res[j] = beta;
    const int act = (beta > gd.tol[j]) && isfinite(beta);
    gd.active[j] = act;
    gd.kdone[j] = 0;
    gd.scale[j] = act ? 1.0 / beta : 0.0;
    if (act) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *gd.k = 0;
    gd.flag[0] = any;
    gd.flag[1] = 0;
    gd.flag[2] = 0;
    *gd.hres = -1.0;
    __threadfence_system();
  }
}

// Arnoldi column k: H[:, k] = h1 + h2, ||w|| from the norm partials; previous
// Givens rotations, a new one, the residual estimate; then k += 1.  One block,
// a warp per column.
__global__ void k_givens(GmresDev gd, const Z* __restrict__ P1, const Z* __restrict__ P2,
                         const double* __restrict__ PN, int nblk) {
  extern __shared__ Z hcol[];      // (m+2) per warp
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  const int k = *gd.k, m = gd.m, r = gd.r;
  Z* hc = hcol + warp * (m + 2);
  for (int j = warp; j < r; j += nw) {
    if (!gd.active[j]) continue;   // warp-uniform
    for (int i = lane; i <= k; i += 32) {
      Z acc = make_double2(0, 0);
      for (int b = 0; b < nblk; ++b) {
        const Z a = P1[((int64_t)i * r + j) * nblk + b], c = P2[((int64_t)i * r + j) * nblk + b];
        acc.x += a.x + c.x;
        acc.y += a.y + c.y;
      }
      hc[i] = acc;
    }
    double s2 = 0;
    for (int b = lane; b < nblk; b += 32) s2 += PN[(int64_t)j * nblk + b];
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, s);
    __syncwarp();
    if (lane == 0) {
      const double hn = sqrt(fmax(0.0, s2));
      Z* H = gd.H + ((int64_t)j * m + k) * (m + 1);
      for (int i = 0; i < k; ++i) {   // previous rotations [[conj c, conj s], [-s, c]]
        const Z c = gd.cs[(int64_t)i * r + j], sg = gd.sn[(int64_t)i * r + j];
        const Z a = hc[i], bb = hc[i + 1];
        const Z t1 = zconjmul(c, a), t2 = zconjmul(sg, bb);
        const Z u1 = zmul(sg, a), u2 = zmul(c, bb);
        hc[i] = make_double2(t1.x + t2.x, t1.y + t2.y);
        hc[i + 1] = make_double2(u2.x - u1.x, u2.y - u1.y);
      }
      const Z a = hc[k];
      const double den = sqrt(a.x * a.x + a.y * a.y + hn * hn);
      const Z c = den > 0 ? make_double2(a.x / den, a.y / den) : make_double2(1, 0);
      const Z sg = den > 0 ? make_double2(hn / den, 0) : make_double2(0, 0);
      gd.cs[(int64_t)k * r + j] = c;
      gd.sn[(int64_t)k * r + j] = sg;
      hc[k] = make_double2(den, 0);
      for (int i = 0; i <= k; ++i) H[i] = hc[i];
      const Z gk = gd.g[(int64_t)k * r + j];
      const Z sgk = zmul(sg, gk);
      gd.g[(int64_t)(k + 1) * r + j] = make_double2(-sgk.x, -sgk.y);
      gd.g[(int64_t)k * r + j] = zconjmul(c, gk);
      const double res = sqrt(sgk.x * sgk.x + sgk.y * sgk.y);
      gd.res[j] = res;
      gd.kdone[j] = k + 1;
      const int stop = !(res > gd.tol[j]) || hn == 0.0 || !isfinite(hn);
      gd.active[j] = stop ? 0 : 1;
      gd.scale[j] = stop ? 0.0 : 1.0 / hn;
    }
    __syncwarp();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0, kd = 0;
    for (int j = 0; j < r; ++j) {
      any |= gd.active[j];
      kd = max(kd, gd.kdone[j]);
    }
    *gd.k = k + 1;
    gd.flag[0] = any;
    gd.flag[1] = k + 1;
    gd.flag[2] = kd;
    *gd.hres = -1.0;
    __threadfence_system();
  }
}

// y_j = H_j^-1 g_j by back substitution over kdone_j columns (lane 0 of a warp per column).
// Back substitution R y = g, a CTA per column.  For k <= kSolveSmemK the CTA
// first stages R's upper triangle in shared memory and every diagonal's
// reciprocal conj(d) / |d|^2 (divisions side by side); warp 0 then runs the
// column-oriented substitution: once y_i is known each lane q < i removes
// R[q, i] y_i from its own right-hand side entry, so the serial chain is a
// shuffle and a complex product per row (serial FP64 divisions and L2 loads
// were the step's cost at GB300's FP64 rate).  Larger k: one thread, global memory.
constexpr int kSolveSmemK = 64;
__global__ void k_solve_y(GmresDev gd) {
  extern __shared__ Z rs[];   // [i][q], q <= i < k: R[q, i]; then k reciprocals
  const int m = gd.m, r = gd.r, j = blockIdx.x;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int kj = gd.kdone[j];
  for (int i = kj + threadIdx.x; i < m; i += blockDim.x) gd.y[(int64_t)i * r + j] = make_double2(0, 0);
  const Z* Hj = gd.H + (int64_t)j * m * (m + 1);   // column c of R at Hj + c (m + 1)
  if (kj <= kSolveSmemK) {
    Z* rinv = rs + kSolveSmemK * kSolveSmemK;
    for (int t = threadIdx.x; t < kj * kj; t += blockDim.x) {
      const int i = t / kj, q = t - i * kj;
      if (q <= i) rs[i * kSolveSmemK + q] = Hj[(int64_t)i * (m + 1) + q];
    }
    for (int i = threadIdx.x; i < kj; i += blockDim.x) {
      const Z d = Hj[(int64_t)i * (m + 1) + i];
      const double inv = 1.0 / (d.x * d.x + d.y * d.y);
      rinv[i] = make_double2(d.x * inv, -d.y * inv);
    }
    __syncthreads();
    if (warp != 0) return;
    Z rhs[2];
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
      const int q = lane + 32 * sl;
      rhs[sl] = q < kj ? gd.g[(int64_t)q * r + j] : make_double2(0, 0);
    }
    for (int i = kj - 1; i >= 0; --i) {
      const int owner = i % 32;
      Z gi = i >= 32 ? rhs[1] : rhs[0];
      gi.x = __shfl_sync(0xffffffffu, gi.x, owner);
      gi.y = __shfl_sync(0xffffffffu, gi.y, owner);
      const Z yi = zmul(gi, rinv[i]);
      if (lane == owner) gd.y[(int64_t)i * r + j] = yi;
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const int q = lane + 32 * sl;
        if (q < i) {
          const Z p = zmul(rs[i * kSolveSmemK + q], yi);
          rhs[sl].x -= p.x;
          rhs[sl].y -= p.y;
        }
      }
    }
  } else if (threadIdx.x == 0) {
    for (int i = kj - 1; i >= 0; --i) {
      Z acc = gd.g[(int64_t)i * r + j];
      for (int q = i + 1; q < kj; ++q) {
        const Z p = zmul(Hj[(int64_t)q * (m + 1) + i], gd.y[(int64_t)q * r + j]);
        acc.x -= p.x;
        acc.y -= p.y;
      }
      const Z d = Hj[(int64_t)i * (m + 1) + i];
      const double dd = d.x * d.x + d.y * d.y;
      gd.y[(int64_t)i * r + j] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
    }
  }
}

// x[n, j] += sum_{i < k} V_i[n, j] y[i r + j], k read from the device.
__global__ void k_add_basis_dev(const Z* __restrict__ V, int64_t vs, GmresDev gd, int64_t n, Z* __restrict__ x) {
  const int k = *gd.k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % gd.r);
    Z acc = x[t];
    for (int i = 0; i < k; ++i) {
      zadd_mul(V[(int64_t)i * vs + t], gd.y[(int64_t)i * gd.r + j], acc);
    }
    x[t] = acc;
  }
}


// Partial ||w_j||^2 over this block's rows into PN[j nblk + blk] (all columns).
__device__ void block_norms(const Z* __restrict__ w, int64_t n0, int64_t n1, int r, int blk, int nblk, Z* ws,
                            double* __restrict__ PN) {
  const int nw = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int j = 0; j < r; ++j) {
    double acc = 0;
    for (int64_t nn = n0 + threadIdx.x; nn < n1; nn += blockDim.x) {
      const Z a = w[nn * r + j];
      acc = fma(a.x, a.x, fma(a.y, a.y, acc));
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    if (lane == 0) ws[warp].x = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t2 = 0;
      for (int q = 0; q < nw; ++q) t2 += ws[q].x;
      PN[(int64_t)j * nblk + blk] = t2;
    }
    __syncthreads();
  }
}

struct DAcc {   // complex FP64 accumulator
  double x, y;
  __device__ DAcc operator+(const DAcc& o) const { return {x + o.x, y + o.y}; }
};
__device__ __forceinline__ double shfl_x(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
__device__ __forceinline__ DAcc shfl_x(DAcc a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o)};
}
__device__ __forceinline__ Z shfl_idx(Z a, int src) {
  return make_double2(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src));
}

// Sums of per-thread values a[q] (q < NQ) over the threads that hold the
// same column (j = tid % r, tid < S = (blockDim / r) r) into out(q, j) for
// j < r, in a fixed thread order (the same result on every run).  When r
// divides 32 the lanes of one column are folded by shuffles first.  red holds
// NQ blockDim values.
// Warp sums of eight values at once: at each butterfly level a lane keeps half
// of its values (the half chosen by its lane bit) and adds the partner's copy of
// that half, so the eight sums take 4 + 2 + 1 + 1 + 1 shuffle-adds instead of
// 8 x 5.  Afterwards lane 4 v (v < 8) holds the warp sum of value v.
__device__ __forceinline__ double warp_sum8(double (&v)[8]) {
  const int lane = threadIdx.x % 32;
#pragma unroll
  for (int q = 0; q < 4; ++q) {   // offset 16: keep values 0-3 (bit clear) or 4-7
    const bool hi = lane & 16;
    const double send = hi ? v[q] : v[q + 4];
    const double got = __shfl_xor_sync(0xffffffffu, send, 16);
    v[q] = (hi ? v[q + 4] : v[q]) + got;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {   // offset 8: keep 0-1 or 2-3 of those
    const bool hi = lane & 8;
    const double send = hi ? v[q] : v[q + 2];
    const double got = __shfl_xor_sync(0xffffffffu, send, 8);
    v[q] = (hi ? v[q + 2] : v[q]) + got;
  }
  {   // offset 4: keep 0 or 1
    const bool hi = lane & 4;
    const double send = hi ? v[0] : v[1];
    const double got = __shfl_xor_sync(0xffffffffu, send, 4);
    v[0] = (hi ? v[1] : v[0]) + got;
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return v[0];
}

template <int NQ, typename T, typename F>
__device__ __forceinline__ void column_reduce(const T (&a)[NQ], int r, T* red, F out) {
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32, nw = blockDim.x / 32, B = blockDim.x;
  const int S = (B / r) * r;
  if constexpr (NQ == 4 && sizeof(T) == 16) {
    if (r == 1) {   // one column: the eight real values of the four sums in one warp pass
      double v[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[2 * q] = a[q].x;
        v[2 * q + 1] = a[q].y;
      }
      const double sum = warp_sum8(v);
      double* rd = reinterpret_cast<double*>(red);
      if ((lane & 3) == 0) rd[(lane >> 2) * nw + warp] = sum;   // value index lane / 4
      __syncthreads();
      if (tid < NQ) {
        T s;
        s.x = 0;
        s.y = 0;
        for (int w = 0; w < nw; ++w) {
          s.x += rd[(2 * tid) * nw + w];
          s.y += rd[(2 * tid + 1) * nw + w];
        }
        out(tid, 0, s);
      }
      __syncthreads();
      return;
    }
  }
  if (r <= 32 && (32 % r) == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T v = a[q];
      for (int o = 16; o >= r; o >>= 1) v = v + shfl_x(v, o);
      if (lane < r) red[q * B + warp * r + lane] = v;
    }
    __syncthreads();
    for (int it = tid; it < NQ * r; it += B) {
      const int q = it / r, j = it - q * r;
      T s = red[q * B + j];
      for (int w = 1; w < nw; ++w) s = s + red[q * B + w * r + j];
      out(q, j, s);
    }
  } else {
    if (tid < S)
#pragma unroll
      for (int q = 0; q < NQ; ++q) red[q * B + tid] = a[q];
    __syncthreads();
    const int G = S / r;
    for (int it = tid; it < NQ * r; it += B) {
      const int q = it / r, j = it - q * r;
      T s = red[q * B + j];
      for (int g = 1; g < G; ++g) s = s + red[q * B + g * r + j];
      out(q, j, s);
    }
  }
  __syncthreads();
}

// Partial <V_i, w_j> over this block's rows for every i <= k and every column
// j in one pass: P[(i r + j) nblk + blk].  Threads stride the flat index
// n r + j by S = (blockDim / r) r, so each keeps one column and the loads of a
// warp are contiguous; basis vectors are taken four at a time.  r <= blockDim.
__device__ void block_dots_all(const Z* __restrict__ V, int64_t vs, const Z* __restrict__ w, int k, int64_t n0,
                               int64_t n1, int r, int blk, int nblk, DAcc* red, Z* __restrict__ P) {
  const int tid = threadIdx.x;
  const int S = (blockDim.x / r) * r;
  const int64_t t1 = n1 * r;
  for (int i0 = 0; i0 <= k; i0 += 4) {
    DAcc acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = {0, 0};
    if (tid < S)
      for (int64_t t = n0 * r + tid; t < t1; t += S) {
        const Z wt = w[t];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (i0 + q <= k) {
            Z a = make_double2(acc[q].x, acc[q].y);
            zconj_fma(V[(int64_t)(i0 + q) * vs + t], wt, a);
            acc[q] = {a.x, a.y};
          }
      }
    column_reduce<4>(acc, r, red, [&](int q, int j, DAcc v) {
      if (i0 + q <= k) P[((int64_t)(i0 + q) * r + j) * nblk + blk] = make_double2(v.x, v.y);
    });
  }
}

// Partial ||w_j||^2 over this block's rows for every column: PN[j nblk + blk].
__device__ void block_norms_all(const Z* __restrict__ w, int64_t n0, int64_t n1, int r, int blk, int nblk, double* red,
                                double* __restrict__ PN) {
  const int tid = threadIdx.x;
  const int S = (blockDim.x / r) * r;
  double acc = 0;
  if (tid < S)
    for (int64_t t = n0 * r + tid; t < n1 * r; t += S) {
      const Z a = w[t];
      acc = fma(a.x, a.x, fma(a.y, a.y, acc));
    }
  const double a1[1] = {acc};
  column_reduce<1>(a1, r, red, [&](int, int j, double v) { PN[(int64_t)j * nblk + blk] = v; });
}

// sum over blocks of PN for column j (same order in every block)
__device__ __forceinline__ double sum_blocks(const double* __restrict__ PN, int j, int nblk) {
  double t = 0;
  for (int b = 0; b < nblk; ++b) t += PN[(int64_t)j * nblk + b];
  return t;
}

// One Arnoldi step for all columns in a single cooperative launch (all blocks
// resident; grid-wide barriers between the phases, no spin-waits of our own).
// Classical Gram-Schmidt with selective reorthogonalisation: the second pass
// runs only for columns whose norm fell below 1/sqrt(2) of its value before
// the first pass (Daniel, Gragg, Kaufman and Stewart 1976; gd.orth = 2), never
// (gd.orth = 1) or always (gd.orth = 3); the decision is the same in every
// block, so every block takes the same grid barriers.
//  0. w = operator output (complex64 -> FP64) on this block's rows;
//  1. partial <V_i, w>, i <= k, and ||w||^2;            [grid sync]
//  2. h = sum of partials; w -= V h; partial ||w||^2;   [grid sync]
//  3. if a column needs it: partial <V_i, w> [grid sync], h2, w -= V h2,
//     partial ||w||^2                                   [grid sync]
//  4. every block: ||w|| per column from the partials; block 0 stores the
//     column h + h2 and ||w||^2 for the Givens update (k_givens_col, launched
//     after the step on a second stream) and sets k += 1;
//  5. V[k+1] = w / ||w||, next operator input.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_arnoldi_step(Z* __restrict__ V, int64_t vs, Z* __restrict__ w,
                                                      const Tin* __restrict__ yin, Tout* __restrict__ xnext,
                                                      GmresDev gd, int64_t N, Z* __restrict__ P1,
                                                      Z* __restrict__ P2, double* __restrict__ PN) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ Z sm[];
  const int m = gd.m, r = gd.r;
  const int nw = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  Z* hs = sm;                        // (m+1) r   h, then h + h2 in block 0
  Z* h2s = hs + (m + 1) * r;         // (m+1) r
  Z* ws = h2s + (m + 1) * r;         // max((m+1) nw, 4 blockDim) warp / column partials
  const int wsn = max((m + 1) * nw, 4 * (int)blockDim.x);
  const bool all_cols = r <= (int)blockDim.x;   // one pass over all columns
  const int k = *gd.k;
  const int nblk = gridDim.x, blk = blockIdx.x;
  const int64_t chunk = (N + nblk - 1) / nblk, n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
  double* PN0 = PN;                              // ||w||^2 before the first pass
  double* PN1 = PN + (int64_t)r * nblk;          // after the first pass
  double* PN2 = PN + 2 * (int64_t)r * nblk;      // after the second pass
  // phase 0
  if (yin != nullptr)
    for (int64_t t = n0 * r + threadIdx.x; t < n1 * r; t += blockDim.x)
      w[t] = make_double2((double)yin[t].x, (double)yin[t].y);
  __syncthreads();
  // phase 1
  if (all_cols) {
    block_dots_all(V, vs, w, k, n0, n1, r, blk, nblk, reinterpret_cast<DAcc*>(ws), P1);
    block_norms_all(w, n0, n1, r, blk, nblk, reinterpret_cast<double*>(ws), PN0);
  } else {
    for (int j = 0; j < r; ++j) block_dots(V, vs, w, k, n0, n1, r, j, blk, nblk, ws, P1), __syncthreads();
    block_norms(w, n0, n1, r, blk, nblk, ws, PN0);
  }
  grid.sync();
  // phase 2 (when r divides the block, a thread keeps one column and sums the
  // new norm as it updates: the same order as a separate pass)
  reduce_all_partials(P1, k, r, nblk, hs);
  const bool fuse_norm = all_cols && (int)blockDim.x % r == 0;
  double nacc = 0;
  for (int64_t t = n0 * r + threadIdx.x; t < n1 * r; t += blockDim.x) {
    const int j = (int)(t % r);
    Z a = w[t];
#pragma unroll 4
    for (int i = 0; i <= k; ++i) {
      zsub_mul(V[(int64_t)i * vs + t], hs[i * r + j], a);
    }
    w[t] = a;
    nacc = fma(a.x, a.x, fma(a.y, a.y, nacc));
  }
  if (fuse_norm) {
    const double a1[1] = {nacc};
    column_reduce<1>(a1, r, reinterpret_cast<double*>(ws),
                     [&](int, int j, double v) { PN1[(int64_t)j * nblk + blk] = v; });
  } else {
    __syncthreads();
    if (all_cols)
      block_norms_all(w, n0, n1, r, blk, nblk, reinterpret_cast<double*>(ws), PN1);
    else
      block_norms(w, n0, n1, r, blk, nblk, ws, PN1);
  }
  grid.sync();
  // phase 3: selective reorthogonalisation.  orth = 2 compares the norms
  // before and after the first pass, a warp per column (lane-strided sums of
  // the block partials, then a butterfly: the same order in every block, so
  // every block takes the same decision)
  int* need = reinterpret_cast<int*>(ws + wsn);   // r flags (shared)
  __shared__ int any_s;
  if (threadIdx.x == 0) any_s = 0;
  __syncthreads();
  if (gd.orth == 2) {
    for (int j = warp; j < r; j += nw) {
      double b0 = 0, b1 = 0;
      for (int b = lane; b < nblk; b += 32) {
        b0 += PN0[(int64_t)j * nblk + b];
        b1 += PN1[(int64_t)j * nblk + b];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        b0 += shfl_x(b0, o);
        b1 += shfl_x(b1, o);
      }
      if (lane == 0) {
        need[j] = gd.active[j] && b1 < 0.5 * b0;
        if (need[j]) atomicOr(&any_s, 1);
      }
    }
  } else {
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
      need[j] = gd.orth == 3 && gd.active[j];
      if (need[j]) atomicOr(&any_s, 1);
    }
  }
  __syncthreads();
  const bool any_reorth = any_s != 0;
  for (int i = threadIdx.x; i < (m + 1) * r; i += blockDim.x) h2s[i] = make_double2(0, 0);
  __syncthreads();
  if (any_reorth) {
    if (all_cols) {
      block_dots_all(V, vs, w, k, n0, n1, r, blk, nblk, reinterpret_cast<DAcc*>(ws), P2);
    } else {
      for (int j = 0; j < r; ++j) {
        if (need[j]) block_dots(V, vs, w, k, n0, n1, r, j, blk, nblk, ws, P2);
        __syncthreads();
      }
    }
    grid.sync();
    for (int p = warp; p < (k + 1) * r; p += nw) {
      const int i = p / r, j = p % r;
      if (!need[j]) continue;
      const Z* src = P2 + ((int64_t)i * r + j) * nblk;
      Z acc = make_double2(0, 0);
      for (int b = lane; b < nblk; b += 32) {
        acc.x += src[b].x;
        acc.y += src[b].y;
      }
      acc = warp_sum(acc);
      if (lane == 0) h2s[i * r + j] = acc;
    }
    __syncthreads();
    for (int64_t t = n0 * r + threadIdx.x; t < n1 * r; t += blockDim.x) {
      const int j = (int)(t % r);
      if (!need[j]) continue;
      Z a = w[t];
#pragma unroll 4
      for (int i = 0; i <= k; ++i) {
        zsub_mul(V[(int64_t)i * vs + t], h2s[i * r + j], a);
      }
      w[t] = a;
    }
    __syncthreads();
    if (all_cols)
      block_norms_all(w, n0, n1, r, blk, nblk, reinterpret_cast<double*>(ws), PN2);
    else
      block_norms(w, n0, n1, r, blk, nblk, ws, PN2);
    grid.sync();
  }
  // phase 4: every block takes ||w|| of each column from the norm partials and
  // scales its own rows; block 0 also stores the Hessenberg column h + h2 and
  // ||w||^2 for the Givens update (k_givens_col), which runs on a second stream
  // beside the next product, and advances k.  A column that met its target keeps
  // producing basis vectors w / ||w||: its Krylov dimension stays where the
  // Givens update stopped it, so they are never used.
  double* scl = reinterpret_cast<double*>(ws);   // r column scales (the partials' space is free)
  for (int j = warp; j < r; j += nw) {
    const double* PNf = (any_reorth && need[j]) ? PN2 : PN1;
    double s2 = 0;
    for (int b = lane; b < nblk; b += 32) s2 += PNf[(int64_t)j * nblk + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += shfl_x(s2, o);
    if (lane == 0) {
      scl[j] = (s2 > 0 && isfinite(s2)) ? 1.0 / sqrt(s2) : 0.0;
      if (blk == 0) gd.hn2[j] = s2;
    }
  }
  if (blk == 0) {
    for (int i = threadIdx.x; i < (k + 1) * r; i += blockDim.x)
      gd.hcol[i] = make_double2(hs[i].x + h2s[i].x, hs[i].y + h2s[i].y);
    if (threadIdx.x == 0) *gd.k = k + 1;
  }
  __syncthreads();
  // phase 5: next basis vector and the next operator input
  for (int64_t t = n0 * r + threadIdx.x; t < n1 * r; t += blockDim.x) {
    const int j = (int)(t % r);
    const double sc = scl[j];
    const Z v = make_double2(w[t].x * sc, w[t].y * sc);
    V[(int64_t)(k + 1) * vs + t] = v;
    Tout o;
    o.x = v.x;
    o.y = v.y;
    xnext[t] = o;
  }
}

// ---------------------------------------------------------------- float-float Krylov basis
// The inner solves of iterative refinement may keep their Krylov basis V and
// work vector w as float-float values (F4 = (re hi, im hi, re lo, im lo), 16
// bytes like complex128) and take the Arnoldi dot products, updates and norms
// in float-float arithmetic on the FP32 pipe (ffops.cuh; GB300 runs FP64 at
// about 1/70 of its FP32 rate).  What crosses the blocks stays FP64: the
// blocks' partial sums, the Hessenberg entries, the norms and the scales.
typedef float4 F4;
struct FFC {   // complex float-float accumulator
  FF re, im;
};
__device__ __forceinline__ FFC ffc_zero() { return FFC{ff_zero(), ff_zero()}; }
__device__ __forceinline__ FFC ffc_of(F4 a) { return FFC{FF{a.x, a.z}, FF{a.y, a.w}}; }
// acc += conj(v) w
__device__ __forceinline__ void ffc_conj_mac(FFC& acc, F4 v, F4 w) {
  ff_mac(acc.re, v.x, v.z, w.x, w.z);
  ff_mac(acc.re, v.y, v.w, w.y, w.w);
  ff_mac(acc.im, v.x, v.z, w.y, w.w);
  ff_mac(acc.im, -v.y, -v.w, w.x, w.z);
}
// acc -= v h
__device__ __forceinline__ void ffc_sub_mul(FFC& acc, F4 v, F4 h) {
  ff_mac(acc.re, -v.x, -v.z, h.x, h.z);
  ff_mac(acc.re, v.y, v.w, h.y, h.w);
  ff_mac(acc.im, -v.x, -v.z, h.y, h.w);
  ff_mac(acc.im, -v.y, -v.w, h.x, h.z);
}
// acc += v h
__device__ __forceinline__ void ffc_add_mul(FFC& acc, F4 v, F4 h) {
  ff_mac(acc.re, v.x, v.z, h.x, h.z);
  ff_mac(acc.re, -v.y, -v.w, h.y, h.w);
  ff_mac(acc.im, v.x, v.z, h.y, h.w);
  ff_mac(acc.im, v.y, v.w, h.x, h.z);
}
__device__ __forceinline__ void ff_norm_mac(FF& acc, F4 a) {   // acc += |a|^2
  ff_mac(acc, a.x, a.z, a.x, a.z);
  ff_mac(acc, a.y, a.w, a.y, a.w);
}
__device__ __forceinline__ F4 ffc_pack(FFC a) {   // renormalised (hi, lo) pairs
  const FF r = ff_add(a.re, ff_zero()), i = ff_add(a.im, ff_zero());
  return make_float4(r.s, i.s, r.c, i.c);
}
__device__ __forceinline__ F4 f4_split(Z z) {
  F4 o;
  ff_split(z.x, o.x, o.z);
  ff_split(z.y, o.y, o.w);
  return o;
}
__device__ __forceinline__ DAcc ffc_dacc(FFC a) { return DAcc{ff_to_double(a.re), ff_to_double(a.im)}; }

// V[k] = w * scale (per column) as float-float; out = its high parts, the
// complex64 operator's input.
__global__ void k_fetch_ff(F4* __restrict__ V, int64_t vs, const Z* __restrict__ w, GmresDev gd, int64_t n,
                           float2* __restrict__ out) {
  const int k = *gd.k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % gd.r);
    const double sc = gd.scale[j];
    const F4 v = f4_split(make_double2(w[t].x * sc, w[t].y * sc));
    V[(int64_t)k * vs + t] = v;
    out[t] = make_float2(v.x, v.y);
  }
}

// yf[i r + j] = gd.y[i r + j] split, i < k (once per cycle, for k_add_basis_ff)
__global__ void k_split_y(GmresDev gd, F4* __restrict__ yf) {
  const int n = *gd.k * gd.r;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) yf[i] = f4_split(gd.y[i]);
}

// x += sum_{i < k} V_i y_i: float-float products and sums, FP64 result.
__global__ void k_add_basis_ff(const F4* __restrict__ V, int64_t vs, GmresDev gd, const F4* __restrict__ yf,
                               int64_t n, Z* __restrict__ x) {
  const int k = *gd.k, r = gd.r;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % r);
    FFC acc = ffc_zero();
    for (int i = 0; i < k; ++i) ffc_add_mul(acc, V[(int64_t)i * vs + t], yf[i * r + j]);
    const Z a = x[t];
    x[t] = make_double2(a.x + ff_to_double(acc.re), a.y + ff_to_double(acc.im));
  }
}

// Rows per thread and round of the float-float Arnoldi loops (RR): all their
// loads are issued before their products, for memory-level parallelism where
// the basis streams from HBM (four rows); where a thread has only a few rows
// (one column at 16x16: about two) the smaller unrolled body of two rows
// keeps the step's code in the instruction cache.

// w[t] -= sum_{i <= k} V_i[t] h_i[t mod r] for the flat rows t in [t0, t1) of
// this block (columns with need[j] == 0 skipped when need is given), RR
// rows per thread and round and four basis vectors per load group; with nacc, the
// thread's sum of |w[t]|^2 after the update (a thread keeps one column when
// r divides the block).
template <int RR>
__device__ __forceinline__ void ff_update_rows(const F4* __restrict__ V, int64_t vs, F4* __restrict__ w,
                                               const F4* hf, int k, int r, int64_t t0, int64_t t1,
                                               const int* need, FF* nacc) {
  const F4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const int B = blockDim.x;
  for (int64_t t = t0 + threadIdx.x; t < t1; t += RR * B) {
    int ju[RR];
    bool uu[RR];
    bool any = false;
    FFC a[RR];
#pragma unroll
    for (int u = 0; u < RR; ++u) {
      const int64_t tu = t + (int64_t)u * B;
      ju[u] = (int)(tu % r);
      uu[u] = tu < t1 && (need == nullptr || need[ju[u]]);
      any |= uu[u];
      a[u] = ffc_of(uu[u] ? w[tu] : z4);
    }
    if (!any) continue;
    for (int i0 = 0; i0 <= k; i0 += 4) {
      F4 vv[RR][4];
#pragma unroll
      for (int u = 0; u < RR; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          vv[u][q] = (uu[u] && i0 + q <= k) ? V[(int64_t)(i0 + q) * vs + t + (int64_t)u * B] : z4;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i0 + q <= k)
#pragma unroll
          for (int u = 0; u < RR; ++u) ffc_sub_mul(a[u], vv[u][q], hf[(i0 + q) * r + ju[u]]);
    }
#pragma unroll
    for (int u = 0; u < RR; ++u)
      if (uu[u]) {
        const F4 o = ffc_pack(a[u]);
        w[t + (int64_t)u * B] = o;
        if (nacc) ff_norm_mac(*nacc, o);
      }
  }
}

// block_dots_all and block_norms_all on the float-float vectors: each thread's
// sums in float-float, the block reduction in FP64 (column_reduce).
template <int RR>
__device__ void block_dots_all_ff(const F4* __restrict__ V, int64_t vs, const F4* __restrict__ w, int k, int64_t n0,
                                  int64_t n1, int r, int blk, int nblk, DAcc* red, Z* __restrict__ P) {
  const int tid = threadIdx.x;
  const int S = (blockDim.x / r) * r;
  const int64_t t1 = n1 * r;
  const F4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int i0 = 0; i0 <= k; i0 += 4) {
    FFC acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = ffc_zero();
    // RR rows per round, every load of the round issued before the
    // products (the basis streams from HBM at large sizes: 5 RR 16-byte
    // loads in flight per thread)
    if (tid < S)
      for (int64_t t = n0 * r + tid; t < t1; t += RR * S) {
        F4 wv[RR], vv[RR][4];
#pragma unroll
        for (int u = 0; u < RR; ++u) {
          const int64_t tu = t + (int64_t)u * S;
          const bool in = tu < t1;
          wv[u] = in ? w[tu] : z4;
#pragma unroll
          for (int q = 0; q < 4; ++q) vv[u][q] = (in && i0 + q <= k) ? V[(int64_t)(i0 + q) * vs + tu] : z4;
        }
#pragma unroll
        for (int u = 0; u < RR; ++u)
#pragma unroll
          for (int q = 0; q < 4; ++q) ffc_conj_mac(acc[q], vv[u][q], wv[u]);
      }
    DAcc ad[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) ad[q] = ffc_dacc(acc[q]);
    column_reduce<4>(ad, r, red, [&](int q, int j, DAcc v) {
      if (i0 + q <= k) P[((int64_t)(i0 + q) * r + j) * nblk + blk] = make_double2(v.x, v.y);
    });
  }
}
__device__ void block_norms_all_ff(const F4* __restrict__ w, int64_t n0, int64_t n1, int r, int blk, int nblk,
                                   double* red, double* __restrict__ PN) {
  const int tid = threadIdx.x;
  const int S = (blockDim.x / r) * r;
  FF acc = ff_zero();
  if (tid < S)
    for (int64_t t = n0 * r + tid; t < n1 * r; t += S) ff_norm_mac(acc, w[t]);
  const double a1[1] = {ff_to_double(acc)};
  column_reduce<1>(a1, r, red, [&](int, int j, double v) { PN[(int64_t)j * nblk + blk] = v; });
}

// The cooperative Arnoldi step of k_arnoldi_step (same phases, barriers,
// orthogonalisation modes and outputs) on the float-float basis, for r <= the
// block's threads.  Shared memory: that of k_arnoldi_step, then (m+1) r F4
// (the Hessenberg column, split for the updates).
template <typename Tin, int RR>
__global__ void __launch_bounds__(256) k_arnoldi_step_ff(F4* __restrict__ V, int64_t vs, F4* __restrict__ w,
                                                         const Tin* __restrict__ yin, float2* __restrict__ xnext,
                                                         GmresDev gd, int64_t N, Z* __restrict__ P1,
                                                         Z* __restrict__ P2, double* __restrict__ PN) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ Z sm[];
  const int m = gd.m, r = gd.r;
  const int nw = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // (m+1) r entries of 16 bytes: the Hessenberg column h (then h2) in FP64,
  // split in place into F4 for the updates once block 0 has stored it
  Z* hs = sm;
  F4* hf = reinterpret_cast<F4*>(sm);
  Z* ws = hs + (m + 1) * r;          // max((m+1) nw, 4 blockDim) warp / column partials
  const int wsn = max((m + 1) * nw, 4 * (int)blockDim.x);
  int* need = reinterpret_cast<int*>(ws + wsn);   // r flags
  const int k = *gd.k;
  const int nblk = gridDim.x, blk = blockIdx.x;
  const int64_t chunk = (N + nblk - 1) / nblk, n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
  double* PN0 = PN;
  double* PN1 = PN + (int64_t)r * nblk;
  double* PN2 = PN + 2 * (int64_t)r * nblk;
  // phase 0: the operator output is complex64, exact as hi parts
  for (int64_t t = n0 * r + threadIdx.x; t < n1 * r; t += blockDim.x)
    w[t] = make_float4((float)yin[t].x, (float)yin[t].y, 0.0f, 0.0f);
  __syncthreads();
  // phase 1
  block_dots_all_ff<RR>(V, vs, w, k, n0, n1, r, blk, nblk, reinterpret_cast<DAcc*>(ws), P1);
  block_norms_all_ff(w, n0, n1, r, blk, nblk, reinterpret_cast<double*>(ws), PN0);
  grid.sync();
  // phase 2
  reduce_all_partials(P1, k, r, nblk, hs);
  for (int i = threadIdx.x; i < (k + 1) * r; i += blockDim.x) {
    const Z z = hs[i];
    if (blk == 0) gd.hcol[i] = z;   // the Hessenberg column for the Givens update (plus h2 below)
    hf[i] = f4_split(z);
  }
  __syncthreads();
  const bool fuse_norm = (int)blockDim.x % r == 0;
  FF nacc = ff_zero();
  ff_update_rows<RR>(V, vs, w, hf, k, r, n0 * r, n1 * r, nullptr, &nacc);
  if (fuse_norm) {
    const double a1[1] = {ff_to_double(nacc)};
    column_reduce<1>(a1, r, reinterpret_cast<double*>(ws),
                     [&](int, int j, double v) { PN1[(int64_t)j * nblk + blk] = v; });
  } else {
    __syncthreads();
    block_norms_all_ff(w, n0, n1, r, blk, nblk, reinterpret_cast<double*>(ws), PN1);
  }
  grid.sync();
  // phase 3: selective reorthogonalisation (the decision as in k_arnoldi_step)
  __shared__ int any_s;
  if (threadIdx.x == 0) any_s = 0;
  __syncthreads();
  if (gd.orth == 2) {
    for (int j = warp; j < r; j += nw) {
      double b0 = 0, b1 = 0;
      for (int b = lane; b < nblk; b += 32) {
        b0 += PN0[(int64_t)j * nblk + b];
        b1 += PN1[(int64_t)j * nblk + b];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        b0 += shfl_x(b0, o);
        b1 += shfl_x(b1, o);
      }
      if (lane == 0) {
        need[j] = gd.active[j] && b1 < 0.5 * b0;
        if (need[j]) atomicOr(&any_s, 1);
      }
    }
  } else {
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
      need[j] = gd.orth == 3 && gd.active[j];
      if (need[j]) atomicOr(&any_s, 1);
    }
  }
  __syncthreads();
  const bool any_reorth = any_s != 0;
  if (any_reorth) {
    for (int i = threadIdx.x; i < (k + 1) * r; i += blockDim.x) hs[i] = make_double2(0, 0);   // h2
    block_dots_all_ff<RR>(V, vs, w, k, n0, n1, r, blk, nblk, reinterpret_cast<DAcc*>(ws), P2);
    grid.sync();
    for (int p = warp; p < (k + 1) * r; p += nw) {
      const int i = p / r, j = p % r;
      if (!need[j]) continue;
      const Z* src = P2 + ((int64_t)i * r + j) * nblk;
      Z acc = make_double2(0, 0);
      for (int b = lane; b < nblk; b += 32) {
        acc.x += src[b].x;
        acc.y += src[b].y;
      }
      acc = warp_sum(acc);
      if (lane == 0) hs[i * r + j] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (k + 1) * r; i += blockDim.x) {
      const Z z = hs[i];
      if (blk == 0) gd.hcol[i] = make_double2(gd.hcol[i].x + z.x, gd.hcol[i].y + z.y);   // h + h2
      hf[i] = f4_split(z);
    }
    __syncthreads();
    ff_update_rows<RR>(V, vs, w, hf, k, r, n0 * r, n1 * r, need, nullptr);
    __syncthreads();
    block_norms_all_ff(w, n0, n1, r, blk, nblk, reinterpret_cast<double*>(ws), PN2);
    grid.sync();
  }
  // phase 4: norms, scales, the Hessenberg column (block 0), k += 1
  double* scl = reinterpret_cast<double*>(ws);
  for (int j = warp; j < r; j += nw) {
    const double* PNf = (any_reorth && need[j]) ? PN2 : PN1;
    double s2 = 0;
    for (int b = lane; b < nblk; b += 32) s2 += PNf[(int64_t)j * nblk + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += shfl_x(s2, o);
    if (lane == 0) {
      scl[j] = (s2 > 0 && isfinite(s2)) ? 1.0 / sqrt(s2) : 0.0;
      if (blk == 0) gd.hn2[j] = s2;
    }
  }
  if (blk == 0 && threadIdx.x == 0) *gd.k = k + 1;
  __syncthreads();
  // phase 5: V[k+1] = w / ||w|| (float-float), the next operator input its high parts
  F4* sclf = hf;   // per column: the scale split (hf is free again)
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    float sh, sl;
    ff_split(scl[j], sh, sl);
    sclf[j] = make_float4(sh, sl, 0.0f, 0.0f);
  }
  __syncthreads();
  for (int64_t t = n0 * r + threadIdx.x; t < n1 * r; t += blockDim.x) {
    const int j = (int)(t % r);
    const F4 a = w[t];
    const FFv sc(sclf[j].x, sclf[j].y);
    const FFv re = ffv_mul(FFv(a.x, a.z), sc), im = ffv_mul(FFv(a.y, a.w), sc);
    V[(int64_t)(k + 1) * vs + t] = make_float4(re.h, im.h, re.l, im.l);
    xnext[t] = make_float2(re.h, im.h);
  }
}

// Givens update of the cooperative step's Hessenberg column (step k = *gd.k - 1:
// the column h + h2 in gd.hcol, ||w||^2 in gd.hn2): previous rotations, the new
// one, the residual estimate and the host flags; one CTA, a warp per column.  The
// lanes load the previous rotations 32 at a time and pass them on by shuffles, so
// the serial chain of rotations waits on no memory; each rotation's four complex
// products are taken by lanes 0-3 in one instruction sequence (lane 0: conj(c)
// h_i, 1: conj(s) h_i+1, 2: s h_i, 3: c h_i+1) and combined by shuffles.
__global__ void __launch_bounds__(256) k_givens_col(GmresDev gd) {
  extern __shared__ Z hs[];   // (k+1) r, column j at hs[i r + j]
  const int m = gd.m, r = gd.r, k = *gd.k - 1;
  const int nw = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __shared__ int any_s, kd_s, rq_s;
  if (threadIdx.x == 0) any_s = 0, kd_s = 0, rq_s = 0;
  for (int i = threadIdx.x; i < (k + 1) * r; i += blockDim.x) hs[i] = gd.hcol[i];
  __syncthreads();
  for (int j = warp; j < r; j += nw) {
    if (!gd.active[j]) continue;
    const Z gk = gd.g[(int64_t)k * r + j];
    const double tolj = gd.tol[j];
    const double s2 = gd.hn2[j];
    Z carry = hs[j];   // entry i of the column after rotations 0 .. i-1
    for (int i0 = 0; i0 < k; i0 += 32) {
      Z cl = make_double2(1, 0), sl = make_double2(0, 0);
      if (i0 + lane < k) {
        cl = gd.cs[(int64_t)(i0 + lane) * r + j];
        sl = gd.sn[(int64_t)(i0 + lane) * r + j];
      }
      const int cnt = min(32, k - i0);
      const int q = lane & 3;
      for (int ii = 0; ii < cnt; ++ii) {   // rotation i: [[conj c, conj s], [-s, c]]
        const int i = i0 + ii;
        const Z c = shfl_idx(cl, ii), sg = shfl_idx(sl, ii);
        const Z bb = hs[(i + 1) * r + j];
        Z f = (q == 0 || q == 3) ? c : sg;
        if (q < 2) f.y = -f.y;
        const Z pq = zmul(f, (q == 0 || q == 2) ? carry : bb);
        const Z t1 = shfl_idx(pq, 0), t2 = shfl_idx(pq, 1), u1 = shfl_idx(pq, 2), u2 = shfl_idx(pq, 3);
        if (lane == 0) hs[i * r + j] = make_double2(t1.x + t2.x, t1.y + t2.y);
        carry = make_double2(u2.x - u1.x, u2.y - u1.y);
      }
    }
    __syncwarp();
    Z* H = gd.H + ((int64_t)j * m + k) * (m + 1);
    for (int i = lane; i < k; i += 32) H[i] = hs[i * r + j];
    if (lane == 0) {
      const Z a = carry;   // rotated entry k; the new rotation pairs it with hn
      const double hn = sqrt(fmax(0.0, s2));
      const double den = sqrt(a.x * a.x + a.y * a.y + hn * hn);
      const double inv = den > 0 ? 1.0 / den : 0.0;
      const Z c = den > 0 ? make_double2(a.x * inv, a.y * inv) : make_double2(1, 0);
      const Z sg = make_double2(hn * inv, 0);
      gd.cs[(int64_t)k * r + j] = c;
      gd.sn[(int64_t)k * r + j] = sg;
      H[k] = make_double2(den, 0);
      const Z sgk = zmul(sg, gk);
      gd.g[(int64_t)(k + 1) * r + j] = make_double2(-sgk.x, -sgk.y);
      gd.g[(int64_t)k * r + j] = zconjmul(c, gk);
      const double res = sqrt(sgk.x * sgk.x + sgk.y * sgk.y);
      gd.res[j] = res;
      gd.kdone[j] = k + 1;
      const int stop = !(res > tolj) || hn == 0.0 || !isfinite(hn);
      gd.active[j] = stop ? 0 : 1;
      gd.scale[j] = stop ? 0.0 : 1.0 / hn;
      if (!stop) {
        atomicOr(&any_s, 2);   // bit 1: a column stays active
        // res / tol >= 0: its float bits order like the values
        atomicMax(&rq_s, __float_as_int((float)fmin(res / tolj, 1e30)));
      }
      atomicMax(&kd_s, k + 1);
    }
    __syncwarp();
  }
  __syncthreads();
  // flags for the host (read after this kernel's event): any column still
  // active, the largest Krylov dimension; kd_s stays 0 only when no column was
  // active on entry, and then comes from the columns' records
  if (kd_s == 0)
    for (int j = threadIdx.x; j < r; j += blockDim.x) atomicMax(&kd_s, gd.kdone[j]);
  __syncthreads();
  if (threadIdx.x == 0) {
    gd.flag[0] = (any_s & 2) ? 1 : 0;
    gd.flag[1] = k + 1;
    gd.flag[2] = kd_s;
    *gd.hres = (any_s & 2) ? (double)__int_as_float(rq_s) : -1.0;
  }
}

static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

#define MM_CK(x)                          \
  do {                                    \
    cudaError_t _e = (x);                 \
    if (_e != cudaSuccess) return {MM_ECUDA, cudaGetErrorString(_e)}; \
  } while (0)

constexpr int kCoopSmemMax = 200 * 1024;   // dynamic shared memory ceiling of the cooperative steps

Status Solver::ensure(int64_t N, int r, int m) {
  if (N == N_ && r == r_ && m <= m_) return {MM_OK, ""};
  release();
  N_ = N; r_ = r; m_ = m;
  {
    // partial-sum blocks: the co-resident grid of the cooperative Arnoldi step
    int dev = 0, sms = 0, per = 0;
    MM_CK(cudaFuncSetAttribute(k_solve_y, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(Z) * (kSolveSmemK * kSolveSmemK + kSolveSmemK))));
    MM_CK(cudaFuncSetAttribute(k_givens_col, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // hs, h2s: (m+1) r each; ws: max((m+1) warps, block threads); need flags
    coop_smem_ = sizeof(Z) * ((size_t)(m + 1) * 2 * r + std::max<size_t>((size_t)(m + 1) * 8, 4 * 256)) +
                 sizeof(int) * (size_t)r + 16;
    coop_ok_ = coop_smem_ <= (size_t)kCoopSmemMax;
    if (coop_ok_) {
      // The attribute is per kernel and process-wide: it is set to the one fixed
      // ceiling (never to this solver's size), so that solvers of other sizes on
      // other threads cannot lower it under a launch of this one.
      MM_CK(cudaFuncSetAttribute(k_arnoldi_step<float2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kCoopSmemMax));
      MM_CK(cudaFuncSetAttribute(k_arnoldi_step<double2, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kCoopSmemMax));
      int p1 = 0, p2 = 0;
      MM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_arnoldi_step<float2, float2>, 256, coop_smem_));
      MM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_arnoldi_step<double2, double2>, 256, coop_smem_));
      // one CTA per SM: the rows per thread double, which halves the share of
      // the FP64 reductions in the step
      per = std::min(std::min(p1, p2), 1);
      coop_ok_ = per >= 1;
    }
    int64_t want = coop_ok_ ? (int64_t)sms * per : 128;
    nblk_ = (int)std::max<int64_t>(1, std::min<int64_t>(want, (N + 63) / 64));
    // the float-float step: one (m+1) r Hessenberg column (split in place), the
    // partial-sum space and the flags; r at most one column per thread
    coop_smem_ff_ = sizeof(Z) * ((size_t)(m + 1) * r + std::max<size_t>((size_t)(m + 1) * 8, 4 * 256)) +
                    sizeof(int) * (size_t)r + 16;
    ffa_ok_ = coop_ok_ && r <= 256 && coop_smem_ff_ <= (size_t)kCoopSmemMax;
    nblk_ff_ = nblk_;
    if (ffa_ok_) {
      MM_CK(cudaFuncSetAttribute(k_arnoldi_step_ff<float2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kCoopSmemMax));
      MM_CK(cudaFuncSetAttribute(k_arnoldi_step_ff<float2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kCoopSmemMax));
      int p3 = 0, p4 = 0;
      MM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p3, k_arnoldi_step_ff<float2, 2>, 256, coop_smem_ff_));
      MM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p4, k_arnoldi_step_ff<float2, 4>, 256, coop_smem_ff_));
      ffa_ok_ = std::min(p3, p4) >= per;
      // where every thread has many rows (the basis streams from HBM), two CTAs
      // per SM when the shared memory allows: twice the loads in flight
      const bool deep = (int64_t)N * r >= (int64_t)sms * 256 * 8;
      const int per_ff = deep ? std::min(std::min(p3, p4), 2) : per;
      nblk_ff_ = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * std::max(per_ff, 1), (N + 63) / 64));
      if (!deep) nblk_ff_ = nblk_;
    }
  }
  size_t vec = sizeof(Z) * (size_t)N * r;
  MM_CK(cudaMalloc(&V_, vec * (m + 1)));
  MM_CK(cudaMalloc(&w_, vec));
  MM_CK(cudaMalloc(&t_, vec));
  MM_CK(cudaMalloc(&x32_, sizeof(float2) * (size_t)N * r));
  MM_CK(cudaMalloc(&y32_, sizeof(float2) * (size_t)N * r));
  MM_CK(cudaMalloc(&partial_, sizeof(double) * 2 * (size_t)(m + 1) * r * nblk_));
  MM_CK(cudaMalloc(&h_, sizeof(Z) * (size_t)(m + 1) * r));
  MM_CK(cudaMalloc(&h2_, sizeof(Z) * (size_t)(m + 1) * r));
  MM_CK(cudaMalloc(&scale_, sizeof(double) * r));
  MM_CK(cudaMalloc(&active_, sizeof(int32_t) * r));
  MM_CK(cudaMalloc(&dx_, vec));
  MM_CK(cudaMalloc(&x64_, vec));
  MM_CK(cudaMalloc(&yf_, sizeof(F4) * (size_t)(m + 1) * r));
  const size_t nbmax = (size_t)std::max(nblk_, nblk_ff_);   // partial sums of either step
  MM_CK(cudaMalloc(&P1_, sizeof(Z) * (size_t)(m + 1) * r * nbmax));
  MM_CK(cudaMalloc(&P2_, sizeof(Z) * (size_t)(m + 1) * r * nbmax));
  MM_CK(cudaMalloc(&PN_, sizeof(double) * 3 * (size_t)r * nbmax));
  {
    // GMRES cycle state: k, active, kdone, tol, res, scale, g, cs, sn, H, y
    size_t b = 0;
    auto take = [&](size_t bytes) { size_t o = b; b += (bytes + 255) / 256 * 256; return o; };
    size_t o_k = take(sizeof(int)), o_act = take(sizeof(int) * r), o_kd = take(sizeof(int) * r);
    size_t o_tol = take(sizeof(double) * r), o_res = take(sizeof(double) * r), o_sc = take(sizeof(double) * r);
    size_t o_g = take(sizeof(Z) * (m + 1) * r), o_cs = take(sizeof(Z) * m * r), o_sn = take(sizeof(Z) * m * r);
    size_t o_H = take(sizeof(Z) * (size_t)r * (m + 1) * m), o_y = take(sizeof(Z) * (size_t)m * r);
    size_t o_hc = take(sizeof(Z) * (size_t)(m + 1) * r), o_hn = take(sizeof(double) * r);
    MM_CK(cudaMalloc(&gstate_, b));
    char* base = static_cast<char*>(gstate_);
    GmresDev& g = *reinterpret_cast<GmresDev*>(gdev_);
    g.k = reinterpret_cast<int*>(base + o_k);
    g.active = reinterpret_cast<int*>(base + o_act);
    g.kdone = reinterpret_cast<int*>(base + o_kd);
    g.tol = reinterpret_cast<double*>(base + o_tol);
    g.res = reinterpret_cast<double*>(base + o_res);
    g.scale = reinterpret_cast<double*>(base + o_sc);
    g.g = reinterpret_cast<Z*>(base + o_g);
    g.cs = reinterpret_cast<Z*>(base + o_cs);
    g.sn = reinterpret_cast<Z*>(base + o_sn);
    g.H = reinterpret_cast<Z*>(base + o_H);
    g.y = reinterpret_cast<Z*>(base + o_y);
    g.hcol = reinterpret_cast<Z*>(base + o_hc);
    g.hn2 = reinterpret_cast<double*>(base + o_hn);
    g.m = m;
    g.r = r;
    MM_CK(cudaHostAlloc(&flag_h_, sizeof(int) * 4 + sizeof(double), cudaHostAllocMapped));
    void* fd = nullptr;
    MM_CK(cudaHostGetDevicePointer(&fd, flag_h_, 0));
    g.flag = static_cast<int*>(fd);
    g.hres = reinterpret_cast<double*>(static_cast<char*>(fd) + sizeof(int) * 4);
    MM_CK(cudaEventCreateWithFlags(&ev_[0], cudaEventDisableTiming));
    MM_CK(cudaEventCreateWithFlags(&ev_[1], cudaEventDisableTiming));
    // the Givens updates of the cooperative steps run on their own stream
    MM_CK(cudaStreamCreateWithFlags(&gst_, cudaStreamNonBlocking));
    for (auto* e : {&eva_, &evg_[0], &evg_[1]}) MM_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  bytes_ = vec * (m + 5) + sizeof(float2) * 2 * (size_t)N * r;
  return {MM_OK, ""};
}

void Solver::release() {
  void* ps[] = {V_, w_, t_, x32_, y32_, partial_, h_, h2_, scale_, active_, dx_, x64_, P1_, P2_, PN_, gstate_, yf_};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (flag_h_) cudaFreeHost(flag_h_);
  for (auto& e : ev_)
    if (e) cudaEventDestroy(e);
  ev_[0] = ev_[1] = nullptr;
  for (auto* e : {&eva_, &evg_[0], &evg_[1]}) {
    if (*e) cudaEventDestroy(*e);
    *e = nullptr;
  }
  if (gst_) cudaStreamDestroy(gst_);
  gst_ = nullptr;
  flag_h_ = nullptr;
  x64_ = P1_ = P2_ = PN_ = gstate_ = yf_ = nullptr;
  V_ = w_ = t_ = nullptr;
  x32_ = y32_ = nullptr;
  partial_ = nullptr;
  h_ = h2_ = nullptr;
  scale_ = nullptr;
  active_ = nullptr;
  dx_ = nullptr;
  N_ = 0; r_ = 0; m_ = 0;
}

// h[i * r + j] = <V_i, w> for i < nvec
Status Solver::dots(const Z* V, int64_t vstride, int nvec, const Z* w, Z* out, cudaStream_t st) {
  if (prof) prof->begin(7, st);
  dim3 g(nblk_, nvec, r_);
  k_dot_partial<<<g, 256, 0, st>>>(V, vstride, w, N_, r_, nblk_, static_cast<double*>(partial_));
  k_dot_final<<<(nvec * r_ + 7) / 8, 256, 0, st>>>(static_cast<const double*>(partial_), nvec, r_, nblk_, out);
  if (prof) prof->end(st, 2);
  MM_CK(cudaGetLastError());
  return {MM_OK, ""};
}

// Applies the operator in double-precision vectors, at precision `prec`.
Status Solver::apply(const Z* in, Z* out, int prec, cudaStream_t st) {
  ++matvecs;
  const int64_t n = N_ * r_;
  if (prec == MM_C128) return op64(in, out, st);
  if (prof) prof->begin(7, st);
  k_to_c64<<<grid_for(n), 256, 0, st>>>(in, static_cast<float2*>(x32_), n);
  if (prof) prof->end(st, 1);
  Status s = op32(x32_, y32_, st);
  if (s.code != MM_OK) return s;
  if (prof) prof->begin(7, st);
  k_to_c128<<<grid_for(n), 256, 0, st>>>(static_cast<const float2*>(y32_), out, n);
  if (prof) prof->end(st, 1);
  MM_CK(cudaGetLastError());
  return {MM_OK, ""};
}

// Restarted GMRES on A x = b; x accumulates.  x_zero: x is 0 on entry, so the
// first residual is b itself (no product).  The cycle runs on the device
// (Arnoldi index, Hessenberg, Givens rotations and residual estimates live in
// device memory); the host issues iteration it while waiting for iteration
// it - 1, so at most one iteration per cycle runs after convergence (its
// columns are inactive and do not change the solution).  tol_abs[j] is the
// absolute residual target of column j.
Status Solver::gmres(const Z* b, Z* x, bool x_zero, const std::vector<double>& tol_abs, int prec, int max_iter,
                     int& iters, std::vector<double>& res, cudaStream_t st) {
  const int64_t N = N_;
  const int r = r_, m = m_;
  const int64_t n = N * r;
  const int64_t vs = n;
  Z* V = static_cast<Z*>(V_);
  Z* w = static_cast<Z*>(w_);
  GmresDev gd = *reinterpret_cast<GmresDev*>(gdev_);
  gd.orth = orth;
  // complex64 inner solves: the float-float basis when asked for and the step fits
  const bool ffk = ff_arnoldi && ffa_ok_ && prec != MM_C128;
  F4* Vf = static_cast<F4*>(V_);
  volatile int* flag = static_cast<volatile int*>(flag_h_);
  volatile double* hres = reinterpret_cast<volatile double*>(static_cast<char*>(flag_h_) + sizeof(int) * 4);
  iters = 0;
  res.assign(r, 0.0);
  MM_CK(cudaMemcpyAsync(gd.tol, tol_abs.data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
  const int nw = 8;
  const size_t sh_dots = sizeof(Z) * (size_t)(m + 1) * nw;
  const size_t sh_upd = sizeof(Z) * (size_t)(m + 1) * (nw + 1);
  const size_t sh_giv = sizeof(Z) * (size_t)(m + 2) * nw;
  bool first = true;
  for (;;) {
    // r0 = b - A x, its norm, cycle initialisation
    if (first && x_zero) {
      MM_CK(cudaMemcpyAsync(w, b, sizeof(Z) * n, cudaMemcpyDeviceToDevice, st));
    } else {
      Status s0 = apply(x, w, prec, st);
      if (s0.code != MM_OK) return s0;
      k_sub<<<grid_for(n), 256, 0, st>>>(b, w, n, w);
    }
    first = false;
    k_norm_partial<<<dim3(nblk_, r), 256, 0, st>>>(w, N, r, nblk_, static_cast<double*>(PN_));
    k_cycle_init<<<1, 256, 0, st>>>(gd, static_cast<const double*>(PN_), nblk_);
    MM_CK(cudaGetLastError());
    // The cycle's first steps are launched without waiting for the initial
    // residual: a cycle whose columns already meet their targets has no active
    // column, its steps change nothing, and the first check stops it.
    if (iters >= max_iter) {
      MM_CK(cudaStreamSynchronize(st));
      std::vector<double> rr(r);
      MM_CK(cudaMemcpy(rr.data(), gd.res, sizeof(double) * r, cudaMemcpyDeviceToHost));
      for (int j = 0; j < r; ++j) {
        res[j] = rr[j];
        if (!std::isfinite(rr[j])) return {MM_EBREAKDOWN, "non-finite residual in GMRES"};
      }
      return {MM_OK, ""};
    }
    bool stopped = false;
    int launched = 0;
    // the events that mark a step's flags as written: the Givens kernel's for
    // cooperative steps, the step's own otherwise
    cudaEvent_t* sev = coop_ok_ ? evg_ : ev_;
    double q_last = -1.0;   // residual / target at the previous check
    // first basis vector V[0] = r0/||r0|| and the operator input
    if (prec == MM_C128)
      k_fetch<Z><<<grid_for(n), 256, 0, st>>>(V, vs, w, gd, n, static_cast<Z*>(x64_));
    else if (ffk)
      k_fetch_ff<<<grid_for(n), 256, 0, st>>>(Vf, vs, w, gd, n, static_cast<float2*>(x32_));
    else
      k_fetch<float2><<<grid_for(n), 256, 0, st>>>(V, vs, w, gd, n, static_cast<float2*>(x32_));
    for (int it = 0; it < m && iters + it < max_iter; ++it) {
      const void* yin = nullptr;
      if (prec == MM_C128) {
        Status s1 = op64(static_cast<const Z*>(x64_), w, st);
        if (s1.code != MM_OK) return s1;
      } else {
        Status s1 = op32(x32_, y32_, st);
        if (s1.code != MM_OK) return s1;
        yin = y32_;
      }
      ++matvecs;
      if (prof) prof->begin(7, st);
      if (coop_ok_) {
        Z* Vp = V;
        int64_t vsp = vs;
        Z* wp = w;
        Z* P1p = static_cast<Z*>(P1_);
        Z* P2p = static_cast<Z*>(P2_);
        double* PNp = static_cast<double*>(PN_);
        int64_t Np = N;
        // the previous step's Givens update (its own stream) wrote the flags this
        // step reads; it has had the whole product to finish
        if (it >= 1) MM_CK(cudaStreamWaitEvent(st, evg_[(it - 1) & 1], 0));
        if (prec == MM_C128) {
          const double2* yp = nullptr;
          double2* xp = static_cast<double2*>(x64_);
          void* args[] = {&Vp, &vsp, &wp, &yp, &xp, &gd, &Np, &P1p, &P2p, &PNp};
          MM_CK(cudaLaunchCooperativeKernel((void*)k_arnoldi_step<double2, double2>, dim3(nblk_), dim3(256), args,
                                            coop_smem_, st));
        } else if (ffk) {
          F4* Vfp = Vf;
          F4* wfp = reinterpret_cast<F4*>(w);
          const float2* yp = static_cast<const float2*>(yin);
          float2* xp = static_cast<float2*>(x32_);
          void* args[] = {&Vfp, &vsp, &wfp, &yp, &xp, &gd, &Np, &P1p, &P2p, &PNp};
          // four rows per round once a thread has eight or more rows
          const bool deep = (int64_t)N * r >= (int64_t)nblk_ff_ * 256 * 8;
          MM_CK(cudaLaunchCooperativeKernel(deep ? (void*)k_arnoldi_step_ff<float2, 4> : (void*)k_arnoldi_step_ff<float2, 2>,
                                            dim3(nblk_ff_), dim3(256), args,
                                            coop_smem_ff_, st));
        } else {
          const float2* yp = static_cast<const float2*>(yin);
          float2* xp = static_cast<float2*>(x32_);
          void* args[] = {&Vp, &vsp, &wp, &yp, &xp, &gd, &Np, &P1p, &P2p, &PNp};
          MM_CK(cudaLaunchCooperativeKernel((void*)k_arnoldi_step<float2, float2>, dim3(nblk_), dim3(256), args,
                                            coop_smem_, st));
        }
        if (prof) prof->end(st, 1);
        // Givens update beside the next product
        MM_CK(cudaEventRecord(eva_, st));
        MM_CK(cudaStreamWaitEvent(gst_, eva_, 0));
        k_givens_col<<<1, 256, sizeof(Z) * (size_t)(m + 1) * r, gst_>>>(gd);
        MM_CK(cudaEventRecord(evg_[it & 1], gst_));
      } else {
        if (yin) k_to_c128<<<grid_for(n), 256, 0, st>>>(static_cast<const float2*>(yin), w, n);
        k_cgs_dots<<<dim3(nblk_, r), 32 * nw, sh_dots, st>>>(V, vs, w, gd, N, nblk_, static_cast<Z*>(P1_));
        k_cgs_update_dots<<<dim3(nblk_, r), 32 * nw, sh_upd, st>>>(V, vs, gd, static_cast<const Z*>(P1_), w, N,
                                                                   nblk_, static_cast<Z*>(P2_));
        k_cgs_update_norm<<<dim3(nblk_, r), 32 * nw, sizeof(Z) * (m + 1), st>>>(
            V, vs, gd, static_cast<const Z*>(P2_), w, N, nblk_, static_cast<double*>(PN_));
        k_givens<<<1, 32 * nw, sh_giv, st>>>(gd, static_cast<const Z*>(P1_), static_cast<const Z*>(P2_),
                                             static_cast<const double*>(PN_), nblk_);
        if (prec == MM_C128)
          k_fetch<Z><<<grid_for(n), 256, 0, st>>>(V, vs, w, gd, n, static_cast<Z*>(x64_));
        else
          k_fetch<float2><<<grid_for(n), 256, 0, st>>>(V, vs, w, gd, n, static_cast<float2*>(x32_));
        if (prof) prof->end(st, yin ? 6 : 5);
      }
      MM_CK(cudaGetLastError());
      MM_CK(cudaEventRecord(ev_[it & 1], st));
      launched = it + 1;
      if (it >= 1) {
        MM_CK(cudaEventSynchronize(sev[(it - 1) & 1]));
        if (!flag[0]) {
          stopped = true;
          break;
        }
        // Steps run one ahead of the host's check, so the step after the last
        // one would be launched for nothing.  When the residual's decay over
        // the last step says this step may end the cycle, wait for it first.
        const double q = *hres;
        if (q > 0 && q_last > 0 && q * (q / q_last) <= 2.0) {
          MM_CK(cudaEventSynchronize(sev[it & 1]));
          if (!flag[0]) {
            stopped = true;
            break;
          }
        }
        q_last = *hres;
      }
    }
    MM_CK(cudaEventSynchronize(sev[(launched - 1) & 1]));
    if (!flag[0]) stopped = true;
    if (coop_ok_) MM_CK(cudaStreamWaitEvent(st, evg_[(launched - 1) & 1], 0));
    k_solve_y<<<r, 256, sizeof(Z) * (kSolveSmemK * kSolveSmemK + kSolveSmemK), st>>>(gd);
    if (prof) prof->begin(7, st);
    if (ffk) {
      k_split_y<<<(unsigned)std::max(1, (m * r + 255) / 256), 256, 0, st>>>(gd, static_cast<F4*>(yf_));
      k_add_basis_ff<<<grid_for(n), 256, 0, st>>>(Vf, vs, gd, static_cast<const F4*>(yf_), n, x);
    } else {
      k_add_basis_dev<<<grid_for(n), 256, 0, st>>>(V, vs, gd, n, x);
    }
    if (prof) prof->end(st, 1);
    MM_CK(cudaGetLastError());
    MM_CK(cudaStreamSynchronize(st));
    iters += flag[2];
    std::vector<double> rr(r);
    MM_CK(cudaMemcpy(rr.data(), gd.res, sizeof(double) * r, cudaMemcpyDeviceToHost));
    for (int j = 0; j < r; ++j) {
      res[j] = rr[j];
      if (!std::isfinite(rr[j])) return {MM_EBREAKDOWN, "non-finite residual in GMRES"};
    }
    if (stopped || iters >= max_iter) return {MM_OK, ""};
  }
}

// Column norms ||a_j|| (synchronous).
Status Solver::norms(const Z* a, std::vector<double>& out, cudaStream_t st) {
  Status s = dots(a, 0, 1, a, static_cast<Z*>(h_), st);
  if (s.code != MM_OK) return s;
  std::vector<Z> hb(r_);
  MM_CK(cudaMemcpyAsync(hb.data(), h_, sizeof(Z) * r_, cudaMemcpyDeviceToHost, st));
  MM_CK(cudaStreamSynchronize(st));
  out.resize(r_);
  for (int j = 0; j < r_; ++j) out[j] = std::sqrt(std::max(0.0, hb[j].x));
  return {MM_OK, ""};
}

Status Solver::solve(const Z* b, Z* x, double tol, int prec, int refine, double inner_tol, int max_iter,
                     int& iters, int& refinements, double& relres, bool& converged, cudaStream_t st) {
  const int64_t n = N_ * r_;
  iters = 0;
  refinements = 0;
  matvecs = 0;
  std::vector<double> bn, rn, res;
  Status s = norms(b, bn, st);
  if (s.code != MM_OK) return s;
  MM_CK(cudaMemsetAsync(x, 0, sizeof(Z) * n, st));
  Z* rr = static_cast<Z*>(t_);
  auto done = [&]() {
    bool d = true;
    for (int j = 0; j < r_; ++j) d &= rn[j] <= tol * bn[j];
    return d;
  };
  if (prec == MM_C128 || !refine) {
    // plain GMRES at one precision; the true residual (same precision) confirms each exit
    std::vector<double> tabs(r_);
    for (int j = 0; j < r_; ++j) tabs[j] = tol * bn[j];
    bool x_zero = true;
    for (;;) {
      int it = 0;
      s = gmres(b, x, x_zero, tabs, prec, max_iter - iters, it, res, st);
      if (s.code != MM_OK) return s;
      iters += it;
      x_zero = false;
      s = apply(x, rr, prec, st);
      if (s.code != MM_OK) return s;
      k_sub<<<grid_for(n), 256, 0, st>>>(b, rr, n, rr);
      s = norms(rr, rn, st);
      if (s.code != MM_OK) return s;
      if (done() || iters >= max_iter || it == 0) break;
    }
  } else {
    // FP64 iterative refinement: GMRES on the complex64 operator solves for the
    // correction of the current residual, computed with the complex128 operator.
    Z* dx = static_cast<Z*>(dx_);
    MM_CK(cudaMemcpyAsync(rr, b, sizeof(Z) * n, cudaMemcpyDeviceToDevice, st));
    rn = bn;
    for (;;) {
      std::vector<double> tabs(r_);
      for (int j = 0; j < r_; ++j) tabs[j] = std::max(inner_tol * rn[j], 0.5 * tol * bn[j]);
      int it = 0;
      MM_CK(cudaMemsetAsync(dx, 0, sizeof(Z) * n, st));
      s = gmres(rr, dx, true, tabs, MM_C64, max_iter - iters, it, res, st);
      if (s.code != MM_OK) return s;
      iters += it;
      ++refinements;
      if (correction32) {
        k_to_c64<<<grid_for(n), 256, 0, st>>>(dx, static_cast<float2*>(x32_), n);
        Status s2 = correction32(x32_, y32_, st);
        if (s2.code != MM_OK) return s2;
        k_to_c128<<<grid_for(n), 256, 0, st>>>(static_cast<const float2*>(y32_), dx, n);
      }
      k_add<<<grid_for(n), 256, 0, st>>>(dx, n, x);
      s = apply(x, rr, MM_C128, st);
      if (s.code != MM_OK) return s;
      k_sub<<<grid_for(n), 256, 0, st>>>(b, rr, n, rr);
      s = norms(rr, rn, st);
      if (s.code != MM_OK) return s;
      if (done() || iters >= max_iter || it == 0) break;
    }
  }
  relres = 0;
  converged = true;
  for (int j = 0; j < r_; ++j) {
    double rel = bn[j] > 0 ? rn[j] / bn[j] : rn[j];
    relres = std::max(relres, rel);
    converged &= rel <= tol * (1.0 + 1e-9);
  }
  if (!std::isfinite(relres)) return {MM_EBREAKDOWN, "non-finite residual"};
  return {MM_OK, ""};
}

// ---------------------------------------------------------------- plane-wave excitation
// V[n, j] = -sum_{T+-} sum_q w_q A f_n(r_q) . p_j exp(-j k khat_j . r_q)  (7-point rule)
// With r_q = o_e + r'_q (o_e the element offset, r'_q in the type's local
// frame) and f_n depending on r_q - (free vertex) only, the phase splits:
// V[n, j] = exp(-j k khat_j . o_e) Vloc[t, n', j], Vloc being the same sum in
// the local frame, which is shared by every element of type t.  So the
// quadrature (14 phase evaluations per basis) runs once per (type, local basis)
// and each element adds one phase: the FP64 sine and cosine, slow at GB300's
// FP64 rate, drop from 14 per unknown to about one per element.
__device__ __forceinline__ void planewave_dirs(double th, double ph, int pol, double* k, double* p) {
  double st, ct, sp, cp;
  sincos(th, &st, &ct);
  sincos(ph, &sp, &cp);
  k[0] = -st * cp; k[1] = -st * sp; k[2] = -ct;
  if (pol == 0) { p[0] = ct * cp; p[1] = ct * sp; p[2] = -st; }
  else { p[0] = -sp; p[1] = cp; p[2] = 0.0; }
}

// Part 1: items (local basis of a type, then element) x right-hand sides.
// vloc[(tbase[t] + n') nrhs + j] = -(local quadrature sum); eph[e nrhs + j] = exp(-j k khat_j . o_e).
// Sixteen lanes per item: lane (side, point) evaluates one quadrature term
// (2 x up to 8 points) and the group adds by shuffles, so the FP64 sine and
// cosine evaluations of one basis run side by side.
__global__ void k_rhs_parts(int ntypes, const int64_t* __restrict__ tbase, int64_t n_elem, int nrhs,
                            const double* const* __restrict__ geo, const double* __restrict__ eoff,
                            const double* __restrict__ theta, const double* __restrict__ phi,
                            const int32_t* __restrict__ pol, double k0, QuadRule q, double2* __restrict__ vloc,
                            double2* __restrict__ eph) {
  const int64_t nloc = tbase[ntypes];
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 16;
  const int sub = threadIdx.x % 16, side = sub / 8, i = sub % 8;
  const unsigned gmask = 0xffffu << (threadIdx.x % 32 & 16);
  if (t >= (nloc + n_elem) * nrhs) return;   // uniform over the 16-lane group
  const int64_t item = t / nrhs;
  const int j = (int)(t - item * nrhs);
  double kh[3], pv[3];
  planewave_dirs(theta[j], phi[j], pol[j], kh, pv);
  if (item >= nloc) {
    if (sub != 0) return;
    const int64_t e = item - nloc;
    double sn, cs;
    sincos(-k0 * (kh[0] * eoff[3 * e] + kh[1] * eoff[3 * e + 1] + kh[2] * eoff[3 * e + 2]), &sn, &cs);
    eph[e * nrhs + j] = make_double2(cs, sn);
    return;
  }
  int ty = 0;
  while (ty + 1 < ntypes && tbase[ty + 1] <= item) ++ty;
  const double* gp = geo[ty] + 13 * (item - tbase[ty]);
  double accr = 0, acci = 0;
  if (i < q.n) {
    const double l = gp[12];
    const double ax = gp[0], ay = gp[1], az = gp[2];
    const double bx = gp[3], by = gp[4], bz = gp[5];
    const double fx = gp[6 + 3 * side], fy = gp[7 + 3 * side], fz = gp[8 + 3 * side];
    const double ux = bx - ax, uy = by - ay, uz = bz - az, vx = fx - ax, vy = fy - ay, vz = fz - az;
    const double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
    const double A = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    const double sg = side == 0 ? 1.0 : -1.0;
    const double rx = q.b0[i] * ax + q.b1[i] * bx + q.b2[i] * fx;
    const double ry = q.b0[i] * ay + q.b1[i] * by + q.b2[i] * fy;
    const double rz = q.b0[i] * az + q.b1[i] * bz + q.b2[i] * fz;
    const double s = sg * l / (2.0 * A);
    const double dotp = s * ((rx - fx) * pv[0] + (ry - fy) * pv[1] + (rz - fz) * pv[2]);
    double sn, cs;
    sincos(-k0 * (kh[0] * rx + kh[1] * ry + kh[2] * rz), &sn, &cs);
    const double wA = q.w[i] * A;
    accr = wA * dotp * cs;
    acci = wA * dotp * sn;
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    accr += __shfl_xor_sync(gmask, accr, o);
    acci += __shfl_xor_sync(gmask, acci, o);
  }
  if (sub == 0) vloc[item * nrhs + j] = make_double2(-accr, -acci);
}

// Part 2: V[n, j] = eph[e, j] Vloc[t, n - off[e], j].
template <typename R>
__global__ void k_rhs_planewave(int64_t N, int nrhs, const int32_t* __restrict__ elem_of,
                                const int32_t* __restrict__ type_of, const int64_t* __restrict__ off,
                                const int64_t* __restrict__ tbase, const double2* __restrict__ vloc,
                                const double2* __restrict__ eph, typename V2<R>::T* __restrict__ V) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  const int64_t n = t / nrhs;
  const int j = (int)(t - n * nrhs);
  const int e = elem_of[n];
  const double2 a = vloc[(tbase[type_of[e]] + n - off[e]) * nrhs + j], b = eph[(int64_t)e * nrhs + j];
  typename V2<R>::T out;
  out.x = (R)(a.x * b.x - a.y * b.y);
  out.y = (R)(a.x * b.y + a.y * b.x);
  V[t] = out;
}

template <typename R>
cudaError_t rhs_planewave(const DevArray& a, const int32_t* elem_of, const double* const* geo, int nrhs,
                          const double* th, const double* ph, const int32_t* pol, double k0, const QuadRule& q,
                          void* V, double2* scratch, cudaStream_t st) {
  int64_t nloc = 0;
  for (int64_t t = 0; t < a.n_types; ++t) nloc += a.Nh[t];
  const int64_t parts = (nloc + a.n_elem) * nrhs;
  if (q.n > 8) return cudaErrorInvalidValue;   // sixteen lanes: two sides of at most 8 points
  k_rhs_parts<<<(unsigned)((16 * parts + 255) / 256), 256, 0, st>>>((int)a.n_types, a.tbase, a.n_elem, nrhs, geo,
                                                                    a.eoff, th, ph, pol, k0, q, scratch,
                                                                    scratch + nloc * nrhs);
  const int64_t tot = a.N * nrhs;
  k_rhs_planewave<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a.N, nrhs, elem_of, a.type_of, a.off, a.tbase,
                                                                     scratch, scratch + nloc * nrhs,
                                                                     static_cast<typename V2<R>::T*>(V));
  return cudaGetLastError();
}
template cudaError_t rhs_planewave<float>(const DevArray&, const int32_t*, const double* const*, int, const double*,
                                          const double*, const int32_t*, double, const QuadRule&, void*, double2*,
                                          cudaStream_t);
template cudaError_t rhs_planewave<double>(const DevArray&, const int32_t*, const double* const*, int, const double*,
                                           const double*, const int32_t*, double, const QuadRule&, void*, double2*,
                                           cudaStream_t);

}  // namespace mm
