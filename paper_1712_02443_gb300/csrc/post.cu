// Post-processing kernels: element currents from a solution (eqs. (JABE), (Tm1))
// and the far-field radiation integral of the equivalent currents.
#include <cmath>

#include "post.h"

namespace mm {

typedef double2 Z;

__device__ __forceinline__ Z zfma(Z acc, Z a, Z b) {   // four fused multiply-adds
  acc.x = __fma_rn(a.x, b.x, acc.x);
  acc.x = __fma_rn(-a.y, b.y, acc.x);
  acc.y = __fma_rn(a.x, b.y, acc.y);
  acc.y = __fma_rn(a.y, b.x, acc.y);
  return acc;
}

// out_e (M x nrhs) = W (M x K) in_e (K x nrhs) for the elements elems[0..nel),
// in_e at in[(in_off[e] + k) nrhs + c], out_e at out[(out_off[e] + i) nrhs + c].
// 32 x 32 output tile per CTA of 256 threads, 2 x 2 outputs each, FP64.
__global__ void __launch_bounds__(256) k_elem_gemm(const Z* __restrict__ W, int M, int K,
                                                   const int32_t* __restrict__ elems, int ncols, int nrhs,
                                                   const int64_t* __restrict__ in_off, const Z* __restrict__ in,
                                                   const int64_t* __restrict__ out_off, Z* __restrict__ out) {
  constexpr int BM = 32, BN = 32, BK = 16;
  __shared__ Z As[BK][BM + 1];
  __shared__ Z Bs[BK][BN + 1];
  __shared__ int64_t cin[BN], cout[BN];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
  for (int c = tid; c < BN; c += 256) {
    const int gc = col0 + c;
    if (gc < ncols) {
      const int e = elems[gc / nrhs], rr = gc % nrhs;
      cin[c] = in_off[e] * nrhs + rr;
      cout[c] = out_off[e] * nrhs + rr;
    } else {
      cin[c] = -1;
      cout[c] = -1;
    }
  }
  Z acc[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0, 0);
  __syncthreads();
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      const int r = e / BK, kk = e % BK, gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? W[(int64_t)gr * K + gk] : make_double2(0, 0);
    }
    for (int e = tid; e < BN * BK; e += 256) {
      const int kk = e % BK, c = e / BK, gk = k0 + kk;
      Bs[kk][c] = (cin[c] >= 0 && gk < K) ? in[cin[c] + (int64_t)gk * nrhs] : make_double2(0, 0);
    }
    __syncthreads();
    for (int kk = 0; kk < BK; ++kk)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) acc[i][j] = zfma(acc[i][j], As[kk][ty * 2 + i], Bs[kk][tx * 2 + j]);
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i) {
    const int gr = row0 + ty * 2 + i;
    if (gr >= M) continue;
    for (int j = 0; j < 2; ++j) {
      const int c = tx * 2 + j;
      if (cout[c] < 0) continue;
      out[cout[c] + (int64_t)gr * nrhs] = acc[i][j];
    }
  }
}

cudaError_t elem_gemm(const void* W, int M, int K, const int32_t* elems, int nel, int nrhs, const int64_t* in_off,
                      const void* in, const int64_t* out_off, void* out, cudaStream_t st) {
  if (nel == 0) return cudaSuccess;
  const int ncols = nel * nrhs;
  dim3 g((M + 31) / 32, (ncols + 31) / 32);
  k_elem_gemm<<<g, 256, 0, st>>>(static_cast<const Z*>(W), M, K, elems, ncols, nrhs, in_off,
                                 static_cast<const Z*>(in), out_off, static_cast<Z*>(out));
  return cudaGetLastError();
}

// F(r^) for one direction (blockIdx.x) and one RHS (blockIdx.y).
__global__ void __launch_bounds__(256) k_farfield(int64_t N, int nrhs, const int32_t* __restrict__ elem_of,
                                                  const int32_t* __restrict__ type_of,
                                                  const int64_t* __restrict__ off,
                                                  const double* const* __restrict__ geo,
                                                  const double* __restrict__ eoff, const Z* __restrict__ J,
                                                  const double* __restrict__ theta, const double* __restrict__ phi,
                                                  double k0, double eta0, QuadRule q, Z* __restrict__ F) {
  const int64_t d = blockIdx.x;
  const int j = blockIdx.y;
  double st, ct, sp, cp;
  sincos(theta[d], &st, &ct);
  sincos(phi[d], &sp, &cp);
  const double rx = st * cp, ry = st * sp, rz = ct;
  const double two_pi = 6.283185307179586476925286766559;
  float ax = 0, ay = 0, az = 0, bx = 0, by = 0, bz = 0;   // sum of J_n int f_n e^{jk r.r'} (re: a, im: b)
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const int e = elem_of[n];
    const double* gp = geo[type_of[e]] + 13 * (n - off[e]);
    const double ox = eoff[3 * e], oy = eoff[3 * e + 1], oz = eoff[3 * e + 2];
    const Z Jn = J[n * nrhs + j];
    const double l = gp[12];
    for (int side = 0; side < 2; ++side) {
      const double pax = gp[0] + ox, pay = gp[1] + oy, paz = gp[2] + oz;
      const double pbx = gp[3] + ox, pby = gp[4] + oy, pbz = gp[5] + oz;
      const double pfx = gp[6 + 3 * side] + ox, pfy = gp[7 + 3 * side] + oy, pfz = gp[8 + 3 * side] + oz;
      const double ux = pbx - pax, uy = pby - pay, uz = pbz - paz, vx = pfx - pax, vy = pfy - pay, vz = pfz - paz;
      const double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
      const double A = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
      const double s = (side == 0 ? 1.0 : -1.0) * l / (2.0 * A);
      for (int i = 0; i < q.n; ++i) {
        const double px = q.b0[i] * pax + q.b1[i] * pbx + q.b2[i] * pfx;
        const double py = q.b0[i] * pay + q.b1[i] * pby + q.b2[i] * pfy;
        const double pz = q.b0[i] * paz + q.b1[i] * pbz + q.b2[i] * pfz;
        double ph = k0 * (rx * px + ry * py + rz * pz);
        ph -= two_pi * rint(ph / two_pi);
        float sn, cs;
        sincosf((float)ph, &sn, &cs);
        const float wA = (float)(q.w[i] * A * s);
        const float fx = (float)(px - pfx) * wA, fy = (float)(py - pfy) * wA, fz = (float)(pz - pfz) * wA;
        // (J e^{j ph}) f
        const float er = (float)Jn.x * cs - (float)Jn.y * sn, ei = (float)Jn.x * sn + (float)Jn.y * cs;
        ax += er * fx; ay += er * fy; az += er * fz;
        bx += ei * fx; by += ei * fy; bz += ei * fz;
      }
    }
  }
  float v[6] = {ax, ay, az, bx, by, bz};
#pragma unroll
  for (int c = 0; c < 6; ++c)
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], s);
  __shared__ float red[8][6];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0)
    for (int c = 0; c < 6; ++c) red[warp][c] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < (int)blockDim.x / 32; ++w)
      for (int c = 0; c < 6; ++c) t[c] += red[w][c];
    // transverse part, then -j k eta0/(4 pi) (re, im) -> (k eta0/(4 pi)) (im, -re)
    const double dr = rx * t[0] + ry * t[1] + rz * t[2], di = rx * t[3] + ry * t[4] + rz * t[5];
    const double tr[3] = {t[0] - rx * dr, t[1] - ry * dr, t[2] - rz * dr};
    const double ti[3] = {t[3] - rx * di, t[4] - ry * di, t[5] - rz * di};
    const double c = k0 * eta0 / (4.0 * M_PI);
    for (int a = 0; a < 3; ++a) F[(d * nrhs + j) * 3 + a] = make_double2(c * ti[a], -c * tr[a]);
  }
}

cudaError_t farfield(const DevArray& a, const int32_t* elem_of, const double* const* geo, int nrhs, const void* J,
                     int64_t ndir, const double* th, const double* ph, double k0, double eta0, const QuadRule& q,
                     void* F, cudaStream_t st) {
  if (ndir == 0) return cudaSuccess;
  k_farfield<<<dim3((unsigned)ndir, nrhs), 256, 0, st>>>(a.N, nrhs, elem_of, a.type_of, a.off, geo, a.eoff,
                                                         static_cast<const Z*>(J), th, ph, k0, eta0, q,
                                                         static_cast<Z*>(F));
  return cudaGetLastError();
}

}  // namespace mm
