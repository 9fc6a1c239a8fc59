// Near-field block fill on the GPU (Sec. V, the precorrected near-field
// operator): for each translation-invariant block, the EFIE Galerkin integrals
// of every (test triangle, source triangle) pair of the two equivalent meshes,
// then for every near pair (m, n) the RWG entry assembled from its four
// triangle pairs, scaled by c_A, minus the grid part
// c_A sum_xyz P_m^T H P_n + c_phi P_m,phi^T H P_n,phi.  FP64 throughout.
//
// The triangle-pair integral is the host fill's (Sec. II, eq. (G3) and the
// Lmat of the EFIE): the 1/R part of G integrated over the source triangle in
// closed form (singularity extraction), tested with the 7-point rule; the
// smooth rest G1 = (exp(-jkR) - 1)/(4 pi R) by the 7 x 7 product rule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "fill_gpu.h"

namespace mm {

namespace {

constexpr double kSnap = 1e-10;
constexpr double kInv4Pi = 0.25 / M_PI;

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 d3(double x, double y, double z) { return D3{x, y, z}; }
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return d3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ D3 operator*(double s, D3 a) { return d3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dotd(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 crossd(D3 a, D3 b) {
  return d3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double normd(D3 a) { return sqrt(dotd(a, a)); }

struct Tri {
  D3 v[3];
  D3 n;
  double area, scale;
};

__device__ __forceinline__ Tri make_tri(const double* c, D3 shift) {
  Tri g;
  for (int i = 0; i < 3; ++i) g.v[i] = d3(c[3 * i], c[3 * i + 1], c[3 * i + 2]) + shift;
  const D3 cr = crossd(g.v[1] - g.v[0], g.v[2] - g.v[0]);
  const double nn = normd(cr);
  g.n = (1.0 / nn) * cr;
  g.area = 0.5 * nn;
  g.scale = sqrt(g.area);
  return g;
}

// ln((R+ + l+)/(R- + l-)) without cancellation; 0 on the edge (principal value)
__device__ __forceinline__ double f2_of(double lp, double lm, double Rp, double Rm, double R0sq) {
  if (lm >= 0.0) {
    const double den = Rm + lm;
    return den > 0.0 ? log((Rp + lp) / den) : 0.0;
  }
  if (lp <= 0.0) {
    const double den = Rp - lp;
    return den > 0.0 ? log((Rm - lm) / den) : 0.0;
  }
  if (R0sq == 0.0) return 0.0;
  return log((Rp + lp) * (Rm - lm) / R0sq);
}

// S0 = int_T 1/R, Sv = int_T (rho' - rho)/R in closed form (rho: projection of r)
__device__ __forceinline__ void static_tri(D3 r, const Tri& g, double& S0, D3& Sv, D3& rho) {
  double d = dotd(r - g.v[0], g.n);
  rho = r - d * g.n;
  if (fabs(d) < kSnap * g.scale) d = 0.0;
  const double ad = fabs(d);
  S0 = 0.0;
  Sv = d3(0, 0, 0);
  for (int i = 0; i < 3; ++i) {
    const D3 Pm = g.v[i], Pp = g.v[(i + 1) % 3];
    D3 s = Pp - Pm;
    s = (1.0 / normd(s)) * s;
    const D3 m = crossd(s, g.n);
    const double lp = dotd(Pp - rho, s), lm = dotd(Pm - rho, s);
    double t0 = dotd(Pm - rho, m);
    if (fabs(t0) < kSnap * g.scale) t0 = 0.0;
    const double R0sq = t0 * t0 + d * d;
    const double Rp = normd(r - Pp), Rm = normd(r - Pm);
    const double f2 = f2_of(lp, lm, Rp, Rm, R0sq);
    double beta = 0.0;
    if (R0sq > 0.0) beta = atan2(t0 * lp, R0sq + ad * Rp) - atan2(t0 * lm, R0sq + ad * Rm);
    S0 += t0 * f2 - ad * beta;
    Sv = Sv + (0.5 * (R0sq * f2 + lp * Rp - lm * Rm)) * m;
  }
}

// (exp(-jkR) - 1)/(4 pi R) as (re, im); -jk/(4 pi) at R = 0
__device__ __forceinline__ void g1_of(double R, double k, double& re, double& im) {
  if (R == 0.0) {
    re = 0.0;
    im = -k * kInv4Pi;
    return;
  }
  const double x = k * R, s = sin(0.5 * x);
  re = -2.0 * s * s * (kInv4Pi / R);
  im = -sin(x) * (kInv4Pi / R);
}

struct Rule7 {
  double b0[7], b1[7], b2[7], w[7];
};

// I[(t nS + s) 9 + 3 i + j]: the EFIE integral of test triangle t (local
// vertex i) against source triangle s (local vertex j), as the host fill's
// per-pair 3 x 3 block (before the RWG signs and lengths).  One thread per pair.
__global__ void __launch_bounds__(128) k_efie_tri_pairs(const double* __restrict__ tc, int nT,
                                                        const double* __restrict__ sc, int nS, D3 shift, double k,
                                                        Rule7 q, double2* __restrict__ I) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)nT * nS) return;
  const int t = (int)(id / nS), s = (int)(id % nS);
  const Tri tg = make_tri(tc + 9 * (int64_t)t, d3(0, 0, 0));
  const Tri g = make_tri(sc + 9 * (int64_t)s, shift);
  double ar[3][3], ai[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) ar[i][j] = ai[i][j] = 0.0;
  const double kk = 1.0 / (k * k * tg.area * g.area);
  D3 tp[7];
  double tw[7];
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    tp[a] = q.b0[a] * tg.v[0] + q.b1[a] * tg.v[1] + q.b2[a] * tg.v[2];
    tw[a] = q.w[a] * tg.area;
  }
  // static part: test quadrature of the closed-form inner integrals
  for (int a = 0; a < 7; ++a) {
    double S0;
    D3 Sv, rho;
    static_tri(tp[a], g, S0, Sv, rho);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const D3 phi = (1.0 / (2.0 * tg.area)) * (tp[a] - tg.v[i]);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const D3 Vj = (1.0 / (2.0 * g.area)) * (Sv + S0 * (rho - g.v[j]));
        ar[i][j] += tw[a] * kInv4Pi * (dotd(phi, Vj) - S0 * kk);
      }
    }
  }
  // smooth part: product quadrature of G1
  for (int a = 0; a < 7; ++a) {
    D3 phi_i[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) phi_i[i] = (1.0 / (2.0 * tg.area)) * (tp[a] - tg.v[i]);
    for (int b = 0; b < 7; ++b) {
      const D3 rs = q.b0[b] * g.v[0] + q.b1[b] * g.v[1] + q.b2[b] * g.v[2];
      double gr, gi;
      g1_of(normd(tp[a] - rs), k, gr, gi);
      const double wgt = tw[a] * q.w[b] * g.area;
      gr *= wgt;
      gi *= wgt;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const D3 phj = (1.0 / (2.0 * g.area)) * (rs - g.v[j]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const double f = dotd(phi_i[i], phj) - kk;
          ar[i][j] += gr * f;
          ai[i][j] += gi * f;
        }
      }
    }
  }
  double2* dst = I + id * 9;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) dst[3 * i + j] = make_double2(ar[i][j], ai[i][j]);
}

// RWG side: triangle, local index of the edge's opposite vertex, sign x length
struct Side {
  int tri, loc;
  double c;
};

// One near entry per thread: the RWG entry from its (up to) four triangle
// pairs, times c_A, minus the grid part.
__global__ void __launch_bounds__(128) k_near_assemble(
    int64_t nent, const int32_t* __restrict__ em, const int32_t* __restrict__ en, const Side* __restrict__ sa,
    const Side* __restrict__ sb, const double2* __restrict__ I, int nS, const int32_t* __restrict__ anca,
    const int32_t* __restrict__ ancb, int dLx, int dLy, int dLz, const double* __restrict__ Pa,
    const double* __restrict__ Pb, int S, const int32_t* __restrict__ so, const double2* __restrict__ H, int HR,
    double2 cA, double2 cphi, double2* __restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nent) return;
  const int m = em[p], n = en[p];
  double lr = 0.0, li = 0.0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const Side A = sa[2 * m + u];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const Side B = sb[2 * n + v];
      const double2 x = I[((int64_t)A.tri * nS + B.tri) * 9 + 3 * A.loc + B.loc];
      const double c = A.c * B.c;
      lr += c * x.x;
      li += c * x.y;
    }
  }
  // grid part: sum_s sum_t P_m[s] H(a_m - (a_n + dL) + o_s - o_t) P_n[t]
  const int w = 2 * HR + 1;
  const int dx = anca[3 * m] - (ancb[3 * n] + dLx), dy = anca[3 * m + 1] - (ancb[3 * n + 1] + dLy),
            dz = anca[3 * m + 2] - (ancb[3 * n + 2] + dLz);
  const double* Pm = Pa + (int64_t)m * S * 4;
  const double* Pn = Pb + (int64_t)n * S * 4;
  double vAr = 0.0, vAi = 0.0, vPr = 0.0, vPi = 0.0;
  for (int s = 0; s < S; ++s) {
    double hxr = 0, hxi = 0, hyr = 0, hyi = 0, hzr = 0, hzi = 0, hpr = 0, hpi = 0;
    const int sx = dx + so[3 * s], sy = dy + so[3 * s + 1], sz = dz + so[3 * s + 2];
    for (int t = 0; t < S; ++t) {
      const int ix = sx - so[3 * t] + HR, iy = sy - so[3 * t + 1] + HR, iz = sz - so[3 * t + 2] + HR;
      const double2 h = H[((int64_t)ix * w + iy) * w + iz];
      const double p0 = Pn[4 * t], p1 = Pn[4 * t + 1], p2 = Pn[4 * t + 2], p3 = Pn[4 * t + 3];
      hxr = fma(h.x, p0, hxr); hxi = fma(h.y, p0, hxi);
      hyr = fma(h.x, p1, hyr); hyi = fma(h.y, p1, hyi);
      hzr = fma(h.x, p2, hzr); hzi = fma(h.y, p2, hzi);
      hpr = fma(h.x, p3, hpr); hpi = fma(h.y, p3, hpi);
    }
    const double q0 = Pm[4 * s], q1 = Pm[4 * s + 1], q2 = Pm[4 * s + 2], q3 = Pm[4 * s + 3];
    vAr += q0 * hxr + q1 * hyr + q2 * hzr;
    vAi += q0 * hxi + q1 * hyi + q2 * hzi;
    vPr += q3 * hpr;
    vPi += q3 * hpi;
  }
  // val = c_A L - (c_A vA + c_phi vP)
  const double Gr = cA.x * lr - cA.y * li, Gi = cA.x * li + cA.y * lr;
  const double gr = cA.x * vAr - cA.y * vAi + cphi.x * vPr - cphi.y * vPi;
  const double gi = cA.x * vAi + cA.y * vAr + cphi.x * vPi + cphi.y * vPr;
  out[p] = make_double2(Gr - gr, Gi - gi);
}

// Full EFIE matrix: out[m Nn + n] = sum over the (up to) four triangle pairs of
// RWG m and RWG n of sign x length products times the pair integral.
__global__ void __launch_bounds__(256) k_efie_assemble(int Nm, int Nn, const Side* __restrict__ sa,
                                                       const Side* __restrict__ sb, const double2* __restrict__ I,
                                                       int nS, double2* __restrict__ out) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)Nm * Nn) return;
  const int m = (int)(id / Nn), n = (int)(id % Nn);
  double lr = 0.0, li = 0.0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const Side A = sa[2 * m + u];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const Side B = sb[2 * n + v];
      const double2 x = I[((int64_t)A.tri * nS + B.tri) * 9 + 3 * A.loc + B.loc];
      const double c = A.c * B.c;
      lr += c * x.x;
      li += c * x.y;
    }
  }
  out[id] = make_double2(lr, li);
}

// grad_r of int_T 1/R in closed form (principal value on the plane of T)
__device__ __forceinline__ D3 static_grad(D3 r, const Tri& g) {
  double d = dotd(r - g.v[0], g.n);
  const D3 rho = r - d * g.n;
  if (fabs(d) < kSnap * g.scale) d = 0.0;
  const double ad = fabs(d);
  D3 gt = d3(0, 0, 0);
  double bsum = 0.0;
  for (int i = 0; i < 3; ++i) {
    const D3 Pm = g.v[i], Pp = g.v[(i + 1) % 3];
    D3 s = Pp - Pm;
    s = (1.0 / normd(s)) * s;
    const D3 m = crossd(s, g.n);
    const double lp = dotd(Pp - rho, s), lm = dotd(Pm - rho, s);
    double t0 = dotd(Pm - rho, m);
    if (fabs(t0) < kSnap * g.scale) t0 = 0.0;
    const double R0sq = t0 * t0 + d * d;
    const double Rp = normd(r - Pp), Rm = normd(r - Pm);
    const double f2 = f2_of(lp, lm, Rp, Rm, R0sq);
    double beta = 0.0;
    if (R0sq > 0.0) beta = atan2(t0 * lp, R0sq + ad * Rp) - atan2(t0 * lm, R0sq + ad * Rm);
    bsum += beta;
    gt = gt - f2 * m;
  }
  const double sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
  return gt - (sg * bsum) * g.n;
}

// c(R) with grad_r G1(|r - r'|) = c(R) (r - r'), as (re, im); 0 at R = 0
__device__ __forceinline__ void g1grad_of(double R, double k, double& re, double& im) {
  if (R == 0.0) {
    re = im = 0.0;
    return;
  }
  const double x = k * R, s = sin(0.5 * x);
  const double a = -2.0 * s * s + x * sin(x);
  const double b = x * cos(x) - sin(x);
  const double f = -kInv4Pi / (R * R * R);
  re = a * f;
  im = b * f;
}

struct Rule3 {
  double b0[3], b1[3], b2[3], w[3];
};

// Dual support entry: refined triangle, alpha, beta (the dual field there is
// alpha r - beta).
struct DualEnt {
  int rt;
  double alpha, bx, by, bz;
};

// rows[(t 3 + i) Nn + n] = <phi_i of test triangle t, curl int G g_n> (the
// host fill_k's rows): one thread per (test triangle, dual function); per test
// point the dual's field on its support entries, with grad int_s G from the
// closed-form static part and the 3-point smooth part.
__global__ void __launch_bounds__(128) k_fillk_rows(const double* __restrict__ tc, int nT,
                                                    const double* __restrict__ rc, int Nn,
                                                    const int32_t* __restrict__ eptr,
                                                    const DualEnt* __restrict__ ent, double k, Rule7 q7, Rule3 q3,
                                                    double2* __restrict__ rows) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)nT * Nn) return;
  const int t = (int)(id / Nn), n = (int)(id % Nn);
  const Tri tg = make_tri(tc + 9 * (int64_t)t, d3(0, 0, 0));
  double accr[3] = {0, 0, 0}, acci[3] = {0, 0, 0};
  const int e0 = eptr[n], e1 = eptr[n + 1];
  for (int a = 0; a < 7; ++a) {
    const D3 r = q7.b0[a] * tg.v[0] + q7.b1[a] * tg.v[1] + q7.b2[a] * tg.v[2];
    const double wq = q7.w[a] * tg.area;
    double Wr[3] = {0, 0, 0}, Wi[3] = {0, 0, 0};
    for (int e = e0; e < e1; ++e) {
      const DualEnt de = ent[e];
      const Tri g = make_tri(rc + 9 * (int64_t)de.rt, d3(0, 0, 0));
      const D3 gs = static_grad(r, g);
      double vr[3] = {kInv4Pi * gs.x, kInv4Pi * gs.y, kInv4Pi * gs.z}, vi[3] = {0, 0, 0};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const D3 rp = q3.b0[p] * g.v[0] + q3.b1[p] * g.v[1] + q3.b2[p] * g.v[2];
        const D3 dd = r - rp;
        double cr, ci;
        g1grad_of(normd(dd), k, cr, ci);
        const double wgt = q3.w[p] * g.area;
        cr *= wgt;
        ci *= wgt;
        vr[0] += cr * dd.x; vr[1] += cr * dd.y; vr[2] += cr * dd.z;
        vi[0] += ci * dd.x; vi[1] += ci * dd.y; vi[2] += ci * dd.z;
      }
      const D3 bt = d3(de.alpha * r.x - de.bx, de.alpha * r.y - de.by, de.alpha * r.z - de.bz);
      // V x bt (complex V, real bt)
      Wr[0] += vr[1] * bt.z - vr[2] * bt.y; Wi[0] += vi[1] * bt.z - vi[2] * bt.y;
      Wr[1] += vr[2] * bt.x - vr[0] * bt.z; Wi[1] += vi[2] * bt.x - vi[0] * bt.z;
      Wr[2] += vr[0] * bt.y - vr[1] * bt.x; Wi[2] += vi[0] * bt.y - vi[1] * bt.x;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const D3 phi = (wq / (2.0 * tg.area)) * (r - tg.v[i]);
      accr[i] += phi.x * Wr[0] + phi.y * Wr[1] + phi.z * Wr[2];
      acci[i] += phi.x * Wi[0] + phi.y * Wi[1] + phi.z * Wi[2];
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) rows[((int64_t)t * 3 + i) * Nn + n] = make_double2(accr[i], acci[i]);
}

// out[m Nn + n] = sum over the two triangles of test RWG m of sign x length x rows
__global__ void __launch_bounds__(256) k_fillk_assemble(int Nm, int Nn, const Side* __restrict__ sa,
                                                        const double2* __restrict__ rows, double2* __restrict__ out) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)Nm * Nn) return;
  const int m = (int)(id / Nn), n = (int)(id % Nn);
  double lr = 0.0, li = 0.0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const Side A = sa[2 * m + u];
    const double2 x = rows[((int64_t)A.tri * 3 + A.loc) * Nn + n];
    lr += A.c * x.x;
    li += A.c * x.y;
  }
  out[id] = make_double2(lr, li);
}

struct DevMesh {
  double* tc = nullptr;   // nT x 9 vertex coordinates
  Side* side = nullptr;   // nRWG x 2 (T+, T-)
  int nT = 0, nR = 0;
};

struct DevType {
  int32_t* anc = nullptr;
  double* Pi = nullptr;
};

template <typename T>
cudaError_t upload(T** d, const T* h, size_t n) {
  *d = nullptr;
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(d, sizeof(T) * n);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d, h, sizeof(T) * n, cudaMemcpyHostToDevice);
}

cudaError_t upload_mesh(const Mesh& m, DevMesh& d) {
  d.nT = (int)m.nt();
  d.nR = (int)m.nrwg();
  std::vector<double> tc(9 * (size_t)d.nT);
  for (int t = 0; t < d.nT; ++t)
    for (int i = 0; i < 3; ++i) {
      const Vec3 v = m.tv(t, i);
      tc[9 * t + 3 * i] = v.x;
      tc[9 * t + 3 * i + 1] = v.y;
      tc[9 * t + 3 * i + 2] = v.z;
    }
  std::vector<Side> sd(2 * (size_t)d.nR, Side{0, 0, 0.0});
  for (int t = 0; t < d.nT; ++t)
    for (int i = 0; i < 3; ++i) {
      const int64_t r = m.tri_rwg[3 * t + i];
      if (r < 0) continue;
      const int sg = m.tri_sign[3 * t + i];
      sd[2 * r + (sg > 0 ? 0 : 1)] = Side{t, i, sg * m.length[r]};
    }
  cudaError_t e = upload(&d.tc, tc.data(), tc.size());
  if (e == cudaSuccess) e = upload(&d.side, sd.data(), sd.size());
  return e;
}

}  // namespace

bool fill_near_blocks_gpu(std::vector<NearFillJob>& jobs, const std::vector<cd>& Hv, int HR,
                          const std::vector<std::array<int, 3>>& so, cd cA, cd cphi, double k, int device,
                          std::string& msg) {
  if (jobs.empty()) return true;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    msg = "cudaSetDevice failed";
    return false;
  }
  std::map<const Mesh*, DevMesh> meshes;
  std::map<const TypeAim*, DevType> types;
  double2* dH = nullptr;
  int32_t* dso = nullptr;
  double2* dI = nullptr;
  int32_t *dm = nullptr, *dn = nullptr;
  double2* dout = nullptr;
  cudaError_t e = cudaSuccess;
  const int S = (int)so.size();
  {
    std::vector<double2> h(Hv.size());
    for (size_t i = 0; i < Hv.size(); ++i) h[i] = make_double2(Hv[i].real(), Hv[i].imag());
    e = upload(&dH, h.data(), h.size());
    std::vector<int32_t> s3(3 * (size_t)S);
    for (int s = 0; s < S; ++s)
      for (int a = 0; a < 3; ++a) s3[3 * s + a] = so[s][a];
    if (e == cudaSuccess) e = upload(&dso, s3.data(), s3.size());
  }
  const Rule r7 = rule_tri7();
  Rule7 q;
  for (int a = 0; a < 7; ++a) {
    q.b0[a] = r7.b0[a];
    q.b1[a] = r7.b1[a];
    q.b2[a] = r7.b2[a];
    q.w[a] = r7.w[a];
  }
  size_t Icap = 0, Ecap = 0;
  for (auto& jb : jobs) {
    if (e != cudaSuccess) break;
    for (const Mesh* mp : {jb.ma, jb.mb})
      if (!meshes.count(mp)) {
        DevMesh dm_;
        e = upload_mesh(*mp, dm_);
        meshes[mp] = dm_;
        if (e != cudaSuccess) break;
      }
    for (const TypeAim* tp : {jb.A, jb.B})
      if (e == cudaSuccess && !types.count(tp)) {
        DevType dt;
        std::vector<int32_t> anc(tp->anc.size());
        for (size_t i = 0; i < anc.size(); ++i) anc[i] = (int32_t)tp->anc[i];
        e = upload(&dt.anc, anc.data(), anc.size());
        if (e == cudaSuccess) e = upload(&dt.Pi, tp->Pi.data(), tp->Pi.size());
        types[tp] = dt;
      }
    if (e != cudaSuccess) break;
    const DevMesh &MA = meshes[jb.ma], &MB = meshes[jb.mb];
    const size_t np = (size_t)MA.nT * MB.nT;
    if (np > Icap) {
      if (dI) cudaFree(dI);
      e = cudaMalloc(&dI, sizeof(double2) * 9 * np);
      if (e != cudaSuccess) {
        dI = nullptr;
        break;
      }
      Icap = np;
    }
    k_efie_tri_pairs<<<(unsigned)((np + 127) / 128), 128>>>(MA.tc, MA.nT, MB.tc, MB.nT,
                                                             D3{jb.rel.x, jb.rel.y, jb.rel.z}, k, q, dI);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    // near entries of the block, row by row
    const auto& ptr = *jb.ptr;
    const auto& col = *jb.col;
    const size_t nent = col.size();
    std::vector<int32_t> hm(nent), hn(nent);
    for (size_t mrow = 0; mrow + 1 < ptr.size(); ++mrow)
      for (int64_t pq = ptr[mrow]; pq < ptr[mrow + 1]; ++pq) {
        hm[pq] = (int32_t)mrow;
        hn[pq] = col[pq];
      }
    if (nent > Ecap) {
      if (dm) cudaFree(dm);
      if (dn) cudaFree(dn);
      if (dout) cudaFree(dout);
      dm = dn = nullptr;
      dout = nullptr;
      e = cudaMalloc(&dm, sizeof(int32_t) * nent);
      if (e == cudaSuccess) e = cudaMalloc(&dn, sizeof(int32_t) * nent);
      if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double2) * nent);
      if (e != cudaSuccess) break;
      Ecap = nent;
    }
    e = cudaMemcpy(dm, hm.data(), sizeof(int32_t) * nent, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dn, hn.data(), sizeof(int32_t) * nent, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
    const DevType &TA = types[jb.A], &TB = types[jb.B];
    k_near_assemble<<<(unsigned)((nent + 127) / 128), 128>>>(
        (int64_t)nent, dm, dn, MA.side, MB.side, dI, MB.nT, TA.anc, TB.anc, (int)jb.dL[0], (int)jb.dL[1],
        (int)jb.dL[2], TA.Pi, TB.Pi, S, dso, dH, HR, make_double2(cA.real(), cA.imag()),
        make_double2(cphi.real(), cphi.imag()), dout);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    std::vector<double2> hv(nent);
    e = cudaMemcpy(hv.data(), dout, sizeof(double2) * nent, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    jb.val->resize(nent);
    for (size_t i = 0; i < nent; ++i) (*jb.val)[i] = cd(hv[i].x, hv[i].y);
  }
  for (auto& kv : meshes) {
    if (kv.second.tc) cudaFree(kv.second.tc);
    if (kv.second.side) cudaFree(kv.second.side);
  }
  for (auto& kv : types) {
    if (kv.second.anc) cudaFree(kv.second.anc);
    if (kv.second.Pi) cudaFree(kv.second.Pi);
  }
  for (void* p : {(void*)dH, (void*)dso, (void*)dI, (void*)dm, (void*)dn, (void*)dout})
    if (p) cudaFree(p);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    msg = std::string("near-field fill on the GPU: ") + cudaGetErrorString(e);
    return false;
  }
  return true;
}

bool fill_efie_gpu(const Mesh& test, const Mesh& src, Vec3 shift, double k, int device, std::vector<cd>& out,
                   std::string& msg) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    msg = "cudaSetDevice failed";
    return false;
  }
  DevMesh MT, MS;
  double2 *dI = nullptr, *dout = nullptr;
  cudaError_t e = upload_mesh(test, MT);
  if (e == cudaSuccess && &src != &test) e = upload_mesh(src, MS);
  const DevMesh& MSr = (&src == &test) ? MT : MS;
  const size_t np = (size_t)MT.nT * MSr.nT, ne = (size_t)MT.nR * MSr.nR;
  if (e == cudaSuccess) e = cudaMalloc(&dI, sizeof(double2) * 9 * np);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double2) * ne);
  if (e == cudaSuccess) {
    const Rule r7 = rule_tri7();
    Rule7 q;
    for (int a = 0; a < 7; ++a) {
      q.b0[a] = r7.b0[a];
      q.b1[a] = r7.b1[a];
      q.b2[a] = r7.b2[a];
      q.w[a] = r7.w[a];
    }
    k_efie_tri_pairs<<<(unsigned)((np + 127) / 128), 128>>>(MT.tc, MT.nT, MSr.tc, MSr.nT, D3{shift.x, shift.y, shift.z},
                                                             k, q, dI);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_efie_assemble<<<(unsigned)((ne + 255) / 256), 256>>>(MT.nR, MSr.nR, MT.side, MSr.side, dI, MSr.nT, dout);
    e = cudaGetLastError();
  }
  std::vector<double2> h;
  if (e == cudaSuccess) {
    h.resize(ne);
    e = cudaMemcpy(h.data(), dout, sizeof(double2) * ne, cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess) {
    out.resize(ne);
    for (size_t i = 0; i < ne; ++i) out[i] = cd(h[i].x, h[i].y);
  }
  for (void* p : {(void*)MT.tc, (void*)MT.side, (void*)MS.tc, (void*)MS.side, (void*)dI, (void*)dout})
    if (p) cudaFree(p);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    msg = std::string("EFIE fill on the GPU: ") + cudaGetErrorString(e);
    return false;
  }
  return true;
}

bool fill_k_gpu(const Mesh& test, const DualSet& d, double k, int device, std::vector<cd>& out, std::string& msg) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    msg = "cudaSetDevice failed";
    return false;
  }
  const int nR = (int)d.rarea.size(), Nn = (int)d.n, E = (int)d.fn.size();
  // refined triangles' vertices; support entries grouped by dual function
  // (entries of one function in increasing entry order, as the host sums them)
  std::vector<double> rc(9 * (size_t)nR);
  for (int r = 0; r < nR; ++r)
    for (int i = 0; i < 3; ++i) {
      const Vec3 v = d.rvert(r, i);
      rc[9 * r + 3 * i] = v.x;
      rc[9 * r + 3 * i + 1] = v.y;
      rc[9 * r + 3 * i + 2] = v.z;
    }
  std::vector<int32_t> eptr(Nn + 1, 0);
  for (int e = 0; e < E; ++e) ++eptr[d.fn[e] + 1];
  for (int n = 0; n < Nn; ++n) eptr[n + 1] += eptr[n];
  std::vector<DualEnt> ent(E);
  {
    std::vector<int32_t> fill(eptr.begin(), eptr.end() - 1);
    for (int e = 0; e < E; ++e) {
      const int64_t r = d.rt[e];
      const double A2 = 2.0 * d.rarea[r];
      const double fs = d.flux[3 * e] + d.flux[3 * e + 1] + d.flux[3 * e + 2];
      Vec3 b{0, 0, 0};
      for (int i = 0; i < 3; ++i) b = b + (d.flux[3 * e + i] / A2) * d.rvert(r, i);
      ent[fill[d.fn[e]]++] = DualEnt{(int)r, fs / A2, b.x, b.y, b.z};
    }
  }
  DevMesh MT;
  double* drc = nullptr;
  int32_t* deptr = nullptr;
  DualEnt* dent = nullptr;
  double2 *drows = nullptr, *dout = nullptr;
  cudaError_t e = upload_mesh(test, MT);
  if (e == cudaSuccess) e = upload(&drc, rc.data(), rc.size());
  if (e == cudaSuccess) e = upload(&deptr, eptr.data(), eptr.size());
  if (e == cudaSuccess) e = upload(&dent, ent.data(), ent.size());
  const size_t nrows = (size_t)MT.nT * 3 * Nn, ne = (size_t)MT.nR * Nn;
  if (e == cudaSuccess) e = cudaMalloc(&drows, sizeof(double2) * nrows);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double2) * ne);
  if (e == cudaSuccess) {
    const Rule r7 = rule_tri7(), r3 = rule_tri3();
    Rule7 q7;
    Rule3 q3;
    for (int a = 0; a < 7; ++a) {
      q7.b0[a] = r7.b0[a];
      q7.b1[a] = r7.b1[a];
      q7.b2[a] = r7.b2[a];
      q7.w[a] = r7.w[a];
    }
    for (int a = 0; a < 3; ++a) {
      q3.b0[a] = r3.b0[a];
      q3.b1[a] = r3.b1[a];
      q3.b2[a] = r3.b2[a];
      q3.w[a] = r3.w[a];
    }
    const size_t nth = (size_t)MT.nT * Nn;
    k_fillk_rows<<<(unsigned)((nth + 127) / 128), 128>>>(MT.tc, MT.nT, drc, Nn, deptr, dent, k, q7, q3, drows);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_fillk_assemble<<<(unsigned)((ne + 255) / 256), 256>>>(MT.nR, Nn, MT.side, drows, dout);
    e = cudaGetLastError();
  }
  std::vector<double2> h;
  if (e == cudaSuccess) {
    h.resize(ne);
    e = cudaMemcpy(h.data(), dout, sizeof(double2) * ne, cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess) {
    out.resize(ne);
    for (size_t i = 0; i < ne; ++i) out[i] = cd(h[i].x, h[i].y);
  }
  for (void* p : {(void*)MT.tc, (void*)MT.side, (void*)drc, (void*)deptr, (void*)dent, (void*)drows, (void*)dout})
    if (p) cudaFree(p);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    msg = std::string("K fill on the GPU: ") + cudaGetErrorString(e);
    return false;
  }
  return true;
}

}  // namespace mm
