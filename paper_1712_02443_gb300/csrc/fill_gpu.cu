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

}  // namespace mm
