// Galerkin fills and the per-type macromodel (Sec. II-D/E/F, Sec. IV), host FP64.
//
//  Lmat[m, n] = int int f_m . f_n G - k^-2 int int (div f_m)(div' f_n) G
//  Kmat_PV[m, n] = <f_m, curl int G g_n>   (principal value on the source plane)
//  D[m, n] = <f^_m, n_in x g_n>
// G = exp(-jkR)/(4 pi R) = 1/(4 pi R) + G1.  The 1/R part is integrated over
// the source triangle in closed form (singularity extraction, the formulas of
// Wilton et al. 1984 / Graglia 1993), G1 by quadrature: 7-point rule on test
// and source primal triangles (L), 7-point test / 3-point refined-source (K).
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "fill_gpu.h"

namespace mm {

static constexpr double SNAP = 1e-10;   // relative height/edge distance treated as exactly 0
static constexpr double INV4PI = 0.25 / M_PI;

struct TriGeo {
  Vec3 v[3];
  Vec3 n;
  double area, scale;
};

static inline TriGeo tri_geo(Vec3 a, Vec3 b, Vec3 c) {
  TriGeo g;
  g.v[0] = a; g.v[1] = b; g.v[2] = c;
  Vec3 cr = cross(b - a, c - a);
  double nn = norm(cr);
  g.n = (1.0 / nn) * cr;
  g.area = 0.5 * nn;
  g.scale = std::sqrt(g.area);
  return g;
}

// ln((R+ + l+)/(R- + l-)) without cancellation, branching on the signs of l+-.
// A point exactly on the edge (segment or end point) takes 0, the principal value.
static inline double f2_of(double lp, double lm, double Rp, double Rm, double R0sq) {
  if (lm >= 0.0) {
    double den = Rm + lm;
    return den > 0.0 ? std::log((Rp + lp) / den) : 0.0;
  }
  if (lp <= 0.0) {
    double den = Rp - lp;
    return den > 0.0 ? std::log((Rm - lm) / den) : 0.0;
  }
  if (R0sq == 0.0) return 0.0;
  return std::log((Rp + lp) * (Rm - lm) / R0sq);
}

// Closed-form S0 = int 1/R, Sv = int (rho' - rho)/R, grad = grad_r int 1/R
// (principal value when r is on the plane), rho = projection of r.
static inline void static_tri(Vec3 r, const TriGeo& g, bool need_sv, bool need_grad, double& S0, Vec3& Sv,
                              Vec3& grad, Vec3& rho) {
  double d = dot(r - g.v[0], g.n);
  rho = r - d * g.n;
  if (std::fabs(d) < SNAP * g.scale) d = 0.0;
  double ad = std::fabs(d);
  S0 = 0.0;
  Sv = {0, 0, 0};
  Vec3 gt{0, 0, 0};
  double bsum = 0.0;
  for (int i = 0; i < 3; ++i) {
    Vec3 Pm = g.v[i], Pp = g.v[(i + 1) % 3];
    Vec3 s = Pp - Pm;
    s = (1.0 / norm(s)) * s;
    Vec3 m = cross(s, g.n);
    double lp = dot(Pp - rho, s), lm = dot(Pm - rho, s);
    double t0 = dot(Pm - rho, m);
    if (std::fabs(t0) < SNAP * g.scale) t0 = 0.0;
    double R0sq = t0 * t0 + d * d;
    double Rp = norm(r - Pp), Rm = norm(r - Pm);
    double f2 = f2_of(lp, lm, Rp, Rm, R0sq);
    double beta = 0.0;
    if (R0sq > 0.0) beta = std::atan2(t0 * lp, R0sq + ad * Rp) - std::atan2(t0 * lm, R0sq + ad * Rm);
    S0 += t0 * f2 - ad * beta;
    bsum += beta;
    if (need_sv) Sv = Sv + (0.5 * (R0sq * f2 + lp * Rp - lm * Rm)) * m;
    if (need_grad) gt = gt - f2 * m;
  }
  if (need_grad) {
    double sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
    grad = gt - (sg * bsum) * g.n;
  }
}

// (exp(-jkR) - 1)/(4 pi R), limit -jk/(4 pi) at R = 0.
static inline cd g1_of(double R, double k) {
  if (R == 0.0) return cd(0.0, -k * INV4PI);
  double x = k * R, s = std::sin(0.5 * x);
  return cd(-2.0 * s * s, -std::sin(x)) * (INV4PI / R);
}

// c(R) with grad_r G1(|r - r'|) = c(R) (r - r'); 0 at R = 0.
static inline cd g1grad_of(double R, double k) {
  if (R == 0.0) return cd(0.0, 0.0);
  double x = k * R, s = std::sin(0.5 * x);
  double re = -2.0 * s * s + x * std::sin(x);
  double im = x * std::cos(x) - std::sin(x);
  return -cd(re, im) * (INV4PI / (R * R * R));
}

static inline Vec3 bary(const Rule& q, int i, const Vec3 v[3]) {
  return q.b0[i] * v[0] + q.b1[i] * v[1] + q.b2[i] * v[2];
}

void fill_efie(const Mesh& test, const Mesh& src, Vec3 shift, const EM& em, std::vector<cd>& out) {
  const double k = em.k;
  int64_t nT = test.nt(), nS = src.nt();
  int64_t Nm = test.nrwg(), Nn = src.nrwg();
  out.assign(Nm * Nn, cd(0, 0));
  Rule q7 = rule_tri7();
  int Q = q7.n();
  std::vector<TriGeo> sg(nS);
  std::vector<Vec3> sp(nS * Q);
  for (int64_t s = 0; s < nS; ++s) {
    sg[s] = tri_geo(src.tv(s, 0) + shift, src.tv(s, 1) + shift, src.tv(s, 2) + shift);
    for (int q = 0; q < Q; ++q) sp[s * Q + q] = bary(q7, q, sg[s].v);
  }
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nT, 32 * std::max(1, em.nthreads)));
  std::vector<cd> I;  // (chunk, nS, 3, 3)
  for (int64_t c0 = 0; c0 < nT; c0 += chunk) {
    int64_t c1 = std::min(nT, c0 + chunk);
    I.assign((c1 - c0) * nS * 9, cd(0, 0));
    parallel_for(c1 - c0, em.nthreads, [&](int64_t a, int64_t b) {
      for (int64_t tt = a; tt < b; ++tt) {
        int64_t t = c0 + tt;
        TriGeo tg = tri_geo(test.tv(t, 0), test.tv(t, 1), test.tv(t, 2));
        Vec3 tp[7];
        double tw[7];
        for (int q = 0; q < Q; ++q) {
          tp[q] = bary(q7, q, tg.v);
          tw[q] = q7.w[q] * tg.area;
        }
        for (int64_t s = 0; s < nS; ++s) {
          const TriGeo& g = sg[s];
          cd acc[3][3];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc[i][j] = 0;
          double kk = 1.0 / (k * k * tg.area * g.area);
          // static part: test quadrature of the closed-form inner integrals
          for (int q = 0; q < Q; ++q) {
            double S0;
            Vec3 Sv, gr, rho;
            static_tri(tp[q], g, true, false, S0, Sv, gr, rho);
            for (int i = 0; i < 3; ++i) {
              Vec3 phi = (1.0 / (2.0 * tg.area)) * (tp[q] - tg.v[i]);
              for (int j = 0; j < 3; ++j) {
                Vec3 Vj = (1.0 / (2.0 * g.area)) * (Sv + S0 * (rho - g.v[j]));
                acc[i][j] += tw[q] * INV4PI * (dot(phi, Vj) - S0 * kk);
              }
            }
          }
          // smooth part: product quadrature of G1
          for (int q = 0; q < Q; ++q) {
            Vec3 phi_i[3];
            for (int i = 0; i < 3; ++i) phi_i[i] = (1.0 / (2.0 * tg.area)) * (tp[q] - tg.v[i]);
            for (int p = 0; p < Q; ++p) {
              Vec3 rs = sp[s * Q + p];
              double R = norm(tp[q] - rs);
              cd wg = g1_of(R, k) * (tw[q] * q7.w[p] * g.area);
              for (int j = 0; j < 3; ++j) {
                Vec3 phj = (1.0 / (2.0 * g.area)) * (rs - g.v[j]);
                for (int i = 0; i < 3; ++i) acc[i][j] += wg * (dot(phi_i[i], phj) - kk);
              }
            }
          }
          cd* dst = &I[((tt * nS) + s) * 9];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) dst[3 * i + j] = acc[i][j];
        }
      }
    });
    for (int64_t tt = 0; tt < c1 - c0; ++tt) {
      int64_t t = c0 + tt;
      for (int i = 0; i < 3; ++i) {
        int64_t m = test.tri_rwg[3 * t + i];
        if (m < 0) continue;
        double cm = test.tri_sign[3 * t + i] * test.length[m];
        for (int64_t s = 0; s < nS; ++s)
          for (int j = 0; j < 3; ++j) {
            int64_t n = src.tri_rwg[3 * s + j];
            if (n < 0) continue;
            double cn = src.tri_sign[3 * s + j] * src.length[n];
            out[m * Nn + n] += (cm * cn) * I[((tt * nS) + s) * 9 + 3 * i + j];
          }
      }
    }
  }
}

void fill_k(const Mesh& test, const Mesh& eq, const DualSet& d, const EM& em, std::vector<cd>& out) {
  const double k = em.k;
  int64_t nT = test.nt(), nR = (int64_t)d.rarea.size(), Nm = test.nrwg(), Nn = d.n;
  int64_t E = (int64_t)d.fn.size();
  out.assign(Nm * Nn, cd(0, 0));
  Rule q7 = rule_tri7(), q3 = rule_tri3();
  std::vector<TriGeo> rg(nR);
  std::vector<Vec3> rp(nR * 3);
  for (int64_t r = 0; r < nR; ++r) {
    rg[r] = tri_geo(d.rvert(r, 0), d.rvert(r, 1), d.rvert(r, 2));
    for (int q = 0; q < 3; ++q) rp[r * 3 + q] = bary(q3, q, rg[r].v);
  }
  // dual field on a support entry: alpha r - beta
  std::vector<double> alpha(E);
  std::vector<Vec3> beta(E);
  for (int64_t e = 0; e < E; ++e) {
    int64_t r = d.rt[e];
    double A2 = 2.0 * d.rarea[r];
    double fs = d.flux[3 * e] + d.flux[3 * e + 1] + d.flux[3 * e + 2];
    alpha[e] = fs / A2;
    Vec3 b{0, 0, 0};
    for (int i = 0; i < 3; ++i) b = b + (d.flux[3 * e + i] / A2) * d.rvert(r, i);
    beta[e] = b;
  }
  std::vector<cd> rows(nT * 3 * Nn);
  parallel_for(nT, em.nthreads, [&](int64_t a, int64_t b) {
    std::vector<CVec3> V(nR);
    std::vector<CVec3> W(Nn);
    for (int64_t t = a; t < b; ++t) {
      TriGeo tg = tri_geo(test.tv(t, 0), test.tv(t, 1), test.tv(t, 2));
      cd* dst = &rows[t * 3 * Nn];
      for (int64_t x = 0; x < 3 * Nn; ++x) dst[x] = 0;
      for (int q = 0; q < q7.n(); ++q) {
        Vec3 r = bary(q7, q, tg.v);
        double wq = q7.w[q] * tg.area;
        for (int64_t s = 0; s < nR; ++s) {
          double S0;
          Vec3 Sv, gr, rho;
          static_tri(r, rg[s], false, true, S0, Sv, gr, rho);
          CVec3 v{INV4PI * gr.x, INV4PI * gr.y, INV4PI * gr.z};
          for (int p = 0; p < 3; ++p) {
            Vec3 dd = r - rp[s * 3 + p];
            cd c = g1grad_of(norm(dd), k) * (q3.w[p] * rg[s].area);
            v.x += c * dd.x; v.y += c * dd.y; v.z += c * dd.z;
          }
          V[s] = v;
        }
        for (int64_t n = 0; n < Nn; ++n) W[n] = {0, 0, 0};
        for (int64_t e = 0; e < E; ++e) {
          Vec3 bt = alpha[e] * r - beta[e];
          CVec3 c = ccross(V[d.rt[e]], bt);
          CVec3& w = W[d.fn[e]];
          w.x += c.x; w.y += c.y; w.z += c.z;
        }
        for (int i = 0; i < 3; ++i) {
          Vec3 phi = (wq / (2.0 * tg.area)) * (r - tg.v[i]);
          for (int64_t n = 0; n < Nn; ++n) dst[i * Nn + n] += cdot(phi, W[n]);
        }
      }
    }
  });
  for (int64_t t = 0; t < nT; ++t)
    for (int i = 0; i < 3; ++i) {
      int64_t m = test.tri_rwg[3 * t + i];
      if (m < 0) continue;
      double cm = test.tri_sign[3 * t + i] * test.length[m];
      for (int64_t n = 0; n < Nn; ++n) out[m * Nn + n] += cm * rows[(t * 3 + i) * Nn + n];
    }
}

void fill_dual_gram(const Mesh& eq, const DualSet& d, std::vector<double>& out) {
  int64_t N = eq.nrwg();
  out.assign(N * N, 0.0);
  Rule q3 = rule_tri3();
  int64_t E = (int64_t)d.fn.size();
  for (int64_t e = 0; e < E; ++e) {
    int64_t r = d.rt[e], T = d.parent[r];
    double A2 = 2.0 * d.rarea[r];
    Vec3 nin = -1.0 * eq.normal[T];
    Vec3 rv[3] = {d.rvert(r, 0), d.rvert(r, 1), d.rvert(r, 2)};
    for (int q = 0; q < 3; ++q) {
      Vec3 x = bary(q3, q, rv);
      Vec3 g{0, 0, 0};
      for (int i = 0; i < 3; ++i) g = g + (d.flux[3 * e + i] / A2) * (x - rv[i]);
      Vec3 ng = cross(nin, g);
      for (int i = 0; i < 3; ++i) {
        int64_t m = eq.tri_rwg[3 * T + i];
        if (m < 0) continue;
        Vec3 f = (eq.tri_sign[3 * T + i] * eq.length[m] / (2.0 * eq.area[T])) * (x - eq.tv(T, i));
        out[m * N + d.fn[e]] += d.rarea[r] * q3.w[q] * dot(f, ng);
      }
    }
  }
}

// ---- dense complex LU -------------------------------------------------------
void lu_factor(LU& lu, std::vector<cd> a, int64_t n) {
  lu.n = n;
  lu.a = std::move(a);
  lu.piv.resize(n);
  auto& A = lu.a;
  for (int64_t j = 0; j < n; ++j) {
    int64_t p = j;
    double best = std::abs(A[j * n + j]);
    for (int64_t i = j + 1; i < n; ++i) {
      double v = std::abs(A[i * n + j]);
      if (v > best) { best = v; p = i; }
    }
    if (!(best > 0)) throw Error{MM_EINVAL, "singular matrix in macromodel build"};
    lu.piv[j] = p;
    if (p != j)
      for (int64_t c = 0; c < n; ++c) std::swap(A[j * n + c], A[p * n + c]);
    cd inv = 1.0 / A[j * n + j];
    for (int64_t i = j + 1; i < n; ++i) {
      cd f = A[i * n + j] * inv;
      A[i * n + j] = f;
      if (f == cd(0, 0)) continue;
      cd* ri = &A[i * n];
      const cd* rj = &A[j * n];
      for (int64_t c = j + 1; c < n; ++c) ri[c] -= f * rj[c];
    }
  }
}

void lu_solve(const LU& lu, std::vector<cd>& b, int64_t nc, int nthreads) {
  int64_t n = lu.n;
  const auto& A = lu.a;
  for (int64_t j = 0; j < n; ++j)
    if (lu.piv[j] != j)
      for (int64_t c = 0; c < nc; ++c) std::swap(b[j * nc + c], b[lu.piv[j] * nc + c]);
  parallel_for(nc, nthreads, [&](int64_t c0, int64_t c1) {
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < i; ++j) {
        cd f = A[i * n + j];
        for (int64_t c = c0; c < c1; ++c) b[i * nc + c] -= f * b[j * nc + c];
      }
    for (int64_t i = n - 1; i >= 0; --i) {
      for (int64_t j = i + 1; j < n; ++j) {
        cd f = A[i * n + j];
        for (int64_t c = c0; c < c1; ++c) b[i * nc + c] -= f * b[j * nc + c];
      }
      cd inv = 1.0 / A[i * n + i];
      for (int64_t c = c0; c < c1; ++c) b[i * nc + c] *= inv;
    }
  });
}

// C (m x n) = A (m x k) B (k x n), row-major.
static void gemm(const std::vector<cd>& A, const std::vector<cd>& B, std::vector<cd>& C, int64_t m, int64_t k,
                 int64_t n, int nthreads) {
  C.assign(m * n, cd(0, 0));
  parallel_for(m, nthreads, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i)
      for (int64_t p = 0; p < k; ++p) {
        cd f = A[i * k + p];
        const cd* rb = &B[p * n];
        cd* rc = &C[i * n];
        for (int64_t j = 0; j < n; ++j) rc[j] += f * rb[j];
      }
  });
}

// Sec. II: G^(E,J) = c L(S,S), G^(E,H^) = c L(S,S^), G^(E^,J) = c L(S^,S),
// G^(E^,H^) = c L(S^,S^), c = -j w mu0; G^(E,E^) = K(S, S^'),
// G^(E^,E^) = K_PV(S^, S^') + D/2 (limit from outside the equivalent surface).
// T = G^(E^,H^)^-1 G^(E^,J) (eq. (Tm1)); A, B of eq. (JM); M = T A^-1 B.
// The fills run on the host; with device >= 0 and a large scatterer the dense
// steps run on that GPU (build_type_dense_gpu), otherwise on the host.
// Scatterers of at least this many RWG functions take the device path: below
// it the host's factorisation is as fast as the device's latency-bound panels.
constexpr int64_t kDenseGpuMinN = 1024;

void build_type(TypeModel& tm, int device) {
  const EM& em = tm.em;
  tm.N = tm.scat.nrwg();
  tm.Nh = tm.eq.nrwg();
  int64_t N = tm.N, Nh = tm.Nh;
  if (N < 1 || Nh < 1) throw Error{MM_EINVAL, "element surfaces carry no RWG functions"};
  build_duals(tm.eq, tm.duals);
  const cd c(0.0, -em.k * em.eta0);
  Vec3 z{0, 0, 0};
  std::vector<cd> Lss, Lse, Les, Lee, Kse, Kee;
  std::vector<double> D;
  // the four EFIE fills on the GPU for large elements of a device context
  // (the same integrals; the host fill otherwise or if the device fails)
  auto efie = [&](const Mesh& t, const Mesh& sm, std::vector<cd>& out) {
    std::string msg;
    if (device >= 0 && N >= kDenseGpuMinN && fill_efie_gpu(t, sm, z, em.k, device, out, msg)) return;
    fill_efie(t, sm, z, em, out);
  };
  efie(tm.scat, tm.scat, Lss);
  efie(tm.scat, tm.eq, Lse);
  efie(tm.eq, tm.scat, Les);
  efie(tm.eq, tm.eq, Lee);
  auto kfill = [&](const Mesh& t, std::vector<cd>& out) {
    std::string msg;
    if (device >= 0 && N >= kDenseGpuMinN && fill_k_gpu(t, tm.duals, em.k, device, out, msg)) return;
    fill_k(t, tm.eq, tm.duals, em, out);
  };
  kfill(tm.scat, Kse);
  kfill(tm.eq, Kee);
  fill_dual_gram(tm.eq, tm.duals, D);
  for (auto& x : Lss) x *= c;
  for (auto& x : Lse) x *= c;
  for (auto& x : Les) x *= c;
  for (auto& x : Lee) x *= c;
  tm.D.resize(Nh * Nh);
  for (int64_t i = 0; i < Nh * Nh; ++i) tm.D[i] = cd(D[i], 0.0);
  tm.GHE = Kee;
  for (int64_t i = 0; i < Nh * Nh; ++i) tm.GHE[i] += 0.5 * D[i];
  tm.GHH = Lee;
  if (device >= 0 && N >= kDenseGpuMinN) {
    // the dense steps (LU factorisations, solves, products) on the device
    std::string msg;
    if (!build_type_dense_gpu(tm, Lss, Lse, Les, Lee, Kse, device, msg)) throw Error{MM_ECUDA, msg};
    return;
  }
  LU lu;
  lu_factor(lu, Lee, Nh);
  tm.T = Les;
  lu_solve(lu, tm.T, N, em.nthreads);           // T = G^(E^,H^)^-1 G^(E^,J)
  std::vector<cd> X1 = tm.GHE;
  lu_solve(lu, X1, Nh, em.nthreads);            // G^(E^,H^)^-1 G^(E^,E^)
  std::vector<cd> tmp;
  gemm(Lse, tm.T, tmp, N, Nh, N, em.nthreads);
  tm.A = Lss;
  for (int64_t i = 0; i < N * N; ++i) tm.A[i] -= tmp[i];
  gemm(Lse, X1, tmp, N, Nh, Nh, em.nthreads);
  tm.B = Kse;
  for (int64_t i = 0; i < N * Nh; ++i) tm.B[i] -= tmp[i];
  LU la;
  lu_factor(la, tm.A, N);
  std::vector<cd> Y = tm.B;
  lu_solve(la, Y, Nh, em.nthreads);             // A^-1 B
  gemm(tm.T, Y, tm.M, Nh, N, Nh, em.nthreads);  // M = T A^-1 B
  tm.JE.resize(Y.size());
  for (size_t i = 0; i < Y.size(); ++i) tm.JE[i] = -Y[i];
  {
    // block-Jacobi preconditioner: the inverse of the element's own block of the
    // array system, D - G^(E^,H^) M (eq. (MV_product1) restricted to one element;
    // G^(E^,H^) is the EFIE operator of the equivalent surface on itself)
    std::vector<cd> GM;
    gemm(tm.GHH, tm.M, GM, Nh, Nh, Nh, em.nthreads);
    std::vector<cd> S(Nh * Nh);
    for (int64_t i = 0; i < Nh * Nh; ++i) S[i] = tm.D[i] - GM[i];
    LU ls;
    lu_factor(ls, S, Nh);
    tm.PJ.assign(Nh * Nh, cd(0, 0));
    for (int64_t i = 0; i < Nh; ++i) tm.PJ[i * Nh + i] = cd(1, 0);
    lu_solve(ls, tm.PJ, Nh, em.nthreads);
    // the right-preconditioned operator Z P^-1 applies M and D to P^-1 x:
    // its macromodel matrices are M PJ and D PJ, formed here in FP64
    std::vector<cd> MD(2 * Nh * Nh);
    std::copy(tm.M.begin(), tm.M.end(), MD.begin());
    std::copy(tm.D.begin(), tm.D.end(), MD.begin() + Nh * Nh);
    gemm(MD, tm.PJ, tm.WPJ, 2 * Nh, Nh, Nh, em.nthreads);
  }
}

}  // namespace mm
