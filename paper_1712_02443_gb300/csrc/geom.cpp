// Geometry set-up: RWG functions, barycentric refinement, Buffa-Christiansen
// duals (Sec. II-A, eqs. (J_expand), (Hhat_expand), (Ehat_expand)), quadrature
// rules and the host thread pool.
#include <algorithm>
#include <cmath>
#include <map>
#include <thread>

#include "internal.h"

namespace mm {

void parallel_for(int64_t n, int nthreads, const std::function<void(int64_t, int64_t)>& body) {
  if (n <= 0) return;
  int T = std::max(1, std::min<int>(nthreads, (int)n));
  if (T == 1) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  std::vector<Error> errs(T);
  std::vector<char> failed(T, 0);
  int64_t chunk = (n + T - 1) / T;
  for (int t = 0; t < T; ++t) {
    int64_t a = t * chunk, b = std::min<int64_t>(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([&, t, a, b] {
      try {
        body(a, b);
      } catch (const Error& e) {
        errs[t] = e;
        failed[t] = 1;
      } catch (...) {
        errs[t] = {MM_EINTERNAL, "exception in worker thread"};
        failed[t] = 1;
      }
    });
  }
  for (auto& x : th) x.join();
  for (int t = 0; t < T; ++t)
    if (failed[t]) throw errs[t];
}

// RWG n lives on interior edge (a, b), a < b, edges in lexicographic order;
// T+ is the adjacent triangle of smaller index; f = +-l/(2A)(r - p_free).
void build_mesh(Mesh& m, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt) {
  if (nv < 3 || nt < 1) throw Error{MM_EINVAL, "mesh needs at least 3 vertices and 1 triangle"};
  m.v.resize(nv);
  for (int64_t i = 0; i < nv; ++i) m.v[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
  m.tri.assign(tri, tri + 3 * nt);
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (m.tri[i] < 0 || m.tri[i] >= nv) throw Error{MM_EINVAL, "triangle vertex index out of range"};
  m.area.resize(nt);
  m.normal.resize(nt);
  double amax = 0;
  for (int64_t t = 0; t < nt; ++t) {
    Vec3 c = cross(m.tv(t, 1) - m.tv(t, 0), m.tv(t, 2) - m.tv(t, 0));
    double n2 = norm(c);
    m.area[t] = 0.5 * n2;
    amax = std::max(amax, m.area[t]);
    m.normal[t] = n2 > 0 ? (1.0 / n2) * c : Vec3{0, 0, 0};
  }
  for (int64_t t = 0; t < nt; ++t)
    if (!(m.area[t] > 1e-14 * amax)) throw Error{MM_EINVAL, "degenerate triangle in mesh"};
  // edge -> list of (triangle, local vertex opposite)
  std::map<std::pair<int64_t, int64_t>, std::vector<std::pair<int64_t, int>>> edges;
  for (int64_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) {
      int64_t a = m.tri[3 * t + (i + 1) % 3], b = m.tri[3 * t + (i + 2) % 3];
      edges[{std::min(a, b), std::max(a, b)}].push_back({t, i});
    }
  m.tri_rwg.assign(3 * nt, -1);
  m.tri_sign.assign(3 * nt, 0);
  m.tri_alledge.assign(3 * nt, -1);
  m.edge_a.clear(); m.edge_b.clear(); m.tplus.clear(); m.tminus.clear();
  m.vplus.clear(); m.vminus.clear(); m.length.clear();
  int64_t all = 0;
  bool closed = true;
  for (auto& kv : edges) {
    auto& lst = kv.second;
    if (lst.size() > 2) throw Error{MM_EINVAL, "non-manifold edge in mesh"};
    for (auto& p : lst) m.tri_alledge[3 * p.first + p.second] = all;
    ++all;
    if (lst.size() != 2) {
      closed = false;
      continue;
    }
    std::sort(lst.begin(), lst.end());
    int64_t e = (int64_t)m.length.size();
    m.edge_a.push_back(kv.first.first);
    m.edge_b.push_back(kv.first.second);
    m.tplus.push_back(lst[0].first);
    m.tminus.push_back(lst[1].first);
    m.vplus.push_back(m.tri[3 * lst[0].first + lst[0].second]);
    m.vminus.push_back(m.tri[3 * lst[1].first + lst[1].second]);
    m.length.push_back(norm(m.v[kv.first.second] - m.v[kv.first.first]));
    m.tri_rwg[3 * lst[0].first + lst[0].second] = e;
    m.tri_sign[3 * lst[0].first + lst[0].second] = 1;
    m.tri_rwg[3 * lst[1].first + lst[1].second] = e;
    m.tri_sign[3 * lst[1].first + lst[1].second] = -1;
  }
  m.n_alledges = all;
  // closed and consistently outward-oriented: every edge appears in opposite
  // directions in its two triangles and the enclosed volume is positive
  if (closed) {
    for (auto& kv : edges) {
      auto& l = kv.second;
      int64_t t0 = l[0].first, t1 = l[1].first;
      int i0 = l[0].second, i1 = l[1].second;
      int64_t a0 = m.tri[3 * t0 + (i0 + 1) % 3], a1 = m.tri[3 * t1 + (i1 + 1) % 3];
      if (a0 == a1) closed = false;  // same traversal direction: inconsistent orientation
    }
    double vol = 0;
    for (int64_t t = 0; t < nt; ++t) vol += dot(m.tv(t, 0), cross(m.tv(t, 1), m.tv(t, 2))) / 6.0;
    if (!(vol > 0)) closed = false;
  }
  m.closed = closed;
}

// Barycentric refinement: primal triangle t = (p0, p1, p2) -> refined
// 6t+2i = (p_i, m_{i,i+1}, g), 6t+2i+1 = (p_i, g, m_{i+2,i}).  Refined vertex
// numbering: primal vertices, then one midpoint per edge, then one centroid per
// triangle.  Dual function of edge e (total flux l_e across g+ -> m_e -> g-,
// from the dual cell of v_s to that of v_t, v_s -> v_t being the traversal
// of e in T+): every refined triangle of the source cell emits l_e/(2 K_s), of
// the sink cell absorbs l_e/(2 K_t), the flux passed symmetrically round each
// cell (no circulation).
void build_duals(const Mesh& m, DualSet& d) {
  if (!m.closed) throw Error{MM_EINVAL, "equivalent surface must be closed and outward-oriented"};
  int64_t nv = (int64_t)m.v.size(), nt = m.nt(), ne = m.n_alledges;
  d.rv.assign(nv + ne + nt, Vec3{0, 0, 0});
  for (int64_t i = 0; i < nv; ++i) d.rv[i] = m.v[i];
  for (int64_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) {
      int64_t e = m.tri_alledge[3 * t + i];
      d.rv[nv + e] = 0.5 * (m.tv(t, (i + 1) % 3) + m.tv(t, (i + 2) % 3));
    }
  for (int64_t t = 0; t < nt; ++t) d.rv[nv + ne + t] = (1.0 / 3.0) * (m.tv(t, 0) + m.tv(t, 1) + m.tv(t, 2));
  d.rtri.resize(3 * 6 * nt);
  d.rarea.resize(6 * nt);
  d.parent.resize(6 * nt);
  for (int64_t t = 0; t < nt; ++t) {
    int64_t g = nv + ne + t;
    for (int i = 0; i < 3; ++i) {
      int j = (i + 1) % 3, k = (i + 2) % 3;
      int64_t mij = nv + m.tri_alledge[3 * t + k];  // edge (i, j) is opposite local vertex k
      int64_t mki = nv + m.tri_alledge[3 * t + j];
      int64_t r0 = 6 * t + 2 * i, r1 = r0 + 1;
      d.rtri[3 * r0] = m.tri[3 * t + i]; d.rtri[3 * r0 + 1] = mij; d.rtri[3 * r0 + 2] = g;
      d.rtri[3 * r1] = m.tri[3 * t + i]; d.rtri[3 * r1 + 1] = g; d.rtri[3 * r1 + 2] = mki;
    }
  }
  for (int64_t r = 0; r < 6 * nt; ++r) {
    d.rarea[r] = 0.5 * norm(cross(d.rvert(r, 1) - d.rvert(r, 0), d.rvert(r, 2) - d.rvert(r, 0)));
    d.parent[r] = r / 6;
  }
  // triangles around each vertex
  std::vector<std::vector<int64_t>> vt(nv);
  for (int64_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) vt[m.tri[3 * t + i]].push_back(t);
  auto local = [&](int64_t t, int64_t v) {
    for (int i = 0; i < 3; ++i)
      if (m.tri[3 * t + i] == v) return i;
    throw Error{MM_EINTERNAL, "vertex not in triangle"};
  };
  // counter-clockwise cycle of refined triangles around a vertex
  std::vector<std::vector<int64_t>> cyc(nv);
  auto cycle = [&](int64_t v) -> const std::vector<int64_t>& {
    auto& c = cyc[v];
    if (!c.empty()) return c;
    const auto& tl = vt[v];
    std::map<int64_t, int64_t> next_of;  // next vertex after v -> triangle
    for (int64_t t : tl) next_of[m.tri[3 * t + (local(t, v) + 1) % 3]] = t;
    int64_t t = tl[0];
    for (size_t s = 0; s < tl.size(); ++s) {
      int i = local(t, v);
      c.push_back(6 * t + 2 * i);
      c.push_back(6 * t + 2 * i + 1);
      int64_t prev_v = m.tri[3 * t + (i + 2) % 3];
      auto it = next_of.find(prev_v);
      if (it == next_of.end()) throw Error{MM_EINVAL, "equivalent surface vertex is not manifold"};
      t = it->second;
    }
    if (t != tl[0]) throw Error{MM_EINVAL, "equivalent surface vertex fan is not a single cycle"};
    return c;
  };
  auto opp = [&](int64_t ra, int64_t rb) {
    for (int i = 0; i < 3; ++i) {
      int64_t x = d.rtri[3 * ra + i];
      bool shared = false;
      for (int j = 0; j < 3; ++j) shared |= (d.rtri[3 * rb + j] == x);
      if (!shared) return i;
    }
    throw Error{MM_EINTERNAL, "refined triangles share no edge"};
  };
  d.n = m.nrwg();
  d.fn.clear(); d.rt.clear(); d.flux.clear();
  for (int64_t e = 0; e < d.n; ++e) {
    int64_t tp = m.tplus[e], tm = m.tminus[e];
    int ip = -1;
    for (int i = 0; i < 3; ++i) {
      int64_t a = m.tri[3 * tp + i], b = m.tri[3 * tp + (i + 1) % 3];
      if ((a == m.edge_a[e] && b == m.edge_b[e]) || (a == m.edge_b[e] && b == m.edge_a[e])) ip = i;
    }
    if (ip < 0) throw Error{MM_EINTERNAL, "edge not found in T+"};
    int64_t vs = m.tri[3 * tp + ip], vtt = m.tri[3 * tp + (ip + 1) % 3];
    double le = m.length[e];
    // sink cell around vt: from T+'s (vt, g+, m_e) clockwise to T-'s (vt, m_e, g-)
    {
      const auto& c = cycle(vtt);
      int64_t K = (int64_t)c.size() / 2, L = (int64_t)c.size();
      int it = (ip + 1) % 3;
      int64_t st = std::find(c.begin(), c.end(), 6 * tp + 2 * it + 1) - c.begin();
      std::vector<int64_t> seq(L);
      for (int64_t j = 0; j < L; ++j) seq[j] = c[((st - j) % L + L) % L];
      if (seq[L - 1] != 6 * tm + 2 * local(tm, vtt)) throw Error{MM_EINTERNAL, "dual walk mismatch (sink)"};
      std::vector<double> fl(3 * L, 0.0);
      fl[0] -= le / 2;
      fl[3 * (L - 1)] -= le / 2;
      for (int64_t j = 0; j + 1 < L; ++j) {
        double F = le * (double)(K - 1 - j) / (2.0 * K);
        fl[3 * j + opp(seq[j], seq[j + 1])] += F;
        fl[3 * (j + 1) + opp(seq[j + 1], seq[j])] -= F;
      }
      for (int64_t j = 0; j < L; ++j) {
        d.fn.push_back(e); d.rt.push_back(seq[j]);
        for (int i = 0; i < 3; ++i) d.flux.push_back(fl[3 * j + i]);
      }
    }
    // source cell around vs: from T+'s (vs, m_e, g+) counter-clockwise to T-'s (vs, g-, m_e)
    {
      const auto& c = cycle(vs);
      int64_t K = (int64_t)c.size() / 2, L = (int64_t)c.size();
      int64_t st = std::find(c.begin(), c.end(), 6 * tp + 2 * ip) - c.begin();
      std::vector<int64_t> seq(L);
      for (int64_t j = 0; j < L; ++j) seq[j] = c[(st + j) % L];
      if (seq[L - 1] != 6 * tm + 2 * local(tm, vs) + 1) throw Error{MM_EINTERNAL, "dual walk mismatch (source)"};
      std::vector<double> fl(3 * L, 0.0);
      fl[0] += le / 2;
      fl[3 * (L - 1)] += le / 2;
      for (int64_t j = 0; j + 1 < L; ++j) {
        double F = le * (double)(K - 1 - j) / (2.0 * K);
        fl[3 * j + opp(seq[j], seq[j + 1])] -= F;
        fl[3 * (j + 1) + opp(seq[j + 1], seq[j])] += F;
      }
      for (int64_t j = 0; j < L; ++j) {
        d.fn.push_back(e); d.rt.push_back(seq[j]);
        for (int i = 0; i < 3; ++i) d.flux.push_back(fl[3 * j + i]);
      }
    }
  }
}

// ---- quadrature rules --------------------------------------------------------
Rule rule_tri3() {
  Rule r;
  double a = 2.0 / 3.0, b = 1.0 / 6.0;
  r.b0 = {a, b, b}; r.b1 = {b, a, b}; r.b2 = {b, b, a};
  r.w = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};
  return r;
}

// Radon's degree-5 formula: centroid (9/40) and two orbits a = (6 -+ sqrt 15)/21
// with weights (155 -+ sqrt 15)/1200.
Rule rule_tri7() {
  Rule r;
  double s = std::sqrt(15.0);
  r.b0.push_back(1.0 / 3.0); r.b1.push_back(1.0 / 3.0); r.b2.push_back(1.0 / 3.0); r.w.push_back(9.0 / 40.0);
  double as[2] = {(6.0 - s) / 21.0, (6.0 + s) / 21.0};
  double ws[2] = {(155.0 - s) / 1200.0, (155.0 + s) / 1200.0};
  for (int o = 0; o < 2; ++o) {
    double a = as[o], c = 1.0 - 2.0 * a;
    double pts[3][3] = {{a, a, c}, {a, c, a}, {c, a, a}};
    for (int p = 0; p < 3; ++p) {
      r.b0.push_back(pts[p][0]); r.b1.push_back(pts[p][1]); r.b2.push_back(pts[p][2]); r.w.push_back(ws[o]);
    }
  }
  return r;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0); w.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1; p1 = p2;
      }
      double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
      double dp = n * (z * pn - pm) / (z * z - 1);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1; p1 = p2;
    }
    double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
    double dp = n * (z * pn - pm) / (z * z - 1);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1 - z * z) * dp * dp);
  }
}

// Degree-`degree` rule: Gauss-Legendre product on [0,1]^2 through the
// collapsed map x = u, y = v (1 - u) with Jacobian (1 - u).
Rule rule_collapsed(int degree) {
  int nu = (degree + 3) / 2, nv = (degree + 2) / 2;
  std::vector<double> xu, wu, xv, wv;
  gauss_legendre(nu, xu, wu);
  gauss_legendre(nv, xv, wv);
  Rule r;
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nv; ++j) {
      double u = 0.5 * (xu[i] + 1.0), v = 0.5 * (xv[j] + 1.0);
      double x = u, y = v * (1.0 - u);
      r.b0.push_back(1.0 - x - y); r.b1.push_back(x); r.b2.push_back(y);
      r.w.push_back(2.0 * (0.5 * wu[i]) * (0.5 * wv[j]) * (1.0 - u));
    }
  return r;
}

}  // namespace mm
