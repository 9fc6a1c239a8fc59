// AIM set-up on the host, FP64 (Sec. V): grid, anchors, projection weights,
// Green's spectrum of the zero-padded grid, precorrected near-field matrix.
//
// Readings of points the paper leaves open:
//  - grid nodes at phase + h*Z^3; a basis' anchor is the node nearest to the
//    area-weighted centroid of its support (round half up) for an odd number
//    of stencil points per axis, the floor for an even number; centroids within
//    1e-9 cell of a rounding tie are rejected;
//  - stencil = anchor + {-N_O/2..N_O/2}^3 (odd) or {-(N_O-1)/2..(N_O+1)/2}^3;
//  - projection weights Pi_{n,psi}[s] = int f_{n,psi} W_s (psi = x, y, z) and
//    Pi_{n,phi}[s] = int div f_n W_s, W_s the tensor Lagrange polynomial of
//    stencil node s (moment matching up to degree N_O per axis), integrated
//    exactly (degree 3 N_O + 1); interpolation is the transpose;
//  - H[u, u'] = G(r_u - r_u'), G(0) := 0, applied as a linear convolution by a
//    zero-padded FFT (each axis padded to an 11-smooth length >= 2N - 1);
//  - near pairs: Chebyshev distance of anchors <= N_NF cells; entry = exact
//    Galerkin G^(E^,J^) minus its grid approximation (precorrection).
// Elements must sit on the grid lattice, so that identical elements share
// weights and (type, type, lattice offset) near-field blocks.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <unordered_map>

#include "aim_setup.h"
#include "fill_gpu.h"

namespace mm {

// ---- host FFT ----------------------------------------------------------------
static int64_t smallest_factor(int64_t n) {
  for (int64_t p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

// Recursive mixed-radix decimation in time: out[k] = sum_j in[j s] W^{jk}.
static void dft_rec(const cd* in, int64_t s, cd* out, int64_t n, int sign, std::vector<cd>& tmp) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  int64_t p = smallest_factor(n), m = n / p;
  for (int64_t q = 0; q < p; ++q) dft_rec(in + q * s, s * p, out + q * m, m, sign, tmp);
  tmp.resize(std::max<size_t>(tmp.size(), (size_t)n));
  std::vector<cd> t(n);
  const double th = sign * 2.0 * M_PI / (double)n;
  for (int64_t kk = 0; kk < m; ++kk)
    for (int64_t r = 0; r < p; ++r) {
      int64_t k = kk + r * m;
      cd acc(0, 0);
      for (int64_t q = 0; q < p; ++q) {
        int64_t e = (q * k) % n;
        acc += out[q * m + kk] * cd(std::cos(th * e), std::sin(th * e));
      }
      t[k] = acc;
    }
  for (int64_t k = 0; k < n; ++k) out[k] = t[k];
}

void fft_inplace(std::vector<cd>& a, int64_t n, int64_t stride, int64_t count, int64_t dist, int sign) {
  std::vector<cd> in(n), out(n), tmp;
  for (int64_t c = 0; c < count; ++c) {
    for (int64_t i = 0; i < n; ++i) in[i] = a[c * dist + i * stride];
    dft_rec(in.data(), 1, out.data(), n, sign, tmp);
    for (int64_t i = 0; i < n; ++i) a[c * dist + i * stride] = out[i];
  }
}

bool fft_length_ok(int64_t n) {
  if (n < 1) return false;
  for (int64_t p : {2, 3, 5, 7, 11})
    while (n % p == 0) n /= p;
  return n == 1;
}

int64_t fft_good_length(int64_t n) {
  int64_t m = std::max<int64_t>(n, 1);
  while (!fft_length_ok(m)) ++m;
  return m;
}

// Padded length of the x and y transforms: the 11-smooth length in [n, 2n]
// with the lowest modelled instruction count of the device's complex64 line
// FFT, L times a per-point cost.  Lines of 32 RR points (RR <= kRegFftMax) run
// in registers: five shuffle butterfly levels plus the RR-point lane DFT,
// modelled as 50 + 1.5 RR per point.  Other lengths take Stockham stages in
// shared memory at about 40 per point and stage, scaled by the radix (4 first,
// then 2, 3, 5, 7, 11).  The weights are rough per-point instruction
// counts of the two forms.
int64_t fft_fast_length(int64_t n) {
  n = std::max<int64_t>(n, 1);
  int64_t best = fft_good_length(n);
  double best_cost = 1e300;
  for (int64_t L = n; L <= 2 * n; ++L) {
    if (!fft_length_ok(L)) continue;
    double per_point;
    if (L % 32 == 0 && L / 32 <= kRegFftMax) {
      per_point = 50.0 + 1.5 * (double)(L / 32);
    } else {
      int64_t m = L;
      double w = 0;
      for (int r : {4, 2, 3, 5, 7, 11}) {
        const double wr = r == 4 ? 1.0 : r == 2 ? 0.8 : r == 3 ? 1.1 : r == 5 ? 1.5 : r == 7 ? 2.0 : 3.0;
        while (m % r == 0) {
          m /= r;
          w += wr;
        }
      }
      per_point = 40.0 * w;
    }
    const double cost = (double)L * per_point;
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = L;
    }
  }
  return best;
}

// ---- stencils and weights ------------------------------------------------------
std::vector<int> stencil_1d(int order) {
  int n = order + 1;
  int lo = (n % 2 == 1) ? -(order / 2) : -((n / 2) - 1);
  std::vector<int> o(n);
  for (int i = 0; i < n; ++i) o[i] = lo + i;
  return o;
}

static inline double lagrange(double s, const std::vector<int>& nodes, int a) {
  double v = 1.0;
  for (size_t b = 0; b < nodes.size(); ++b)
    if ((int)b != a) v *= (s - nodes[b]) / (double)(nodes[a] - nodes[b]);
  return v;
}

// Anchors and weights of one type, with the element placed at `pos`.
void type_aim(const Mesh& eq, Vec3 pos, const AimOpts& o, TypeAim& ta) {
  int64_t N = eq.nrwg();
  auto o1 = stencil_1d(o.order);
  int n1 = (int)o1.size();
  int S = n1 * n1 * n1;
  ta.Nh = N;
  ta.S = S;
  ta.anc.assign(3 * N, 0);
  ta.Pi.assign(N * S * 4, 0.0);
  bool odd = (n1 % 2) == 1;
  double ph[3] = {o.phase.x, o.phase.y, o.phase.z};
  for (int64_t n = 0; n < N; ++n) {
    int64_t tp = eq.tplus[n], tm = eq.tminus[n];
    Vec3 gp = (1.0 / 3.0) * (eq.tv(tp, 0) + eq.tv(tp, 1) + eq.tv(tp, 2));
    Vec3 gm = (1.0 / 3.0) * (eq.tv(tm, 0) + eq.tv(tm, 1) + eq.tv(tm, 2));
    double ap = eq.area[tp], am = eq.area[tm];
    Vec3 c = (1.0 / (ap + am)) * (ap * gp + am * gm);
    c = c + pos;
    double cc[3] = {c.x, c.y, c.z};
    for (int a = 0; a < 3; ++a) {
      double s = (cc[a] - ph[a]) / o.h;
      double fr = s - std::floor(s);
      if (odd) {
        if (std::fabs(fr - 0.5) < 1e-9)
          throw Error{MM_EINVAL, "a basis centroid lies on a rounding tie of the AIM grid; shift the grid phase"};
        ta.anc[3 * n + a] = (int64_t)std::floor(s + 0.5);
      } else {
        if (std::min(fr, 1.0 - fr) < 1e-9)
          throw Error{MM_EINVAL, "a basis centroid lies on an AIM grid plane; shift the grid phase"};
        ta.anc[3 * n + a] = (int64_t)std::floor(s);
      }
    }
  }
  Rule q = rule_collapsed(3 * o.order + 1);
  for (int64_t n = 0; n < N; ++n) {
    for (int side = 0; side < 2; ++side) {
      int64_t t = side == 0 ? eq.tplus[n] : eq.tminus[n];
      int64_t fv = side == 0 ? eq.vplus[n] : eq.vminus[n];
      double sg = side == 0 ? 1.0 : -1.0;
      double A = eq.area[t];
      Vec3 v[3] = {eq.tv(t, 0), eq.tv(t, 1), eq.tv(t, 2)};
      double div = sg * eq.length[n] / A;
      for (int p = 0; p < q.n(); ++p) {
        Vec3 r = q.b0[p] * v[0] + q.b1[p] * v[1] + q.b2[p] * v[2];
        Vec3 f = (sg * eq.length[n] / (2.0 * A)) * (r - eq.v[fv]);
        Vec3 rr = r + pos;
        double loc[3] = {(rr.x - ph[0]) / o.h - ta.anc[3 * n], (rr.y - ph[1]) / o.h - ta.anc[3 * n + 1],
                         (rr.z - ph[2]) / o.h - ta.anc[3 * n + 2]};
        double Lx[16], Ly[16], Lz[16];
        for (int a = 0; a < n1; ++a) {
          Lx[a] = lagrange(loc[0], o1, a);
          Ly[a] = lagrange(loc[1], o1, a);
          Lz[a] = lagrange(loc[2], o1, a);
        }
        double wA = q.w[p] * A;
        for (int iz = 0; iz < n1; ++iz)
          for (int iy = 0; iy < n1; ++iy)
            for (int ix = 0; ix < n1; ++ix) {
              int s = (iz * n1 + iy) * n1 + ix;
              double W = Lz[iz] * Ly[iy] * Lx[ix] * wA;
              double* P = &ta.Pi[(n * S + s) * 4];
              P[0] += W * f.x;
              P[1] += W * f.y;
              P[2] += W * f.z;
              P[3] += W * div;
            }
      }
    }
  }
  // stencil bounding box of the type (in reference anchor coordinates)
  for (int a = 0; a < 3; ++a) {
    int64_t lo = INT64_MAX, hi = INT64_MIN;
    for (int64_t n = 0; n < N; ++n) {
      lo = std::min(lo, ta.anc[3 * n + a] + o1.front());
      hi = std::max(hi, ta.anc[3 * n + a] + o1.back());
    }
    ta.box_lo[a] = lo;
    ta.box_dim[a] = hi - lo + 1;
  }
}

// Process-wide cache of Green's spectra (bounded number of entries).
struct GhatKey {
  int64_t n[6];
  double h, k;
  bool operator<(const GhatKey& o) const {
    for (int i = 0; i < 6; ++i)
      if (n[i] != o.n[i]) return n[i] < o.n[i];
    if (h != o.h) return h < o.h;
    return k < o.k;
  }
};
static std::mutex g_ghat_mu;
static std::map<GhatKey, std::shared_ptr<const std::vector<cd>>> g_ghat;
constexpr size_t kGhatCacheEntries = 32;

static bool ghat_cache_get(const GhatKey& key, std::vector<cd>& out) {
  std::shared_ptr<const std::vector<cd>> v;
  {
    std::lock_guard<std::mutex> lk(g_ghat_mu);
    auto it = g_ghat.find(key);
    if (it == g_ghat.end()) return false;
    v = it->second;
  }
  out = *v;
  return true;
}

static void ghat_cache_put(const GhatKey& key, const std::vector<cd>& v) {
  auto p = std::make_shared<const std::vector<cd>>(v);
  std::lock_guard<std::mutex> lk(g_ghat_mu);
  if (g_ghat.size() >= kGhatCacheEntries) g_ghat.erase(g_ghat.begin());
  g_ghat[key] = std::move(p);
}

static inline cd green(double R, double k) {
  return std::exp(cd(0.0, -k * R)) / (4.0 * M_PI * R);
}

// Grid-approximation entry c_A sum_{xyz} Pi_m H Pi_n + c_phi Pi_m,phi H Pi_n,phi for anchor
// difference da = a_m - a_n, using the offset table Htab over [-R, R]^3.
struct HTable {
  int R = 0;
  std::vector<cd> v;
  cd at(int64_t dx, int64_t dy, int64_t dz) const {
    int w = 2 * R + 1;
    return v[((dx + R) * w + (dy + R)) * w + (dz + R)];
  }
};

void build_array_host(ArrayHost& ah, const std::vector<const TypeModel*>& types, const std::vector<int32_t>& type_of,
                      const std::vector<Vec3>& offsets, const AimOpts& o, const EM& em) {
  int64_t ne = (int64_t)type_of.size();
  int64_t nty = (int64_t)types.size();
  if (ne < 1) throw Error{MM_EINVAL, "array has no elements"};
  if (!(o.h > 0) || o.order < 1 || o.order > 8 || o.n_nf < -1) throw Error{MM_EINVAL, "invalid AIM options"};
  ah.opts = o;
  ah.type_of = type_of;
  ah.n_elem = ne;
  ah.off.assign(ne + 1, 0);
  for (int64_t e = 0; e < ne; ++e) ah.off[e + 1] = ah.off[e] + types[type_of[e]]->Nh;
  ah.N = ah.off[ne];
  ah.c_A = cd(0.0, -em.k * em.eta0);
  ah.c_phi = cd(0.0, em.eta0 / em.k);
  // lattice positions relative to element 0
  Vec3 o0 = offsets[0];
  ah.L.assign(3 * ne, 0);
  for (int64_t e = 0; e < ne; ++e) {
    double d[3] = {(offsets[e].x - o0.x) / o.h, (offsets[e].y - o0.y) / o.h, (offsets[e].z - o0.z) / o.h};
    for (int a = 0; a < 3; ++a) {
      double r = std::nearbyint(d[a]);
      if (std::fabs(d[a] - r) > 1e-9 * std::max(1.0, std::fabs(d[a])))
        throw Error{MM_EINVAL, "element offsets must differ by integer multiples of the AIM grid spacing"};
      ah.L[3 * e + a] = (int64_t)r;
    }
  }
  // per-type anchors and weights at the reference position o0
  ah.tai.resize(nty);
  for (int64_t t = 0; t < nty; ++t) type_aim(types[t]->eq, o0, o, ah.tai[t]);
  const int S = ah.tai[0].S;
  auto o1 = stencil_1d(o.order);
  // global grid
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) { lo[a] = INT64_MAX; hi[a] = INT64_MIN; }
  for (int64_t e = 0; e < ne; ++e) {
    const TypeAim& ta = ah.tai[type_of[e]];
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], ta.box_lo[a] + ah.L[3 * e + a]);
      hi[a] = std::max(hi[a], ta.box_lo[a] + ta.box_dim[a] - 1 + ah.L[3 * e + a]);
    }
  }
  for (int a = 0; a < 3; ++a) {
    ah.grid[a] = hi[a] - lo[a] + 1;
    ah.fft[a] = a < 2 ? fft_fast_length(2 * ah.grid[a] - 1) : fft_good_length(2 * ah.grid[a] - 1);
    ah.lo[a] = lo[a];
  }
  ah.base.assign(3 * ne, 0);
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a) ah.base[3 * e + a] = ah.L[3 * e + a] - lo[a];
  // Green's spectrum: circulant embedding of H on the padded grid, FFT, / (Px Py Pz).
  // It depends only on the grid and padded sizes, h and k: spectra are kept in a
  // process-wide cache (arrays of equal grid size share one computation).
  const GhatKey gkey{{ah.grid[0], ah.grid[1], ah.grid[2], ah.fft[0], ah.fft[1], ah.fft[2]}, o.h, em.k};
  if (ghat_cache_get(gkey, ah.Ghat)) {
    // cached
  } else {
    int64_t Px = ah.fft[0], Py = ah.fft[1], Pz = ah.fft[2];
    int64_t Nx = ah.grid[0], Ny = ah.grid[1], Nz = ah.grid[2];
    std::vector<cd> K(Px * Py * Pz, cd(0, 0));
    auto wrap = [](int64_t i, int64_t N, int64_t P, bool& used) -> int64_t {
      if (i < N) { used = true; return i; }
      if (i > P - N) { used = true; return i - P; }
      used = false;
      return 0;
    };
    for (int64_t i = 0; i < Px; ++i)
      for (int64_t j = 0; j < Py; ++j)
        for (int64_t l = 0; l < Pz; ++l) {
          bool ux, uy, uz;
          int64_t dx = wrap(i, Nx, Px, ux), dy = wrap(j, Ny, Py, uy), dz = wrap(l, Nz, Pz, uz);
          if (!(ux && uy && uz)) continue;
          if (dx == 0 && dy == 0 && dz == 0) continue;
          double R = o.h * std::sqrt((double)(dx * dx + dy * dy + dz * dz));
          K[(i * Py + j) * Pz + l] = green(R, em.k);
        }
    // 3D FFT (forward, exp(-i...)): along z, y, x
    parallel_for(Px, em.nthreads, [&](int64_t a, int64_t b) {
      for (int64_t i = a; i < b; ++i) {
        std::vector<cd> slab(K.begin() + i * Py * Pz, K.begin() + (i + 1) * Py * Pz);
        fft_inplace(slab, Pz, 1, Py, Pz, -1);
        fft_inplace(slab, Py, Pz, Pz, 1, -1);
        std::copy(slab.begin(), slab.end(), K.begin() + i * Py * Pz);
      }
    });
    parallel_for(Py * Pz, em.nthreads, [&](int64_t a, int64_t b) {
      std::vector<cd> line(Px);
      for (int64_t c = a; c < b; ++c) {
        for (int64_t i = 0; i < Px; ++i) line[i] = K[i * Py * Pz + c];
        fft_inplace(line, Px, 1, 1, Px, -1);
        for (int64_t i = 0; i < Px; ++i) K[i * Py * Pz + c] = line[i];
      }
    });
    double inv = 1.0 / (double)(Px * Py * Pz);
    for (auto& x : K) x *= inv;
    ah.Ghat = std::move(K);
    ghat_cache_put(gkey, ah.Ghat);
  }
  // near field: blocks per (type, type, lattice offset)
  const int nnf = o.n_nf;   // -1: no near-field correction
  int64_t ext[3] = {0, 0, 0};
  for (int64_t t = 0; t < nty; ++t)
    for (int a = 0; a < 3; ++a) ext[a] = std::max(ext[a], ah.tai[t].box_dim[a]);
  struct KeyHash {
    size_t operator()(const std::array<int64_t, 3>& k) const {
      return (size_t)(k[0] * 73856093LL) ^ (size_t)(k[1] * 19349663LL) ^ (size_t)(k[2] * 83492791LL);
    }
  };
  std::unordered_map<std::array<int64_t, 3>, int64_t, KeyHash> at;
  for (int64_t e = 0; e < ne; ++e) {
    std::array<int64_t, 3> key{ah.L[3 * e], ah.L[3 * e + 1], ah.L[3 * e + 2]};
    if (at.count(key)) throw Error{MM_EINVAL, "two elements at the same position"};
    at[key] = e;
  }
  int64_t Rs[3];
  for (int a = 0; a < 3; ++a) Rs[a] = ext[a] + nnf;
  // offset table for the grid part: |a_m - a_n| <= nnf, stencil offsets <= order
  HTable H;
  H.R = std::max(nnf, 0) + o1.back() - o1.front();
  {
    int w = 2 * H.R + 1;
    H.v.assign((size_t)w * w * w, cd(0, 0));
    for (int dx = -H.R; dx <= H.R; ++dx)
      for (int dy = -H.R; dy <= H.R; ++dy)
        for (int dz = -H.R; dz <= H.R; ++dz) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          H.v[((dx + H.R) * w + (dy + H.R)) * w + (dz + H.R)] =
              green(o.h * std::sqrt((double)(dx * dx + dy * dy + dz * dz)), em.k);
        }
  }
  std::vector<std::array<int, 3>> so(S);
  {
    int n1 = (int)o1.size();
    for (int iz = 0; iz < n1; ++iz)
      for (int iy = 0; iy < n1; ++iy)
        for (int ix = 0; ix < n1; ++ix) so[(iz * n1 + iy) * n1 + ix] = {o1[ix], o1[iy], o1[iz]};
  }
  // distinct blocks: key (ta, tb, dL) with dL = L_b - L_a
  struct Block {
    std::vector<int64_t> ptr;   // Nh_a + 1
    std::vector<int32_t> col;   // local columns
    std::vector<cd> val;
  };
  std::map<std::array<int64_t, 5>, int64_t> block_index;
  std::vector<Block> blocks;
  std::vector<std::array<int64_t, 5>> block_keys;
  std::vector<Vec3> block_rel;
  // neighbour lists per element: (neighbour element, block id), ascending neighbour
  std::vector<std::vector<std::pair<int64_t, int64_t>>> nbr(ne);
  for (int64_t e = 0; e < ne; ++e) {
    for (int64_t dx = -Rs[0]; dx <= Rs[0]; ++dx)
      for (int64_t dy = -Rs[1]; dy <= Rs[1]; ++dy)
        for (int64_t dz = -Rs[2]; dz <= Rs[2]; ++dz) {
          auto it = at.find({ah.L[3 * e] + dx, ah.L[3 * e + 1] + dy, ah.L[3 * e + 2] + dz});
          if (it == at.end()) continue;
          int64_t f = it->second;
          const TypeAim &A = ah.tai[type_of[e]], &B = ah.tai[type_of[f]];
          // bounding-box test on anchors (conservative)
          bool cand = true;
          int64_t d3[3] = {dx, dy, dz};
          for (int a = 0; a < 3; ++a) {
            int64_t alo = A.box_lo[a] - o1.front(), ahi = A.box_lo[a] + A.box_dim[a] - 1 - o1.back();
            int64_t blo = B.box_lo[a] - o1.front() + d3[a], bhi = B.box_lo[a] + B.box_dim[a] - 1 - o1.back() + d3[a];
            if (blo - ahi > nnf || alo - bhi > nnf) cand = false;
          }
          if (!cand) continue;
          std::array<int64_t, 5> key{type_of[e], type_of[f], dx, dy, dz};
          auto bi = block_index.find(key);
          int64_t id;
          if (bi == block_index.end()) {
            id = (int64_t)blocks.size();
            block_index[key] = id;
            blocks.emplace_back();
            block_keys.push_back(key);
            block_rel.push_back(offsets[f] - offsets[e]);
          } else {
            id = bi->second;
          }
          nbr[e].push_back({f, id});
        }
    std::sort(nbr[e].begin(), nbr[e].end());
  }
  // fill each distinct block: exact Galerkin entries minus the grid part, near
  // pairs only; a block computed by an earlier array with the same types and
  // AIM options is taken from the row type's cache.  Patterns first (host);
  // the values on the GPU for device contexts (fill_gpu.cu), else on the host.
  auto cache_key = [&](size_t id) {
    const auto& key = block_keys[id];
    const TypeModel* tb = types[key[1]];
    return NearBlockKey{tb, {key[2], key[3], key[4]}, o.h, {o.phase.x, o.phase.y, o.phase.z}, o.order, o.n_nf};
  };
  std::vector<size_t> todo;
  for (size_t id = 0; id < blocks.size(); ++id) {
    auto key = block_keys[id];
    const TypeModel* ta = types[key[0]];
    const TypeAim &A = ah.tai[key[0]], &B = ah.tai[key[1]];
    int64_t Na = ta->Nh, Nb = types[key[1]]->Nh;
    int64_t dL[3] = {key[2], key[3], key[4]};
    Block& blk = blocks[id];
    const NearBlockKey ck = cache_key(id);
    {
      std::lock_guard<std::mutex> lk(ta->nf_mu);
      auto it = ta->nf_cache.find(ck);
      if (it != ta->nf_cache.end()) {
        blk.ptr = it->second->ptr;
        blk.col = it->second->col;
        blk.val = it->second->val;
        continue;
      }
    }
    blk.ptr.assign(Na + 1, 0);
    std::vector<int32_t> cols;
    for (int64_t m = 0; m < Na; ++m) {
      for (int64_t n = 0; n < Nb; ++n) {
        int64_t cheb = 0;
        for (int a = 0; a < 3; ++a)
          cheb = std::max<int64_t>(cheb, std::llabs(A.anc[3 * m + a] - (B.anc[3 * n + a] + dL[a])));
        if (cheb <= nnf) cols.push_back((int32_t)n);
      }
      blk.ptr[m + 1] = (int64_t)cols.size();
    }
    if (cols.empty()) {   // no near pairs: remembered as an empty block
      blk.ptr.clear();
      std::lock_guard<std::mutex> lk(ta->nf_mu);
      ta->nf_cache.emplace(ck, std::make_shared<NearBlockData>());
      continue;
    }
    blk.col = std::move(cols);
    todo.push_back(id);
  }
  std::vector<char> done(blocks.size(), 0);
  if (o.device >= 0 && !todo.empty()) {
    std::vector<NearFillJob> jobs;
    for (size_t id : todo) {
      const auto& key = block_keys[id];
      NearFillJob jb;
      jb.ma = &types[key[0]]->eq;
      jb.mb = &types[key[1]]->eq;
      jb.rel = block_rel[id];
      jb.A = &ah.tai[key[0]];
      jb.B = &ah.tai[key[1]];
      for (int a = 0; a < 3; ++a) jb.dL[a] = key[2 + a];
      jb.ptr = &blocks[id].ptr;
      jb.col = &blocks[id].col;
      jb.val = &blocks[id].val;
      jobs.push_back(jb);
    }
    std::string msg;
    if (fill_near_blocks_gpu(jobs, H.v, H.R, so, ah.c_A, ah.c_phi, em.k, o.device, msg))
      for (size_t id : todo) done[id] = 1;
  }
  for (size_t id : todo) {
    if (done[id]) continue;
    auto key = block_keys[id];
    const TypeModel* ta = types[key[0]];
    const TypeModel* tb = types[key[1]];
    const TypeAim &A = ah.tai[key[0]], &B = ah.tai[key[1]];
    int64_t Na = ta->Nh, Nb = tb->Nh;
    int64_t dL[3] = {key[2], key[3], key[4]};
    Block& blk = blocks[id];
    std::vector<cd> G;
    fill_efie(ta->eq, tb->eq, block_rel[id], em, G);
    for (auto& x : G) x *= ah.c_A;   // G^(E^,J^) = -j w mu0 Lmat
    blk.val.resize(blk.ptr[Na]);
    parallel_for(Na, em.nthreads, [&](int64_t m0, int64_t m1) {
      for (int64_t m = m0; m < m1; ++m) {
        for (int64_t p = blk.ptr[m]; p < blk.ptr[m + 1]; ++p) {
          const int32_t n = blk.col[p];
          int64_t da[3];
          for (int a = 0; a < 3; ++a) da[a] = A.anc[3 * m + a] - (B.anc[3 * n + a] + dL[a]);
          cd vA(0, 0), vP(0, 0);
          const double* Pm = &A.Pi[(size_t)m * S * 4];
          const double* Pn = &B.Pi[(size_t)n * S * 4];
          for (int s = 0; s < S; ++s) {
            cd hx(0, 0), hy(0, 0), hz(0, 0), hp(0, 0);
            for (int t = 0; t < S; ++t) {
              cd h = H.at(da[0] + so[s][0] - so[t][0], da[1] + so[s][1] - so[t][1], da[2] + so[s][2] - so[t][2]);
              hx += h * Pn[4 * t]; hy += h * Pn[4 * t + 1]; hz += h * Pn[4 * t + 2]; hp += h * Pn[4 * t + 3];
            }
            vA += Pm[4 * s] * hx + Pm[4 * s + 1] * hy + Pm[4 * s + 2] * hz;
            vP += Pm[4 * s + 3] * hp;
          }
          blk.val[p] = G[m * Nb + n] - (ah.c_A * vA + ah.c_phi * vP);
        }
      }
    });
  }
  for (size_t id : todo) {
    const TypeModel* ta = types[block_keys[id][0]];
    auto d = std::make_shared<NearBlockData>();
    d->ptr = blocks[id].ptr;
    d->col = blocks[id].col;
    d->val = blocks[id].val;
    std::lock_guard<std::mutex> lk(ta->nf_mu);
    ta->nf_cache.emplace(cache_key(id), std::move(d));
  }
  ah.nnz_near = 0;
  for (int64_t e = 0; e < ne; ++e)
    for (auto& pr : nbr[e])
      if (!blocks[pr.second].ptr.empty()) ah.nnz_near += blocks[pr.second].ptr.back();
  if (o.csr_max_nnz >= 0 && ah.nnz_near > o.csr_max_nnz) {
    ah.rowptr.clear();
    ah.col.clear();
    ah.val.clear();
  } else {
  // assemble the global CSR, rows element-major, columns ascending
  ah.rowptr.assign(ah.N + 1, 0);
  for (int64_t e = 0; e < ne; ++e) {
    int64_t Na = types[type_of[e]]->Nh;
    for (int64_t m = 0; m < Na; ++m) {
      int64_t c = 0;
      for (auto& pr : nbr[e]) {
        const Block& b = blocks[pr.second];
        if (b.ptr.empty()) continue;
        c += b.ptr[m + 1] - b.ptr[m];
      }
      ah.rowptr[ah.off[e] + m + 1] = c;
    }
  }
  for (int64_t i = 0; i < ah.N; ++i) ah.rowptr[i + 1] += ah.rowptr[i];
  int64_t nnz = ah.rowptr[ah.N];
  ah.col.resize(nnz);
  ah.val.resize(nnz);
  parallel_for(ne, em.nthreads, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      int64_t Na = types[type_of[e]]->Nh;
      for (int64_t m = 0; m < Na; ++m) {
        int64_t p = ah.rowptr[ah.off[e] + m];
        for (auto& pr : nbr[e]) {
          const Block& b = blocks[pr.second];
          if (b.ptr.empty()) continue;
          for (int64_t q = b.ptr[m]; q < b.ptr[m + 1]; ++q) {
            ah.col[p] = (int32_t)(ah.off[pr.first] + b.col[q]);
            ah.val[p] = b.val[q];
            ++p;
          }
        }
      }
    }
  });
  }
  ah.n_blocks = (int64_t)blocks.size();
  ah.nf_blocks.resize(blocks.size());
  for (size_t id = 0; id < blocks.size(); ++id) {
    auto& d = ah.nf_blocks[id];
    const auto& key = block_keys[id];
    d.ta = (int32_t)key[0];
    d.tb = (int32_t)key[1];
    for (int a = 0; a < 3; ++a) d.dL[a] = key[2 + a];
    d.Na = types[key[0]]->Nh;
    d.Nb = types[key[1]]->Nh;
    d.ptr = std::move(blocks[id].ptr);
    d.col = std::move(blocks[id].col);
    d.val = std::move(blocks[id].val);
  }
  ah.nf_nbr = std::move(nbr);
}

}  // namespace mm
