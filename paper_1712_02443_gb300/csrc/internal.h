// Internal data structures of libmacroaim (host side).
#pragma once

#include <complex>
#include <cstdint>
#include <functional>
#include <string>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "fft_plan.h"
#include "macroaim.h"

namespace mm {

using cd = std::complex<double>;

struct Vec3 {
  double x, y, z;
};
inline Vec3 operator+(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline Vec3 operator-(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline Vec3 operator*(double s, Vec3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline Vec3 cross(Vec3 a, Vec3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(Vec3 a) { return std::sqrt(dot(a, a)); }

struct CVec3 {
  cd x, y, z;
};
inline CVec3 ccross(CVec3 a, Vec3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline cd cdot(Vec3 a, CVec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Error carrier used inside the library; converted to mm_status at the ABI.
struct Error {
  mm_status code;
  std::string msg;
};

// ---- mesh and RWG functions (Sec. II-A) ----------------------------------
struct Mesh {
  std::vector<Vec3> v;
  std::vector<int32_t> tri;          // 3 per triangle
  std::vector<double> area;
  std::vector<Vec3> normal;          // unit, from vertex order
  // RWG on interior edges, lexicographic (min, max) order
  std::vector<int64_t> edge_a, edge_b;
  std::vector<int64_t> tplus, tminus, vplus, vminus;
  std::vector<double> length;
  std::vector<int64_t> tri_rwg;      // 3 per triangle: RWG of the edge opposite local vertex i, -1 if none
  std::vector<int32_t> tri_sign;     // 3 per triangle: +1 T+, -1 T-, 0 none
  std::vector<int64_t> tri_alledge;  // 3 per triangle: index among all edges (boundary included)
  int64_t n_alledges = 0;
  bool closed = false;
  int64_t nt() const { return (int64_t)tri.size() / 3; }
  int64_t nrwg() const { return (int64_t)length.size(); }
  Vec3 tv(int64_t t, int i) const { return v[tri[3 * t + i]]; }
};

// Builds RWG data and validates; throws Error.
void build_mesh(Mesh& m, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt);

// Barycentric refinement and Buffa-Christiansen duals on a closed mesh.
struct DualSet {
  std::vector<Vec3> rv;        // refined vertices
  std::vector<int64_t> rtri;   // 3 per refined triangle
  std::vector<double> rarea;
  std::vector<int64_t> parent; // primal triangle of each refined triangle
  // support entries: function fn[e] on refined triangle rt[e] with outward fluxes flux[3e+i]
  std::vector<int64_t> fn, rt;
  std::vector<double> flux;
  int64_t n = 0;
  Vec3 rvert(int64_t r, int i) const { return rv[rtri[3 * r + i]]; }
};
void build_duals(const Mesh& m, DualSet& d);

// ---- quadrature ------------------------------------------------------------
struct Rule {
  std::vector<double> b0, b1, b2, w;  // barycentric coordinates, weights summing to 1
  int n() const { return (int)w.size(); }
};
Rule rule_tri3();
Rule rule_tri7();
Rule rule_collapsed(int degree);

// ---- threading -------------------------------------------------------------
void parallel_for(int64_t n, int nthreads, const std::function<void(int64_t, int64_t)>& body);

// ---- fills (Sec. II-IV) ----------------------------------------------------
struct EM {
  double k;
  double eta0;
  int nthreads;
};
// Lmat[m, n] (row-major test x source) between RWG sets, translated source by `shift`.
void fill_efie(const Mesh& test, const Mesh& src, Vec3 shift, const EM& em, std::vector<cd>& out);
// Kmat_PV[m, n] = <f_m, K g_n> (principal value), g = duals of the closed mesh.
void fill_k(const Mesh& test, const Mesh& eq, const DualSet& d, const EM& em, std::vector<cd>& out);
// D[m, n] = <f^_m, n_in x g_n>.
void fill_dual_gram(const Mesh& eq, const DualSet& d, std::vector<double>& out);

// Dense complex LU with partial pivoting (row-major, in place); throws on singular.
struct LU {
  int64_t n = 0;
  std::vector<cd> a;
  std::vector<int64_t> piv;
};
void lu_factor(LU& lu, std::vector<cd> a, int64_t n);
// Solves A X = B in place for B (n x ncols, row-major).
void lu_solve(const LU& lu, std::vector<cd>& b, int64_t ncols, int nthreads);

// A near-field block of a row type against a column type at one lattice
// offset (sparse rows, local columns): exact Galerkin entries minus the grid
// part over the near pairs.
struct NearBlockData {
  std::vector<int64_t> ptr;   // rows + 1 (empty: no near pairs)
  std::vector<int32_t> col;
  std::vector<cd> val;
};
// Key of a cached block: column type, lattice offset, AIM options.
struct NearBlockKey {
  const void* col_type;
  int64_t dL[3];
  double h, phase[3];
  int order, n_nf;
  bool operator<(const NearBlockKey& o) const {
    if (col_type != o.col_type) return col_type < o.col_type;
    for (int a = 0; a < 3; ++a)
      if (dL[a] != o.dL[a]) return dL[a] < o.dL[a];
    if (h != o.h) return h < o.h;
    for (int a = 0; a < 3; ++a)
      if (phase[a] != o.phase[a]) return phase[a] < o.phase[a];
    if (order != o.order) return order < o.order;
    return n_nf < o.n_nf;
  }
};

struct TypeModel {
  Mesh scat, eq;
  DualSet duals;
  EM em;
  int64_t N = 0, Nh = 0;
  std::vector<cd> M, D, T, A, B, GHH, GHE;   // row-major
  std::vector<cd> JE;                         // -A^-1 B (N x N^): scatterer currents from E^, eq. (JABE)
  std::vector<cd> PJ;                         // (D - G^(E^,H^) M)^-1 (N^ x N^): inverse of the element's self block
  std::vector<cd> WPJ;                        // [M PJ; D PJ] (2 N^ x N^): macromodel of the preconditioned operator
  // near-field blocks with this type as the row type, computed by earlier
  // arrays (identical for every array with the same AIM options): arrays built
  // from the same types, on any thread, reuse them
  mutable std::mutex nf_mu;
  mutable std::map<NearBlockKey, std::shared_ptr<const NearBlockData>> nf_cache;
};
// device >= 0: the dense linear algebra of the build on that GPU.
void build_type(TypeModel& tm, int device = -1);
bool build_type_dense_gpu(TypeModel& tm, const std::vector<cd>& Lss, const std::vector<cd>& Lse,
                          const std::vector<cd>& Les, const std::vector<cd>& Lee, const std::vector<cd>& Kse,
                          int device, std::string& msg);

// ---- host FFT (mixed radix, FP64), used for the Green's spectrum ------------
void fft_inplace(std::vector<cd>& a, int64_t n, int64_t stride, int64_t count, int64_t dist, int sign);
bool fft_length_ok(int64_t n);
int64_t fft_good_length(int64_t n);
int64_t fft_fast_length(int64_t n);

}  // namespace mm
