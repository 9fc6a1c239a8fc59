// Near-field block fill on the GPU (Sec. V): exact Galerkin EFIE entries of
// the near pairs minus the grid part, FP64, for device contexts.
#pragma once

#include <array>
#include <string>
#include <vector>

#include "aim_setup.h"

namespace mm {

// One translation-invariant near-field block: rows of type a (its equivalent
// mesh ma, anchors and weights A), columns of type b (mb shifted by rel,
// anchors B shifted by dL grid cells), near pairs (ptr: Na + 1, col).  val
// receives ptr.back() entries.
struct NearFillJob {
  const Mesh* ma = nullptr;
  const Mesh* mb = nullptr;
  Vec3 rel{0, 0, 0};
  const TypeAim* A = nullptr;
  const TypeAim* B = nullptr;
  int64_t dL[3] = {0, 0, 0};
  const std::vector<int64_t>* ptr = nullptr;
  const std::vector<int32_t>* col = nullptr;
  std::vector<cd>* val = nullptr;
};

// Fills every job on `device`: val = c_A L_mn - (c_A sum_xyz P^T H P + c_phi
// P_phi^T H P_phi) for the near pairs, with L the EFIE Galerkin entry of the
// shifted meshes (the same closed-form static part and 7 x 7 product
// quadrature of the smooth part as the host fill) and H the grid Green's
// function table (Hv, half width HR, stencil offsets so).  Returns false with
// msg set on a CUDA error; the caller then fills on the host.
bool fill_near_blocks_gpu(std::vector<NearFillJob>& jobs, const std::vector<cd>& Hv, int HR,
                          const std::vector<std::array<int, 3>>& so, cd cA, cd cphi, double k, int device,
                          std::string& msg);

// The full EFIE Galerkin matrix (Nm x Nn, row-major, before the -j k eta0
// factor) of the test mesh against the source mesh shifted by `shift`, the
// host fill_efie's integrals on `device`.  False with msg set on a CUDA error.
bool fill_efie_gpu(const Mesh& test, const Mesh& src, Vec3 shift, double k, int device, std::vector<cd>& out,
                   std::string& msg);

// The K matrix <f_m, curl int G g_n> of the test mesh's RWG functions against
// the dual functions d (principal value), the host fill_k's integrals on
// `device`.  False with msg set on a CUDA error.
bool fill_k_gpu(const Mesh& test, const DualSet& d, double k, int device, std::vector<cd>& out, std::string& msg);

}  // namespace mm
