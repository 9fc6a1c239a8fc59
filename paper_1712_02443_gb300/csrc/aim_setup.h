// Host-side AIM set-up structures (Sec. V).
#pragma once

#include <array>

#include "internal.h"

namespace mm {

struct AimOpts {
  double h;
  int order;
  int n_nf;
  Vec3 phase;
  int64_t csr_max_nnz = -1;   // assemble the expanded near-field CSR up to this many non-zeros (-1: always)
  int device = -1;            // CUDA device of the array's context: near-field blocks filled there (-1: host)
};

// Anchors and projection weights of one element type, placed at the array's
// reference position (identical elements on the grid lattice share them).
struct TypeAim {
  int64_t Nh = 0;
  int S = 0;                   // stencil nodes (order+1)^3
  std::vector<int64_t> anc;    // Nh x 3 grid anchors at the reference position
  std::vector<double> Pi;      // Nh x S x 4 (psi = x, y, z, phi), s = (iz*n+iy)*n+ix
  int64_t box_lo[3] = {0, 0, 0};
  int64_t box_dim[3] = {0, 0, 0};
};

struct ArrayHost {
  AimOpts opts{};
  int64_t n_elem = 0, N = 0;
  std::vector<int32_t> type_of;
  std::vector<int64_t> off;     // n_elem + 1 unknown offsets
  std::vector<int64_t> L;       // lattice position of each element (grid cells, relative to element 0)
  std::vector<int64_t> base;    // per element: L - grid origin (add to reference anchors)
  std::vector<TypeAim> tai;
  int64_t grid[3] = {0, 0, 0}, fft[3] = {0, 0, 0}, lo[3] = {0, 0, 0};
  std::vector<cd> Ghat;         // fft[0] x fft[1] x fft[2] (x slowest), already divided by Px Py Pz
  std::vector<int64_t> rowptr;  // near field CSR
  std::vector<int32_t> col;
  std::vector<cd> val;
  int64_t nnz_near = 0;         // near-field non-zeros (whether or not the CSR is assembled)
  cd c_A, c_phi;
  int64_t n_blocks = 0;
  // the near field before expansion: distinct (type, type, lattice offset)
  // blocks (sparse rows, local columns) and, per element, its neighbours with
  // the block that couples them (rows of element e, columns of the neighbour)
  struct NearBlock {
    int32_t ta = 0, tb = 0;
    int64_t dL[3] = {0, 0, 0};
    int64_t Na = 0, Nb = 0;
    std::vector<int64_t> ptr;   // Na + 1 (empty: no near pairs)
    std::vector<int32_t> col;
    std::vector<cd> val;
  };
  std::vector<NearBlock> nf_blocks;
  std::vector<std::vector<std::pair<int64_t, int64_t>>> nf_nbr;   // (neighbour element, block id)
};

std::vector<int> stencil_1d(int order);
void type_aim(const Mesh& eq, Vec3 pos, const AimOpts& o, TypeAim& ta);
void build_array_host(ArrayHost& ah, const std::vector<const TypeModel*>& types, const std::vector<int32_t>& type_of,
                      const std::vector<Vec3>& offsets, const AimOpts& o, const EM& em);

}  // namespace mm
