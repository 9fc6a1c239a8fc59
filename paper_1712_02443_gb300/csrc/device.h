// Device-side structures and kernel launchers of libmacroaim.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <vector>

#include "fft_plan.h"

namespace mm {

template <typename R> struct V2;
template <> struct V2<float> { typedef float2 T; };
template <> struct V2<double> { typedef double2 T; };
// The float-float form of the complex128 FFT stages (kernels.cu): complex
// values CF (ffops.cuh) inside, FP64 grids outside.
struct FFTag {};
struct CF;
template <> struct V2<FFTag> { typedef CF T; };
// element type of the grids the FFT stages read and write
template <typename R> struct GridT { typedef typename V2<R>::T T; };
template <> struct GridT<FFTag> { typedef double2 T; };

// Stage profiler: CUDA events around stages on the launching stream.
struct Profiler {
  bool on = false;
  struct Rec {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int64_t launches[16] = {0};   // slots 0-7: complex64 stages (7 = Krylov), 8-14: complex128 stages
  int open_stage = -1;
  cudaEvent_t open_ev = nullptr;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  uint32_t mask = 0xFFu;          // stages that record (bit s: stage s of either precision)
  void begin(int stage, cudaStream_t st) {
    if (!on || !((mask >> (stage % 8)) & 1u)) {
      open_stage = -1;
      return;
    }
    open_stage = stage;
    open_ev = get();
    cudaEventRecord(open_ev, st);
  }
  void end(cudaStream_t st, int nlaunch) {
    if (!on || open_stage < 0) return;
    cudaEvent_t b = get();
    cudaEventRecord(b, st);
    recs.push_back({open_stage, open_ev, b});
    launches[open_stage] += nlaunch;
  }
  void reset() {
    for (auto& r : recs) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
    for (auto& l : launches) l = 0;
  }
  ~Profiler() {
    reset();
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// Element pairs coupled by one near-field block, as the kernels read them (the
// device copy of DevArray::NfGroup, same layout).
struct NearGroupDev {
  int q, Na;
  int64_t first_pair, npairs;
};

// Per-type parameters of the table-driven projection (device copy).
struct PrjTypeDev {
  const unsigned char* tab;     // E float4 weights, then E uint16 basis indices (16-byte padded)
  const int32_t* inv_ptr;       // box node -> first entry (nodes + 1)
  const int32_t* elems;         // the type's element ids
  int E, Nh, bx, by, bz;
  int64_t ne;                   // number of elements of the type
};

// Per-type parameters of the table-driven interpolation (device copy).
struct ItpTypeDev {
  const float* Pi;              // S x Nh x 4 weights (stencil node outermost)
  const int32_t* anc;           // per basis: stencil anchor in the type's box (3 ints)
  const int32_t* elems;
  int Nh, bx, by, bz;
  int64_t ne;
};

// Radix plan of one FFT length (radices from {4, 2, 3, 5, 7, 11}).
struct FftPlan {
  int L = 1;
  int nst = 0;
  int rad[16] = {0};
};
FftPlan make_plan(int L);

// Operator data in one precision (R = float for MM_C64, double for MM_C128).
template <typename R>
struct DevPrec {
  bool ready = false;
  std::vector<void*> W;   // per type: stacked [M_t; D_t], 2 Nh x Nh complex, row-major
  std::vector<R*> Pi;     // per type: S x Nh x 4 projection weights (stencil node outermost)
  // complex64 only: per type the projection weights in the order of the inverse
  // stencil lists (inv_ent): E float4 weights, then E uint16 basis indices
  // (padded to 16 bytes); the table of the shared-memory projection
  std::vector<void*> prj_tab;
  PrjTypeDev* prj_types = nullptr;   // per type (n_types), when every type has a table
  size_t prj_smem = 0;               // shared memory of the largest type's tables, u chunk and box
  int64_t prj_total = 0;             // elements of all types
  ItpTypeDev* itp_types = nullptr;   // the same for the table-driven interpolation
  size_t itp_smem = 0;
  void* val = nullptr;    // near-field values (nnz complex)
  void* Ghat = nullptr;   // Green's spectrum [ky][kz][kx] complex, divided by Px Py Pz
  void* twx = nullptr;    // exp(-2 pi i k / Px), k < Px
  void* twy = nullptr;
  void* twz = nullptr;
  // tensor-core macromodel operands (complex64 modes): per type packed [M; D]
  std::vector<void*> Atc[2];   // [0] BF16, [1] FP16; (Mp x Kp) 16-bit
  std::vector<int> Mp, Kp;
  void* nfb_val = nullptr;     // near-field blocks, dense row-major, at DevArray::nfb_off
  // complex64 only: the blocks for the tensor-core near field, complex rows of
  // interleaved (re, im) FP32 at DevArray::nfb_arow, row pitch nfb_tc_pitch
  // floats; TF32 hi parts in rows [0, nfb_tc_rows), lo parts below them
  void* nfb_tc = nullptr;
  CUtensorMap nfb_tmap;        // 2-D map over nfb_tc: box 32 floats x 128 rows, 128-byte swizzle
  std::vector<void*> PJ;       // per type: block-Jacobi operator (Nh x Nh), uploaded on first use
  // the right-preconditioned operator's macromodel matrices [M PJ; D PJ] (same
  // layouts as W and Atc), uploaded with PJ: Z P^-1 x takes one GEMM
  std::vector<void*> WP;
  std::vector<void*> AtcP[2];
  // FP64 only: W and WP with (Re, Im, Re + Im) per entry for the three-multiplication GEMM
  std::vector<void*> W3, WP3;
  // FP64 only, the float-float contractions (kMvFF): per type [M; D] as F6
  // entries (2 Nh x Nh, row-major), and the near-field blocks as F6 in the
  // dense layout of nfb_val; uploaded on first use
  std::vector<void*> ffW;
  void* ff_nfb = nullptr;
  // ... and the FFT stages' twiddles and Green's spectrum as CF (same layouts as twx, twy, twz, Ghat)
  void *ff_twx = nullptr, *ff_twy = nullptr, *ff_twz = nullptr, *ff_Ghat = nullptr;
  // ... and per type the projection / interpolation weights as float pairs:
  // float4 hi, float4 lo (x, y, z, phi) per (stencil node s, basis n), s outermost
  std::vector<void*> ff_Pi;
  bool ff_ready = false;
};

// Work buffers for one (precision, nrhs) pair.
struct Work {
  int nrhs = 0;
  void* u = nullptr;      // N x nrhs   macromodel product T A^-1 B x
  void* v = nullptr;      // N x nrhs   D x
  void* grid = nullptr;   // 4 nrhs x Nx x Ny x Nz   grid charges/currents, then potentials
  void* spec = nullptr;   // 4 nrhs x Nx x Py x Pz   partial spectra
  void* bt = nullptr;     // packed right-hand sides of the tensor-core GEMM
  size_t bt_cap = 0;      // elements
  int* err = nullptr;     // device error flag of bounded waits
  void* pt = nullptr;     // N x nrhs   preconditioned vector (block-Jacobi)
  double* us = nullptr;   // N x nrhs   FP64 only: Re u + Im u for the three-product near field
  void* np = nullptr;     // complex64 only: partial sums of the tensor-core near field (np_parts x nfg_prows x nrhs)
  int np_parts = 1;       // planes of np: 2 lets the tensor-core near field split its k tiles in two
  void* boxbuf = nullptr; // from 8 RHS on: per-element projection boxes (n_elem x 4 nrhs x box_nodes_max)
  void* x6 = nullptr;     // FP64 only, float-float products: x and u split into F6 entries (N x nrhs)
  void* u6 = nullptr;
  size_t bytes = 0;
};

// Grid-stage tuner's choice for one (right-hand-side count, precision): the
// projection and interpolation variants and the times of every variant (ms).
struct GridTune {
  int project = 0, interp = 0;
  std::vector<float> project_ms, interp_ms;
};

struct DevArray {
  int device = 0;
  int64_t N = 0, n_elem = 0, n_types = 0, nnz = 0;
  int grid[3] = {0, 0, 0}, fft[3] = {0, 0, 0};
  int S = 0, n1 = 0, o1lo = 0;
  double cA[2] = {0, 0}, cphi[2] = {0, 0};
  // per type (host mirrors + device pointers)
  std::vector<int64_t> Nh;
  std::vector<int> box;                 // 3 per type
  std::vector<int32_t*> anc;            // per type: Nh x 3 box-local anchors
  std::vector<double*> geo;             // per type: Nh x 13 (pa, pb, p+, p-, length), local coordinates
  std::vector<int32_t*> elems;          // per type: element ids of that type
  std::vector<int32_t*> inv_ptr;        // per type: box node -> first stencil entry touching it (nodes + 1)
  std::vector<int32_t*> inv_ent;        // per type: stencil entries n | (s << 16), grouped by box node
  std::vector<int32_t> inv_len;         // per type: number of those entries
  std::vector<int64_t> n_of_type;
  // per element
  int64_t* off = nullptr;               // n_elem + 1
  int64_t* tbase = nullptr;             // n_types + 1: prefix of the types' N^_t (local bases of all types)
  int32_t* boxorg = nullptr;            // n_elem x 3: global grid coordinates of the type box origin
  int box_nodes_max = 1;                // largest stencil box (nodes) over the types
  int32_t* gptr = nullptr;              // grid nodes + 1: the two-pass projection's gather lists ...
  int64_t* gent = nullptr;              // ... entries element * box_nodes_max + local node
  int32_t* type_of = nullptr;
  double* eoff = nullptr;               // n_elem x 3 element offsets
  // near field pattern (shared by both precisions)
  int64_t* rowptr = nullptr;            // rows padded to multiples of 4 entries (zero values)
  int32_t* col = nullptr;
  int64_t nnz_padded = 0;
  // near field as translation-invariant blocks (used for 8 or more right-hand
  // sides): per distinct block its shape and dense offset; per (block, 64-row
  // tile) the 16-column k tiles that hold a non-zero; element pairs grouped by
  // lattice offset so that each group touches every output element at most once
  int nfb_nmt = 0;                      // 64-row tiles of the tallest block
  int32_t* nfb_na = nullptr;            // per block: rows (N^ of the row type)
  int32_t* nfb_nb = nullptr;            // per block: columns
  int64_t* nfb_off = nullptr;           // per block: first entry in the dense values
  int32_t* nfb_tptr = nullptr;          // blocks x nfb_nmt + 1
  int32_t* nfb_tlist = nullptr;         // k-tile indices
  int nfb_nmt32 = 0;                    // the same for 32-row tiles
  int32_t* nfb_tptr32 = nullptr;
  int32_t* nfb_tlist32 = nullptr;
  int nfb_nmt128 = 0;                   // the same for 128-row tiles (tensor-core near field)
  int32_t* nfb_tptr128 = nullptr;
  int32_t* nfb_tlist128 = nullptr;
  int32_t* nfb_arow = nullptr;          // per block: its first row in the tensor-core block rows
  int nfb_tc_rows = 0;                  // rows of all blocks (tensor-core layout)
  int nfb_tc_pitch = 0;                 // floats per row (2 Nb of the widest block, rounded up to 32)
  int* near_err = nullptr;              // device flag of the tensor-core near field's bounded waits
  int64_t* nfg_prow = nullptr;          // per pair: first row of its slice in the partial-sum buffer
  int64_t nfg_prows = 0;                // rows of the partial-sum buffer (sum over pairs of the row type's N^)
  int32_t* nfe_ptr = nullptr;           // per element: its pairs as row element (n_elem + 1) ...
  int32_t* nfe_pair = nullptr;          // ... and the pair indices
  longlong2* nfe_qb = nullptr;          // per entry of nfe_pair: (block q, unknown offset of the column element)
  int32_t* nfe_order = nullptr;         // element ids sorted by type, then id (the direct near field's unit order)
  int32_t* nfb_tperm = nullptr;         // per type: offset of its anchor ordering in nfb_perm
  int32_t* nfb_perm = nullptr;          // per type (concatenated): sorted position -> local basis
  int32_t* nfb_pa = nullptr;            // per block: offset of its row type's ordering in nfb_perm
  int32_t* nfb_pb = nullptr;            // per block: offset of its column type's ordering
  int64_t nfb_entries = 0;              // dense complex entries over all blocks
  struct NfGroup {                      // the element pairs coupled by one block (host mirror)
    int q = 0;                          // block id
    int Na = 0;                         // its rows
    int64_t first_pair = 0, npairs = 0; // range in nfg_poff
  };
  std::vector<NfGroup> nfg;
  void* nfg_dev = nullptr;              // device copy of nfg (same layout)
  longlong2* nfg_poff = nullptr;        // per pair: unknown offsets of (row element, column element), grouped by block
  int near_mode = 0;                    // 0 blocks; 2 CSR rows (when assembled)
  // autotuned block near-field shape per (right-hand sides, sizeof(R)): (kernel shape, k split)
  std::map<std::pair<int, int>, std::pair<int, int>> near_tune;
  int near_force_shape = -1, near_force_ks = 1;   // MACROAIM_NEAR_SHAPE="shape,ksplit": no tuning
  // tile shapes of the float-float GEMM (0: 32 x 32, 1: 16 x 32, the default,
  // 2: 32 x 64) and block near field (0: 32 x 32, 1: the same held to three CTAs
  // per SM, the default, 2: 32 rows x 64 columns, 3: 32 x 16);
  // MACROAIM_FF_SHAPE="gemm,near" (16x16 loop array, one column, alone: GEMM 97,
  // 81, 161 us; near field 172, 162, 199, 183 us)
  int ff_gemm_shape = 1, ff_near_shape = 1;
  std::map<std::pair<int, int>, GridTune> grid_tune;   // per (right-hand sides, sizeof(R))
  bool tune_grid = true;                           // MACROAIM_GRID_TUNE=0: variant 0, no timing
  int grid_force_p = -1, grid_force_i = -1;        // MACROAIM_GRID_SCHED="p,i": fixed variants
  // streams of the product: the near field runs on `side` beside the far-field
  // chain (projection, convolution, interpolation) on `chain`, which has the
  // higher priority; fork / join events order both against the caller's stream
  cudaStream_t side = nullptr, chain = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_done = nullptr;
  FftPlan px, py;
  DevPrec<float> pf;
  DevPrec<double> pd;
  Work wf, wd;
  Profiler prof;
  size_t bytes = 0;                     // resident operator bytes
  // host copies kept for lazy upload of the other precision
  std::vector<std::vector<double>> hW;  // per type: 2 Nh x Nh complex128 interleaved
  std::vector<std::vector<double>> hPi;
  std::vector<double> hval, hGhat;      // complex128 interleaved
};

// Shapes of the block near field: 0-4 CUDA-core tiles (k_near_blocks), 5-6
// tensor-core tiles with partial sums, 7-9 the tensor-core direct form
// (near_tc.cu, complex64).
constexpr int kNearShapes = 10;
// Flags of matvec: kMvNoTune never times near-field kernel shapes (an untuned
// right-hand-side count takes the size rule and is not remembered);
// kMvNoProfile records no stage events (the array's profiler is left alone).
// kMvUInput takes x as u (the macromodel stage skipped) and v = 0: y = -G x.
// kMvFF (complex128 only): every stage in float-float arithmetic on the FP32
// pipe (DevPrec::ffW and the other ff_ operands, Work::x6 and u6 must be in
// place); the stages exchange FP64 vectors and grids.
constexpr unsigned kMvNoTune = 1u, kMvNoProfile = 2u, kMvUInput = 4u, kMvFF = 8u;
// gemm_mode: 0 CUDA-core GEMM; 1 BF16 / 2 FP16 tensor-core GEMM (complex64 only)
// pre: apply Z P^-1 (the block-Jacobi right-preconditioned operator) through
// the fused macromodel matrices p.WP / p.AtcP
template <typename R>
cudaError_t matvec(DevArray& a, DevPrec<R>& p, Work& w, int nrhs, const void* x, void* y, cudaStream_t st,
                   int gemm_mode = 0, bool pre = false, unsigned flags = 0);
// y = P^-1 x with P^-1 the per-type block-Jacobi operators (p.PJ).
template <typename R>
cudaError_t precond_apply(DevArray& a, DevPrec<R>& p, int nrhs, const void* x, void* y, cudaStream_t st);
template <typename R>
size_t fft_smem_bytes(const DevArray& a, int which);
cudaError_t kernels_init(DevArray& a);
// shared memory the table-driven projection needs for one type
size_t project_tab_smem(int E, int nodes, int Nh);
// ... and the table-driven interpolation (weights, box of eight right-hand sides)
size_t interp_tab_smem(int S, int Nh, int nodes);

}  // namespace mm
