// C ABI of libmacroaim (see include/macroaim.h for the contract of each call).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <set>
#include <functional>
#include <map>
#include <memory>
#include <cstdio>
#include <mutex>
#include <new>
#include <string>
#include <thread>

#include "aim_setup.h"
#include "device.h"
#include "ffops.cuh"
#include "internal.h"
#include "macroaim.h"
#include "post.h"
#include "solver.h"
#include "drive.h"
#include "near_tc.h"
#include "tc_gemm.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

struct mm_ctx {
  int device = -1;
  int nthreads = 1;
  std::string err;
};
struct mm_mesh {
  mm_ctx* ctx;
  mm::Mesh m;
};
struct mm_type {
  mm_ctx* ctx;
  mm::TypeModel tm;
  // delta-gap feed (mm_type_set_feed): J_f = -A^-1 f (N) and J^_f = T J_f (N^)
  // of one volt, f the gap's MoM right-hand side
  bool fed = false;
  std::vector<mm::cd> feed_Jf, feed_Jhf;
};
struct mm_array {
  mm_ctx* ctx = nullptr;
  std::vector<const mm_type*> types;
  mm::ArrayHost ah;
  mm::DevArray da;
  bool on_device = false;
  double k0 = 0, eta0 = 0;
  int32_t* elem_of = nullptr;     // device: element of each unknown
  double** geo_ptrs = nullptr;    // device: per-type geometry pointers
  double* d_ang = nullptr;        // device: theta, phi scratch for the excitation
  int32_t* d_pol = nullptr;
  int ang_cap = 0;
  cudaEvent_t ang_ev = nullptr;   // the last excitation kernels (they use d_ang, d_pol, d_pw)
  double2* d_pw = nullptr;        // excitation scratch: local sums and element phases
  int64_t pw_cap = 0;             // its capacity (complex128 entries)
  void* hx = nullptr;             // device staging for mm_apply_host
  void* hy = nullptr;
  size_t h_cap = 0;
  std::unique_ptr<mm::Solver> solver;
  // post-processing operators (uploaded on first use): per type -A^-1 B and T, scatterer offsets
  std::vector<void*> d_JE, d_T;
  int64_t* d_offs = nullptr;
  std::vector<int64_t> offs;      // host: scatterer unknown offsets (n_elem + 1)
  double* d_dir = nullptr;        // device: theta, phi of the far-field directions
  int64_t dir_cap = 0;
  // host: per type, the near-field block ordering of its bases (sorted position ->
  // basis) and its inverse
  std::vector<std::vector<int32_t>> nf_perm, nf_iperm;
  std::vector<int32_t> nfb_arow_h;   // per block: first row in the tensor-core block layout
  std::vector<std::vector<int32_t>> inv_ent_h;   // per type: the inverse stencil lists (host copy)
  std::vector<void*> d_Jf, d_Jhf;    // per type: device copies of the feed vectors (nullptr: not fed)
  void* d_volts = nullptr;           // driven elements' volts (n_elem x nrhs complex128)
  void* d_fu = nullptr;              // the driven elements' equivalent currents J^_f V (N^ x nrhs)
  size_t fu_cap = 0;
  size_t volts_cap = 0;
  void* d_pw2 = nullptr;             // ground plane: the image wave's excitation
  size_t pw2_cap = 0;
  double* d_gc = nullptr;            // ground plane: per right-hand side factor of the image wave
  int gc_cap = 0;
  cudaStream_t bst = nullptr;        // mm_apply_batch: this array's product stream and its event
  cudaEvent_t bev_done = nullptr, bev_fork = nullptr;
  uint64_t epoch = 0;                // bumped whenever a work buffer a product uses is reallocated
  std::set<std::pair<int, int>> settled;   // (nrhs, precision) with a product done (tuners run)
  void* pv_V = nullptr;              // mm_solve_planewave_host: excitation and solution on the device
  void* pv_E = nullptr;
  size_t pv_cap = 0;
  ~mm_array();
};

namespace {

// Batch products replayed as one CUDA graph: once every array of a batch has
// done a product of its width and precision (tuners run, work buffers
// allocated), the batch's launch sequence is captured into a graph on a
// library stream and later calls with the same arrays, widths, buffers,
// precision and work-buffer epochs launch that graph instead of every kernel.
// A graph is dropped when one of its arrays is destroyed.
struct BatchGraph {
  std::vector<const mm_array*> arrays;
  std::vector<int32_t> nrhs;
  std::vector<const void*> x, y;
  std::vector<uint64_t> epochs;
  int32_t precision = 0;
  int device = 0;
  cudaGraphExec_t exec = nullptr;
};
std::mutex g_graph_mu;
std::vector<BatchGraph> g_graphs;
constexpr size_t kMaxGraphs = 16;
cudaStream_t g_cap_stream[64] = {nullptr};
cudaEvent_t g_cap_in[64] = {nullptr}, g_cap_out[64] = {nullptr};

void drop_graphs_of(const mm_array* a) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (size_t i = 0; i < g_graphs.size();) {
    const auto& g = g_graphs[i];
    if (std::find(g.arrays.begin(), g.arrays.end(), a) != g.arrays.end()) {
      cudaGraphExecDestroy(g.exec);
      g_graphs.erase(g_graphs.begin() + i);
    } else {
      ++i;
    }
  }
}


mm_status fail(mm_ctx* ctx, mm_status code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define API_TRY try {
#define API_CATCH(ctx)                                             \
  }                                                                \
  catch (const mm::Error& e) {                                     \
    return fail(ctx, e.code, e.msg);                               \
  }                                                                \
  catch (const std::bad_alloc&) {                                  \
    return fail(ctx, MM_ENOMEM, "host allocation failed");         \
  }                                                                \
  catch (...) {                                                    \
    return fail(ctx, MM_EINTERNAL, "unexpected exception");        \
  }

#define CU(x)                                                                              \
  do {                                                                                     \
    cudaError_t _e = (x);                                                                  \
    if (_e != cudaSuccess) throw mm::Error{MM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(_e)}; \
  } while (0)

template <typename T>
T* dev_upload(const T* h, size_t n, size_t& acc) {
  T* d = nullptr;
  const size_t cap = n == 0 ? 1 : n;   // empty arrays still get a valid pointer
  CU(cudaMalloc(&d, sizeof(T) * cap));
  acc += sizeof(T) * cap;
  if (h && n > 0) CU(cudaMemcpy(d, h, sizeof(T) * n, cudaMemcpyHostToDevice));
  return d;
}

template <typename R>
void upload_precision(mm_array* a, mm::DevPrec<R>& p) {
  if (p.ready) return;
  auto& da = a->da;
  const auto& ah = a->ah;
  typedef typename mm::V2<R>::T C;
  p.W.resize(da.n_types);
  p.Pi.resize(da.n_types);
  for (int64_t t = 0; t < da.n_types; ++t) {
    const auto& tm = a->types[t]->tm;
    int64_t Nh = tm.Nh;
    std::vector<C> W(2 * Nh * Nh);
    for (int64_t i = 0; i < Nh * Nh; ++i) {
      W[i].x = (R)tm.M[i].real(); W[i].y = (R)tm.M[i].imag();
      W[Nh * Nh + i].x = (R)tm.D[i].real(); W[Nh * Nh + i].y = (R)tm.D[i].imag();
    }
    p.W[t] = dev_upload(W.data(), W.size(), da.bytes);
    if (sizeof(R) == 8) {
      // three-multiplication form of the FP64 GEMM: (Re, Im, Re + Im) per entry
      std::vector<double> W3(3 * 2 * Nh * Nh);
      for (int64_t i = 0; i < 2 * Nh * Nh; ++i) {
        const mm::cd w = i < Nh * Nh ? tm.M[i] : tm.D[i - Nh * Nh];
        W3[3 * i] = w.real();
        W3[3 * i + 1] = w.imag();
        W3[3 * i + 2] = w.real() + w.imag();
      }
      p.W3.push_back(dev_upload(W3.data(), W3.size(), da.bytes));
    }
    // device layout [s][n][4]: consecutive bases of one stencil node are contiguous
    const auto& Pi = ah.tai[t].Pi;
    const int S = ah.tai[t].S;
    std::vector<R> P(Pi.size());
    for (int64_t n = 0; n < Nh; ++n)
      for (int sn = 0; sn < S; ++sn)
        for (int c = 0; c < 4; ++c) P[((size_t)sn * Nh + n) * 4 + c] = (R)Pi[((size_t)n * S + sn) * 4 + c];
    p.Pi[t] = dev_upload(P.data(), P.size(), da.bytes);
    if (sizeof(R) == 4 && (size_t)t < a->inv_ent_h.size()) {
      // the same weights in inverse-list order, with the basis indices as uint16
      const auto& ent = a->inv_ent_h[t];
      const size_t E = ent.size(), nb = (2 * E + 15) / 16 * 16;
      std::vector<unsigned char> tab(16 * E + nb, 0);
      for (size_t q = 0; q < E; ++q) {
        const int n = ent[q] & 0xffff, sn = ent[q] >> 16;
        float w[4];
        for (int c = 0; c < 4; ++c) w[c] = (float)Pi[((size_t)n * S + sn) * 4 + c];
        std::memcpy(&tab[16 * q], w, 16);
        const uint16_t n16 = (uint16_t)n;
        std::memcpy(&tab[16 * E + 2 * q], &n16, 2);
      }
      p.prj_tab.push_back(dev_upload(tab.data(), tab.size(), da.bytes));
    }
  }
  if (sizeof(R) == 4 && (int64_t)p.prj_tab.size() == da.n_types && da.n_types > 0) {
    std::vector<mm::PrjTypeDev> pt(da.n_types);
    size_t smem = 0;
    int64_t total = 0;
    for (int64_t t = 0; t < da.n_types; ++t) {
      pt[t].tab = static_cast<const unsigned char*>(p.prj_tab[t]);
      pt[t].inv_ptr = da.inv_ptr[t];
      pt[t].elems = da.elems[t];
      pt[t].E = da.inv_len[t];
      pt[t].Nh = (int)da.Nh[t];
      pt[t].bx = da.box[3 * t];
      pt[t].by = da.box[3 * t + 1];
      pt[t].bz = da.box[3 * t + 2];
      pt[t].ne = da.n_of_type[t];
      smem = std::max(smem, mm::project_tab_smem(pt[t].E, pt[t].bx * pt[t].by * pt[t].bz, pt[t].Nh));
      total += pt[t].ne;
    }
    p.prj_types = dev_upload(pt.data(), pt.size(), da.bytes);
    p.prj_smem = smem;
    p.prj_total = total;
    std::vector<mm::ItpTypeDev> it(da.n_types);
    size_t ismem = 0;
    for (int64_t t = 0; t < da.n_types; ++t) {
      it[t].Pi = reinterpret_cast<const float*>(p.Pi[t]);
      it[t].anc = da.anc[t];
      it[t].elems = da.elems[t];
      it[t].Nh = (int)da.Nh[t];
      it[t].bx = da.box[3 * t];
      it[t].by = da.box[3 * t + 1];
      it[t].bz = da.box[3 * t + 2];
      it[t].ne = da.n_of_type[t];
      ismem = std::max(ismem, mm::interp_tab_smem((int)da.S, it[t].Nh, it[t].bx * it[t].by * it[t].bz));
    }
    p.itp_types = dev_upload(it.data(), it.size(), da.bytes);
    p.itp_smem = ismem;
  }
  if (da.nnz > 0) {
    // near-field values in the padded row layout of da.rowptr (pad entries are
    // 0); complex64 interleaved, FP64 as (Re, Im, Re + Im) for the
    // three-product form of the FP64 SpMV
    const int per = sizeof(R) == 8 ? 3 : 2;
    std::vector<R> v((size_t)per * da.nnz_padded, (R)0);
    int64_t q = 0;
    for (int64_t i = 0; i < ah.N; ++i) {
      int64_t len = ah.rowptr[i + 1] - ah.rowptr[i];
      for (int64_t k = 0; k < len; ++k) {
        const auto& z = ah.val[ah.rowptr[i] + k];
        R* d = v.data() + (size_t)per * (q + k);
        d[0] = (R)z.real();
        d[1] = (R)z.imag();
        if (per == 3) d[2] = (R)(z.real() + z.imag());
      }
      q += (len + 3) / 4 * 4;
    }
    p.val = dev_upload(v.data(), v.size(), da.bytes);
  }
  if (da.nfb_entries > 0) {
    // near-field blocks, dense row-major (zeros outside the near pairs)
    std::vector<C> d((size_t)da.nfb_entries);
    for (auto& z : d) { z.x = 0; z.y = 0; }
    int64_t o = 0;
    for (const auto& b : ah.nf_blocks) {
      if (b.ptr.empty()) continue;
      const auto &ia = a->nf_iperm[b.ta], &ib = a->nf_iperm[b.tb];   // original -> sorted position
      for (int64_t m = 0; m < b.Na; ++m)
        for (int64_t q = b.ptr[m]; q < b.ptr[m + 1]; ++q) {
          C& z = d[(size_t)(o + (int64_t)ia[m] * b.Nb + ib[b.col[q]])];
          z.x = (R)b.val[q].real();
          z.y = (R)b.val[q].imag();
        }
      o += b.Na * b.Nb;
    }
    p.nfb_val = dev_upload(d.data(), d.size(), da.bytes);
    if (sizeof(R) == 4 && da.nfb_tc_rows > 0 && !a->nfb_arow_h.empty()) {
      // the same blocks for the tensor-core near field: complex rows of
      // interleaved FP32 (row pitch nfb_tc_pitch), TF32 hi parts in rows
      // [0, rows), lo parts in rows [rows, 2 rows)
      const int64_t rows = da.nfb_tc_rows, pitch = da.nfb_tc_pitch;
      std::vector<float> A((size_t)(2 * rows * pitch), 0.0f);
      int64_t q = 0;
      for (const auto& b : ah.nf_blocks) {
        if (!b.ptr.empty()) {
          const auto &ia = a->nf_iperm[b.ta], &ib = a->nf_iperm[b.tb];
          for (int64_t m = 0; m < b.Na; ++m)
            for (int64_t e = b.ptr[m]; e < b.ptr[m + 1]; ++e) {
              const int64_t row = a->nfb_arow_h[q] + ia[m], kc = ib[b.col[e]];
              float hi[2], lo[2];
              mm::near_tc_split(b.val[e].real(), b.val[e].imag(), hi, lo);
              float* dh = A.data() + (size_t)(row * pitch + 2 * kc);
              float* dl = A.data() + (size_t)((rows + row) * pitch + 2 * kc);
              dh[0] = hi[0];
              dh[1] = hi[1];
              dl[0] = lo[0];
              dl[1] = lo[1];
            }
        }
        ++q;
      }
      CU(mm::tc_gemm_init());
      void* dA = dev_upload(A.data(), A.size(), da.bytes);
      if (mm::tc_encode_2d(&p.nfb_tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, dA, (uint64_t)pitch, (uint64_t)(2 * rows),
                           (uint64_t)pitch * 4, 32, 128))
        p.nfb_tc = dA;
      else
        cudaFree(dA);   // no tensor-map encoder: the CUDA-core block kernels apply the near field
    }
  }
  {
    const int64_t Px = ah.fft[0], Py = ah.fft[1], Pz = ah.fft[2];
    std::vector<C> g(Px * Py * Pz);
    for (int64_t i = 0; i < Px; ++i)
      for (int64_t j = 0; j < Py; ++j)
        for (int64_t l = 0; l < Pz; ++l) {
          const auto& z = ah.Ghat[(i * Py + j) * Pz + l];
          C& o = g[(j * Pz + l) * Px + i];
          o.x = (R)z.real(); o.y = (R)z.imag();
        }
    p.Ghat = dev_upload(g.data(), g.size(), da.bytes);
  }
  auto tw = [&](int64_t L) {
    std::vector<C> t(L);
    for (int64_t k = 0; k < L; ++k) {
      double th = -2.0 * M_PI * (double)k / (double)L;
      t[k].x = (R)std::cos(th); t[k].y = (R)std::sin(th);
    }
    return dev_upload(t.data(), t.size(), da.bytes);
  };
  p.twx = tw(ah.fft[0]);
  p.twy = tw(ah.fft[1]);
  p.twz = tw(ah.fft[2]);
  p.ready = true;
}

// Packed real operand of the tensor-core GEMM for one 16-bit format (mode 1 BF16,
// 2 FP16): per type, row 2i = [Re W_i, -Im W_i], row 2i+1 = [Im W_i, Re W_i]
// for W = [M; D], padded to the tile sizes.
// pre: the preconditioned operator's matrices [M PJ; D PJ] (p.AtcP) instead of [M; D]
void upload_tc(mm_array* a, int mode, bool pre = false) {
  auto& p = a->da.pf;
  const int slot = mode - 1;
  auto& dst = pre ? p.AtcP[slot] : p.Atc[slot];
  if (!dst.empty()) return;
  auto& da = a->da;
  const int TM = mm::tc_tile_m(), TK = mm::tc_tile_k();
  p.Mp.resize(da.n_types);
  p.Kp.resize(da.n_types);
  for (int64_t t = 0; t < da.n_types; ++t) {
    const auto& tm = a->types[t]->tm;
    const int64_t Nh = tm.Nh;
    const int64_t Nhp = mm::tc_k_split((int)Nh);   // the imaginary half starts here
    const int Mp = (int)((4 * Nh + TM - 1) / TM * TM), Kp = (int)((Nhp + Nh + TK - 1) / TK * TK);
    p.Mp[t] = Mp;
    p.Kp[t] = Kp;
    std::vector<uint16_t> A((size_t)Mp * Kp, 0);
    auto cvt = [&](double v) -> uint16_t {
      if (mode == 1) {
        __nv_bfloat16 b = __float2bfloat16_rn((float)v);
        return *reinterpret_cast<uint16_t*>(&b);
      }
      __half h = __float2half_rn((float)v);
      return *reinterpret_cast<uint16_t*>(&h);
    };
    for (int64_t i = 0; i < 2 * Nh; ++i) {
      const std::vector<mm::cd>& W = pre ? tm.WPJ : (i < Nh ? tm.M : tm.D);
      const int64_t ii = (pre || i < Nh) ? i : i - Nh;
      for (int64_t k = 0; k < Nh; ++k) {
        const mm::cd w = W[ii * Nh + k];
        A[(size_t)(2 * i) * Kp + k] = cvt(w.real());
        A[(size_t)(2 * i) * Kp + Nhp + k] = cvt(-w.imag());
        A[(size_t)(2 * i + 1) * Kp + k] = cvt(w.imag());
        A[(size_t)(2 * i + 1) * Kp + Nhp + k] = cvt(w.real());
      }
    }
    dst.push_back(dev_upload(A.data(), A.size(), da.bytes));
  }
}

// Block-Jacobi operators per type (inverse self blocks), uploaded on first use.
template <typename R>
void upload_pj(mm_array* a, mm::DevPrec<R>& p) {
  if (!p.PJ.empty()) return;
  typedef typename mm::V2<R>::T C;
  for (int64_t t = 0; t < a->da.n_types; ++t) {
    const auto& tm = a->types[t]->tm;
    std::vector<C> W(tm.PJ.size());
    for (size_t i = 0; i < W.size(); ++i) {
      W[i].x = (R)tm.PJ[i].real();
      W[i].y = (R)tm.PJ[i].imag();
    }
    p.PJ.push_back(dev_upload(W.data(), W.size(), a->da.bytes));
    std::vector<C> WP(tm.WPJ.size());
    for (size_t i = 0; i < WP.size(); ++i) {
      WP[i].x = (R)tm.WPJ[i].real();
      WP[i].y = (R)tm.WPJ[i].imag();
    }
    p.WP.push_back(dev_upload(WP.data(), WP.size(), a->da.bytes));
    if (sizeof(R) == 8) {
      std::vector<double> W3(3 * tm.WPJ.size());
      for (size_t i = 0; i < tm.WPJ.size(); ++i) {
        W3[3 * i] = tm.WPJ[i].real();
        W3[3 * i + 1] = tm.WPJ[i].imag();
        W3[3 * i + 2] = tm.WPJ[i].real() + tm.WPJ[i].imag();
      }
      p.WP3.push_back(dev_upload(W3.data(), W3.size(), a->da.bytes));
    }
  }
}

// Operands of the float-float complex128 product (matvec flag kMvFF): [M; D]
// per type and the near-field blocks, each complex entry as re, im and re + im
// split into a float and the float nearest to the remainder.
mm::F6 f6_host(mm::cd z) {
  auto split = [](double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  };
  mm::F6 f;
  split(z.real(), f.rh, f.rl);
  split(z.imag(), f.ih, f.il);
  split(z.real() + z.imag(), f.sh, f.sl);
  return f;
}

void upload_ff(mm_array* a) {
  auto& p = a->da.pd;
  if (p.ff_ready) return;
  auto& da = a->da;
  const auto& ah = a->ah;
  for (int64_t t = 0; t < da.n_types; ++t) {
    const auto& tm = a->types[t]->tm;
    const int64_t Nh = tm.Nh;
    std::vector<mm::F6> W(2 * Nh * Nh);
    for (int64_t i = 0; i < Nh * Nh; ++i) {
      W[i] = f6_host(tm.M[i]);
      W[Nh * Nh + i] = f6_host(tm.D[i]);
    }
    p.ffW.push_back(dev_upload(W.data(), W.size(), da.bytes));
    // projection / interpolation weights: [s][n] -> (hi x, y, z, phi), (lo x, y, z, phi)
    const auto& Pi = ah.tai[t].Pi;
    const int S = ah.tai[t].S;
    std::vector<float> P((size_t)S * Nh * 8);
    for (int64_t n = 0; n < Nh; ++n)
      for (int sn = 0; sn < S; ++sn)
        for (int c = 0; c < 4; ++c) {
          const double w = Pi[((size_t)n * S + sn) * 4 + c];
          const float hi = (float)w;
          float* d = P.data() + ((size_t)sn * Nh + n) * 8;
          d[c] = hi;
          d[4 + c] = (float)(w - (double)hi);
        }
    p.ff_Pi.push_back(dev_upload(P.data(), P.size(), da.bytes));
  }
  if (da.nfb_entries > 0) {
    std::vector<mm::F6> d((size_t)da.nfb_entries, f6_host(mm::cd(0.0, 0.0)));
    int64_t o = 0;
    for (const auto& b : ah.nf_blocks) {
      if (b.ptr.empty()) continue;
      const auto &ia = a->nf_iperm[b.ta], &ib = a->nf_iperm[b.tb];   // original -> sorted position
      for (int64_t m = 0; m < b.Na; ++m)
        for (int64_t q = b.ptr[m]; q < b.ptr[m + 1]; ++q)
          d[(size_t)(o + (int64_t)ia[m] * b.Nb + ib[b.col[q]])] = f6_host(b.val[q]);
      o += b.Na * b.Nb;
    }
    p.ff_nfb = dev_upload(d.data(), d.size(), da.bytes);
  }
  auto ffv = [](double x) {
    const float hi = (float)x;
    return mm::FFv(hi, (float)(x - (double)hi));
  };
  {
    // the Green's spectrum [ky][kz][kx] and the twiddles of the FFT stages
    const int64_t Px = ah.fft[0], Py = ah.fft[1], Pz = ah.fft[2];
    std::vector<mm::CF> g(Px * Py * Pz);
    for (int64_t i = 0; i < Px; ++i)
      for (int64_t j = 0; j < Py; ++j)
        for (int64_t l = 0; l < Pz; ++l) {
          const auto& z = ah.Ghat[(i * Py + j) * Pz + l];
          g[(j * Pz + l) * Px + i] = mm::CF{ffv(z.real()), ffv(z.imag())};
        }
    p.ff_Ghat = dev_upload(g.data(), g.size(), da.bytes);
    auto tw = [&](int64_t L) {
      std::vector<mm::CF> t(L);
      for (int64_t k = 0; k < L; ++k) {
        const double th = -2.0 * M_PI * (double)k / (double)L;
        t[k] = mm::CF{ffv(std::cos(th)), ffv(std::sin(th))};
      }
      return dev_upload(t.data(), t.size(), da.bytes);
    };
    p.ff_twx = tw(Px);
    p.ff_twy = tw(Py);
    p.ff_twz = tw(Pz);
  }
  p.ff_ready = true;
}

// x and u as F6 for the float-float product (after ensure_work<double>)
void ensure_ff_work(mm_array* a, mm::Work& w, int nrhs) {
  if (w.x6 && w.u6) return;
  ++a->epoch;
  const size_t b = sizeof(mm::F6) * (size_t)a->da.N * nrhs;
  CU(cudaMalloc(&w.x6, b));
  CU(cudaMalloc(&w.u6, b));
  w.bytes += 2 * b;
}

template <typename R>
void ensure_pt(mm_array* a, mm::Work& w, int nrhs) {
  if (w.pt) return;
  ++a->epoch;
  CU(cudaMalloc(&w.pt, sizeof(typename mm::V2<R>::T) * (size_t)a->da.N * nrhs));
}

void ensure_tc_work(mm_array* a, mm::Work& w, int nrhs) {
  auto& da = a->da;
  size_t need = 0;
  const int TN = mm::tc_tile_n(), TK = mm::tc_tile_k();
  for (int64_t t = 0; t < da.n_types; ++t) {
    const int64_t ncols = da.n_of_type[t] * nrhs;
    const int64_t Np = (ncols + TN - 1) / TN * TN;
    const int64_t Kp = (mm::tc_k_split((int)da.Nh[t]) + da.Nh[t] + TK - 1) / TK * TK;
    need = std::max(need, (size_t)(Np * Kp));
  }
  if (w.bt_cap < need) {
    ++a->epoch;
    if (w.bt) cudaFree(w.bt);
    w.bt = nullptr;
    CU(cudaMalloc(&w.bt, sizeof(uint16_t) * need));
    // entries the packing never writes (between the halves) meet zero columns
    // of A; they start at zero so that they are finite
    CU(cudaMemset(w.bt, 0, sizeof(uint16_t) * need));
    w.bt_cap = need;
  }
  if (!w.err) {
    CU(cudaMalloc(&w.err, sizeof(int)));
    CU(cudaMemset(w.err, 0, sizeof(int)));
  }
}

// A bounded wait of the tensor-core GEMM or near field expired (checked where
// the call synchronises).  Both flags are read and cleared before either is
// reported, so that a later call does not report this call's expiry.
mm_status check_tc(mm_array* a) {
  int hg = 0, hn = 0;
  if (a->da.wf.err) {
    if (cudaMemcpy(&hg, a->da.wf.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MM_ECUDA;
    if (hg) cudaMemset(a->da.wf.err, 0, sizeof(int));
  }
  if (a->da.near_err) {
    if (cudaMemcpy(&hn, a->da.near_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MM_ECUDA;
    if (hn) cudaMemset(a->da.near_err, 0, sizeof(int));
  }
  if (hg) return fail(a->ctx, MM_ETIMEOUT, "a tensor-core GEMM wait expired; results of that product are invalid");
  if (hn)
    return fail(a->ctx, MM_ETIMEOUT, "a tensor-core near-field wait expired; results of that product are invalid");
  return MM_OK;
}

template <typename R>
void ensure_work(mm_array* a, mm::Work& w, int nrhs) {
  if (w.nrhs == nrhs) return;
  typedef typename mm::V2<R>::T C;
  ++a->epoch;
  for (void* q : {w.u, w.v, w.grid, w.spec, w.bt, (void*)w.err, w.pt, (void*)w.us, w.np, w.boxbuf, w.x6, w.u6})
    if (q) cudaFree(q);
  w = mm::Work();
  auto& da = a->da;
  size_t vec = sizeof(C) * (size_t)da.N * nrhs;
  size_t g = sizeof(C) * (size_t)4 * nrhs * da.grid[0] * da.grid[1] * da.grid[2];
  size_t s = sizeof(C) * (size_t)4 * nrhs * da.grid[0] * da.fft[1] * da.fft[2];
  CU(cudaMalloc(&w.u, vec));
  CU(cudaMalloc(&w.v, vec));
  CU(cudaMalloc(&w.grid, g));
  CU(cudaMalloc(&w.spec, s));
  w.bytes = 2 * vec + g + s;
  if (sizeof(R) == 8 && da.nnz > 0) {
    CU(cudaMalloc(&w.us, sizeof(double) * (size_t)da.N * nrhs));
    w.bytes += sizeof(double) * (size_t)da.N * nrhs;
  }
  if (nrhs >= 8 && da.gptr) {
    // the two-pass projection's per-element boxes (a tuner variant from 8 RHS on)
    const size_t bb = sizeof(C) * (size_t)da.n_elem * 4 * nrhs * da.box_nodes_max;
    CU(cudaMalloc(&w.boxbuf, bb));
    w.bytes += bb;
  }
  if (sizeof(R) == 4 && da.pf.nfb_tc && da.nfg_prows > 0) {
    // two planes for few right-hand sides (the k split of the tensor-core near field)
    w.np_parts = nrhs <= 8 ? 2 : 1;
    CU(cudaMalloc(&w.np, sizeof(float2) * (size_t)da.nfg_prows * nrhs * w.np_parts));
    w.bytes += sizeof(float2) * (size_t)da.nfg_prows * nrhs * w.np_parts;
  }
  w.nrhs = nrhs;
}

void free_prec_f(mm::DevPrec<float>& p) {
  if (p.nfb_tc) cudaFree(p.nfb_tc);
  for (auto& v : p.Atc)
    for (void* q : v) cudaFree(q);
  for (void* q : p.W) cudaFree(q);
  for (void* q : p.Pi) cudaFree(q);
  for (void* q : p.prj_tab) cudaFree(q);
  if (p.prj_types) cudaFree(p.prj_types);
  if (p.itp_types) cudaFree(p.itp_types);
  for (void* q : {p.val, p.Ghat, p.twx, p.twy, p.twz, p.nfb_val})
    if (q) cudaFree(q);
  for (void* q : p.PJ) cudaFree(q);
  for (void* q : p.WP) cudaFree(q);
  for (auto& v : p.AtcP)
    for (void* q : v) cudaFree(q);
}
void free_prec_d(mm::DevPrec<double>& p) {
  for (void* q : p.ffW) cudaFree(q);
  for (void* q : p.ff_Pi) cudaFree(q);
  for (void* q : {p.ff_nfb, p.ff_twx, p.ff_twy, p.ff_twz, p.ff_Ghat})
    if (q) cudaFree(q);
  for (void* q : p.PJ) cudaFree(q);
  for (void* q : p.WP) cudaFree(q);
  for (void* q : p.W3) cudaFree(q);
  for (void* q : p.WP3) cudaFree(q);
  for (void* q : p.W) cudaFree(q);
  for (void* q : p.Pi) cudaFree(q);
  for (void* q : {p.val, p.Ghat, p.twx, p.twy, p.twz, p.nfb_val})
    if (q) cudaFree(q);
}

}  // namespace

mm_array::~mm_array() {
  solver.reset();
  if (!on_device) return;
  cudaSetDevice(da.device);
  free_prec_f(da.pf);
  free_prec_d(da.pd);
  for (mm::Work* w : {&da.wf, &da.wd})
    for (void* q : {w->u, w->v, w->grid, w->spec, w->bt, (void*)w->err, w->pt, (void*)w->us, w->np, w->boxbuf,
                    w->x6, w->u6})
      if (q) cudaFree(q);
  for (auto* p : da.anc) cudaFree(p);
  for (auto* p : da.geo) cudaFree(p);
  for (auto* p : da.elems) cudaFree(p);
  for (auto* p : da.inv_ptr) cudaFree(p);
  for (auto* p : da.inv_ent) cudaFree(p);
  for (void* q : {(void*)da.gptr, (void*)da.gent})
    if (q) cudaFree(q);
  for (void* q : {(void*)da.off, (void*)da.boxorg, (void*)da.type_of, (void*)da.eoff, (void*)da.rowptr,
                  (void*)da.col, (void*)elem_of, (void*)geo_ptrs, (void*)d_ang, (void*)d_pol, hx, hy, (void*)d_offs,
                  (void*)d_dir})
    if (q) cudaFree(q);
  for (void* q : d_JE) cudaFree(q);
  for (void* q : d_T) cudaFree(q);
  for (void* q : {(void*)da.nfb_tptr32, (void*)da.nfb_tlist32, (void*)da.nfb_tptr128, (void*)da.nfb_tlist128,
                  (void*)da.nfb_arow})
    if (q) cudaFree(q);
  for (void* q : {(void*)da.nfb_na, (void*)da.nfb_nb, (void*)da.nfb_off, (void*)da.nfb_tptr, (void*)da.nfb_tlist,
                  (void*)da.nfb_perm, (void*)da.nfb_pa, (void*)da.nfb_pb})
    if (q) cudaFree(q);
  for (void* q : {da.nfg_dev, (void*)da.nfg_poff, (void*)da.nfg_prow, (void*)da.nfe_ptr, (void*)da.nfe_pair,
                  (void*)da.nfe_qb, (void*)da.nfe_order, (void*)da.nfb_tperm})
    if (q) cudaFree(q);
  if (da.side) cudaStreamDestroy(da.side);
  if (da.chain) cudaStreamDestroy(da.chain);
  if (ang_ev) cudaEventDestroy(ang_ev);
  if (d_pw) cudaFree(d_pw);
  for (void* q : d_Jf)
    if (q) cudaFree(q);
  for (void* q : d_Jhf)
    if (q) cudaFree(q);
  for (void* q : {d_volts, d_fu, d_pw2, (void*)d_gc})
    if (q) cudaFree(q);
  if (bst) cudaStreamDestroy(bst);
  for (cudaEvent_t e : {bev_done, bev_fork})
    if (e) cudaEventDestroy(e);
  if (pv_V) cudaFree(pv_V);
  if (pv_E) cudaFree(pv_E);
  if (da.tbase) cudaFree(da.tbase);
  for (cudaEvent_t e : {da.ev_fork, da.ev_join, da.ev_done})
    if (e) cudaEventDestroy(e);
}

extern "C" {

mm_status mm_ctx_create(int device, mm_ctx** out) {
  if (!out) return MM_EINVAL;
  *out = nullptr;
  auto* c = new (std::nothrow) mm_ctx();
  if (!c) return MM_ENOMEM;
  c->nthreads = std::max(1u, std::thread::hardware_concurrency());
  c->device = device;
  if (device >= 0) {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device >= n) {
      delete c;
      return MM_ECUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
      delete c;
      return MM_ECUDA;
    }
    if (!(prop.major == 10 && prop.minor == 3)) {  // built for sm_103a only
      delete c;
      return MM_EINVAL;
    }
  } else if (device != -1) {
    delete c;
    return MM_EINVAL;
  }
  *out = c;
  return MM_OK;
}

void mm_ctx_destroy(mm_ctx* ctx) { delete ctx; }

const char* mm_last_error(const mm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mm_status mm_ctx_set_threads(mm_ctx* ctx, int nthreads) {
  if (!ctx || nthreads < 1) return MM_EINVAL;
  ctx->nthreads = nthreads;
  return MM_OK;
}

mm_status mm_mesh_create(mm_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, mm_mesh** out) {
  if (!ctx || !xyz || !tri || !out) return fail(ctx, MM_EINVAL, "null argument");
  API_TRY
  auto m = std::make_unique<mm_mesh>();
  m->ctx = ctx;
  mm::build_mesh(m->m, xyz, nv, tri, nt);
  *out = m.release();
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_mesh_info(const mm_mesh* mesh, int64_t* n_rwg, int32_t* closed) {
  if (!mesh) return MM_EINVAL;
  if (n_rwg) *n_rwg = mesh->m.nrwg();
  if (closed) *closed = mesh->m.closed ? 1 : 0;
  return MM_OK;
}

void mm_mesh_destroy(mm_mesh* mesh) { delete mesh; }

mm_status mm_element_type_create(mm_ctx* ctx, const mm_mesh* scatterer, const mm_mesh* equiv, const mm_em_opts* opts,
                                 mm_type** out) {
  if (!ctx || !scatterer || !equiv || !opts || !out) return fail(ctx, MM_EINVAL, "null argument");
  if (!(opts->k0 > 0)) return fail(ctx, MM_EINVAL, "k0 must be positive");
  if (!equiv->m.closed) return fail(ctx, MM_EINVAL, "equivalent surface must be closed and outward-oriented");
  API_TRY
  auto t = std::make_unique<mm_type>();
  t->ctx = ctx;
  t->tm.scat = scatterer->m;
  t->tm.eq = equiv->m;
  t->tm.em.k = opts->k0;
  t->tm.em.eta0 = opts->eta0 > 0 ? opts->eta0 : 376.730313668;
  t->tm.em.nthreads = ctx->nthreads;
  mm::build_type(t->tm, ctx->device);
  *out = t.release();
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_type_matrix(const mm_type* type, int32_t which, double* out_host, int64_t* rows, int64_t* cols) {
  if (!type) return MM_EINVAL;
  const auto& tm = type->tm;
  const std::vector<mm::cd>* M = nullptr;
  int64_t r = 0, c = 0;
  switch (which) {
    case MM_MAT_M: M = &tm.M; r = tm.Nh; c = tm.Nh; break;
    case MM_MAT_D: M = &tm.D; r = tm.Nh; c = tm.Nh; break;
    case MM_MAT_T: M = &tm.T; r = tm.Nh; c = tm.N; break;
    case MM_MAT_A: M = &tm.A; r = tm.N; c = tm.N; break;
    case MM_MAT_B: M = &tm.B; r = tm.N; c = tm.Nh; break;
    case MM_MAT_GHH: M = &tm.GHH; r = tm.Nh; c = tm.Nh; break;
    case MM_MAT_GHE: M = &tm.GHE; r = tm.Nh; c = tm.Nh; break;
    case MM_MAT_PJ: M = &tm.PJ; r = tm.Nh; c = tm.Nh; break;
    default: return MM_EINVAL;
  }
  if (rows) *rows = r;
  if (cols) *cols = c;
  if (out_host) std::memcpy(out_host, M->data(), sizeof(mm::cd) * r * c);
  return MM_OK;
}

mm_status mm_type_info(const mm_type* type, int64_t* n_scat, int64_t* n_equiv) {
  if (!type) return MM_EINVAL;
  if (n_scat) *n_scat = type->tm.N;
  if (n_equiv) *n_equiv = type->tm.Nh;
  return MM_OK;
}

void mm_type_destroy(mm_type* type) { delete type; }

mm_status mm_array_create(mm_ctx* ctx, int64_t n_elem, const mm_type* const* types, const double* offsets_xyz,
                          const mm_aim_opts* opts, mm_array** out) {
  if (!ctx || !types || !offsets_xyz || !opts || !out || n_elem < 1) return fail(ctx, MM_EINVAL, "invalid argument");
  API_TRY
  auto a = std::make_unique<mm_array>();
  a->ctx = ctx;
  std::vector<int32_t> type_of(n_elem);
  std::vector<const mm::TypeModel*> tms;
  for (int64_t e = 0; e < n_elem; ++e) {
    if (!types[e]) return fail(ctx, MM_EINVAL, "null element type");
    auto it = std::find(a->types.begin(), a->types.end(), types[e]);
    if (it == a->types.end()) {
      type_of[e] = (int32_t)a->types.size();
      a->types.push_back(types[e]);
      tms.push_back(&types[e]->tm);
    } else {
      type_of[e] = (int32_t)(it - a->types.begin());
    }
  }
  mm::EM em = tms[0]->em;
  for (auto* t : tms)
    if (t->em.k != em.k || t->em.eta0 != em.eta0) return fail(ctx, MM_EINVAL, "element types differ in k0 or eta0");
  em.nthreads = ctx->nthreads;
  a->k0 = em.k;
  a->eta0 = em.eta0;
  a->offs.assign(n_elem + 1, 0);
  for (int64_t e = 0; e < n_elem; ++e) a->offs[e + 1] = a->offs[e] + tms[type_of[e]]->N;
  std::vector<mm::Vec3> offs(n_elem);
  for (int64_t e = 0; e < n_elem; ++e) offs[e] = {offsets_xyz[3 * e], offsets_xyz[3 * e + 1], offsets_xyz[3 * e + 2]};
  if (opts->near_csr < 0 || opts->near_csr > 2) return fail(ctx, MM_EINVAL, "near_csr must be 0, 1 or 2");
  mm::AimOpts ao{opts->h, opts->order, opts->n_nf, {opts->phase[0], opts->phase[1], opts->phase[2]}};
  {
    // tuning override: MACROAIM_NEAR=csr applies the near field as CSR rows (and needs them)
    const char* nm = std::getenv("MACROAIM_NEAR");
    const bool want = nm && std::string(nm) == "csr";
    // automatic on a device: a moderate CSR (values of both precisions and
    // columns within 8 GiB) is assembled for the complex128 products, which run
    // faster from CSR rows at GB300's FP64 rate than from the dense blocks
    if (opts->near_csr == 1 || (opts->near_csr == 0 && (ctx->device < 0 || want)))
      ao.csr_max_nnz = -1;
    else if (opts->near_csr == 2)
      ao.csr_max_nnz = 0;
    else
      ao.csr_max_nnz = ((int64_t)8 << 30) / 36;   // 8 + 24 value bytes + 4 column bytes
  }
  // near-field blocks filled on the context's device (host contexts: on the host;
  // MACROAIM_NEAR_FILL=host keeps the host fill on a device context)
  {
    const char* nf = std::getenv("MACROAIM_NEAR_FILL");
    ao.device = (nf && std::string(nf) == "host") ? -1 : ctx->device;
  }
  mm::build_array_host(a->ah, tms, type_of, offs, ao, em);
  auto& ah = a->ah;
  auto& da = a->da;
  da.N = ah.N;
  da.n_elem = n_elem;
  da.n_types = (int64_t)tms.size();
  da.nnz = ah.rowptr.empty() ? 0 : ah.rowptr[ah.N];
  for (int i = 0; i < 3; ++i) {
    da.grid[i] = (int)ah.grid[i];
    da.fft[i] = (int)ah.fft[i];
  }
  auto o1 = mm::stencil_1d(opts->order);
  da.n1 = (int)o1.size();
  da.S = da.n1 * da.n1 * da.n1;
  da.o1lo = o1.front();
  da.cA[0] = ah.c_A.real(); da.cA[1] = ah.c_A.imag();
  da.cphi[0] = ah.c_phi.real(); da.cphi[1] = ah.c_phi.imag();
  da.px = mm::make_plan(da.fft[0]);
  da.py = mm::make_plan(da.fft[1]);
  if (da.px.nst < 0 || da.py.nst < 0) throw mm::Error{MM_EINTERNAL, "FFT length without a radix plan"};
  if (da.fft[2] > 64 || da.grid[2] > 32)
    throw mm::Error{MM_EINVAL, "grid extent along z too large for the direct z transform (<= 32 nodes)"};
  if (ctx->device >= 0) {
    CU(cudaSetDevice(ctx->device));
    da.device = ctx->device;
    a->on_device = true;
    size_t& acc = da.bytes;
    std::vector<std::vector<int32_t>> elems(da.n_types);
    for (int64_t e = 0; e < n_elem; ++e) elems[type_of[e]].push_back((int32_t)e);
    std::vector<double*> gptr(da.n_types);
    for (int64_t t = 0; t < da.n_types; ++t) {
      const auto& ta = ah.tai[t];
      const auto& eq = tms[t]->eq;
      int64_t Nh = tms[t]->Nh;
      da.Nh.push_back(Nh);
      for (int i = 0; i < 3; ++i) da.box.push_back((int)ta.box_dim[i]);
      std::vector<int32_t> anc(3 * Nh);
      for (int64_t n = 0; n < Nh; ++n)
        for (int i = 0; i < 3; ++i) anc[3 * n + i] = (int32_t)(ta.anc[3 * n + i] - ta.box_lo[i]);
      da.anc.push_back(dev_upload(anc.data(), anc.size(), acc));
      std::vector<double> geo(13 * Nh);
      for (int64_t n = 0; n < Nh; ++n) {
        mm::Vec3 pa = eq.v[eq.edge_a[n]], pb = eq.v[eq.edge_b[n]], pp = eq.v[eq.vplus[n]], pm = eq.v[eq.vminus[n]];
        double g[13] = {pa.x, pa.y, pa.z, pb.x, pb.y, pb.z, pp.x, pp.y, pp.z, pm.x, pm.y, pm.z, eq.length[n]};
        std::copy(g, g + 13, &geo[13 * n]);
      }
      da.geo.push_back(dev_upload(geo.data(), geo.size(), acc));
      gptr[t] = da.geo.back();
      da.elems.push_back(dev_upload(elems[t].data(), elems[t].size(), acc));
      da.n_of_type.push_back((int64_t)elems[t].size());
      {
        // inverse stencil lists: for each node of the type's box, the (basis, stencil node) pairs touching it
        const int bx = (int)ta.box_dim[0], by = (int)ta.box_dim[1], bz = (int)ta.box_dim[2];
        const int nodes = bx * by * bz, n1 = da.n1, S = da.S;
        if (Nh >= 65536 || S >= 65536) throw mm::Error{MM_EINVAL, "element type too large for the projection lists"};
        std::vector<std::vector<int32_t>> lists(nodes);
        for (int64_t n = 0; n < Nh; ++n)
          for (int sn = 0; sn < S; ++sn) {
            const int ix = sn % n1, iy = (sn / n1) % n1, iz = sn / (n1 * n1);
            const int x = anc[3 * n] + da.o1lo + ix, y = anc[3 * n + 1] + da.o1lo + iy, z = anc[3 * n + 2] + da.o1lo + iz;
            lists[(x * by + y) * bz + z].push_back((int32_t)(n | (sn << 16)));
          }
        std::vector<int32_t> ptr(nodes + 1, 0), ent;
        for (int q = 0; q < nodes; ++q) {
          ptr[q + 1] = ptr[q] + (int32_t)lists[q].size();
          ent.insert(ent.end(), lists[q].begin(), lists[q].end());
        }
        da.inv_ptr.push_back(dev_upload(ptr.data(), ptr.size(), acc));
        da.inv_ent.push_back(dev_upload(ent.data(), ent.size(), acc));
        da.inv_len.push_back((int32_t)ent.size());
        a->inv_ent_h.push_back(ent);
      }
    }
    a->geo_ptrs = dev_upload(gptr.data(), gptr.size(), acc);
    da.off = dev_upload(ah.off.data(), ah.off.size(), acc);
    std::vector<int64_t> tbase(da.n_types + 1, 0);
    for (int64_t t = 0; t < da.n_types; ++t) tbase[t + 1] = tbase[t] + da.Nh[t];
    da.tbase = dev_upload(tbase.data(), tbase.size(), acc);
    std::vector<int32_t> boxorg(3 * n_elem), eo;
    std::vector<double> eoff(3 * n_elem);
    for (int64_t e = 0; e < n_elem; ++e) {
      const auto& ta = ah.tai[type_of[e]];
      for (int i = 0; i < 3; ++i) boxorg[3 * e + i] = (int32_t)(ta.box_lo[i] + ah.base[3 * e + i]);
      eoff[3 * e] = offs[e].x; eoff[3 * e + 1] = offs[e].y; eoff[3 * e + 2] = offs[e].z;
    }
    da.boxorg = dev_upload(boxorg.data(), boxorg.size(), acc);
    {
      // the two-pass projection's gather lists: per grid node, the (element,
      // local box node) pairs whose box covers it, for box nodes that receive
      // a projection weight
      int nmax = 1;
      std::vector<std::vector<char>> live(da.n_types);
      for (int64_t t = 0; t < da.n_types; ++t) {
        const auto& ta = ah.tai[t];
        const int nodes = (int)(ta.box_dim[0] * ta.box_dim[1] * ta.box_dim[2]);
        nmax = std::max(nmax, nodes);
        live[t].assign(nodes, 0);
      }
      {
        // a node is live if some (basis, stencil point) of the type lands on it
        for (int64_t t = 0; t < da.n_types; ++t) {
          const auto& ta = ah.tai[t];
          const int by = (int)ta.box_dim[1], bz = (int)ta.box_dim[2], n1 = da.n1;
          for (int64_t n = 0; n < ta.Nh; ++n)
            for (int sn = 0; sn < da.S; ++sn) {
              const int ix = sn % n1, iy = (sn / n1) % n1, iz = sn / (n1 * n1);
              const int x = (int)(ta.anc[3 * n] - ta.box_lo[0]) + da.o1lo + ix;
              const int y = (int)(ta.anc[3 * n + 1] - ta.box_lo[1]) + da.o1lo + iy;
              const int z = (int)(ta.anc[3 * n + 2] - ta.box_lo[2]) + da.o1lo + iz;
              live[t][(x * by + y) * bz + z] = 1;
            }
        }
      }
      const int64_t Ny = ah.grid[1], Nz = ah.grid[2], ng = ah.grid[0] * Ny * Nz;
      std::vector<int32_t> cnt(ng + 1, 0);
      auto each = [&](const std::function<void(int64_t, int64_t)>& f) {
        for (int64_t e = 0; e < n_elem; ++e) {
          const int t = type_of[e];
          const auto& ta = ah.tai[t];
          const int bx = (int)ta.box_dim[0], by = (int)ta.box_dim[1], bz = (int)ta.box_dim[2];
          for (int lx = 0; lx < bx; ++lx)
            for (int ly = 0; ly < by; ++ly)
              for (int lz = 0; lz < bz; ++lz) {
                const int node = (lx * by + ly) * bz + lz;
                if (!live[t][node]) continue;
                const int64_t g = ((boxorg[3 * e] + lx) * Ny + (boxorg[3 * e + 1] + ly)) * Nz + boxorg[3 * e + 2] + lz;
                f(g, e * nmax + node);
              }
        }
      };
      each([&](int64_t g, int64_t) { ++cnt[g + 1]; });
      for (int64_t g = 0; g < ng; ++g) cnt[g + 1] += cnt[g];
      std::vector<int64_t> ent(cnt[ng]);
      std::vector<int32_t> fillp(cnt.begin(), cnt.end() - 1);
      each([&](int64_t g, int64_t v) { ent[fillp[g]++] = v; });
      da.box_nodes_max = nmax;
      da.gptr = dev_upload(cnt.data(), cnt.size(), acc);
      da.gent = dev_upload(ent.data(), ent.size(), acc);
    }
    da.type_of = dev_upload(type_of.data(), type_of.size(), acc);
    da.eoff = dev_upload(eoff.data(), eoff.size(), acc);
    std::vector<int32_t> eof(ah.N);
    for (int64_t e = 0; e < n_elem; ++e)
      for (int64_t n = ah.off[e]; n < ah.off[e + 1]; ++n) eof[n] = (int32_t)e;
    a->elem_of = dev_upload(eof.data(), eof.size(), acc);
    if (!ah.rowptr.empty()) {
      // rows padded to multiples of 4 entries; pad columns point at the row itself
      std::vector<int64_t> rp(ah.N + 1, 0);
      for (int64_t i = 0; i < ah.N; ++i) rp[i + 1] = rp[i] + (ah.rowptr[i + 1] - ah.rowptr[i] + 3) / 4 * 4;
      std::vector<int32_t> cl(rp[ah.N]);
      for (int64_t i = 0; i < ah.N; ++i) {
        int64_t len = ah.rowptr[i + 1] - ah.rowptr[i];
        for (int64_t k = 0; k < rp[i + 1] - rp[i]; ++k) cl[rp[i] + k] = k < len ? ah.col[ah.rowptr[i] + k] : (int32_t)i;
      }
      da.nnz_padded = rp[ah.N];
      da.rowptr = dev_upload(rp.data(), rp.size(), acc);
      da.col = dev_upload(cl.data(), cl.size(), acc);
    }
    {
      // near field as blocks: shapes, dense offsets, non-zero k tiles per
      // 64-row tile, and the element pairs of each lattice offset
      const auto& nb = ah.nf_blocks;
      const int64_t nbk = (int64_t)nb.size();
      // per type: bases sorted by anchor (y, then x, then z), so that the near
      // pairs of a block gather into fewer 64 x 16 tiles
      a->nf_perm.assign(da.n_types, {});
      a->nf_iperm.assign(da.n_types, {});
      std::vector<int32_t> perm_all, perm_off(da.n_types, 0);
      for (int64_t t = 0; t < da.n_types; ++t) {
        const auto& ta = ah.tai[t];
        std::vector<int32_t> pm(ta.Nh);
        for (int64_t i = 0; i < ta.Nh; ++i) pm[i] = (int32_t)i;
        std::stable_sort(pm.begin(), pm.end(), [&](int32_t x, int32_t y) {
          const int64_t* ax = &ta.anc[3 * x];
          const int64_t* ay = &ta.anc[3 * y];
          if (ax[1] != ay[1]) return ax[1] < ay[1];
          if (ax[0] != ay[0]) return ax[0] < ay[0];
          return ax[2] < ay[2];
        });
        std::vector<int32_t> ip(ta.Nh);
        for (int64_t i = 0; i < ta.Nh; ++i) ip[pm[i]] = (int32_t)i;
        perm_off[t] = (int32_t)perm_all.size();
        perm_all.insert(perm_all.end(), pm.begin(), pm.end());
        a->nf_perm[t] = std::move(pm);
        a->nf_iperm[t] = std::move(ip);
      }
      int64_t maxNa = 0;
      for (const auto& b : nb)
        if (!b.ptr.empty()) maxNa = std::max(maxNa, b.Na);
      std::vector<int32_t> na(nbk, 0), nbv(nbk, 0);
      std::vector<int64_t> boff(nbk, 0);
      int64_t o = 0;
      for (int64_t q = 0; q < nbk; ++q) {
        const auto& b = nb[q];
        na[q] = (int32_t)b.Na;
        nbv[q] = (int32_t)b.Nb;
        boff[q] = o;
        if (!b.ptr.empty()) o += b.Na * b.Nb;
      }
      // per (block, row tile of TM rows) the 16-column k tiles holding a non-zero,
      // for the kernel's two row-tile heights (64 and 32)
      auto tile_lists = [&](int TM, int& nmt, std::vector<int32_t>& tptr, std::vector<int32_t>& tl) {
        nmt = (int)((maxNa + TM - 1) / TM);
        tptr.assign(nbk * std::max(nmt, 1) + 1, 0);
        tl.clear();
        std::vector<char> used;
        for (int64_t q = 0; q < nbk; ++q) {
          const auto& b = nb[q];
          for (int mt = 0; mt < nmt; ++mt) {
            tptr[q * nmt + mt] = (int32_t)tl.size();
            if (b.ptr.empty() || (int64_t)mt * TM >= b.Na) continue;
            used.assign((size_t)((b.Nb + 15) / 16), 0);
            const auto &pa = a->nf_perm[b.ta], &ib = a->nf_iperm[b.tb];
            for (int64_t m = (int64_t)mt * TM; m < std::min<int64_t>(b.Na, (int64_t)mt * TM + TM); ++m)
              for (int64_t e = b.ptr[pa[m]]; e < b.ptr[pa[m] + 1]; ++e) used[ib[b.col[e]] / 16] = 1;
            for (size_t kt = 0; kt < used.size(); ++kt)
              if (used[kt]) tl.push_back((int32_t)kt);
          }
        }
        tptr[nbk * nmt] = (int32_t)tl.size();
      };
      int nmt = 0, nmt32 = 0, nmt128 = 0;
      std::vector<int32_t> tptr, tl, tptr32, tl32, tptr128, tl128;
      tile_lists(64, nmt, tptr, tl);
      tile_lists(32, nmt32, tptr32, tl32);
      tile_lists(128, nmt128, tptr128, tl128);
      // rows of the tensor-core block layout: the non-empty blocks one after another
      a->nfb_arow_h.assign(nbk, 0);
      int64_t trows = 0, tpitch = 0;
      for (int64_t q = 0; q < nbk; ++q) {
        a->nfb_arow_h[q] = (int32_t)trows;
        if (nb[q].ptr.empty()) continue;
        trows += nb[q].Na;
        tpitch = std::max<int64_t>(tpitch, (2 * nb[q].Nb + 31) / 32 * 32);
      }
      da.nfb_entries = o;
      if (o > 0) {
        da.nfb_nmt = nmt;
        da.nfb_na = dev_upload(na.data(), na.size(), acc);
        da.nfb_nb = dev_upload(nbv.data(), nbv.size(), acc);
        da.nfb_off = dev_upload(boff.data(), boff.size(), acc);
        da.nfb_tptr = dev_upload(tptr.data(), tptr.size(), acc);
        da.nfb_tlist = dev_upload(tl.data(), tl.size(), acc);
        da.nfb_nmt32 = nmt32;
        da.nfb_tptr32 = dev_upload(tptr32.data(), tptr32.size(), acc);
        da.nfb_tlist32 = dev_upload(tl32.data(), tl32.size(), acc);
        if (2 * trows <= 0x7fffffffLL && tpitch * 4 < ((int64_t)1 << 40)) {
          da.nfb_nmt128 = nmt128;
          da.nfb_tptr128 = dev_upload(tptr128.data(), tptr128.size(), acc);
          da.nfb_tlist128 = dev_upload(tl128.data(), tl128.size(), acc);
          da.nfb_arow = dev_upload(a->nfb_arow_h.data(), a->nfb_arow_h.size(), acc);
          da.nfb_tc_rows = (int)trows;
          da.nfb_tc_pitch = (int)tpitch;
        }
        std::vector<int32_t> bpa(nbk, 0), bpb(nbk, 0);
        for (int64_t q = 0; q < nbk; ++q) {
          bpa[q] = perm_off[nb[q].ta];
          bpb[q] = perm_off[nb[q].tb];
        }
        da.nfb_perm = dev_upload(perm_all.data(), perm_all.size(), acc);
        da.nfb_pa = dev_upload(bpa.data(), bpa.size(), acc);
        da.nfb_pb = dev_upload(bpb.data(), bpb.size(), acc);
        std::vector<std::vector<int2>> groups(nbk);
        for (int64_t e = 0; e < n_elem; ++e)
          for (const auto& pr : ah.nf_nbr[e])
            if (!nb[pr.second].ptr.empty()) groups[pr.second].push_back(make_int2((int)e, (int)pr.first));
        std::vector<int2> allp;
        for (int64_t q = 0; q < nbk; ++q) {
          if (groups[q].empty()) continue;
          mm::DevArray::NfGroup ng;
          ng.q = (int)q;
          ng.Na = (int)nb[q].Na;
          ng.first_pair = (int64_t)allp.size();
          ng.npairs = (int64_t)groups[q].size();
          allp.insert(allp.end(), groups[q].begin(), groups[q].end());
          da.nfg.push_back(ng);
        }
        static_assert(sizeof(mm::DevArray::NfGroup) == 24, "group record layout shared with the kernel");
        std::vector<longlong2> poff(allp.size());
        for (size_t i = 0; i < allp.size(); ++i) {
          poff[i].x = ah.off[allp[i].x];
          poff[i].y = ah.off[allp[i].y];
        }
        da.nfg_poff = dev_upload(poff.data(), poff.size(), acc);
        {
          // partial sums of the tensor-core near field: one slice of the row
          // type's N^ rows per pair, and per element the pairs it is the row of
          std::vector<int64_t> prow(allp.size());
          std::vector<int32_t> eptr(n_elem + 1, 0), epair(allp.size());
          int64_t rows = 0;
          for (const auto& ng : da.nfg)
            for (int64_t k = 0; k < ng.npairs; ++k) {
              prow[ng.first_pair + k] = rows;
              rows += ng.Na;
            }
          for (const auto& pr : allp) ++eptr[pr.x + 1];
          for (int64_t e = 0; e < n_elem; ++e) eptr[e + 1] += eptr[e];
          std::vector<int32_t> fillp(eptr.begin(), eptr.end() - 1);
          for (size_t k = 0; k < allp.size(); ++k) epair[fillp[allp[k].x]++] = (int32_t)k;
          std::vector<int32_t> tperm(perm_off.begin(), perm_off.end());
          // per entry of epair: (block q, column element's unknown offset), for
          // the direct form that walks an element's pairs in this order
          std::vector<int32_t> pair_q(allp.size());
          for (const auto& ng : da.nfg)
            for (int64_t k = 0; k < ng.npairs; ++k) pair_q[ng.first_pair + k] = ng.q;
          std::vector<longlong2> qb(allp.size());
          for (size_t i = 0; i < allp.size(); ++i) {
            qb[i].x = pair_q[epair[i]];
            qb[i].y = ah.off[allp[epair[i]].y];
          }
          da.nfe_qb = dev_upload(qb.data(), qb.size(), acc);
          std::vector<int32_t> order(n_elem);
          for (int64_t e = 0; e < n_elem; ++e) order[e] = (int32_t)e;
          std::stable_sort(order.begin(), order.end(),
                           [&](int32_t x, int32_t y) { return ah.type_of[x] < ah.type_of[y]; });
          da.nfe_order = dev_upload(order.data(), order.size(), acc);
          da.nfg_prows = rows;
          da.nfg_prow = dev_upload(prow.data(), prow.size(), acc);
          da.nfe_ptr = dev_upload(eptr.data(), eptr.size(), acc);
          da.nfe_pair = dev_upload(epair.data(), epair.size(), acc);
          da.nfb_tperm = dev_upload(tperm.data(), tperm.size(), acc);
        }
        da.nfg_dev = dev_upload(reinterpret_cast<const unsigned char*>(da.nfg.data()),
                                sizeof(mm::DevArray::NfGroup) * da.nfg.size(), acc);
        // tuning override: MACROAIM_NEAR=csr (CSR rows, when assembled)
        if (const char* nm = std::getenv("MACROAIM_NEAR"))
          if (std::string(nm) == "csr") da.near_mode = 2;
        // tuning override: MACROAIM_NEAR_SHAPE="shape,ksplit" fixes the block kernel's shape
        if (const char* ns = std::getenv("MACROAIM_NEAR_SHAPE")) {
          int sh = -1, ks = 1;
          if (std::sscanf(ns, "%d,%d", &sh, &ks) >= 1 && sh >= 0 && sh < mm::kNearShapes && ks >= 1 && ks <= 16) {
            da.near_force_shape = sh;
            da.near_force_ks = ks;
          }
        }
      }
    }
    // tuning override: MACROAIM_GRID_TUNE=0 keeps the grid stages' default schedules
    if (const char* gt = std::getenv("MACROAIM_GRID_TUNE"))
      if (std::string(gt) == "0") da.tune_grid = false;
    // tuning override: MACROAIM_GRID_SCHED="p,i" fixes the projection and interpolation variants
    if (const char* gs = std::getenv("MACROAIM_GRID_SCHED")) {
      int gp = -1, gi = -1;
      if (std::sscanf(gs, "%d,%d", &gp, &gi) == 2 && gp >= 0 && gp <= 3 && gi >= 0 && gi <= 3) {
        da.grid_force_p = gp;
        da.grid_force_i = gi;
      }
    }
    // tuning override: MACROAIM_FF_SHAPE="gemm,near" fixes the float-float kernels' tile shapes
    if (const char* fs = std::getenv("MACROAIM_FF_SHAPE")) {
      int fg = 0, fn = 0;
      if (std::sscanf(fs, "%d,%d", &fg, &fn) == 2 && fg >= 0 && fg <= 2 && fn >= 0 && fn <= 3) {
        da.ff_gemm_shape = fg;
        da.ff_near_shape = fn;
      }
    }
    upload_precision<float>(a.get(), da.pf);
    CU(mm::kernels_init(da));
    // the near field's own stream (MACROAIM_NEAR_OVERLAP=0: one stream, in order)
    const char* ov = std::getenv("MACROAIM_NEAR_OVERLAP");
    if ((da.nfb_entries > 0 || da.nnz > 0) && !(ov && std::string(ov) == "0")) {
      int lo = 0, hi = 0;   // numerically lower = served first
      CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      CU(cudaStreamCreateWithPriority(&da.side, cudaStreamNonBlocking, lo));
      CU(cudaStreamCreateWithPriority(&da.chain, cudaStreamNonBlocking, hi));
      CU(cudaEventCreateWithFlags(&da.ev_fork, cudaEventDisableTiming));
      CU(cudaEventCreateWithFlags(&da.ev_join, cudaEventDisableTiming));
      CU(cudaEventCreateWithFlags(&da.ev_done, cudaEventDisableTiming));
    }
  }
  *out = a.release();
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_array_info_get(const mm_array* a, mm_array_info* info) {
  if (!a || !info) return MM_EINVAL;
  info->n_unknowns = a->ah.N;
  info->n_elem = a->ah.n_elem;
  info->n_types = (int64_t)a->types.size();
  for (int i = 0; i < 3; ++i) {
    info->grid[i] = a->ah.grid[i];
    info->fft[i] = a->ah.fft[i];
  }
  info->nnz_near = a->ah.nnz_near;
  info->device_bytes = (int64_t)a->da.bytes;
  info->n_scat_unknowns = a->offs.empty() ? 0 : a->offs.back();
  info->n_near_blocks = 0;
  info->near_block_entries = 0;
  for (const auto& b : a->ah.nf_blocks)
    if (!b.ptr.empty()) {
      ++info->n_near_blocks;
      info->near_block_entries += b.Na * b.Nb;
    }
  info->near_format = (a->da.near_mode == 2 && a->da.nnz > 0) ? 1 : 0;
  return MM_OK;
}

mm_status mm_array_footprint(const mm_array* a, int32_t nrhs, int32_t precision, int32_t restart, size_t* bytes) {
  if (!a || !bytes || nrhs < 1 || restart < 1) return MM_EINVAL;
  const auto& da = a->da;
  size_t cs = (precision == MM_C128 || precision == MM_C128_FF) ? 16 : 8;
  size_t vec = cs * (size_t)da.N * nrhs;
  size_t g = cs * (size_t)4 * nrhs * da.grid[0] * da.grid[1] * da.grid[2];
  size_t s = cs * (size_t)4 * nrhs * da.grid[0] * da.fft[1] * da.fft[2];
  size_t kry = 16 * (size_t)da.N * nrhs * (restart + 4) + 16 * (size_t)da.N * nrhs;
  // partial sums of the tensor-core near field (complex64 products)
  size_t np = da.pf.nfb_tc ? sizeof(float) * 2 * (size_t)da.nfg_prows * nrhs : 0;
  size_t bb = nrhs >= 8 ? cs * (size_t)da.n_elem * 4 * nrhs * da.box_nodes_max : 0;   // two-pass projection
  // x and u as F6 (float-float products: MM_C128_FF, and the refinement residuals of complex64 solves)
  size_t f6 = precision != MM_C128 ? 2 * sizeof(mm::F6) * (size_t)da.N * nrhs : 0;
  *bytes = 2 * vec + g + s + kry + np + bb + f6;
  return MM_OK;
}

mm_status mm_array_export(const mm_array* a, int32_t which, void* out, int64_t* count) {
  if (!a || !count) return MM_EINVAL;
  const auto& ah = a->ah;
  switch (which) {
    case MM_EXPORT_ANCHORS: {
      *count = 3 * ah.N;
      if (out) {
        int64_t* o = static_cast<int64_t*>(out);
        for (int64_t e = 0; e < ah.n_elem; ++e) {
          const auto& ta = ah.tai[ah.type_of[e]];
          for (int64_t n = 0; n < ta.Nh; ++n)
            for (int i = 0; i < 3; ++i) o[3 * (ah.off[e] + n) + i] = ta.anc[3 * n + i] + ah.base[3 * e + i];
        }
      }
      return MM_OK;
    }
    case MM_EXPORT_PI: {
      const int S = ah.tai[0].S;
      *count = ah.N * S * 4;
      if (out) {
        double* o = static_cast<double*>(out);
        for (int64_t e = 0; e < ah.n_elem; ++e) {
          const auto& ta = ah.tai[ah.type_of[e]];
          std::memcpy(o + ah.off[e] * S * 4, ta.Pi.data(), sizeof(double) * ta.Pi.size());
        }
      }
      return MM_OK;
    }
    case MM_EXPORT_NEAR_PTR:
    case MM_EXPORT_NEAR_COL:
    case MM_EXPORT_NEAR_VAL:
      if (ah.rowptr.empty() && ah.nnz_near > 0)
        return fail(a->ctx, MM_EINVAL, "near-field CSR not assembled (create the array with near_csr = 1)");
      break;
    default:
      break;
  }
  switch (which) {
    case MM_EXPORT_NEAR_PTR:
      *count = (int64_t)ah.rowptr.size();
      if (out) std::memcpy(out, ah.rowptr.data(), sizeof(int64_t) * ah.rowptr.size());
      return MM_OK;
    case MM_EXPORT_NEAR_COL:
      *count = (int64_t)ah.col.size();
      if (out) std::memcpy(out, ah.col.data(), sizeof(int32_t) * ah.col.size());
      return MM_OK;
    case MM_EXPORT_NEAR_VAL:
      *count = 2 * (int64_t)ah.val.size();
      if (out) std::memcpy(out, ah.val.data(), sizeof(mm::cd) * ah.val.size());
      return MM_OK;
    case MM_EXPORT_GHAT:
      *count = 2 * (int64_t)ah.Ghat.size();
      if (out) std::memcpy(out, ah.Ghat.data(), sizeof(mm::cd) * ah.Ghat.size());
      return MM_OK;
    default:
      return MM_EINVAL;
  }
}

void mm_array_destroy(mm_array* a) {
  if (a) drop_graphs_of(a);
  delete a;
}

mm_status mm_batch_graphs(const mm_array* array, int32_t* count) {
  if (!count) return MM_EINVAL;
  std::lock_guard<std::mutex> lk(g_graph_mu);
  int32_t n = 0;
  for (const auto& g : g_graphs)
    if (!array || std::find(g.arrays.begin(), g.arrays.end(), array) != g.arrays.end()) ++n;
  *count = n;
  return MM_OK;
}

mm_status mm_apply(mm_array* a, int32_t nrhs, const void* x_dev, void* y_dev, int32_t precision, void* stream) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || !x_dev || !y_dev || x_dev == y_dev) return fail(ctx, MM_EINVAL, "invalid apply arguments");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (precision == MM_C64 || precision == MM_C64_BF16 || precision == MM_C64_F16) {
    const int mode = precision == MM_C64 ? 0 : (precision == MM_C64_BF16 ? 1 : 2);
    ensure_work<float>(a, a->da.wf, nrhs);
    if (mode) {
      upload_tc(a, mode);
      ensure_tc_work(a, a->da.wf, nrhs);
    }
    e = mm::matvec<float>(a->da, a->da.pf, a->da.wf, nrhs, x_dev, y_dev, st, mode);
  } else if (precision == MM_C128 || precision == MM_C128_FF) {
    upload_precision<double>(a, a->da.pd);
    ensure_work<double>(a, a->da.wd, nrhs);
    unsigned fl = 0;
    if (precision == MM_C128_FF) {
      upload_ff(a);
      ensure_ff_work(a, a->da.wd, nrhs);
      fl = mm::kMvFF;
    }
    e = mm::matvec<double>(a->da, a->da.pd, a->da.wd, nrhs, x_dev, y_dev, st, 0, false, fl);
  } else {
    return fail(ctx, MM_EINVAL, "unknown precision");
  }
  if (e != cudaSuccess) return fail(ctx, MM_ECUDA, std::string("matvec: ") + cudaGetErrorString(e));
  a->settled.insert({nrhs, precision});
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_apply_batch(mm_array* const* arrays, int32_t count, const int32_t* nrhs, const void* const* x_dev,
                         void* const* y_dev, int32_t precision, void* stream) {
  if (!arrays || count < 1 || !nrhs || !x_dev || !y_dev) return MM_EINVAL;
  for (int32_t i = 0; i < count; ++i) {
    if (!arrays[i] || !arrays[i]->on_device || nrhs[i] < 1 || !x_dev[i] || !y_dev[i] || x_dev[i] == y_dev[i])
      return arrays[i] ? fail(arrays[i]->ctx, MM_EINVAL, "invalid batch entry " + std::to_string(i)) : MM_EINVAL;
    for (int32_t j = 0; j < i; ++j)
      if (arrays[j] == arrays[i])
        return fail(arrays[i]->ctx, MM_EINVAL, "an array appears twice in the batch (it serves one product at a time)");
    if (arrays[i]->da.device != arrays[0]->da.device)
      return fail(arrays[i]->ctx, MM_EINVAL, "the arrays of a batch must be on one device");
  }
  mm_ctx* ctx = arrays[0]->ctx;
  API_TRY
  const int dev = arrays[0]->da.device;
  if (dev < 0 || dev >= 64) return fail(ctx, MM_EINVAL, "device index out of range");
  CU(cudaSetDevice(dev));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // fork (from stream `from`): every array's product on its own stream, joined back into `from`
  auto launch_all = [&](cudaStream_t from) -> mm_status {
    if (!arrays[0]->bev_fork) CU(cudaEventCreateWithFlags(&arrays[0]->bev_fork, cudaEventDisableTiming));
    CU(cudaEventRecord(arrays[0]->bev_fork, from));
    for (int32_t i = 0; i < count; ++i) {
      mm_array* a = arrays[i];
      if (!a->bst) {
        CU(cudaStreamCreateWithFlags(&a->bst, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&a->bev_done, cudaEventDisableTiming));
      }
      CU(cudaStreamWaitEvent(a->bst, arrays[0]->bev_fork, 0));
      const mm_status s = mm_apply(a, nrhs[i], x_dev[i], y_dev[i], precision, a->bst);
      if (s != MM_OK) {
        if (a != arrays[0]) ctx->err = a->ctx->err;
        return s;
      }
      CU(cudaEventRecord(a->bev_done, a->bst));
    }
    for (int32_t i = 0; i < count; ++i) CU(cudaStreamWaitEvent(from, arrays[i]->bev_done, 0));
    return MM_OK;
  };
  // a graph applies when no array records stage events and every array has
  // done a product of this width and precision
  bool graphable = true;
  for (int32_t i = 0; i < count && graphable; ++i)
    graphable = !arrays[i]->da.prof.on && arrays[i]->settled.count({nrhs[i], precision}) > 0;
  auto matches = [&](const BatchGraph& g) {
    if (g.precision != precision || g.device != dev || (int32_t)g.arrays.size() != count) return false;
    for (int32_t i = 0; i < count; ++i)
      if (g.arrays[i] != arrays[i] || g.nrhs[i] != nrhs[i] || g.x[i] != x_dev[i] || g.y[i] != y_dev[i] ||
          g.epochs[i] != arrays[i]->epoch)
        return false;
    return true;
  };
  if (graphable) {
    cudaGraphExec_t exec = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_graph_mu);
      for (const auto& g : g_graphs)
        if (matches(g)) {
          exec = g.exec;
          break;
        }
    }
    if (!g_cap_stream[dev]) {
      CU(cudaStreamCreateWithFlags(&g_cap_stream[dev], cudaStreamNonBlocking));
      CU(cudaEventCreateWithFlags(&g_cap_in[dev], cudaEventDisableTiming));
      CU(cudaEventCreateWithFlags(&g_cap_out[dev], cudaEventDisableTiming));
    }
    cudaStream_t cs = g_cap_stream[dev];
    if (exec == nullptr) {
      // capture the launch sequence (nothing runs during capture), then replay it below
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      mm_status ls = MM_OK;
      if (ce == cudaSuccess) {
        ls = launch_all(cs);
        ce = cudaStreamEndCapture(cs, &graph);
      }
      if (ce == cudaSuccess && ls == MM_OK && graph != nullptr &&
          cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        BatchGraph g;
        for (int32_t i = 0; i < count; ++i) {
          g.arrays.push_back(arrays[i]);
          g.nrhs.push_back(nrhs[i]);
          g.x.push_back(x_dev[i]);
          g.y.push_back(y_dev[i]);
          g.epochs.push_back(arrays[i]->epoch);
        }
        g.precision = precision;
        g.device = dev;
        g.exec = exec;
        std::lock_guard<std::mutex> lk(g_graph_mu);
        if (g_graphs.size() >= kMaxGraphs) {
          cudaGraphExecDestroy(g_graphs.front().exec);
          g_graphs.erase(g_graphs.begin());
        }
        g_graphs.push_back(g);
      } else {
        exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();   // a failed capture leaves no error behind: the kernels run below
    }
    if (exec != nullptr) {
      CU(cudaEventRecord(g_cap_in[dev], st));
      CU(cudaStreamWaitEvent(cs, g_cap_in[dev], 0));
      CU(cudaGraphLaunch(exec, cs));
      CU(cudaEventRecord(g_cap_out[dev], cs));
      CU(cudaStreamWaitEvent(st, g_cap_out[dev], 0));
      return MM_OK;
    }
  }
  return launch_all(st);
  API_CATCH(ctx)
}

mm_status mm_apply_host(mm_array* a, int32_t nrhs, const void* x_host, void* y_host, int32_t precision) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || !x_host || !y_host) return fail(ctx, MM_EINVAL, "invalid apply arguments");
  if (precision < MM_C64 || precision > MM_C128_FF) return fail(ctx, MM_EINVAL, "unknown precision");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  size_t bytes = ((precision == MM_C128 || precision == MM_C128_FF) ? 16 : 8) * (size_t)a->da.N * nrhs;
  if (a->h_cap < bytes) {
    if (a->hx) cudaFree(a->hx);
    if (a->hy) cudaFree(a->hy);
    a->hx = a->hy = nullptr;
    CU(cudaMalloc(&a->hx, bytes));
    CU(cudaMalloc(&a->hy, bytes));
    a->h_cap = bytes;
  }
  CU(cudaMemcpyAsync(a->hx, x_host, bytes, cudaMemcpyHostToDevice, 0));
  mm_status s = mm_apply(a, nrhs, a->hx, a->hy, precision, nullptr);
  if (s != MM_OK) return s;
  CU(cudaMemcpyAsync(y_host, a->hy, bytes, cudaMemcpyDeviceToHost, 0));
  CU(cudaStreamSynchronize(0));
  return check_tc(a);
  API_CATCH(ctx)
}

mm_status mm_rhs_planewave(mm_array* a, int32_t nrhs, const double* theta, const double* phi, const int32_t* pol,
                           void* V_dev, int32_t precision, void* stream) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || !theta || !phi || !pol || !V_dev) return fail(ctx, MM_EINVAL, "invalid excitation arguments");
  for (int j = 0; j < nrhs; ++j)
    if (pol[j] != 0 && pol[j] != 1) return fail(ctx, MM_EINVAL, "pol must be 0 (theta) or 1 (phi)");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (a->ang_cap < nrhs) {
    if (a->d_ang) cudaFree(a->d_ang);
    if (a->d_pol) cudaFree(a->d_pol);
    a->d_ang = nullptr;
    a->d_pol = nullptr;
    CU(cudaMalloc(&a->d_ang, sizeof(double) * 2 * nrhs));
    CU(cudaMalloc(&a->d_pol, sizeof(int32_t) * nrhs));
    a->ang_cap = nrhs;
  }
  // the copies come from pageable staging (copied out before the calls
  // return), after the previous excitation kernel, on whatever stream it ran
  if (a->ang_ev) CU(cudaStreamWaitEvent(st, a->ang_ev, 0));
  std::vector<double> ang(2 * nrhs);
  std::copy(theta, theta + nrhs, ang.begin());
  std::copy(phi, phi + nrhs, ang.begin() + nrhs);
  std::vector<int32_t> pl(pol, pol + nrhs);
  CU(cudaMemcpyAsync(a->d_ang, ang.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(a->d_pol, pl.data(), sizeof(int32_t) * nrhs, cudaMemcpyHostToDevice, st));
  int64_t nloc = 0;
  for (int64_t t = 0; t < a->da.n_types; ++t) nloc += a->da.Nh[t];
  const int64_t pw_need = (nloc + a->da.n_elem) * nrhs;
  if (a->pw_cap < pw_need) {
    if (a->d_pw) cudaFree(a->d_pw);
    a->d_pw = nullptr;
    a->pw_cap = 0;
    CU(cudaMalloc(&a->d_pw, sizeof(double2) * (size_t)pw_need));
    a->pw_cap = pw_need;
  }
  mm::Rule r7 = mm::rule_tri7();
  mm::QuadRule q;
  q.n = r7.n();
  for (int i = 0; i < q.n; ++i) {
    q.b0[i] = r7.b0[i]; q.b1[i] = r7.b1[i]; q.b2[i] = r7.b2[i]; q.w[i] = r7.w[i];
  }
  cudaError_t e;
  if (precision == MM_C64)
    e = mm::rhs_planewave<float>(a->da, a->elem_of, a->geo_ptrs, nrhs, a->d_ang, a->d_ang + nrhs, a->d_pol, a->k0, q,
                                 V_dev, a->d_pw, st);
  else if (precision == MM_C128)
    e = mm::rhs_planewave<double>(a->da, a->elem_of, a->geo_ptrs, nrhs, a->d_ang, a->d_ang + nrhs, a->d_pol, a->k0,
                                  q, V_dev, a->d_pw, st);
  else
    return fail(ctx, MM_EINVAL, "unknown precision");
  if (e != cudaSuccess) return fail(ctx, MM_ECUDA, std::string("excitation: ") + cudaGetErrorString(e));
  if (!a->ang_ev) CU(cudaEventCreateWithFlags(&a->ang_ev, cudaEventDisableTiming));
  CU(cudaEventRecord(a->ang_ev, st));
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_solve(mm_array* a, int32_t nrhs, const void* V_dev, void* E_dev, const mm_solve_opts* opts,
                   mm_solve_stats* stats, void* stream) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || !V_dev || !E_dev || !opts || V_dev == E_dev) return fail(ctx, MM_EINVAL, "invalid solve arguments");
  if (!(opts->tol > 0) || opts->restart < 1 || opts->max_iter < 1) return fail(ctx, MM_EINVAL, "invalid solve options");
  if (opts->precision < MM_C64 || opts->precision > MM_C64_F16) return fail(ctx, MM_EINVAL, "unknown precision");
  if (opts->orth < 0 || opts->orth > 3) return fail(ctx, MM_EINVAL, "orth must be 0, 1, 2 or 3");
  if (opts->precond < 0 || opts->precond > 1) return fail(ctx, MM_EINVAL, "precond must be 0 or 1");
  if (opts->fp64 < 0 || opts->fp64 > 1) return fail(ctx, MM_EINVAL, "fp64 must be 0 or 1");
  if (opts->refine && opts->precision == MM_C128)
    return fail(ctx, MM_EINVAL, "refinement needs a complex64 operator precision");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!a->solver) a->solver = std::make_unique<mm::Solver>();
  mm::Solver& S = *a->solver;
  S.prof = &a->da.prof;
  // Arnoldi mode of the kernel: 1 one pass, 2 selective second pass, 3 two passes
  S.orth = opts->orth != 0 ? opts->orth : (opts->refine ? 1 : 2);
  mm::Status s = S.ensure(a->da.N, nrhs, opts->restart);
  if (s.code != MM_OK) return fail(ctx, s.code, s.msg);
  upload_precision<double>(a, a->da.pd);
  ensure_work<double>(a, a->da.wd, nrhs);
  ensure_work<float>(a, a->da.wf, nrhs);
  // refinement residuals and the inner Arnoldi products in float-float
  // arithmetic (the default) or FP64
  const bool ff_res = opts->refine && opts->fp64 == 0;
  // tuning override: MACROAIM_FF_ARNOLDI=0 keeps the inner Arnoldi in FP64 (the residual stays float-float)
  {
    const char* fa = std::getenv("MACROAIM_FF_ARNOLDI");
    S.ff_arnoldi = ff_res && !(fa && std::string(fa) == "0");
  }
  if (ff_res) {
    upload_ff(a);
    ensure_ff_work(a, a->da.wd, nrhs);
  }
  const int mode = opts->precision == MM_C64_BF16 ? 1 : (opts->precision == MM_C64_F16 ? 2 : 0);
  if (mode) {
    upload_tc(a, mode);
    ensure_tc_work(a, a->da.wf, nrhs);
  }
  mm_array* arr = a;
  const bool pj = opts->precond == 1;
  if (pj) {
    // right preconditioning: GMRES runs on Z P^-1 (P = the elements' own blocks)
    upload_pj<double>(a, a->da.pd);
    upload_pj<float>(a, a->da.pf);
    if (mode) upload_tc(a, mode, true);
    ensure_pt<double>(a, a->da.wd, nrhs);
  }
  // With refinement the solution itself is kept (the FP64 residual uses the
  // plain operator) and each inner correction y is mapped to P^-1 y in
  // complex64, the precision it was solved in; without refinement GMRES runs on
  // Z P^-1 throughout and the result is mapped once at the end.
  const bool pj_outer = pj && !opts->refine;
  // Z P^-1 x is one product with the fused macromodel matrices [M PJ; D PJ]
  S.op64 = [arr, nrhs, pj_outer, ff_res](const double2* in, double2* out, cudaStream_t s2) -> mm::Status {
    cudaError_t e = mm::matvec<double>(arr->da, arr->da.pd, arr->da.wd, nrhs, in, out, s2, 0, pj_outer,
                                       ff_res ? mm::kMvFF : 0u);
    if (e != cudaSuccess) return {MM_ECUDA, cudaGetErrorString(e)};
    return {MM_OK, ""};
  };
  S.op32 = [arr, nrhs, mode, pj](const void* in, void* out, cudaStream_t s2) -> mm::Status {
    cudaError_t e = mm::matvec<float>(arr->da, arr->da.pf, arr->da.wf, nrhs, in, out, s2, mode, pj);
    if (e != cudaSuccess) return {MM_ECUDA, cudaGetErrorString(e)};
    return {MM_OK, ""};
  };
  S.correction32 = nullptr;
  if (pj && opts->refine)
    S.correction32 = [arr, nrhs](const void* in, void* out, cudaStream_t s2) -> mm::Status {
      cudaError_t e = mm::precond_apply<float>(arr->da, arr->da.pf, nrhs, in, out, s2);
      if (e != cudaSuccess) return {MM_ECUDA, cudaGetErrorString(e)};
      return {MM_OK, ""};
    };
  int iters = 0, refs = 0;
  double relres = 0;
  bool conv = false;
  s = S.solve(static_cast<const double2*>(V_dev), static_cast<double2*>(E_dev), opts->tol,
              opts->precision == MM_C128 ? MM_C128 : MM_C64,
              opts->refine, opts->inner_tol > 0 ? opts->inner_tol : 1e-2, opts->max_iter, iters, refs, relres, conv,
              st);
  if (pj_outer && (s.code == MM_OK || s.code == MM_ENOCONV)) {
    // the solution of Z P^-1 y = V is y; E = P^-1 y
    CU(mm::precond_apply<double>(a->da, a->da.pd, nrhs, E_dev, a->da.wd.pt, st));
    CU(cudaMemcpyAsync(E_dev, a->da.wd.pt, sizeof(double2) * (size_t)a->da.N * nrhs, cudaMemcpyDeviceToDevice, st));
  }
  if (stats) {
    stats->iterations = iters;
    stats->matvecs = S.matvecs;
    stats->refinements = refs;
    stats->converged = conv ? 1 : 0;
    stats->rel_residual = relres;
  }
  if (s.code != MM_OK) return fail(ctx, s.code, s.msg);
  {
    // bounded waits of the tensor-core GEMM and near field
    const mm_status t = check_tc(a);
    if (t != MM_OK) return t;
  }
  if (!conv) return fail(ctx, MM_ENOCONV, "GMRES reached max_iter before the tolerance");
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_solve_planewave_host(mm_array* a, int32_t nrhs, const double* theta, const double* phi,
                                  const int32_t* pol, double* E_host, const mm_solve_opts* opts,
                                  mm_solve_stats* stats) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || !theta || !phi || !pol || !E_host || !opts) return fail(ctx, MM_EINVAL, "invalid solve arguments");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  const size_t bytes = sizeof(double2) * (size_t)a->da.N * nrhs;
  if (a->pv_cap < bytes) {
    if (a->pv_V) cudaFree(a->pv_V);
    if (a->pv_E) cudaFree(a->pv_E);
    a->pv_V = a->pv_E = nullptr;
    a->pv_cap = 0;
    CU(cudaMalloc(&a->pv_V, bytes));
    CU(cudaMalloc(&a->pv_E, bytes));
    a->pv_cap = bytes;
  }
  mm_status s = mm_rhs_planewave(a, nrhs, theta, phi, pol, a->pv_V, MM_C128, nullptr);
  if (s != MM_OK) return s;
  s = mm_solve(a, nrhs, a->pv_V, a->pv_E, opts, stats, nullptr);
  if (s != MM_OK && s != MM_ENOCONV) return s;
  const std::string msg = s == MM_ENOCONV ? ctx->err : std::string();
  CU(cudaMemcpy(E_host, a->pv_E, bytes, cudaMemcpyDeviceToHost));
  if (s == MM_ENOCONV) return fail(ctx, s, msg);
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_array_tuning(const mm_array* a, int32_t nrhs, int32_t precision, int32_t* choices, float* project_ms,
                          float* interp_ms) {
  if (!a || !choices || nrhs < 1) return MM_EINVAL;
  if (precision != MM_C64 && precision != MM_C128) return MM_EINVAL;
  const auto key = std::make_pair((int)nrhs, precision == MM_C128 ? 8 : 4);
  const auto nt = a->da.near_tune.find(key);
  const auto gt = a->da.grid_tune.find(key);
  if (nt == a->da.near_tune.end() && gt == a->da.grid_tune.end()) return MM_EINVAL;
  choices[0] = nt != a->da.near_tune.end() ? nt->second.first : -1;
  choices[1] = nt != a->da.near_tune.end() ? nt->second.second : -1;
  choices[2] = gt != a->da.grid_tune.end() ? gt->second.project : -1;
  choices[3] = gt != a->da.grid_tune.end() ? gt->second.interp : -1;
  const bool has = gt != a->da.grid_tune.end();
  for (int i = 0; i < 4; ++i)
    if (project_ms)
      project_ms[i] = has && i < (int)gt->second.project_ms.size() ? gt->second.project_ms[i] : -1.f;
  for (int i = 0; i < 4; ++i)
    if (interp_ms)
      interp_ms[i] = has && i < (int)gt->second.interp_ms.size() ? gt->second.interp_ms[i] : -1.f;
  return MM_OK;
}

mm_status mm_array_near_shape(const mm_array* a, int32_t nrhs, int32_t precision, int32_t* shape,
                              int32_t* ksplit) {
  if (!a || !shape || !ksplit || nrhs < 1) return MM_EINVAL;
  if (precision != MM_C64 && precision != MM_C128) return MM_EINVAL;
  const auto it = a->da.near_tune.find(std::make_pair((int)nrhs, precision == MM_C128 ? 8 : 4));
  if (it == a->da.near_tune.end()) return MM_EINVAL;
  *shape = it->second.first;
  *ksplit = it->second.second;
  return MM_OK;
}

mm_status mm_currents(mm_array* a, int32_t nrhs, const void* E_dev, void* J_dev, void* Jhat_dev, void* stream) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || !E_dev) return fail(ctx, MM_EINVAL, "invalid currents arguments");
  if (!J_dev && !Jhat_dev) return MM_OK;
  API_TRY
  CU(cudaSetDevice(a->da.device));
  auto& da = a->da;
  if (a->d_JE.empty()) {
    size_t acc = 0;
    for (int64_t t = 0; t < da.n_types; ++t) {
      const auto& tm = a->types[t]->tm;
      a->d_JE.push_back(dev_upload(tm.JE.data(), tm.JE.size(), acc));
      a->d_T.push_back(dev_upload(tm.T.data(), tm.T.size(), acc));
    }
    if (!a->d_offs) a->d_offs = dev_upload(a->offs.data(), a->offs.size(), acc);
    da.bytes += acc;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* J = J_dev;
  void* tmp = nullptr;
  if (!J) {   // J^ alone still needs J
    CU(cudaMallocAsync(&tmp, sizeof(double2) * (size_t)a->offs.back() * nrhs, st));
    J = tmp;
  }
  cudaError_t e = cudaSuccess;
  for (int64_t t = 0; t < da.n_types && e == cudaSuccess; ++t) {
    const auto& tm = a->types[t]->tm;
    e = mm::elem_gemm(a->d_JE[t], (int)tm.N, (int)tm.Nh, da.elems[t], (int)da.n_of_type[t], nrhs, da.off, E_dev,
                      a->d_offs, J, st);
    if (e == cudaSuccess && Jhat_dev)
      e = mm::elem_gemm(a->d_T[t], (int)tm.Nh, (int)tm.N, da.elems[t], (int)da.n_of_type[t], nrhs, a->d_offs, J,
                        da.off, Jhat_dev, st);
  }
  if (tmp) cudaFreeAsync(tmp, st);
  if (e != cudaSuccess) return fail(ctx, MM_ECUDA, std::string("currents: ") + cudaGetErrorString(e));
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_type_set_feed(mm_type* type, int32_t n_edges, const int64_t* rwg, const double* direction) {
  if (!type) return MM_EINVAL;
  mm_ctx* ctx = type->ctx;
  auto& tm = type->tm;
  if (n_edges < 1 || !rwg || !direction) return fail(ctx, MM_EINVAL, "invalid feed arguments");
  const mm::Mesh& ms = tm.scat;
  const mm::Vec3 d{direction[0], direction[1], direction[2]};
  if (!(mm::norm(d) > 0)) return fail(ctx, MM_EINVAL, "feed direction must be non-zero");
  API_TRY
  const int64_t N = tm.N;
  std::vector<mm::cd> f(N, mm::cd(0, 0));
  for (int32_t i = 0; i < n_edges; ++i) {
    const int64_t g = rwg[i];
    if (g < 0 || g >= N) return fail(ctx, MM_EINVAL, "feed edge out of range");
    // s = sign(d . n_g), n_g the in-plane normal of edge g from its T+ to its T- triangle
    const mm::Vec3 a = ms.v[ms.edge_a[g]], b = ms.v[ms.edge_b[g]];
    const mm::Vec3 e = (1.0 / mm::norm(b - a)) * (b - a);
    const int64_t tp = ms.tplus[g], tq = ms.tminus[g];
    const mm::Vec3 cp = (1.0 / 3.0) * (ms.tv(tp, 0) + ms.tv(tp, 1) + ms.tv(tp, 2));
    const mm::Vec3 cq = (1.0 / 3.0) * (ms.tv(tq, 0) + ms.tv(tq, 1) + ms.tv(tq, 2));
    const mm::Vec3 c = cq - cp;
    const mm::Vec3 n = c - mm::dot(c, e) * e;
    const double sd = mm::dot(n, d);
    if (sd == 0) return fail(ctx, MM_EINVAL, "feed direction parallel to a gap edge");
    f[g] += (sd > 0 ? 1.0 : -1.0) * ms.length[g];
  }
  // J_f = -A^-1 f, J^_f = T J_f (FP64)
  mm::LU lu;
  mm::lu_factor(lu, tm.A, N);
  std::vector<mm::cd> Jf(f);
  mm::lu_solve(lu, Jf, 1, ctx->nthreads);
  for (auto& z : Jf) z = -z;
  std::vector<mm::cd> Jhf(tm.Nh, mm::cd(0, 0));
  for (int64_t m = 0; m < tm.Nh; ++m) {
    mm::cd acc(0, 0);
    for (int64_t n = 0; n < N; ++n) acc += tm.T[m * N + n] * Jf[n];
    Jhf[m] = acc;
  }
  type->feed_Jf = std::move(Jf);
  type->feed_Jhf = std::move(Jhf);
  type->fed = true;
  return MM_OK;
  API_CATCH(ctx)
}

namespace {

// Device copies of the feed vectors of the array's types and of the volts.
void upload_feeds(mm_array* a, const double* volts, int nrhs, cudaStream_t st) {
  auto& da = a->da;
  if (a->d_Jf.empty()) {
    size_t acc = 0;
    for (int64_t t = 0; t < da.n_types; ++t) {
      const mm_type* ty = a->types[t];
      a->d_Jf.push_back(ty->fed ? dev_upload(ty->feed_Jf.data(), ty->feed_Jf.size(), acc) : nullptr);
      a->d_Jhf.push_back(ty->fed ? dev_upload(ty->feed_Jhf.data(), ty->feed_Jhf.size(), acc) : nullptr);
    }
    da.bytes += acc;
  }
  if (a->d_offs == nullptr) {
    size_t acc = 0;
    a->d_offs = dev_upload(a->offs.data(), a->offs.size(), acc);
    da.bytes += acc;
  }
  const size_t vb = sizeof(double2) * (size_t)da.n_elem * nrhs;
  if (a->volts_cap < vb) {
    if (a->d_volts) cudaFree(a->d_volts);
    a->d_volts = nullptr;
    a->volts_cap = 0;
    CU(cudaMalloc(&a->d_volts, vb));
    a->volts_cap = vb;
  }
  CU(cudaMemcpyAsync(a->d_volts, volts, vb, cudaMemcpyHostToDevice, st));
}

bool any_fed(const mm_array* a) {
  for (const mm_type* t : a->types)
    if (t->fed) return true;
  return false;
}

}  // namespace

mm_status mm_rhs_deltagap(mm_array* a, int32_t nrhs, const double* volts, void* V_dev, void* stream) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || !volts || !V_dev) return fail(ctx, MM_EINVAL, "invalid excitation arguments");
  if (!any_fed(a)) return fail(ctx, MM_EINVAL, "no element type of the array has a feed (mm_type_set_feed)");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto& da = a->da;
  upload_precision<double>(a, da.pd);
  ensure_work<double>(a, da.wd, nrhs);
  upload_feeds(a, volts, nrhs, st);
  // u = J^_f V per driven element (zero elsewhere), then V^_eff = -G u
  const size_t ub = sizeof(double2) * (size_t)da.N * nrhs;
  if (a->fu_cap < ub) {
    if (a->d_fu) cudaFree(a->d_fu);
    a->d_fu = nullptr;
    a->fu_cap = 0;
    CU(cudaMalloc(&a->d_fu, ub));
    a->fu_cap = ub;
  }
  void* u = a->d_fu;
  CU(cudaMemsetAsync(u, 0, ub, st));
  for (int64_t t = 0; t < da.n_types; ++t)
    if (a->d_Jhf[t]) CU(mm::feed_axpy(a->d_Jhf[t], (int)da.Nh[t], da.elems[t], (int)da.n_of_type[t], nrhs, da.off,
                                      a->d_volts, u, false, st));
  CU(mm::matvec<double>(da, da.pd, da.wd, nrhs, u, V_dev, st, 0, false, mm::kMvUInput));
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_currents_fed(mm_array* a, int32_t nrhs, const void* E_dev, const double* volts, void* J_dev,
                          void* Jhat_dev, void* stream) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!volts) return fail(ctx, MM_EINVAL, "invalid currents arguments");
  mm_status s = mm_currents(a, nrhs, E_dev, J_dev, Jhat_dev, stream);
  if (s != MM_OK) return s;
  if (!J_dev && !Jhat_dev) return MM_OK;
  API_TRY
  CU(cudaSetDevice(a->da.device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto& da = a->da;
  upload_feeds(a, volts, nrhs, st);
  for (int64_t t = 0; t < da.n_types; ++t) {
    if (!a->d_Jf[t]) continue;
    if (J_dev)
      CU(mm::feed_axpy(a->d_Jf[t], (int)a->types[t]->tm.N, da.elems[t], (int)da.n_of_type[t], nrhs, a->d_offs,
                       a->d_volts, J_dev, true, st));
    if (Jhat_dev)
      CU(mm::feed_axpy(a->d_Jhf[t], (int)da.Nh[t], da.elems[t], (int)da.n_of_type[t], nrhs, da.off, a->d_volts,
                       Jhat_dev, true, st));
  }
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_rhs_planewave_ground(mm_array* a, int32_t nrhs, const double* theta, const double* phi,
                                  const int32_t* pol, double z_ground, void* V_dev, int32_t precision, void* stream) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || !theta || !phi || !pol || !V_dev) return fail(ctx, MM_EINVAL, "invalid excitation arguments");
  if (precision != MM_C64 && precision != MM_C128) return fail(ctx, MM_EINVAL, "unknown precision");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t cs = precision == MM_C128 ? 16 : 8;
  const size_t bytes = cs * (size_t)a->da.N * nrhs;
  if (a->pw2_cap < bytes) {
    if (a->d_pw2) cudaFree(a->d_pw2);
    a->d_pw2 = nullptr;
    a->pw2_cap = 0;
    CU(cudaMalloc(&a->d_pw2, bytes));
    a->pw2_cap = bytes;
  }
  if (a->gc_cap < nrhs) {
    if (a->d_gc) cudaFree(a->d_gc);
    a->d_gc = nullptr;
    a->gc_cap = 0;
    CU(cudaMalloc(&a->d_gc, sizeof(double) * 2 * nrhs));
    a->gc_cap = nrhs;
  }
  // the image of a plane wave arriving from (theta, phi) with polarisation p is
  // the plane wave arriving from (pi - theta, phi) with polarisation S p =
  // +theta^ (p = theta^) or -phi^ (p = phi^), times exp(2 j k0 z_g cos theta)
  std::vector<double> th2(nrhs), c(2 * nrhs);
  for (int j = 0; j < nrhs; ++j) {
    th2[j] = M_PI - theta[j];
    const double s = pol[j] == 0 ? 1.0 : -1.0;
    const double arg = 2.0 * a->k0 * z_ground * std::cos(theta[j]);
    c[2 * j] = s * std::cos(arg);
    c[2 * j + 1] = s * std::sin(arg);
  }
  mm_status r = mm_rhs_planewave(a, nrhs, theta, phi, pol, V_dev, precision, stream);
  if (r != MM_OK) return r;
  r = mm_rhs_planewave(a, nrhs, th2.data(), phi, pol, a->d_pw2, precision, stream);
  if (r != MM_OK) return r;
  CU(cudaMemcpyAsync(a->d_gc, c.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, st));
  CU(mm::rhs_combine(precision == MM_C64, a->da.N, nrhs, a->d_gc, a->d_pw2, V_dev, st));
  // the factors come from pageable host memory: the copy is staged before the
  // call returns, so c may go out of scope
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_farfield(mm_array* a, int32_t nrhs, const void* Jhat_dev, int64_t ndir, const double* theta,
                      const double* phi, void* F_dev, void* stream) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || nrhs > 65535 || !Jhat_dev || ndir < 0 || ndir > 2147483647LL || (ndir > 0 && (!theta || !phi)) ||
      !F_dev)
    return fail(ctx, MM_EINVAL, "invalid far-field arguments");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (a->dir_cap < ndir) {
    if (a->d_dir) cudaFree(a->d_dir);
    a->d_dir = nullptr;
    CU(cudaMalloc(&a->d_dir, sizeof(double) * 2 * (size_t)ndir));
    a->dir_cap = ndir;
  }
  std::vector<double> dirs(2 * (size_t)ndir);
  std::copy(theta, theta + ndir, dirs.begin());
  std::copy(phi, phi + ndir, dirs.begin() + ndir);
  CU(cudaMemcpyAsync(a->d_dir, dirs.data(), sizeof(double) * 2 * (size_t)ndir, cudaMemcpyHostToDevice, st));
  int64_t nloc = 0;
  for (int64_t t = 0; t < a->da.n_types; ++t) nloc += a->da.Nh[t];
  const int64_t pw_need = (nloc + a->da.n_elem) * nrhs;
  if (a->pw_cap < pw_need) {
    if (a->d_pw) cudaFree(a->d_pw);
    a->d_pw = nullptr;
    a->pw_cap = 0;
    CU(cudaMalloc(&a->d_pw, sizeof(double2) * (size_t)pw_need));
    a->pw_cap = pw_need;
  }
  mm::Rule r7 = mm::rule_tri7();
  mm::QuadRule q;
  q.n = r7.n();
  for (int i = 0; i < q.n; ++i) {
    q.b0[i] = r7.b0[i]; q.b1[i] = r7.b1[i]; q.b2[i] = r7.b2[i]; q.w[i] = r7.w[i];
  }
  cudaError_t e = mm::farfield(a->da, a->elem_of, a->geo_ptrs, nrhs, Jhat_dev, ndir, a->d_dir, a->d_dir + ndir, a->k0,
                               a->eta0, q, F_dev, st);
  if (e != cudaSuccess) return fail(ctx, MM_ECUDA, std::string("far field: ") + cudaGetErrorString(e));
  CU(cudaStreamSynchronize(st));   // the host staging of the directions is released on return
  return MM_OK;
  API_CATCH(ctx)
}

mm_status mm_rcs(mm_array* a, int32_t nrhs, const void* Jhat_dev, int64_t ndir, const double* theta, const double* phi,
                 double* sigma_host) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!sigma_host) return fail(ctx, MM_EINVAL, "null sigma");
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  void* F = nullptr;
  CU(cudaMalloc(&F, sizeof(double2) * 3 * (size_t)std::max<int64_t>(ndir, 1) * nrhs));
  mm_status s = mm_farfield(a, nrhs, Jhat_dev, ndir, theta, phi, F, nullptr);
  if (s == MM_OK) {
    std::vector<double2> h(3 * (size_t)ndir * nrhs);
    cudaError_t e = cudaMemcpy(h.data(), F, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      cudaFree(F);
      return fail(ctx, MM_ECUDA, std::string("rcs copy: ") + cudaGetErrorString(e));
    }
    for (int64_t i = 0; i < ndir * nrhs; ++i) {
      double p = 0;
      for (int c = 0; c < 3; ++c) p += h[3 * i + c].x * h[3 * i + c].x + h[3 * i + c].y * h[3 * i + c].y;
      sigma_host[i] = 4.0 * M_PI * p;
    }
  }
  cudaFree(F);
  return s;
  API_CATCH(ctx)
}

mm_status mm_profile_enable(mm_array* a, int32_t enable) {
  if (!a) return MM_EINVAL;
  if (!a->on_device) return fail(a->ctx, MM_EINVAL, "array has no device (host-only context)");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  for (auto& r : a->da.prof.recs) {
    cudaEventSynchronize(r.b);
  }
  a->da.prof.reset();
  a->da.prof.on = enable != 0;
  return MM_OK;
  API_CATCH(a->ctx)
}

mm_status mm_profile_stages(mm_array* a, uint32_t stage_mask) {
  if (!a) return MM_EINVAL;
  a->da.prof.mask = stage_mask & 0xFFu;
  return MM_OK;
}

mm_status mm_profile_read(mm_array* a, int32_t precision, double* ms, int64_t* launches) {
  if (!a || !ms || !launches || precision < -1 || precision > 1) return MM_EINVAL;
  if (!a->on_device) return fail(a->ctx, MM_EINVAL, "array has no device (host-only context)");
  API_TRY
  CU(cudaSetDevice(a->da.device));
  // slots 0-7: complex64 stages and the (FP64) Krylov stage; 8-14: complex128 stages
  auto wanted = [&](int slot) {
    if (slot == MM_STAGE_KRYLOV) return true;
    if (precision == MM_C64) return slot < 8;
    if (precision == MM_C128) return slot >= 8;
    return true;
  };
  for (int i = 0; i < MM_STAGE_COUNT; ++i) {
    ms[i] = 0;
    launches[i] = 0;
  }
  for (int slot = 0; slot < 16; ++slot)
    if (wanted(slot)) launches[slot % 8] += a->da.prof.launches[slot];
  for (auto& r : a->da.prof.recs) {
    if (!wanted(r.stage)) continue;
    CU(cudaEventSynchronize(r.b));
    float t = 0;
    CU(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.stage % 8] += t;
  }
  return MM_OK;
  API_CATCH(a->ctx)
}

}  // extern "C"

// ---- allocation-free product ---------------------------------------------------
// Scratch for mm_apply_noalloc: a static device array in this translation unit.
// Host code must not take its address directly (that is a host-side stand-in);
// the device address comes from cudaGetSymbolAddress, looked up once per device.
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::mutex g_noalloc_mutex;
std::map<int, void*> g_noalloc_ptr;

size_t align256(size_t b) { return (b + 255) / 256 * 256; }
}  // namespace

extern "C" mm_status mm_apply_noalloc(mm_array* a, int32_t nrhs, const void* x_dev, void* y_dev, int32_t precision,
                                      void* stream) {
  if (!a) return MM_EINVAL;
  mm_ctx* ctx = a->ctx;
  if (!a->on_device) return fail(ctx, MM_EINVAL, "array has no device (host-only context)");
  if (nrhs < 1 || !x_dev || !y_dev || x_dev == y_dev) return fail(ctx, MM_EINVAL, "invalid apply arguments");
  if (precision != MM_C64 && precision != MM_C128) return fail(ctx, MM_EINVAL, "unknown precision");
  if (precision == MM_C128 && !a->da.pd.ready)
    return fail(ctx, MM_EINVAL,
                "complex128 operator not resident: call mm_apply or mm_solve at complex128 once before");
  API_TRY
  const auto& da = a->da;
  const size_t cs = precision == MM_C128 ? 16 : 8;
  const size_t vec = align256(cs * (size_t)da.N * nrhs);
  const size_t grid = align256(cs * (size_t)4 * nrhs * da.grid[0] * da.grid[1] * da.grid[2]);
  const size_t spec = align256(cs * (size_t)4 * nrhs * da.grid[0] * da.fft[1] * da.fft[2]);
  // complex64 with tensor-core near-field blocks: their partial sums too
  const size_t npart1 = precision == MM_C64 && da.pf.nfb_tc && da.nfg_prows > 0
                            ? align256(sizeof(float2) * (size_t)da.nfg_prows * nrhs)
                            : 0;
  // a second plane (the k split of the tensor-core near field) when it fits
  const int parts = nrhs <= 8 && 2 * vec + grid + spec + 2 * npart1 <= kNoAllocScratchBytes ? 2 : 1;
  const size_t npart = npart1 * parts;
  const size_t need = 2 * vec + grid + spec + npart;
  if (need > kNoAllocScratchBytes)
    return fail(ctx, MM_EINVAL,
                "mm_apply_noalloc needs " + std::to_string(need) + " bytes of scratch; the static maximum is " +
                    std::to_string(kNoAllocScratchBytes) + " bytes (use mm_apply)");
  cudaError_t e = cudaSetDevice(da.device);
  if (e != cudaSuccess) return fail(ctx, MM_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    auto it = g_noalloc_ptr.find(da.device);
    if (it == g_noalloc_ptr.end()) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(ctx, MM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      it = g_noalloc_ptr.emplace(da.device, p).first;
    }
    base = static_cast<unsigned char*>(it->second);
  }
  mm::Work w;
  w.nrhs = nrhs;
  w.u = base;
  w.v = base + vec;
  w.grid = base + 2 * vec;
  w.spec = base + 2 * vec + grid;
  w.np = npart ? base + 2 * vec + grid + spec : nullptr;
  w.np_parts = parts;
  w.bytes = need;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // no stage events (they are created on demand) and no timing of near-field
  // kernel shapes (it synchronises): an untuned right-hand-side count takes
  // the size rule
  const unsigned flags = mm::kMvNoTune | mm::kMvNoProfile;
  if (precision == MM_C64)
    e = mm::matvec<float>(a->da, a->da.pf, w, nrhs, x_dev, y_dev, st, 0, false, flags);
  else
    e = mm::matvec<double>(a->da, a->da.pd, w, nrhs, x_dev, y_dev, st, 0, false, flags);
  if (e != cudaSuccess) return fail(ctx, MM_ECUDA, std::string("matvec: ") + cudaGetErrorString(e));
  return MM_OK;
  API_CATCH(ctx)
}

// ---- testing hook of the bounded tensor-core waits ------------------------------
extern "C" mm_status mm_test_tc_stall(int32_t ms) {
  if (ms < 0) return MM_EINVAL;
  mm::tc_set_stall(ms);
  return MM_OK;
}
