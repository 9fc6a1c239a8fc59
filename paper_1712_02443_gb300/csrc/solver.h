// Batched GMRES with FP64 Arnoldi and FP64 iterative refinement (device side).
#pragma once

#include <complex>
#include <functional>
#include <string>
#include <vector>

#include "device.h"
#include "macroaim.h"

namespace mm {

struct Status {
  mm_status code;
  std::string msg;
};

// Quadrature rule passed by value to kernels (at most 16 points).
struct QuadRule {
  int n;
  double b0[16], b1[16], b2[16], w[16];
};

class Solver {
 public:
  // operators on device vectors of the current (N, r): complex128 and complex64
  std::function<Status(const double2*, double2*, cudaStream_t)> op64;
  std::function<Status(const void*, void*, cudaStream_t)> op32;
  // optional: maps each refinement correction (complex64 in -> out) before it is
  // added to the solution, e.g. a right preconditioner applied to the inner
  // GMRES's solution in the precision of the inner solve
  std::function<Status(const void*, void*, cudaStream_t)> correction32;
  int matvecs = 0;
  Profiler* prof = nullptr;   // optional stage profiler (Krylov kernels)
  int orth = 2;               // 1 one pass, 2 selective second pass, 3 two passes
  // complex64 inner solves keep the Krylov basis as float-float values and take
  // the Arnoldi products on the FP32 pipe (when the cooperative step fits)
  bool ff_arnoldi = true;

  ~Solver() { release(); }
  Status ensure(int64_t N, int r, int m);
  void release();
  Status solve(const double2* b, double2* x, double tol, int prec, int refine, double inner_tol, int max_iter,
               int& iters, int& refinements, double& relres, bool& converged, cudaStream_t st);
  size_t bytes() const { return bytes_; }

 private:
  Status apply(const double2* in, double2* out, int prec, cudaStream_t st);
  Status dots(const double2* V, int64_t vstride, int nvec, const double2* w, double2* out, cudaStream_t st);
  Status norms(const double2* a, std::vector<double>& out, cudaStream_t st);
  Status gmres(const double2* b, double2* x, bool x_zero, const std::vector<double>& tol_abs, int prec, int max_iter,
               int& iters, std::vector<double>& res, cudaStream_t st);
  int64_t N_ = 0;
  int r_ = 0, m_ = 0, nblk_ = 1;
  int nblk_ff_ = 1;            // blocks of the float-float step (two per SM at large sizes when they fit)
  void *V_ = nullptr, *w_ = nullptr, *t_ = nullptr, *x32_ = nullptr, *y32_ = nullptr;
  void *partial_ = nullptr, *h_ = nullptr, *h2_ = nullptr, *scale_ = nullptr, *active_ = nullptr, *dx_ = nullptr;
  void *x64_ = nullptr, *P1_ = nullptr, *P2_ = nullptr, *PN_ = nullptr, *gstate_ = nullptr, *flag_h_ = nullptr;
  alignas(16) unsigned char gdev_[160] = {0};   // GmresDev (device pointers of the cycle state)
  cudaEvent_t ev_[2] = {nullptr, nullptr};
  cudaStream_t gst_ = nullptr;                    // Givens updates of the cooperative steps
  cudaEvent_t eva_ = nullptr, evg_[2] = {nullptr, nullptr};
  bool coop_ok_ = false;       // the Arnoldi step runs as one cooperative launch
  size_t coop_smem_ = 0;
  bool ffa_ok_ = false;        // ... and its float-float form fits (r <= 256, shared memory, occupancy)
  size_t coop_smem_ff_ = 0;
  void* yf_ = nullptr;         // the cycle's y split for the float-float basis sum
  size_t bytes_ = 0;
};

// scratch: (sum of the types' N^_t + n_elem) x nrhs complex128 (local sums, element phases)
template <typename R>
cudaError_t rhs_planewave(const DevArray& a, const int32_t* elem_of, const double* const* geo, int nrhs,
                          const double* th, const double* ph, const int32_t* pol, double k0, const QuadRule& q,
                          void* V, double2* scratch, cudaStream_t st);

}  // namespace mm
