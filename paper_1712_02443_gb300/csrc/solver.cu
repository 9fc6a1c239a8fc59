// GMRES (Sec. V; Saad and Schultz 1986) for the final system (eq. (finalsystem)),
// with FP64 Arnoldi (classical Gram-Schmidt applied twice) and Givens rotations,
// independent columns for several right-hand sides, and FP64 iterative
// refinement around a complex64 inner operator.  Also the plane-wave
// excitation kernel (Sec. IV, eq. (V1)).
#include <cmath>
#include <cstdio>
#include <vector>

#include "solver.h"

namespace mm {

typedef double2 Z;

__device__ __forceinline__ Z zmul(Z a, Z b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ Z zconjmul(Z a, Z b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__global__ void k_to_c64(const Z* __restrict__ s, float2* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = make_float2((float)s[i].x, (float)s[i].y);
}
__global__ void k_to_c128(const float2* __restrict__ s, Z* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = make_double2((double)s[i].x, (double)s[i].y);
}

// partial[(i * r + j) * nblk + blk] = sum over this block's rows of conj(V_i[n, j]) w[n, j]
__global__ void k_dot_partial(const Z* __restrict__ V, int64_t vstride, const Z* __restrict__ w, int64_t N, int r,
                              int nblk, double* __restrict__ partial) {
  const int i = blockIdx.y, j = blockIdx.z, blk = blockIdx.x;
  const Z* vi = V + (int64_t)i * vstride;
  const int64_t chunk = (N + nblk - 1) / nblk;
  const int64_t n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
  double sr = 0, si = 0;
  for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    Z p = zconjmul(vi[n * r + j], w[n * r + j]);
    sr += p.x;
    si += p.y;
  }
  __shared__ double s_r[256], s_i[256];
  s_r[threadIdx.x] = sr;
  s_i[threadIdx.x] = si;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s_r[threadIdx.x] += s_r[threadIdx.x + s];
      s_i[threadIdx.x] += s_i[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int64_t o = ((int64_t)i * r + j) * nblk + blk;
    partial[2 * o] = s_r[0];
    partial[2 * o + 1] = s_i[0];
  }
}

// out[i * r + j] = sum_blk partial (fixed order: deterministic)
__global__ void k_dot_final(const double* __restrict__ partial, int nvec, int r, int nblk, Z* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nvec * r) return;
  double sr = 0, si = 0;
  for (int b = 0; b < nblk; ++b) {
    sr += partial[2 * ((int64_t)t * nblk + b)];
    si += partial[2 * ((int64_t)t * nblk + b) + 1];
  }
  out[t] = make_double2(sr, si);
}

// w[n, j] -= sum_{i < nvec} V_i[n, j] h[i * r + j]
__global__ void k_orth_update(const Z* __restrict__ V, int64_t vstride, const Z* __restrict__ h, int nvec, int64_t N,
                              int r, Z* __restrict__ w) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % r);
    Z acc = w[t];
    for (int i = 0; i < nvec; ++i) {
      Z p = zmul(V[(int64_t)i * vstride + t], h[i * r + j]);
      acc.x -= p.x;
      acc.y -= p.y;
    }
    w[t] = acc;
  }
}

// dst[n, j] = active[j] ? src[n, j] * scale[j] : 0
__global__ void k_scale_cols(const Z* __restrict__ src, const double* __restrict__ scale,
                             const int32_t* __restrict__ active, int64_t N, int r, Z* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % r);
    Z v = src[t];
    double s = active[j] ? scale[j] : 0.0;
    dst[t] = make_double2(v.x * s, v.y * s);
  }
}

// x[n, j] += sum_i V_i[n, j] y[i * r + j]
__global__ void k_add_basis(const Z* __restrict__ V, int64_t vstride, const Z* __restrict__ y, int nvec, int64_t N,
                            int r, Z* __restrict__ x) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % r);
    Z acc = x[t];
    for (int i = 0; i < nvec; ++i) {
      Z p = zmul(V[(int64_t)i * vstride + t], y[i * r + j]);
      acc.x += p.x;
      acc.y += p.y;
    }
    x[t] = acc;
  }
}

// d = a - b
__global__ void k_sub(const Z* a, const Z* b, int64_t n, Z* d) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    d[t] = make_double2(a[t].x - b[t].x, a[t].y - b[t].y);
}
// x += d
__global__ void k_add(const Z* __restrict__ d, int64_t n, Z* __restrict__ x) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    x[t] = make_double2(x[t].x + d[t].x, x[t].y + d[t].y);
}

static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

#define MM_CK(x)                          \
  do {                                    \
    cudaError_t _e = (x);                 \
    if (_e != cudaSuccess) return {MM_ECUDA, cudaGetErrorString(_e)}; \
  } while (0)

Status Solver::ensure(int64_t N, int r, int m) {
  if (N == N_ && r == r_ && m <= m_) return {MM_OK, ""};
  release();
  N_ = N; r_ = r; m_ = m;
  nblk_ = (int)std::min<int64_t>(128, std::max<int64_t>(1, N / 2048));
  size_t vec = sizeof(Z) * (size_t)N * r;
  MM_CK(cudaMalloc(&V_, vec * (m + 1)));
  MM_CK(cudaMalloc(&w_, vec));
  MM_CK(cudaMalloc(&t_, vec));
  MM_CK(cudaMalloc(&x32_, sizeof(float2) * (size_t)N * r));
  MM_CK(cudaMalloc(&y32_, sizeof(float2) * (size_t)N * r));
  MM_CK(cudaMalloc(&partial_, sizeof(double) * 2 * (size_t)(m + 1) * r * nblk_));
  MM_CK(cudaMalloc(&h_, sizeof(Z) * (size_t)(m + 1) * r));
  MM_CK(cudaMalloc(&h2_, sizeof(Z) * (size_t)(m + 1) * r));
  MM_CK(cudaMalloc(&scale_, sizeof(double) * r));
  MM_CK(cudaMalloc(&active_, sizeof(int32_t) * r));
  MM_CK(cudaMalloc(&dx_, vec));
  bytes_ = vec * (m + 4) + sizeof(float2) * 2 * (size_t)N * r;
  return {MM_OK, ""};
}

void Solver::release() {
  void* ps[] = {V_, w_, t_, x32_, y32_, partial_, h_, h2_, scale_, active_, dx_};
  for (void* p : ps)
    if (p) cudaFree(p);
  V_ = w_ = t_ = nullptr;
  x32_ = y32_ = nullptr;
  partial_ = nullptr;
  h_ = h2_ = nullptr;
  scale_ = nullptr;
  active_ = nullptr;
  dx_ = nullptr;
  N_ = 0; r_ = 0; m_ = 0;
}

// h[i * r + j] = <V_i, w> for i < nvec
Status Solver::dots(const Z* V, int64_t vstride, int nvec, const Z* w, Z* out, cudaStream_t st) {
  if (prof) prof->begin(7, st);
  dim3 g(nblk_, nvec, r_);
  k_dot_partial<<<g, 256, 0, st>>>(V, vstride, w, N_, r_, nblk_, static_cast<double*>(partial_));
  k_dot_final<<<(nvec * r_ + 127) / 128, 128, 0, st>>>(static_cast<const double*>(partial_), nvec, r_, nblk_, out);
  if (prof) prof->end(st, 2);
  MM_CK(cudaGetLastError());
  return {MM_OK, ""};
}

// Applies the operator in double-precision vectors, at precision `prec`.
Status Solver::apply(const Z* in, Z* out, int prec, cudaStream_t st) {
  ++matvecs;
  const int64_t n = N_ * r_;
  if (prec == MM_C128) return op64(in, out, st);
  if (prof) prof->begin(7, st);
  k_to_c64<<<grid_for(n), 256, 0, st>>>(in, static_cast<float2*>(x32_), n);
  if (prof) prof->end(st, 1);
  Status s = op32(x32_, y32_, st);
  if (s.code != MM_OK) return s;
  if (prof) prof->begin(7, st);
  k_to_c128<<<grid_for(n), 256, 0, st>>>(static_cast<const float2*>(y32_), out, n);
  if (prof) prof->end(st, 1);
  MM_CK(cudaGetLastError());
  return {MM_OK, ""};
}

// Restarted GMRES on A x = b; x accumulates.  x_zero: x is 0 on entry, so the
// first residual is b itself (no product).  A cycle stops at the restart length
// or when every column's Givens residual estimate meets tol_abs; in the latter
// case GMRES returns (the caller checks the true residual).  tol_abs[j] is the
// absolute residual target of column j.
Status Solver::gmres(const Z* b, Z* x, bool x_zero, const std::vector<double>& tol_abs, int prec, int max_iter,
                     int& iters, std::vector<double>& res, cudaStream_t st) {
  const int64_t N = N_;
  const int r = r_, m = m_;
  const int64_t n = N * r;
  const int64_t vs = n;
  Z* V = static_cast<Z*>(V_);
  Z* w = static_cast<Z*>(w_);
  Z* h = static_cast<Z*>(h_);
  Z* h2 = static_cast<Z*>(h2_);
  iters = 0;
  res.assign(r, 0.0);
  std::vector<std::complex<double>> Hh((size_t)(m + 1) * m * r), cs((size_t)m * r), sn((size_t)m * r),
      g((size_t)(m + 1) * r);
  std::vector<Z> hbuf((size_t)(m + 1) * r), hb2((size_t)(m + 1) * r);
  std::vector<int32_t> active(r), kdone(r);
  std::vector<double> sc(r);
  bool first = true;
  for (;;) {
    // r0 = b - A x
    if (first && x_zero) {
      MM_CK(cudaMemcpyAsync(w, b, sizeof(Z) * n, cudaMemcpyDeviceToDevice, st));
    } else {
      Status s0 = apply(x, w, prec, st);
      if (s0.code != MM_OK) return s0;
      k_sub<<<grid_for(n), 256, 0, st>>>(b, w, n, w);
    }
    first = false;
    Status s = dots(w, 0, 1, w, h, st);
    if (s.code != MM_OK) return s;
    MM_CK(cudaMemcpyAsync(hbuf.data(), h, sizeof(Z) * r, cudaMemcpyDeviceToHost, st));
    MM_CK(cudaStreamSynchronize(st));
    bool any = false;
    for (int j = 0; j < r; ++j) {
      double beta = std::sqrt(std::max(0.0, hbuf[j].x));
      res[j] = beta;
      if (!std::isfinite(beta)) return {MM_EBREAKDOWN, "non-finite residual in GMRES"};
      active[j] = beta > tol_abs[j];
      any |= (bool)active[j];
      sc[j] = beta > 0 ? 1.0 / beta : 0.0;
      for (int i = 0; i <= m; ++i) g[(size_t)i * r + j] = 0;
      g[j] = beta;
      kdone[j] = 0;
    }
    if (!any || iters >= max_iter) return {MM_OK, ""};
    MM_CK(cudaMemcpyAsync(scale_, sc.data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
    MM_CK(cudaMemcpyAsync(active_, active.data(), sizeof(int32_t) * r, cudaMemcpyHostToDevice, st));
    k_scale_cols<<<grid_for(n), 256, 0, st>>>(w, static_cast<double*>(scale_), static_cast<int32_t*>(active_), N, r, V);
    bool all_met = false;
    for (int k = 0; k < m && iters < max_iter; ++k) {
      s = apply(V + (int64_t)k * vs, w, prec, st);
      if (s.code != MM_OK) return s;
      // classical Gram-Schmidt, twice
      s = dots(V, vs, k + 1, w, h, st);
      if (s.code != MM_OK) return s;
      if (prof) prof->begin(7, st);
      k_orth_update<<<grid_for(n), 256, 0, st>>>(V, vs, h, k + 1, N, r, w);
      if (prof) prof->end(st, 1);
      s = dots(V, vs, k + 1, w, h2, st);
      if (s.code != MM_OK) return s;
      if (prof) prof->begin(7, st);
      k_orth_update<<<grid_for(n), 256, 0, st>>>(V, vs, h2, k + 1, N, r, w);
      if (prof) prof->end(st, 1);
      s = dots(w, 0, 1, w, h2 + (size_t)(k + 1) * r, st);
      if (s.code != MM_OK) return s;
      MM_CK(cudaMemcpyAsync(hbuf.data(), h, sizeof(Z) * (size_t)(k + 1) * r, cudaMemcpyDeviceToHost, st));
      MM_CK(cudaMemcpyAsync(hb2.data(), h2, sizeof(Z) * (size_t)(k + 2) * r, cudaMemcpyDeviceToHost, st));
      MM_CK(cudaStreamSynchronize(st));
      ++iters;
      bool still = false;
      for (int j = 0; j < r; ++j) {
        if (!active[j]) {
          sc[j] = 0.0;
          continue;
        }
        std::complex<double>* H = &Hh[(size_t)j * (m + 1) * m];   // column-major (m+1) x m per column j
        for (int i = 0; i <= k; ++i)
          H[(size_t)k * (m + 1) + i] = std::complex<double>(hbuf[(size_t)i * r + j].x + hb2[(size_t)i * r + j].x,
                                                            hbuf[(size_t)i * r + j].y + hb2[(size_t)i * r + j].y);
        double hn = std::sqrt(std::max(0.0, hb2[(size_t)(k + 1) * r + j].x));
        if (!std::isfinite(hn)) return {MM_EBREAKDOWN, "non-finite Arnoldi norm"};
        H[(size_t)k * (m + 1) + k + 1] = hn;
        for (int i = 0; i < k; ++i) {
          std::complex<double> c = cs[(size_t)i * r + j], sg = sn[(size_t)i * r + j];
          std::complex<double> a = H[(size_t)k * (m + 1) + i], bb = H[(size_t)k * (m + 1) + i + 1];
          H[(size_t)k * (m + 1) + i] = std::conj(c) * a + std::conj(sg) * bb;
          H[(size_t)k * (m + 1) + i + 1] = -sg * a + c * bb;
        }
        std::complex<double> a = H[(size_t)k * (m + 1) + k], bb = H[(size_t)k * (m + 1) + k + 1];
        double den = std::sqrt(std::norm(a) + std::norm(bb));
        std::complex<double> c = den > 0 ? a / den : 1.0, sg = den > 0 ? bb / den : 0.0;
        cs[(size_t)k * r + j] = c;
        sn[(size_t)k * r + j] = sg;
        H[(size_t)k * (m + 1) + k] = den;
        H[(size_t)k * (m + 1) + k + 1] = 0.0;
        std::complex<double> gk = g[(size_t)k * r + j];
        g[(size_t)(k + 1) * r + j] = -sg * gk;
        g[(size_t)k * r + j] = std::conj(c) * gk;
        kdone[j] = k + 1;
        res[j] = std::abs(g[(size_t)(k + 1) * r + j]);
        if (res[j] <= tol_abs[j] || hn == 0.0) {
          active[j] = 0;
          sc[j] = 0.0;
        } else {
          sc[j] = 1.0 / hn;
          still = true;
        }
      }
      if (!still) {
        all_met = true;
        break;
      }
      MM_CK(cudaMemcpyAsync(scale_, sc.data(), sizeof(double) * r, cudaMemcpyHostToDevice, st));
      MM_CK(cudaMemcpyAsync(active_, active.data(), sizeof(int32_t) * r, cudaMemcpyHostToDevice, st));
      k_scale_cols<<<grid_for(n), 256, 0, st>>>(w, static_cast<double*>(scale_), static_cast<int32_t*>(active_), N, r,
                                                V + (int64_t)(k + 1) * vs);
    }
    // y_j = H_j^-1 g_j (upper triangular), x += V y
    int kmax = 0;
    for (int j = 0; j < r; ++j) kmax = std::max(kmax, kdone[j]);
    std::vector<Z> y((size_t)std::max(kmax, 1) * r, make_double2(0, 0));
    for (int j = 0; j < r; ++j) {
      int kj = kdone[j];
      std::complex<double>* H = &Hh[(size_t)j * (m + 1) * m];
      std::vector<std::complex<double>> yy(kj);
      for (int i = kj - 1; i >= 0; --i) {
        std::complex<double> acc = g[(size_t)i * r + j];
        for (int q = i + 1; q < kj; ++q) acc -= H[(size_t)q * (m + 1) + i] * yy[q];
        yy[i] = acc / H[(size_t)i * (m + 1) + i];
      }
      for (int i = 0; i < kj; ++i) y[(size_t)i * r + j] = make_double2(yy[i].real(), yy[i].imag());
    }
    if (kmax > 0) {
      MM_CK(cudaMemcpyAsync(h, y.data(), sizeof(Z) * (size_t)kmax * r, cudaMemcpyHostToDevice, st));
      if (prof) prof->begin(7, st);
      k_add_basis<<<grid_for(n), 256, 0, st>>>(V, vs, h, kmax, N, r, x);
      if (prof) prof->end(st, 1);
      MM_CK(cudaGetLastError());
    }
    // the synchronous copy of y must complete before the host vector goes away
    MM_CK(cudaStreamSynchronize(st));
    if (all_met || iters >= max_iter) return {MM_OK, ""};
  }
}

// Column norms ||a_j|| (synchronous).
Status Solver::norms(const Z* a, std::vector<double>& out, cudaStream_t st) {
  Status s = dots(a, 0, 1, a, static_cast<Z*>(h_), st);
  if (s.code != MM_OK) return s;
  std::vector<Z> hb(r_);
  MM_CK(cudaMemcpyAsync(hb.data(), h_, sizeof(Z) * r_, cudaMemcpyDeviceToHost, st));
  MM_CK(cudaStreamSynchronize(st));
  out.resize(r_);
  for (int j = 0; j < r_; ++j) out[j] = std::sqrt(std::max(0.0, hb[j].x));
  return {MM_OK, ""};
}

Status Solver::solve(const Z* b, Z* x, double tol, int prec, int refine, double inner_tol, int max_iter,
                     int& iters, int& refinements, double& relres, bool& converged, cudaStream_t st) {
  const int64_t n = N_ * r_;
  iters = 0;
  refinements = 0;
  matvecs = 0;
  std::vector<double> bn, rn, res;
  Status s = norms(b, bn, st);
  if (s.code != MM_OK) return s;
  MM_CK(cudaMemsetAsync(x, 0, sizeof(Z) * n, st));
  Z* rr = static_cast<Z*>(t_);
  auto done = [&]() {
    bool d = true;
    for (int j = 0; j < r_; ++j) d &= rn[j] <= tol * bn[j];
    return d;
  };
  if (prec == MM_C128 || !refine) {
    // plain GMRES at one precision; the true residual (same precision) confirms each exit
    std::vector<double> tabs(r_);
    for (int j = 0; j < r_; ++j) tabs[j] = tol * bn[j];
    bool x_zero = true;
    for (;;) {
      int it = 0;
      s = gmres(b, x, x_zero, tabs, prec, max_iter - iters, it, res, st);
      if (s.code != MM_OK) return s;
      iters += it;
      x_zero = false;
      s = apply(x, rr, prec, st);
      if (s.code != MM_OK) return s;
      k_sub<<<grid_for(n), 256, 0, st>>>(b, rr, n, rr);
      s = norms(rr, rn, st);
      if (s.code != MM_OK) return s;
      if (done() || iters >= max_iter || it == 0) break;
    }
  } else {
    // FP64 iterative refinement: GMRES on the complex64 operator solves for the
    // correction of the current residual, computed with the complex128 operator.
    Z* dx = static_cast<Z*>(dx_);
    MM_CK(cudaMemcpyAsync(rr, b, sizeof(Z) * n, cudaMemcpyDeviceToDevice, st));
    rn = bn;
    for (;;) {
      std::vector<double> tabs(r_);
      for (int j = 0; j < r_; ++j) tabs[j] = std::max(inner_tol * rn[j], 0.5 * tol * bn[j]);
      int it = 0;
      MM_CK(cudaMemsetAsync(dx, 0, sizeof(Z) * n, st));
      s = gmres(rr, dx, true, tabs, MM_C64, max_iter - iters, it, res, st);
      if (s.code != MM_OK) return s;
      iters += it;
      ++refinements;
      k_add<<<grid_for(n), 256, 0, st>>>(dx, n, x);
      s = apply(x, rr, MM_C128, st);
      if (s.code != MM_OK) return s;
      k_sub<<<grid_for(n), 256, 0, st>>>(b, rr, n, rr);
      s = norms(rr, rn, st);
      if (s.code != MM_OK) return s;
      if (done() || iters >= max_iter || it == 0) break;
    }
  }
  relres = 0;
  converged = true;
  for (int j = 0; j < r_; ++j) {
    double rel = bn[j] > 0 ? rn[j] / bn[j] : rn[j];
    relres = std::max(relres, rel);
    converged &= rel <= tol * (1.0 + 1e-9);
  }
  if (!std::isfinite(relres)) return {MM_EBREAKDOWN, "non-finite residual"};
  return {MM_OK, ""};
}

// ---------------------------------------------------------------- plane-wave excitation
// V[n, j] = -sum_{T+-} sum_q w_q A f_n(r_q) . p_j exp(-j k khat_j . r_q)  (7-point rule)
template <typename R>
__global__ void k_rhs_planewave(int64_t N, int nrhs, const int32_t* __restrict__ elem_of,
                                const int32_t* __restrict__ type_of, const int64_t* __restrict__ off,
                                const double* const* __restrict__ geo, const double* __restrict__ eoff,
                                const double* __restrict__ theta, const double* __restrict__ phi,
                                const int32_t* __restrict__ pol, double k0, QuadRule q,
                                typename V2<R>::T* __restrict__ V) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * nrhs) return;
  const int64_t n = t / nrhs;
  const int j = (int)(t % nrhs);
  const int e = elem_of[n];
  const int ty = type_of[e];
  const double* gp = geo[ty] + 13 * (n - off[e]);
  const double ox = eoff[3 * e], oy = eoff[3 * e + 1], oz = eoff[3 * e + 2];
  double st, ct, sp, cp;
  sincos(theta[j], &st, &ct);
  sincos(phi[j], &sp, &cp);
  const double kx = -st * cp, ky = -st * sp, kz = -ct;
  double px, py, pz;
  if (pol[j] == 0) { px = ct * cp; py = ct * sp; pz = -st; }
  else { px = -sp; py = cp; pz = 0.0; }
  double accr = 0, acci = 0;
  const double l = gp[12];
  for (int side = 0; side < 2; ++side) {
    const double ax = gp[0] + ox, ay = gp[1] + oy, az = gp[2] + oz;
    const double bx = gp[3] + ox, by = gp[4] + oy, bz = gp[5] + oz;
    const double fx = gp[6 + 3 * side] + ox, fy = gp[7 + 3 * side] + oy, fz = gp[8 + 3 * side] + oz;
    const double ux = bx - ax, uy = by - ay, uz = bz - az, vx = fx - ax, vy = fy - ay, vz = fz - az;
    const double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
    const double A = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    const double sg = side == 0 ? 1.0 : -1.0;
    for (int i = 0; i < q.n; ++i) {
      const double rx = q.b0[i] * ax + q.b1[i] * bx + q.b2[i] * fx;
      const double ry = q.b0[i] * ay + q.b1[i] * by + q.b2[i] * fy;
      const double rz = q.b0[i] * az + q.b1[i] * bz + q.b2[i] * fz;
      const double s = sg * l / (2.0 * A);
      const double dotp = s * ((rx - fx) * px + (ry - fy) * py + (rz - fz) * pz);
      double sn, cs;
      sincos(-k0 * (kx * rx + ky * ry + kz * rz), &sn, &cs);
      const double wA = q.w[i] * A;
      accr += wA * dotp * cs;
      acci += wA * dotp * sn;
    }
  }
  typename V2<R>::T out;
  out.x = (R)(-accr);
  out.y = (R)(-acci);
  V[t] = out;
}

template <typename R>
cudaError_t rhs_planewave(const DevArray& a, const int32_t* elem_of, const double* const* geo, int nrhs,
                          const double* th, const double* ph, const int32_t* pol, double k0, const QuadRule& q,
                          void* V, cudaStream_t st) {
  const int64_t tot = a.N * nrhs;
  k_rhs_planewave<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
      a.N, nrhs, elem_of, a.type_of, a.off, geo, a.eoff, th, ph, pol, k0, q, static_cast<typename V2<R>::T*>(V));
  return cudaGetLastError();
}
template cudaError_t rhs_planewave<float>(const DevArray&, const int32_t*, const double* const*, int, const double*,
                                          const double*, const int32_t*, double, const QuadRule&, void*, cudaStream_t);
template cudaError_t rhs_planewave<double>(const DevArray&, const int32_t*, const double* const*, int, const double*,
                                           const double*, const int32_t*, double, const QuadRule&, void*,
                                           cudaStream_t);

}  // namespace mm
