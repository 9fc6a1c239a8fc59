// Dense complex128 linear algebra of the macromodel build on the device
// (Sec. II: eq. (Hdiscretized1), eq. (JM), eq. (JABE), eq. (Tm1)): the LU
// factorisations of G^(E^,H^) and of A, the solves for T, A^-1 B and the
// block-Jacobi inverse, and the products forming A, B, M, [M PJ; D PJ].
//
// Matrices are row-major, as on the host.  LU with partial pivoting, blocked
// right-looking: a panel of kNb columns is factorised by one CTA (pivot search
// by a block reduction, row swaps within the panel, scaling, rank-1 updates),
// its row swaps are applied to the other columns, the block row of U is a
// unit-lower triangular solve, and the trailing matrix is updated with one
// cuBLAS ZGEMM (a plain library GEMM).  Triangular solves with many right-hand
// sides are blocked the same way.  A row-major matrix is the column-major
// transpose of the same buffer, so every row-major product C = A B is the
// column-major product C^T = B^T A^T.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"

namespace mm {

namespace {

constexpr int kNb = 32;          // panel width
constexpr int kPanelThreads = 512;

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 csub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cinv2(double2 a) {
  const double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}

// Panel [k, k + nb) of the n x n row-major matrix A: partial pivoting over rows
// [j, n) of each column j, swaps within the panel's columns only; piv[j] = the
// row swapped with row j.  *err = 1 on an exactly zero pivot column.
__global__ void __launch_bounds__(kPanelThreads) k_lu_panel(double2* __restrict__ A, int n, int k, int nb,
                                                            int* __restrict__ piv, int* __restrict__ err) {
  __shared__ double sv[kPanelThreads];
  __shared__ int si[kPanelThreads];
  __shared__ int s_p;
  const int tid = threadIdx.x;
  for (int j = k; j < k + nb; ++j) {
    double best = -1.0;
    int bi = n;
    for (int i = j + tid; i < n; i += blockDim.x) {
      const double2 a = A[(int64_t)i * n + j];
      const double v = hypot(a.x, a.y);
      if (v > best || (v == best && i < bi)) {
        best = v;
        bi = i;
      }
    }
    sv[tid] = best;
    si[tid] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (tid < s) {
        const double v = sv[tid + s];
        const int i = si[tid + s];
        if (v > sv[tid] || (v == sv[tid] && i < si[tid])) {
          sv[tid] = v;
          si[tid] = i;
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      s_p = si[0];
      piv[j] = si[0];
      if (!(sv[0] > 0.0)) *err = 1;
    }
    __syncthreads();
    const int p = s_p;
    if (!(sv[0] > 0.0)) return;   // uniform
    if (p != j)
      for (int c = k + tid; c < k + nb; c += blockDim.x) {
        const double2 t = A[(int64_t)j * n + c];
        A[(int64_t)j * n + c] = A[(int64_t)p * n + c];
        A[(int64_t)p * n + c] = t;
      }
    __syncthreads();
    const double2 inv = cinv2(A[(int64_t)j * n + j]);
    for (int i = j + 1 + tid; i < n; i += blockDim.x) A[(int64_t)i * n + j] = cmul2(A[(int64_t)i * n + j], inv);
    __syncthreads();
    const int w = k + nb - j - 1;   // panel columns right of j
    if (w > 0) {
      const int64_t items = (int64_t)(n - j - 1) * w;
      for (int64_t t = tid; t < items; t += blockDim.x) {
        const int i = j + 1 + (int)(t / w), c = j + 1 + (int)(t % w);
        A[(int64_t)i * n + c] = csub2(A[(int64_t)i * n + c], cmul2(A[(int64_t)i * n + j], A[(int64_t)j * n + c]));
      }
    }
    __syncthreads();
  }
}

// The panel's row swaps applied to columns outside [k, k + nb) (one thread per column).
__global__ void k_lu_swaps(double2* __restrict__ A, int n, int k, int nb, const int* __restrict__ piv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n - nb) return;
  const int c = t < k ? t : t + nb;
  for (int j = k; j < k + nb; ++j) {
    const int p = piv[j];
    if (p != j) {
      const double2 x = A[(int64_t)j * n + c];
      A[(int64_t)j * n + c] = A[(int64_t)p * n + c];
      A[(int64_t)p * n + c] = x;
    }
  }
}

// X = L^-1 X for the nb rows of X (row-major, ld ldx, ncol columns) with L the
// unit lower triangle of the nb x nb block of A at (k, k) (one thread per column).
__global__ void k_trsm_lower_unit(const double2* __restrict__ A, int n, int k, int nb, double2* __restrict__ X,
                                  int64_t ldx, int ncol) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  for (int i = 1; i < nb; ++i) {
    double2 acc = X[(int64_t)i * ldx + c];
    for (int r = 0; r < i; ++r) acc = csub2(acc, cmul2(A[(int64_t)(k + i) * n + k + r], X[(int64_t)r * ldx + c]));
    X[(int64_t)i * ldx + c] = acc;
  }
}

// X = U^-1 X for the nb rows of X with U the upper triangle (with its diagonal)
// of the nb x nb block of A at (k, k).
__global__ void k_trsm_upper(const double2* __restrict__ A, int n, int k, int nb, double2* __restrict__ X,
                             int64_t ldx, int ncol) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  for (int i = nb - 1; i >= 0; --i) {
    double2 acc = X[(int64_t)i * ldx + c];
    for (int r = i + 1; r < nb; ++r)
      acc = csub2(acc, cmul2(A[(int64_t)(k + i) * n + k + r], X[(int64_t)r * ldx + c]));
    X[(int64_t)i * ldx + c] = cmul2(acc, cinv2(A[(int64_t)(k + i) * n + k + i]));
  }
}

// Row swaps of an LU's pivots applied, in order, to B (n x ncol, row-major).
__global__ void k_apply_piv(double2* __restrict__ B, int n, int ncol, const int* __restrict__ piv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  for (int j = 0; j < n; ++j) {
    const int p = piv[j];
    if (p != j) {
      const double2 x = B[(int64_t)j * ncol + c];
      B[(int64_t)j * ncol + c] = B[(int64_t)p * ncol + c];
      B[(int64_t)p * ncol + c] = x;
    }
  }
}

__global__ void k_set_identity(double2* __restrict__ A, int n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  A[t] = make_double2(t / n == t % n ? 1.0 : 0.0, 0.0);
}

struct Dense {
  cublasHandle_t h = nullptr;
  cudaStream_t st = nullptr;
  std::vector<void*> bufs;
  int* err = nullptr;
  std::string msg;
  bool ok = true;

  ~Dense() {
    if (st) cudaStreamSynchronize(st);
    for (void* p : bufs) cudaFree(p);
    if (err) cudaFree(err);
    if (h) cublasDestroy(h);
    if (st) cudaStreamDestroy(st);
  }
  bool check(cudaError_t e, const char* what) {
    if (e != cudaSuccess && ok) {
      ok = false;
      msg = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return ok;
  }
  bool checkb(cublasStatus_t s, const char* what) {
    if (s != CUBLAS_STATUS_SUCCESS && ok) {
      ok = false;
      msg = std::string(what) + ": cuBLAS status " + std::to_string((int)s);
    }
    return ok;
  }
  double2* alloc(size_t n) {
    void* p = nullptr;
    if (!check(cudaMalloc(&p, sizeof(double2) * (n ? n : 1)), "cudaMalloc")) return nullptr;
    bufs.push_back(p);
    return static_cast<double2*>(p);
  }
  double2* upload(const std::vector<cd>& v) {
    double2* d = alloc(v.size());
    if (d) check(cudaMemcpyAsync(d, v.data(), sizeof(double2) * v.size(), cudaMemcpyHostToDevice, st), "upload");
    return d;
  }
  void download(const double2* d, std::vector<cd>& v, size_t n) {
    v.resize(n);
    if (ok) check(cudaMemcpyAsync(v.data(), d, sizeof(double2) * n, cudaMemcpyDeviceToHost, st), "download");
  }
  // C (m x n) = alpha A (m x k) B (k x n) + beta C, row-major with leading dims
  void gemm(int m, int n, int k, cd alpha, const double2* A, int64_t lda, const double2* B, int64_t ldb, cd beta,
            double2* C, int64_t ldc) {
    if (!ok || m <= 0 || n <= 0 || k <= 0) return;
    const cuDoubleComplex al = make_cuDoubleComplex(alpha.real(), alpha.imag());
    const cuDoubleComplex be = make_cuDoubleComplex(beta.real(), beta.imag());
    checkb(cublasZgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, n, m, k, &al, reinterpret_cast<const cuDoubleComplex*>(B),
                       (int)ldb, reinterpret_cast<const cuDoubleComplex*>(A), (int)lda, &be,
                       reinterpret_cast<cuDoubleComplex*>(C), (int)ldc),
           "cublasZgemm");
  }
  // In-place LU with partial pivoting of the n x n matrix A; piv (n ints, device).
  void lu(double2* A, int n, int* piv) {
    for (int k = 0; k < n && ok; k += kNb) {
      const int nb = n - k < kNb ? n - k : kNb;
      k_lu_panel<<<1, kPanelThreads, 0, st>>>(A, n, k, nb, piv, err);
      if (n - nb > 0) k_lu_swaps<<<(n - nb + 255) / 256, 256, 0, st>>>(A, n, k, nb, piv);
      const int rest = n - k - nb;
      if (rest > 0) {
        k_trsm_lower_unit<<<(rest + 127) / 128, 128, 0, st>>>(A, n, k, nb, A + (int64_t)k * n + k + nb, n, rest);
        // A22 -= L21 U12
        gemm(rest, rest, nb, cd(-1, 0), A + (int64_t)(k + nb) * n + k, n, A + (int64_t)k * n + k + nb, n, cd(1, 0),
             A + (int64_t)(k + nb) * n + k + nb, n);
      }
      check(cudaGetLastError(), "LU kernels");
    }
  }
  // B = A^-1 B for the LU (A, piv) of lu(); B n x ncol row-major.
  void solve(const double2* A, int n, const int* piv, double2* B, int ncol) {
    if (!ok || ncol <= 0) return;
    const int g = (ncol + 127) / 128;
    k_apply_piv<<<g, 128, 0, st>>>(B, n, ncol, piv);
    for (int k = 0; k < n && ok; k += kNb) {   // forward: unit lower
      const int nb = n - k < kNb ? n - k : kNb;
      k_trsm_lower_unit<<<g, 128, 0, st>>>(A, n, k, nb, B + (int64_t)k * ncol, ncol, ncol);
      const int rest = n - k - nb;
      if (rest > 0)
        gemm(rest, ncol, nb, cd(-1, 0), A + (int64_t)(k + nb) * n + k, n, B + (int64_t)k * ncol, ncol, cd(1, 0),
             B + (int64_t)(k + nb) * ncol, ncol);
    }
    const int nblk = (n + kNb - 1) / kNb;
    for (int b = nblk - 1; b >= 0 && ok; --b) {   // backward: upper
      const int k = b * kNb, nb = n - k < kNb ? n - k : kNb;
      k_trsm_upper<<<g, 128, 0, st>>>(A, n, k, nb, B + (int64_t)k * ncol, ncol, ncol);
      if (k > 0)
        gemm(k, ncol, nb, cd(-1, 0), A + k, n, B + (int64_t)k * ncol, ncol, cd(1, 0), B, ncol);
    }
    check(cudaGetLastError(), "solve kernels");
  }
};

}  // namespace

// The dense steps of build_type on the device; the fills (host) are inputs.
// Returns false with a message on a CUDA or cuBLAS error or a zero pivot.
bool build_type_dense_gpu(TypeModel& tm, const std::vector<cd>& Lss, const std::vector<cd>& Lse,
                          const std::vector<cd>& Les, const std::vector<cd>& Lee, const std::vector<cd>& Kse,
                          int device, std::string& msg) {
  const int N = (int)tm.N, Nh = (int)tm.Nh;
  Dense d;
  if (!d.check(cudaSetDevice(device), "cudaSetDevice") ||
      !d.check(cudaStreamCreateWithFlags(&d.st, cudaStreamNonBlocking), "cudaStreamCreate") ||
      !d.checkb(cublasCreate(&d.h), "cublasCreate") || !d.checkb(cublasSetStream(d.h, d.st), "cublasSetStream") ||
      !d.check(cudaMalloc(&d.err, sizeof(int)), "cudaMalloc") ||
      !d.check(cudaMemsetAsync(d.err, 0, sizeof(int), d.st), "cudaMemset")) {
    msg = d.msg;
    return false;
  }
  int *piv1 = nullptr, *piv2 = nullptr, *piv3 = nullptr;
  d.check(cudaMalloc(&piv1, sizeof(int) * Nh), "cudaMalloc");
  d.check(cudaMalloc(&piv2, sizeof(int) * N), "cudaMalloc");
  d.check(cudaMalloc(&piv3, sizeof(int) * Nh), "cudaMalloc");
  d.bufs.push_back(piv1);
  d.bufs.push_back(piv2);
  d.bufs.push_back(piv3);
  double2* dLee = d.upload(Lee);                 // G^(E^,H^), factorised in place
  double2* dT = d.upload(Les);                   // -> T = G^(E^,H^)^-1 G^(E^,J)
  double2* dX1 = d.upload(tm.GHE);               // -> G^(E^,H^)^-1 G^(E^,E^)
  double2* dLse = d.upload(Lse);
  double2* dA = d.upload(Lss);                   // -> A
  double2* dB = d.upload(Kse);                   // -> B
  if (!d.ok) {
    msg = d.msg;
    return false;
  }
  d.lu(dLee, Nh, piv1);
  d.solve(dLee, Nh, piv1, dT, N);
  d.solve(dLee, Nh, piv1, dX1, Nh);
  d.gemm(N, N, Nh, cd(-1, 0), dLse, Nh, dT, N, cd(1, 0), dA, N);     // A = G^(E,J) - G^(E,H^) T
  d.gemm(N, Nh, Nh, cd(-1, 0), dLse, Nh, dX1, Nh, cd(1, 0), dB, Nh); // B = G^(E,E^) - G^(E,H^) X1
  d.download(dT, tm.T, (size_t)Nh * N);
  d.download(dA, tm.A, (size_t)N * N);
  d.download(dB, tm.B, (size_t)N * Nh);
  double2* dY = d.alloc((size_t)N * Nh);
  if (dY) d.check(cudaMemcpyAsync(dY, dB, sizeof(double2) * (size_t)N * Nh, cudaMemcpyDeviceToDevice, d.st), "copy");
  d.lu(dA, N, piv2);
  d.solve(dA, N, piv2, dY, Nh);                                        // Y = A^-1 B
  double2* dM = d.alloc((size_t)Nh * Nh);
  d.gemm(Nh, Nh, N, cd(1, 0), dT, N, dY, Nh, cd(0, 0), dM, Nh);        // M = T A^-1 B
  std::vector<cd> Y;
  d.download(dY, Y, (size_t)N * Nh);
  d.download(dM, tm.M, (size_t)Nh * Nh);
  // block-Jacobi: PJ = (D - G^(E^,H^) M)^-1, WPJ = [M; D] PJ
  double2* dS = d.upload(tm.D);
  double2* dG = d.upload(Lee);
  d.gemm(Nh, Nh, Nh, cd(-1, 0), dG, Nh, dM, Nh, cd(1, 0), dS, Nh);
  double2* dP = d.alloc((size_t)Nh * Nh);
  if (dP) k_set_identity<<<(unsigned)(((int64_t)Nh * Nh + 255) / 256), 256, 0, d.st>>>(dP, Nh);
  d.lu(dS, Nh, piv3);
  d.solve(dS, Nh, piv3, dP, Nh);
  double2* dMD = d.alloc((size_t)2 * Nh * Nh);
  if (dMD) {
    d.check(cudaMemcpyAsync(dMD, dM, sizeof(double2) * (size_t)Nh * Nh, cudaMemcpyDeviceToDevice, d.st), "copy");
    d.check(cudaMemcpyAsync(dMD + (size_t)Nh * Nh, tm.D.data(), sizeof(double2) * (size_t)Nh * Nh,
                            cudaMemcpyHostToDevice, d.st),
            "copy");
  }
  double2* dW = d.alloc((size_t)2 * Nh * Nh);
  d.gemm(2 * Nh, Nh, Nh, cd(1, 0), dMD, Nh, dP, Nh, cd(0, 0), dW, Nh);
  d.download(dP, tm.PJ, (size_t)Nh * Nh);
  d.download(dW, tm.WPJ, (size_t)2 * Nh * Nh);
  int herr = 0;
  if (d.ok) d.check(cudaMemcpyAsync(&herr, d.err, sizeof(int), cudaMemcpyDeviceToHost, d.st), "download");
  if (d.ok) d.check(cudaStreamSynchronize(d.st), "synchronize");
  if (!d.ok) {
    msg = d.msg;
    return false;
  }
  if (herr) {
    msg = "singular matrix in macromodel build";
    return false;
  }
  tm.JE.resize(Y.size());
  for (size_t i = 0; i < Y.size(); ++i) tm.JE[i] = -Y[i];
  return true;
}

}  // namespace mm
