// Tensor-core (tcgen05) form of the macromodel contraction, BF16 or FP16 inputs
// with FP32 accumulation in tensor memory (Sec. III / eq. (MV_product1): the
// per-type products u = M x, v = D x of identical elements).
//
// The complex product is a real GEMM with interleaved real/imaginary rows:
//   A (4 Nh x 2 Nh): row 2i = [Re W_i, -Im W_i], row 2i+1 = [Im W_i, Re W_i]
//                    (W = [M; D] stacked, so i runs over 2 Nh output rows);
//   B (ncols x 2 Nh): column (element, rhs) = [Re x_e, Im x_e];
//   C = A B^T: row 2i = Re out_i, row 2i+1 = Im out_i.
// Both operands are K-major in global memory, padded to multiples of the tile.
//
// Kernel: one CTA per 128 x 128 output tile, 128 threads.  K slices of 64
// elements (128 bytes per row) are staged in shared memory in the 128-byte
// swizzled K-major layout, double-buffered; thread 0 issues four
// tcgen05.mma (K = 16 each) per slice and commits them to an mbarrier; the
// accumulator lives in 128 TMEM columns.  Every mbarrier wait is bounded: on
// expiry the kernel records an error and stops issuing work.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "tc_gemm.h"

namespace mm {

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64;
constexpr uint32_t kTmemCols = 128;
constexpr long long kSpinLimit = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 1024-byte atoms.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 bytes
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor for kind::f16: FP32 accumulate, K-major A and B.
__host__ __device__ constexpr uint32_t make_idesc(bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(TBN >> 3) << 17) |
         ((uint32_t)(TBM >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Copies a 128 x 64 tile (K-major rows of 128 bytes) into the swizzled layout.
__device__ __forceinline__ void load_tile(const uint16_t* __restrict__ g, int64_t ld, int row0, int k0,
                                          unsigned char* s) {
  for (int c = threadIdx.x; c < 128 * 8; c += blockDim.x) {
    const int r = c >> 3, ch = c & 7;
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(g + (int64_t)(row0 + r) * ld + k0 + ch * 8));
    *reinterpret_cast<uint4*>(s + r * 128 + ((ch ^ (r & 7)) << 4)) = v;
  }
}

}  // namespace

// C (Mp x Np, FP32) = A (Mp x Kp) B^T (Np x Kp); epilogue writes complex rows
// (2i, 2i+1) of C to out_u (i < Nh) or out_v (i >= Nh) for column n = j*nrhs+c.
template <bool BF16>
__global__ void __launch_bounds__(128) k_tc_gemm(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B,
                                                 int Kp, int Nh, int ncols, int nrhs, const int32_t* __restrict__ elems,
                                                 const int64_t* __restrict__ off, float2* __restrict__ out_u,
                                                 float2* __restrict__ out_v, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned stage buffers
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA[2] = {base, base + 16384};
  unsigned char* sB[2] = {base + 32768, base + 49152};
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * TBN;
  const int nk = Kp / TBK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
  }
  load_tile(A, Kp, m0, 0, sA[0]);
  load_tile(B, Kp, n0, 0, sB[0]);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = make_idesc(BF16);
  bool ok = true;
  int uses[2] = {0, 0};
  for (int kt = 0; kt < nk && ok; ++kt) {
    const int s = kt & 1;
    if (tid == 0) {
      const uint64_t da = make_desc(smem_u32(sA[s])), db = make_desc(smem_u32(sB[s]));
#pragma unroll
      for (int kk = 0; kk < TBK / 16; ++kk) {
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        const uint64_t a = da + (uint64_t)((kk * 32) >> 4), b = db + (uint64_t)((kk * 32) >> 4);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[s]))
                   : "memory");
    }
    ++uses[s];
    if (kt + 1 < nk) {
      const int s1 = s ^ 1;
      // the products that read stage s1 must be done before it is overwritten;
      // thread 0 waits (bounded) and the barrier makes the outcome block-uniform
      bool w_ok = true;
      if (uses[s1] > 0 && tid == 0) w_ok = mbar_wait(smem_u32(&mbar[s1]), (uses[s1] - 1) & 1);
      ok = __syncthreads_and(w_ok) != 0;
      if (ok) {
        load_tile(A, Kp, m0, (kt + 1) * TBK, sA[s1]);
        load_tile(B, Kp, n0, (kt + 1) * TBK, sB[s1]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
  }
  // wait for the last slice's products (they complete after all earlier ones)
  {
    bool w_ok = ok;
    if (ok && nk > 0 && tid == 0) {
      const int sl = (nk - 1) & 1;
      w_ok = mbar_wait(smem_u32(&mbar[sl]), (uses[sl] - 1) & 1);
    }
    ok = __syncthreads_and(w_ok) != 0;
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // epilogue: warp w holds rows 32w..32w+31; lane pairs (2i, 2i+1) are (Re, Im)
    const int row = m0 + warp * 32 + lane;
    const int orow = row >> 1;                 // complex output row in the stacked [M; D]
    for (int c0 = 0; c0 < TBN; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float v = __uint_as_float(r[q]);
        const float im = __shfl_down_sync(0xffffffffu, v, 1);
        const int n = n0 + c0 + q;
        if ((lane & 1) == 0 && n < ncols && orow < 2 * Nh) {
          const int j = n / nrhs, cc = n % nrhs;
          const int64_t e0 = off[elems[j]];
          const float2 o = make_float2(v, im);
          if (orow < Nh)
            out_u[(e0 + orow) * nrhs + cc] = o;
          else
            out_v[(e0 + orow - Nh) * nrhs + cc] = o;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// B^T operand: column n = (element elems[n / nrhs], rhs n % nrhs) -> [Re x, Im x], padded.
template <bool BF16>
__global__ void k_pack_b(const float2* __restrict__ x, int Nh, int ncols, int nrhs, const int32_t* __restrict__ elems,
                         const int64_t* __restrict__ off, int Np, int Kp, uint16_t* __restrict__ Bt) {
  const int64_t total = (int64_t)Np * Kp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(t / Kp), kq = (int)(t % Kp);
    float v = 0.f;
    if (n < ncols && kq < 2 * Nh) {
      const int j = n / nrhs, c = n % nrhs;
      const int kk = kq < Nh ? kq : kq - Nh;
      const float2 xv = x[(off[elems[j]] + kk) * nrhs + c];
      v = kq < Nh ? xv.x : xv.y;
    }
    uint16_t h;
    if (BF16) {
      const __nv_bfloat16 b = __float2bfloat16_rn(v);
      h = *reinterpret_cast<const uint16_t*>(&b);
    } else {
      const __half b = __float2half_rn(v);
      h = *reinterpret_cast<const uint16_t*>(&b);
    }
    Bt[t] = h;
  }
}

size_t tc_smem_bytes() { return 4 * 16384 + 1024; }

cudaError_t tc_gemm_init() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes());
}

cudaError_t tc_macro_gemm(bool bf16, const uint16_t* A, int Mp, int Kp, int Nh, const int32_t* elems, int nel,
                          int nrhs, const int64_t* off, const float2* x, uint16_t* Bt, size_t bt_cap, float2* u,
                          float2* v, int* err, cudaStream_t st) {
  const int ncols = nel * nrhs;
  const int Np = (ncols + TBN - 1) / TBN * TBN;
  if ((size_t)Np * Kp > bt_cap) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)Np * Kp;
  const unsigned pb = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
  if (bf16)
    k_pack_b<true><<<pb, 256, 0, st>>>(x, Nh, ncols, nrhs, elems, off, Np, Kp, Bt);
  else
    k_pack_b<false><<<pb, 256, 0, st>>>(x, Nh, ncols, nrhs, elems, off, Np, Kp, Bt);
  dim3 g(Mp / TBM, Np / TBN);
  if (bf16)
    k_tc_gemm<true><<<g, 128, tc_smem_bytes(), st>>>(A, Bt, Kp, Nh, ncols, nrhs, elems, off, u, v, err);
  else
    k_tc_gemm<false><<<g, 128, tc_smem_bytes(), st>>>(A, Bt, Kp, Nh, ncols, nrhs, elems, off, u, v, err);
  return cudaGetLastError();
}

int tc_tile_m() { return TBM; }
int tc_tile_k() { return TBK; }
int tc_tile_n() { return TBN; }

}  // namespace mm
